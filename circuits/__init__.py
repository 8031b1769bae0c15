"""Seeded synthetic circuit generators shared by the oracle, the GPU library, the tests and the bench.

This module only *describes* circuits: it builds gate records (2x2 matrices, target, controls) from seeds.
It never applies a gate to a state, so it holds none of the simulation arithmetic; both the FP64 oracle
and the CUDA path consume the records it produces, byte for byte.

Qubit convention (the paper's stride rule, Sec. V.A, Eq. for the strided pair update): qubit ``t`` is bit
``t`` of the amplitude index, so a gate on qubit ``t`` pairs indices ``k`` and ``k + 2**t``.

Gate record (96 bytes, identical to ``sv_gate`` in ``include/sv.h``)::

    U[8]        float64   row-major q11, q12, q21, q22 as (re, im) pairs (a row of V for GATE_U4 / GATE_U4_ROW)
    kind        int32     GATE_U (0), GATE_SWAP (1), GATE_U4 (2) or GATE_U4_ROW (3)
    target      int32     target qubit (first qubit of a SWAP; qubit of index bit b0 of a two-qubit gate)
    target2     int32     second qubit of a SWAP or two-qubit gate (bit b1), -1 otherwise
    ncontrols   int32     number of control qubits (0..4)
    controls[4] int32     control qubits; a gate acts only where every control bit is 1 (Sec. V.B)

A dense two-qubit gate V (4x4, entry order b0 + 2 b1) takes four consecutive records: GATE_U4 with row 0,
then three GATE_U4_ROW records with rows 1..3 (same targets, no controls).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

GATE_U = 0
GATE_SWAP = 1
GATE_U4 = 2
GATE_U4_ROW = 3
MAX_CONTROLS = 4

GATE_DTYPE = np.dtype(
    [
        ("U", "<f8", (8,)),
        ("kind", "<i4"),
        ("target", "<i4"),
        ("target2", "<i4"),
        ("ncontrols", "<i4"),
        ("controls", "<i4", (MAX_CONTROLS,)),
    ],
    align=True,
)
assert GATE_DTYPE.itemsize == 96

# Gate constants (Sec. II.A: Pauli X and Hadamard; the others are standard single-qubit gates).
SQRT1_2 = 1.0 / math.sqrt(2.0)
I2 = np.eye(2, dtype=np.complex128)
X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)
H = np.array([[SQRT1_2, SQRT1_2], [SQRT1_2, -SQRT1_2]], dtype=np.complex128)
S = np.array([[1, 0], [0, 1j]], dtype=np.complex128)
T = np.array([[1, 0], [0, np.exp(1j * math.pi / 4)]], dtype=np.complex128)


def phase(theta: float) -> np.ndarray:
    """diag(1, e^{i theta}); the QFT's controlled rotation R_k is phase(2 pi / 2^k)."""
    return np.array([[1, 0], [0, complex(math.cos(theta), math.sin(theta))]], dtype=np.complex128)


def rx(theta: float) -> np.ndarray:
    c, s = math.cos(theta / 2), math.sin(theta / 2)
    return np.array([[c, -1j * s], [-1j * s, c]], dtype=np.complex128)


def ry(theta: float) -> np.ndarray:
    c, s = math.cos(theta / 2), math.sin(theta / 2)
    return np.array([[c, -s], [s, c]], dtype=np.complex128)


def rz(theta: float) -> np.ndarray:
    return np.array([[np.exp(-0.5j * theta), 0], [0, np.exp(0.5j * theta)]], dtype=np.complex128)


def _pack_u(u: np.ndarray) -> np.ndarray:
    u = np.asarray(u, dtype=np.complex128).reshape(2, 2)
    return np.array([u[0, 0].real, u[0, 0].imag, u[0, 1].real, u[0, 1].imag,
                     u[1, 0].real, u[1, 0].imag, u[1, 1].real, u[1, 1].imag], dtype=np.float64)


def unpack_u(rec) -> np.ndarray:
    """2x2 complex matrix of a gate record."""
    v = np.asarray(rec["U"], dtype=np.float64)
    return np.array([[v[0] + 1j * v[1], v[2] + 1j * v[3]], [v[4] + 1j * v[5], v[6] + 1j * v[7]]])


@dataclass
class Gate:
    """One gate before packing: a 2x2 unitary on ``target`` under ``controls``, a SWAP, or a dense 4x4 unitary
    on (``target``, ``target2``) under ``controls``."""
    kind: int
    target: int
    u: np.ndarray | None = None
    target2: int = -1
    controls: tuple = ()


def gate_u(u, target: int, controls=()) -> Gate:
    return Gate(GATE_U, int(target), np.asarray(u, dtype=np.complex128).reshape(2, 2), -1, tuple(int(c) for c in controls))


def gate_u4(v, q0: int, q1: int, controls=()) -> Gate:
    """Dense two-qubit gate: v (4x4) indexed by b0 + 2 b1, b0 = bit of q0, b1 = bit of q1."""
    return Gate(GATE_U4, int(q0), np.asarray(v, dtype=np.complex128).reshape(4, 4), int(q1),
                tuple(int(c) for c in controls))


def gate_swap(a: int, b: int) -> Gate:
    return Gate(GATE_SWAP, int(a), None, int(b), ())


def cnot(control: int, target: int) -> Gate:
    return gate_u(X, target, (control,))


def _row(v: np.ndarray, r: int) -> np.ndarray:
    return np.array([[x.real, x.imag] for x in v[r]], dtype=np.float64).ravel()


def pack(gates) -> np.ndarray:
    """List of :class:`Gate` -> contiguous structured array of 96-byte records (four per two-qubit gate)."""
    count = sum(4 if g.kind == GATE_U4 else 1 for g in gates)
    out = np.zeros(count, dtype=GATE_DTYPE)
    i = 0
    for g in gates:
        r = out[i]
        r["kind"] = g.kind
        r["target"] = g.target
        r["target2"] = g.target2
        r["ncontrols"] = len(g.controls)
        if len(g.controls) > MAX_CONTROLS:
            raise ValueError("too many controls")
        ctl = list(g.controls) + [-1] * (MAX_CONTROLS - len(g.controls))
        r["controls"] = ctl
        if g.kind == GATE_U:
            r["U"] = _pack_u(g.u)
        elif g.kind == GATE_U4:
            r["U"] = _row(g.u, 0)
            for row in range(1, 4):
                c = out[i + row]
                c["kind"] = GATE_U4_ROW
                c["target"], c["target2"], c["ncontrols"] = g.target, g.target2, 0
                c["controls"] = [-1] * MAX_CONTROLS
                c["U"] = _row(g.u, row)
            i += 3
        i += 1
    return out


def unpack_u4(recs) -> np.ndarray:
    """4x4 matrix of a two-qubit gate from its four records."""
    return np.array([[recs[r]["U"][2 * c] + 1j * recs[r]["U"][2 * c + 1] for c in range(4)] for r in range(4)])


def unpack(arr: np.ndarray):
    """Structured array -> list of :class:`Gate`."""
    res = []
    i = 0
    while i < len(arr):
        r = arr[i]
        kind = int(r["kind"])
        nc = int(r["ncontrols"])
        if kind == GATE_SWAP:
            res.append(gate_swap(int(r["target"]), int(r["target2"])))
        elif kind == GATE_U4:
            res.append(gate_u4(unpack_u4(arr[i:i + 4]), int(r["target"]), int(r["target2"]),
                               tuple(int(c) for c in r["controls"][:nc])))
            i += 3
        else:
            res.append(gate_u(unpack_u(r), int(r["target"]), tuple(int(c) for c in r["controls"][:nc])))
        i += 1
    return res


def inverse(arr: np.ndarray) -> np.ndarray:
    """Circuit inverse: gates in reverse order, each U replaced by its conjugate transpose (SWAP is its own inverse)."""
    gates = unpack(arr)[::-1]
    inv = []
    for g in gates:
        if g.kind == GATE_SWAP:
            inv.append(g)
        else:
            inv.append(Gate(g.kind, g.target, g.u.conj().T.copy(), g.target2, g.controls))
    return pack(inv)


# ----------------------------------------------------------------------------------------------------------------
# Circuits
# ----------------------------------------------------------------------------------------------------------------

def haar_u4(rng: np.random.Generator) -> np.ndarray:
    """Haar-random 4x4 unitary: QR of a complex Ginibre matrix with the phases of R's diagonal moved into Q
    (Mezzadri 2007)."""
    z = (rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4))) / math.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diag(r)
    return q * (d / np.abs(d))


def haar_u2(rng: np.random.Generator) -> np.ndarray:
    """Haar-distributed U(2): QR of a complex Ginibre matrix with the phases of R's diagonal divided out
    (Mezzadri 2007, "How to generate random matrices from the classical compact groups")."""
    z = (rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))) / math.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diagonal(r)
    return q * (d / np.abs(d))


def qft(n: int) -> list:
    """Textbook QFT on n qubits, little-endian: for j = n-1 .. 0, H(j) then controlled phase 2 pi / 2^(j-m+1)
    from every lower qubit m onto j; the closing SWAPs reverse the qubit order.  Maps |x> to
    sum_y e^{2 pi i x y / 2^n} |y> / sqrt(2^n).  n H + n(n-1)/2 controlled phases + floor(n/2) SWAPs."""
    gates = []
    for j in range(n - 1, -1, -1):
        gates.append(gate_u(H, j))
        for m in range(j - 1, -1, -1):
            gates.append(gate_u(phase(2.0 * math.pi / 2 ** (j - m + 1)), j, (m,)))
    for i in range(n // 2):
        gates.append(gate_swap(i, n - 1 - i))
    return gates


def random_layers(n: int, depth: int, rng: np.random.Generator) -> list:
    """``depth`` layers; each is a Haar-random U(2) on qubits 0..n-1 in order, then a CNOT on every pair of a
    seeded random perfect matching (control perm[2i], target perm[2i+1]; with odd n the last qubit idles)."""
    gates = []
    for _ in range(depth):
        for q in range(n):
            gates.append(gate_u(haar_u2(rng), q))
        perm = rng.permutation(n)
        for i in range(n // 2):
            gates.append(cnot(int(perm[2 * i]), int(perm[2 * i + 1])))
    return gates


def ghz(n: int) -> list:
    """H on qubit 0 then a CNOT chain 0->1->...->n-1: (|0...0> + |1...1>)/sqrt(2)."""
    return [gate_u(H, 0)] + [cnot(i, i + 1) for i in range(n - 1)]


def hadamard_all(n: int) -> list:
    return [gate_u(H, q) for q in range(n)]


@dataclass
class Workload:
    """A seeded circuit: qubit count, start basis state |x0>, packed gates."""
    name: str
    n: int
    x0: int
    gates: np.ndarray


def qft_workload(n: int = 20, seed: int = 1001) -> Workload:
    """QFT on n qubits from a seeded basis state |x>."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x = int(rng.integers(0, 2 ** n))
    return Workload(f"qft_n{n}", n, x, pack(qft(n)))


def random_workload(n: int = 30, depth: int = 20, seed: int = 1002) -> Workload:
    """``depth`` random layers on n qubits from |0...0>."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return Workload(f"random_n{n}_d{depth}", n, 0, pack(random_layers(n, depth, rng)))


def qft_random_workload(n: int = 33, depth: int = 10, seed: int = 1003) -> Workload:
    """QFT on n qubits followed by ``depth`` random layers, from a seeded basis state."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x = int(rng.integers(0, 2 ** n))
    return Workload(f"qft_random_n{n}_d{depth}", n, x, pack(qft(n) + random_layers(n, depth, rng)))


def random_layers_packed(n: int, depth: int, rng: np.random.Generator) -> np.ndarray:
    """The same layer structure as :func:`random_layers`, drawn in bulk and packed directly (batched QR for the
    Haar unitaries), for workloads with millions of gates.  Per layer: n U(2) records, then n // 2 CNOTs."""
    per = n + n // 2
    out = np.zeros(depth * per, dtype=GATE_DTYPE)
    z = (rng.standard_normal((depth, n, 2, 2)) + 1j * rng.standard_normal((depth, n, 2, 2))) / math.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diagonal(r, axis1=-2, axis2=-1)
    u = q * (d / np.abs(d))[..., None, :]
    flat = np.stack([u.real, u.imag], axis=-1).reshape(depth, n, 8)
    xrec = _pack_u(X)
    for L in range(depth):
        base = L * per
        blk = out[base:base + n]
        blk["U"] = flat[L]
        blk["target"] = np.arange(n)
        blk["target2"] = -1
        blk["controls"] = -1
        perm = rng.permutation(n)
        c = out[base + n:base + per]
        c["U"] = xrec
        c["target"] = perm[1:2 * (n // 2):2]
        c["target2"] = -1
        c["ncontrols"] = 1
        ctl = np.full((n // 2, MAX_CONTROLS), -1, dtype=np.int32)
        ctl[:, 0] = perm[0:2 * (n // 2):2]
        c["controls"] = ctl
    return out


def batched_workloads(count: int = 4096, n_lo: int = 10, n_hi: int = 22, d_lo: int = 10, d_hi: int = 40,
                      seed: int = 1004) -> list:
    """``count`` independent random circuits; n = round(exp(U(ln n_lo, ln n_hi))), depth uniform in
    [d_lo, d_hi] inclusive; each from |0...0>."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ns = np.rint(np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), size=count))).astype(int)
    ds = rng.integers(d_lo, d_hi + 1, size=count)
    out = []
    for i in range(count):
        out.append(Workload(f"b{i}_n{ns[i]}_d{ds[i]}", int(ns[i]), 0,
                            random_layers_packed(int(ns[i]), int(ds[i]), rng)))
    return out


def served_stream(count: int, rate_hz: float, n_lo: int = 12, n_hi: int = 28, d_lo: int = 10, d_hi: int = 30,
                  seed: int = 1005):
    """Poisson arrival stream: (arrival time in s, Workload) pairs; n log-uniform in [n_lo, n_hi], depth uniform."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate_hz, size=count)
    t = np.cumsum(gaps) - gaps[0]
    ns = np.rint(np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), size=count))).astype(int)
    ds = rng.integers(d_lo, d_hi + 1, size=count)
    out = []
    for i in range(count):
        out.append((float(t[i]), Workload(f"s{i}_n{ns[i]}_d{ds[i]}", int(ns[i]), 0,
                                          random_layers_packed(int(ns[i]), int(ds[i]), rng))))
    return out


def random_state(n: int, seed: int) -> np.ndarray:
    """A seeded normalised complex128 state (for tests that start from a dense state)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    v = rng.standard_normal(2 ** n) + 1j * rng.standard_normal(2 ** n)
    return v / np.linalg.norm(v)
