"""FP64 CPU oracle (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg use this package; the
library in ``paper_1801_01037_gb300`` never imports it, and it imports nothing from the library.

The arithmetic lives in ``sv_oracle.c`` (plain C, IEEE double, no FMA contraction): Algorithm 1's pair
loop from Sec. V.B of the paper, with the controlled-gate rule of the same section.  This wrapper only
marshals numpy arrays to it.  The probabilities (|alpha_k|^2, Sec. II.A) are computed here in numpy.

Parity status: every function is pinned by tests in ``tests/test_oracle_pins.py`` (dense Kronecker
operator of Sec. II.A/V.A by brute force, the paper's worked examples under ``tests/golden/``, and closed
forms); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sv_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

GATE_RECORD_BYTES = 96


def build(force: bool = False) -> str:
    """Compile ``sv_oracle.c`` into ``oracle/_build/liboracle.so`` (gcc, -O2, no fast-math, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-fno-fast-math", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
           _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            lib.oracle_gate_size.restype = ctypes.c_int
            lib.oracle_init_basis.argtypes = [ctypes.c_int, P, ctypes.c_uint64]
            lib.oracle_apply_gate.argtypes = [ctypes.c_int, P, P, ctypes.c_int, P, ctypes.c_int]
            lib.oracle_apply_gate4.argtypes = [ctypes.c_int, P, P, ctypes.c_int, ctypes.c_int, P, ctypes.c_int]
            lib.oracle_apply_swap.argtypes = [ctypes.c_int, P, ctypes.c_int, ctypes.c_int]
            lib.oracle_apply_circuit.argtypes = [ctypes.c_int, P, P, ctypes.c_uint64, ctypes.c_int]
            lib.oracle_apply_circuit_collapse.argtypes = [ctypes.c_int, P, P, ctypes.c_uint64, ctypes.c_int]
            lib.oracle_norm2.argtypes = [ctypes.c_int, P]
            lib.oracle_norm2.restype = ctypes.c_double
            lib.oracle_max_threads.restype = ctypes.c_int
            if lib.oracle_gate_size() != GATE_RECORD_BYTES:
                raise RuntimeError("oracle gate record size mismatch")
            _lib = lib
    return _lib


def _nqubits(psi: np.ndarray) -> int:
    n = int(psi.size).bit_length() - 1
    if psi.dtype != np.complex128 or not psi.flags.c_contiguous or psi.size != (1 << n) or n < 1:
        raise ValueError("state must be a C-contiguous complex128 array of length 2^n, n >= 1")
    return n


def basis_state(n: int, x: int = 0) -> np.ndarray:
    psi = np.empty(1 << n, dtype=np.complex128)
    rc = _load().oracle_init_basis(n, psi.ctypes.data, int(x))
    if rc != 0:
        raise ValueError(f"oracle_init_basis({n}, {x}) failed: {rc}")
    return psi


def product_state(factors) -> np.ndarray:
    """The product state of Sec. V, |psi_0 ... psi_{n-1}>, with qubit t in alpha_t|0> + beta_t|1>
    (factors[t] = (alpha_t, beta_t)): the Kronecker product of the one-qubit vectors, qubit 0 on the
    least significant index bit (stride 2^t, Sec. V.A), so amplitude k = prod_t (bit t of k ? beta_t : alpha_t)."""
    f = np.asarray(factors, dtype=np.complex128).reshape(-1, 2)
    psi = np.ones(1, dtype=np.complex128)
    for t in range(f.shape[0]):
        psi = np.kron(f[t], psi)  # qubit t becomes the most significant bit so far
    return psi


def apply_gate(psi: np.ndarray, u, target: int, controls=()) -> np.ndarray:
    """Apply a (controlled) 2x2 unitary in place; returns ``psi``."""
    n = _nqubits(psi)
    u = np.asarray(u, dtype=np.complex128).reshape(2, 2)
    U = np.ascontiguousarray(np.stack([u.real, u.imag], axis=-1).reshape(8))
    ctl = np.ascontiguousarray(np.asarray(controls, dtype=np.int32))
    rc = _load().oracle_apply_gate(n, psi.ctypes.data, U.ctypes.data, int(target),
                                   ctl.ctypes.data if ctl.size else None, int(ctl.size))
    if rc != 0:
        raise ValueError(f"oracle_apply_gate rejected the gate (rc={rc})")
    return psi


def apply_gate4(psi: np.ndarray, v, q0: int, q1: int, controls=()) -> np.ndarray:
    """Apply a (controlled) dense two-qubit gate in place (v: 4x4, entry order b0 + 2 b1); returns ``psi``."""
    n = _nqubits(psi)
    v = np.asarray(v, dtype=np.complex128).reshape(4, 4)
    V = np.ascontiguousarray(np.stack([v.real, v.imag], axis=-1).reshape(32))
    ctl = np.ascontiguousarray(np.asarray(controls, dtype=np.int32))
    rc = _load().oracle_apply_gate4(n, psi.ctypes.data, V.ctypes.data, int(q0), int(q1),
                                    ctl.ctypes.data if ctl.size else None, int(ctl.size))
    if rc != 0:
        raise ValueError(f"oracle_apply_gate4 rejected the gate (rc={rc})")
    return psi


def apply_swap(psi: np.ndarray, a: int, b: int) -> np.ndarray:
    n = _nqubits(psi)
    rc = _load().oracle_apply_swap(n, psi.ctypes.data, int(a), int(b))
    if rc != 0:
        raise ValueError(f"oracle_apply_swap rejected ({a}, {b})")
    return psi


def apply_circuit(psi: np.ndarray, gates: np.ndarray, threads: int = 1, collapse: bool = False) -> np.ndarray:
    """Apply packed gate records (96-byte structured array) in order, in place; returns ``psi``.

    threads > 1 splits Algorithm 1's outer loop over OpenMP threads (the paper's "outer" variant), or with
    ``collapse`` both loops (its collapse(2) variant, which keeps gates on high qubits parallel too).  Every
    pair is independent, so the result is the same bit for bit in every case."""
    n = _nqubits(psi)
    g = np.ascontiguousarray(gates)
    if g.dtype.itemsize != GATE_RECORD_BYTES:
        raise ValueError("gate records must be 96 bytes")
    fn = _load().oracle_apply_circuit_collapse if collapse else _load().oracle_apply_circuit
    rc = fn(n, psi.ctypes.data, g.ctypes.data if g.size else None, int(g.size), int(threads))
    if rc != 0:
        raise ValueError(f"oracle_apply_circuit: bad gate at index {-rc - 2}" if rc <= -2 else "bad argument")
    return psi


def simulate(n: int, gates: np.ndarray, x0: int = 0, threads: int = 1, collapse: bool = False) -> np.ndarray:
    """|x0> followed by the circuit: the final complex128 state vector in index order."""
    return apply_circuit(basis_state(n, x0), gates, threads, collapse)


def norm2(psi: np.ndarray) -> float:
    n = _nqubits(psi)
    return float(_load().oracle_norm2(n, psi.ctypes.data))


def probabilities(psi: np.ndarray) -> np.ndarray:
    """|alpha_k|^2 for every k (Sec. II.A's probability interpretation), FP64."""
    return psi.real * psi.real + psi.imag * psi.imag


def sample(psi: np.ndarray, u) -> np.ndarray:
    """Measurement outcomes for uniform numbers u in [0, 1): the smallest index k whose cumulative probability
    (|alpha_0|^2 + ... + |alpha_k|^2, FP64, index order) exceeds u times the total."""
    c = np.cumsum(probabilities(psi))
    return np.searchsorted(c, np.asarray(u, dtype=np.float64) * c[-1], side="right").astype(np.uint64)


def expect_z(psi: np.ndarray, mask: int) -> float:
    """sum_k |alpha_k|^2 (-1)^popcount(k & mask): the Pauli-Z product on the qubits in `mask`."""
    k = np.arange(psi.size, dtype=np.uint64) & np.uint64(mask)
    par = np.zeros(psi.size, dtype=np.uint64)
    while np.any(k):
        par ^= k & np.uint64(1)
        k >>= np.uint64(1)
    return float(np.sum(probabilities(psi) * (1.0 - 2.0 * par)))


def max_threads() -> int:
    return int(_load().oracle_max_threads())
