"""The pins are sharp: each plausible slip planted in a copy of the oracle's C source (a transposed operand,
a wrong sign, a dropped term, a wrong stride, a wrong control rule, an update that reads an already-written
value, a wrong SWAP condition) makes the brute-force Kronecker comparison fail.  The mutants are built
from a temporary copy on the CPU; the oracle itself is untouched."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import circuits as C
import oracle
from test_oracle_pins import dense_gate, dense_gate4, dense_swap

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "sv_oracle.c")

MUTANTS = {
    "transposed_q12_q21": ("const double q21r = U[4], q21i = U[5]", "const double q21r = U[2], q21i = U[3]"),
    "sign_flip": ("(q11r * ar - q11i * ai)", "(q11r * ar + q11i * ai)"),
    "dropped_term": ("+ (q12r * bi + q12i * br);", "+ (q12r * bi);"),
    "wrong_stride": ("const uint64_t stride = (uint64_t)1 << t;", "const uint64_t stride = (uint64_t)1 << (t + 1);"),
    "any_control_instead_of_all": ("return (k & cmask) == cmask;", "return cmask == 0 || (k & cmask) != 0;"),
    "reads_updated_value": ("b[0] = (q21r * ar - q21i * ai)", "b[0] = (q21r * a[0] - q21i * ai)"),
    "swap_condition": ("if ((k & ma) && !(k & mb)) {", "if (k & ma) {"),
    "u4_qubit_roles": ("idx[j] = k | ((j & 1) ? m0 : 0) | ((j & 2) ? m1 : 0);",
                       "idx[j] = k | ((j & 1) ? m1 : 0) | ((j & 2) ? m0 : 0);"),
    "u4_transposed": ("const double vr = V[8 * r + 2 * j], vi = V[8 * r + 2 * j + 1];",
                      "const double vr = V[8 * j + 2 * r], vi = V[8 * j + 2 * r + 1];"),
    "u4_controls_ignored": ("if (cmask != (k & cmask)) continue;", "if (0) continue;"),
    "u4_conjugated": ("si = si + (vr * ai[j] + vi * ar[j]);", "si = si + (vr * ai[j] - vi * ar[j]);"),
}


def build_mutant(tmp_path, name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / f"{name}.so"
    subprocess.run(["gcc", "-O1", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared", str(path), "-o", str(so)],
                   check=True)
    lib = ctypes.CDLL(str(so))
    P = ctypes.c_void_p
    lib.oracle_apply_gate.argtypes = [ctypes.c_int, P, P, ctypes.c_int, P, ctypes.c_int]
    lib.oracle_apply_gate4.argtypes = [ctypes.c_int, P, P, ctypes.c_int, ctypes.c_int, P, ctypes.c_int]
    lib.oracle_apply_swap.argtypes = [ctypes.c_int, P, ctypes.c_int, ctypes.c_int]
    return lib


def pins_detect(lib) -> bool:
    """Run the brute-force pins against ``lib``; True if any of them fails."""
    rng = np.random.Generator(np.random.PCG64(5))
    n = 4
    for t in range(n):
        for ctl in [(), ((t + 1) % n,), ((t + 1) % n, (t + 2) % n)]:
            u = C.haar_u2(rng)
            psi = rng.standard_normal(2 ** n) + 1j * rng.standard_normal(2 ** n)
            want = dense_gate(n, u, t, ctl) @ psi
            got = psi.copy()
            U = np.ascontiguousarray(np.stack([u.real, u.imag], axis=-1).reshape(8))
            c = np.array(ctl, dtype=np.int32)
            lib.oracle_apply_gate(n, got.ctypes.data, U.ctypes.data, t, c.ctypes.data if c.size else None, c.size)
            if np.max(np.abs(got - want)) > 1e-12:
                return True
    for q0, q1, ctl in [(0, 2, ()), (3, 1, ()), (1, 2, (0,)), (2, 0, (3, 1))]:
        v = C.haar_u4(rng)
        psi = rng.standard_normal(2 ** n) + 1j * rng.standard_normal(2 ** n)
        want = dense_gate4(n, v, q0, q1, ctl) @ psi
        got = psi.copy()
        V = np.ascontiguousarray(np.stack([v.real, v.imag], axis=-1).reshape(32))
        c = np.array(ctl, dtype=np.int32)
        lib.oracle_apply_gate4(n, got.ctypes.data, V.ctypes.data, q0, q1, c.ctypes.data if c.size else None, c.size)
        if np.max(np.abs(got - want)) > 1e-12:
            return True
    for a, b in [(0, 2), (3, 1)]:
        psi = rng.standard_normal(2 ** n) + 1j * rng.standard_normal(2 ** n)
        got = psi.copy()
        lib.oracle_apply_swap(n, got.ctypes.data, a, b)
        if not np.array_equal(got, dense_swap(n, a, b) @ psi):
            return True
    return False


def test_unmutated_copy_passes(tmp_path):
    src = open(SRC).read()
    path = tmp_path / "clean.c"
    path.write_text(src)
    so = tmp_path / "clean.so"
    subprocess.run(["gcc", "-O1", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared", str(path), "-o", str(so)],
                   check=True)
    lib = ctypes.CDLL(str(so))
    P = ctypes.c_void_p
    lib.oracle_apply_gate.argtypes = [ctypes.c_int, P, P, ctypes.c_int, P, ctypes.c_int]
    lib.oracle_apply_gate4.argtypes = [ctypes.c_int, P, P, ctypes.c_int, ctypes.c_int, P, ctypes.c_int]
    lib.oracle_apply_swap.argtypes = [ctypes.c_int, P, ctypes.c_int, ctypes.c_int]
    assert not pins_detect(lib)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(tmp_path, name):
    assert pins_detect(build_mutant(tmp_path, name))


# ---- product_state (numpy): plausible slips in the Kronecker order or the factor layout ----------------------
def _product_msb_first(factors):
    f = np.asarray(factors, dtype=np.complex128).reshape(-1, 2)
    psi = np.ones(1, dtype=np.complex128)
    for t in range(f.shape[0]):
        psi = np.kron(psi, f[t])  # qubit 0 ends up on the most significant bit
    return psi


def _product_alpha_beta_swapped(factors):
    f = np.asarray(factors, dtype=np.complex128).reshape(-1, 2)[:, ::-1]
    psi = np.ones(1, dtype=np.complex128)
    for t in range(f.shape[0]):
        psi = np.kron(f[t], psi)
    return psi


def _product_conjugated(factors):
    return np.conj(oracle.product_state(factors))


def product_pins_detect(fn):
    """The product-state pins of test_oracle_pins (one-qubit preparations through the pair update, basis
    factors), replayed against `fn`; True if any fails."""
    rng = np.random.Generator(np.random.PCG64(11))
    n = 3
    us = [C.haar_u2(rng) for _ in range(n)]
    want = oracle.basis_state(n, 0)
    for t, u in enumerate(us):
        oracle.apply_gate(want, u, t)
    if np.max(np.abs(fn([u[:, 0] for u in us]) - want)) >= 1e-14:
        return True
    x = 0b110
    return not np.array_equal(fn([(0, 1) if (x >> t) & 1 else (1, 0) for t in range(n)]), oracle.basis_state(n, x))


def test_product_state_pins_pass_and_catch_slips():
    assert not product_pins_detect(oracle.product_state)
    for fn in (_product_msb_first, _product_alpha_beta_swapped, _product_conjugated):
        assert product_pins_detect(fn), fn.__name__
