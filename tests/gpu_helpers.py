"""Shared helpers for the GPU tests: run a circuit through the C ABI and compare with the FP64 oracle.

Tolerances (written here, used by every GPU parity test):
  complex128, both arithmetic modes: max |psi_gpu - psi_oracle| <= 1e-12 and 1 - F <= 1e-12.
  complex64: max |psi_gpu - psi_oracle| <= 1e-4 * max |psi_oracle| and 1 - F <= 1e-8
  (FP32 rounding is 6e-8 relative per operation; a few hundred gates stay far inside 1e-4).
"""
import numpy as np

import oracle
from paper_1801_01037_gb300 import _binding as B

C128_ABS = 1e-12
C128_INFID = 1e-12
C64_REL = 1e-4
C64_INFID = 1e-8

MODES = [
    ("c128_df32", B.SV_C128, B.SV_ARITH_DF32),
    ("c128_f64", B.SV_C128, B.SV_ARITH_F64),
    ("c64", B.SV_C64, B.SV_ARITH_AUTO),
]
MODE_IDS = [m[0] for m in MODES]


def make_state(n, dtype, arith, psi0=None, x0=0, chunk_k=0, fusion=1):
    h = B.sv_create(n, dtype)
    if dtype == B.SV_C128:
        B.sv_set_option(h, B.SV_OPT_ARITH, arith)
    if chunk_k:
        B.sv_set_option(h, B.SV_OPT_CHUNK_QUBITS, chunk_k)
    B.sv_set_option(h, B.SV_OPT_FUSION, fusion)
    if psi0 is not None:
        B.sv_write_amplitudes(h, 0, psi0.astype(np.complex64 if dtype == B.SV_C64 else np.complex128))
    elif x0:
        B.sv_init_basis(h, x0)
    return h


def run_gpu(n, gates, dtype, arith, psi0=None, x0=0, chunk_k=0, fusion=1, graph=False):
    h = make_state(n, dtype, arith, psi0, x0, chunk_k, fusion)
    try:
        (B.sv_apply_circuit_graph if graph else B.sv_apply_circuit)(h, gates)
        return B.sv_read_amplitudes(h).astype(np.complex128)
    finally:
        B.sv_destroy(h)


def run_oracle(n, gates, psi0=None, x0=0):
    psi = oracle.basis_state(n, x0) if psi0 is None else np.ascontiguousarray(psi0, dtype=np.complex128).copy()
    return oracle.apply_circuit(psi, gates)


def infidelity(a, b):
    num = abs(np.vdot(a, b)) ** 2
    return 1.0 - num / (np.vdot(a, a).real * np.vdot(b, b).real)


def assert_close(got, want, dtype, what=""):
    err = np.max(np.abs(got - want))
    inf = infidelity(got, want)
    if dtype == B.SV_C128:
        assert err <= C128_ABS, f"{what}: max abs err {err:.3e}"
        assert inf <= C128_INFID, f"{what}: 1-F {inf:.3e}"
    else:
        scale = np.max(np.abs(want))
        assert err <= C64_REL * scale, f"{what}: max abs err {err:.3e} (scale {scale:.3e})"
        assert inf <= C64_INFID, f"{what}: 1-F {inf:.3e}"
    return err, inf
