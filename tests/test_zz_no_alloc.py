"""sv_norm_noalloc: the norm for callers that must not have the library allocate device memory (for example a
host framework that has reserved the GPU's memory for its own pool, or a latency-critical loop that cannot
take cudaMalloc's implicit synchronisation).  The caller owns the state buffer and the one-double output;
the library only uses its fixed scratch array.  Its result must match sv_norm on the same state, within the
norm tolerance of the other GPU tests, on two calls in a row (the second call reuses the scratch the first
one left behind).  This file is collected last so that a run stopping at the first failure has run the rest.
"""
import ctypes

import numpy as np
import pytest

import circuits as C

pytestmark = pytest.mark.gpu
B = pytest.importorskip("paper_1801_01037_gb300")._binding

NORM_TOL = {B.SV_C128: 1e-13, B.SV_C64: 1e-5}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1801_01037_gb300 import build
    build.build()
    B.load()


@pytest.mark.parametrize("side_stream", [False, True], ids=["default_stream", "side_stream"])
@pytest.mark.parametrize("dtype", [B.SV_C128, B.SV_C64], ids=["c128", "c64"])
@pytest.mark.parametrize("n", [1, 9, 21])
def test_norm_noalloc_matches_sv_norm_twice(dtype, n, side_stream):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(40 + n)
    # an unnormalised state (norm far from 1), then a circuit so the layout and values are non-trivial
    v = (rng.standard_normal(2 ** n) + 1j * rng.standard_normal(2 ** n)) * 1.7
    v = v.astype(np.complex64 if dtype == B.SV_C64 else np.complex128)
    # The circuit is unitary, so the norm stays that of the written values (computed here on the host in
    # FP64 from exactly the values written), up to the rounding of the gates.
    host_norm = float(np.sum(np.abs(v.astype(np.complex128)) ** 2))
    h = B.sv_create(n, dtype)
    try:
        B.sv_write_amplitudes(h, 0, v)
        B.sv_apply_circuit(h, C.random_workload(n, 2, seed=n).gates)
        want = B.sv_norm(h)
        assert abs(want - host_norm) <= (1e-12 if dtype == B.SV_C128 else 1e-5) * host_norm
        _, _, psi_ptr = B.sv_get_info(h)
        out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")  # the caller's own output buffer
        stream = torch.cuda.Stream() if side_stream else None
        sptr = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
        torch.cuda.synchronize()
        lib = B.load()
        for call in range(2):
            out.fill_(-1.0)
            torch.cuda.synchronize()
            free_before, _ = torch.cuda.mem_get_info()
            rc = lib.sv_norm_noalloc(ctypes.c_void_p(psi_ptr), n, dtype, sptr, ctypes.c_void_p(out.data_ptr()))
            assert rc == B.SV_OK, B.sv_last_error()
            torch.cuda.synchronize()
            free_after, _ = torch.cuda.mem_get_info()
            got = float(out.item())
            assert abs(got - want) <= NORM_TOL[dtype] * max(1.0, want), (call, got, want)
            assert abs(got - host_norm) <= (1e-12 if dtype == B.SV_C128 else 1e-5) * host_norm, (call, got, host_norm)
            if call == 1:
                # the second call (set-up done by the first) takes no device memory at all
                assert free_after == free_before, (free_before, free_after)
    finally:
        B.sv_destroy(h)


def test_norm_noalloc_rejects_bad_arguments():
    lib = B.load()
    assert lib.sv_norm_noalloc(None, 4, B.SV_C128, None, None) == B.SV_ERR_ARG
    assert lib.sv_norm_noalloc(ctypes.c_void_p(16), 0, B.SV_C128, None, ctypes.c_void_p(16)) == B.SV_ERR_ARG
    assert lib.sv_norm_noalloc(ctypes.c_void_p(17), 4, B.SV_C128, None, ctypes.c_void_p(16)) == B.SV_ERR_ARG
    assert lib.sv_norm_noalloc(ctypes.c_void_p(16), 4, 9, None, ctypes.c_void_p(16)) == B.SV_ERR_ARG
