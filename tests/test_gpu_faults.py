"""Failure handling, injected on the host (no GPU fault is ever caused): an allocation that fails, a request
that can never fit, a malformed request; the library reports each as a status and keeps working."""
import os
import time

import numpy as np
import pytest

import circuits as C
from gpu_helpers import assert_close, run_oracle

pytestmark = pytest.mark.gpu
B = pytest.importorskip("paper_1801_01037_gb300")._binding


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1801_01037_gb300 import build
    build.build()
    B.load()


def test_injected_allocation_failure_is_reported_and_recoverable():
    os.environ["SV_FAULT_ALLOC"] = "1"
    try:
        with pytest.raises(B.SvError) as e:
            B.sv_create(10, B.SV_C128)
        assert e.value.code == B.SV_ERR_OOM and "injected" in str(e.value)
    finally:
        del os.environ["SV_FAULT_ALLOC"]
    h = B.sv_create(10, B.SV_C128)   # the library still works afterwards
    B.sv_destroy(h)


def test_injected_allocation_failure_of_a_batch():
    """The batch's single state allocation fails as if out of memory: nothing is returned or leaked, and the
    next batch runs."""
    import circuits as C
    ws = C.batched_workloads(6, n_lo=3, n_hi=9, d_lo=2, d_hi=4, seed=5)
    os.environ["SV_FAULT_ALLOC"] = "1"
    try:
        with pytest.raises(B.SvError) as e:
            B.sv_run_batch([w.n for w in ws], B.SV_C64, [w.gates for w in ws])
        assert e.value.code == B.SV_ERR_OOM and "injected" in str(e.value)
    finally:
        del os.environ["SV_FAULT_ALLOC"]
    handles = B.sv_run_batch([w.n for w in ws], B.SV_C64, [w.gates for w in ws])
    for h in handles:
        B.sv_destroy(h)


def poll_until(srv, t, timeout_s=60.0):
    t0 = time.time()
    while time.time() - t0 < timeout_s:
        done, h = B.sv_poll(srv, t)
        if done:
            return h
        time.sleep(0.001)
    raise AssertionError("request did not finish")


def test_server_survives_a_failed_admission():
    srv = B.sv_server_create(1 << 30, 4)
    try:
        os.environ["SV_FAULT_ALLOC"] = "1"
        try:
            t_bad = B.sv_submit(srv, 8, B.SV_C128, C.pack(C.ghz(8)))
            with pytest.raises(B.SvError) as e:
                poll_until(srv, t_bad)
            assert e.value.code == B.SV_ERR_OOM
        finally:
            del os.environ["SV_FAULT_ALLOC"]
        g = C.random_workload(9, 3, seed=2).gates
        h = poll_until(srv, B.sv_submit(srv, 9, B.SV_C128, g))
        assert_close(B.sv_read_amplitudes(h).astype(np.complex128), run_oracle(9, g), B.SV_C128)
        B.sv_destroy(h)
        bad = C.pack([C.gate_u(np.array([[1, 1], [1, 1]]), 0)])
        with pytest.raises(B.SvError) as e:
            B.sv_submit(srv, 3, B.SV_C128, bad)
        assert e.value.code == B.SV_ERR_NOT_UNITARY
    finally:
        B.sv_server_destroy(srv)
