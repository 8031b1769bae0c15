"""Host-side guards around the device path: the graph cache never replays a graph captured for other gate
records, even when two circuits hash to the same key, and amplitude writes refuse values the arithmetic
cannot hold.  Each refusal is a status code returned before any device work."""
import os

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


def test_graph_cache_survives_a_key_collision(monkeypatch):
    # the test hook gives every circuit the same cache key, as a 64-bit hash collision would
    monkeypatch.setenv("SV_TEST_GRAPH_KEY_COLLIDE", "1")
    n = 12
    wa = C.random_workload(n, 3, seed=31)
    wb = C.random_workload(n, 3, seed=32)
    h = B.sv_create(n, B.SV_C128)
    try:
        for w in (wa, wb, wa, wb):
            B.sv_init_basis(h, 0)
            B.sv_apply_circuit_graph(h, w.gates)
            assert_close(B.sv_read_amplitudes(h).astype(np.complex128), run_oracle(n, w.gates), B.SV_C128,
                         "graph replay under a colliding key")
    finally:
        B.sv_destroy(h)
    assert os.environ.get("SV_TEST_GRAPH_KEY_COLLIDE") == "1"


@pytest.mark.parametrize("dtype", [B.SV_C128, B.SV_C64], ids=["c128", "c64"])
def test_write_amplitudes_rejects_values_outside_the_arithmetic(dtype):
    n = 6
    npdt = np.complex128 if dtype == B.SV_C128 else np.complex64
    good = C.random_state(n, seed=3).astype(npdt)
    h = B.sv_create(n, dtype)
    try:
        B.sv_write_amplitudes(h, 0, good)
        bad_values = [complex(np.nan, 0), complex(0, np.inf), complex(-np.inf, 1)]
        if dtype == B.SV_C128:
            bad_values += [complex(2.0 ** 126, 0), complex(0, -2.0 ** 130)]
        for bad in bad_values:
            v = good.copy()
            v[17] = bad
            with pytest.raises(B.SvError) as e:
                B.sv_write_amplitudes(h, 0, v)
            assert e.value.code == B.SV_ERR_ARG
        # nothing of a refused write reaches the device
        assert np.array_equal(B.sv_read_amplitudes(h), good)
        if dtype == B.SV_C128:
            ok = good.copy()
            ok[3] = 2.0 ** 125  # large but inside the range
            B.sv_write_amplitudes(h, 0, ok)
            assert B.sv_read_amplitudes(h)[3] == 2.0 ** 125
    finally:
        B.sv_destroy(h)


def test_tensor_core_wait_that_runs_out_is_reported(monkeypatch):
    # With SV_TEST_TC_NO_MMA set, the tensor-core pass issues no MMA, so the mbarrier it waits on never
    # completes: every wait is bounded (2 s), the kernel records the time-out, skips its remaining blocks and
    # returns, and the state's next read reports SV_ERR_TIMEOUT.  The context stays usable: the same circuit
    # on a new state afterwards matches the oracle.
    n = 13
    w = C.random_workload(n, 4, seed=31)
    monkeypatch.setenv("SV_TEST_TC_NO_MMA", "1")
    h = B.sv_create(n, B.SV_C128)
    try:
        B.sv_set_option(h, B.SV_OPT_TENSOR_BLOCKS, 1)
        B.sv_apply_circuit(h, w.gates)
        assert B.sv_last_plan_blocks(h)["blocks"] > 0
        with pytest.raises(B.SvError) as ei:
            B.sv_read_amplitudes(h)
        assert ei.value.code == B.SV_ERR_TIMEOUT
    finally:
        B.sv_destroy(h)
    monkeypatch.delenv("SV_TEST_TC_NO_MMA")
    h = B.sv_create(n, B.SV_C128)
    try:
        B.sv_set_option(h, B.SV_OPT_TENSOR_BLOCKS, 1)
        B.sv_apply_circuit(h, w.gates)
        got = B.sv_read_amplitudes(h)
    finally:
        B.sv_destroy(h)
    assert_close(got, run_oracle(n, w.gates), B.SV_C128, "after a time-out")
