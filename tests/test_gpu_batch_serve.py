"""Batched circuits and the serving loop against the oracle; each result is the same alone and in the mix."""
import time

import numpy as np
import pytest

import circuits as C
from gpu_helpers import assert_close, run_gpu, run_oracle

pytestmark = pytest.mark.gpu
B = pytest.importorskip("paper_1801_01037_gb300")._binding


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1801_01037_gb300 import build
    build.build()
    B.load()


@pytest.mark.parametrize("dtype", [B.SV_C128, B.SV_C64], ids=["c128", "c64"])
def test_batch_matches_oracle_and_single_runs(dtype):
    ws = C.batched_workloads(24, n_lo=3, n_hi=17, d_lo=2, d_hi=6, seed=77)
    handles = B.sv_run_batch([w.n for w in ws], dtype, [w.gates for w in ws])
    try:
        for w, h in zip(ws, handles):
            got = B.sv_read_amplitudes(h).astype(np.complex128)
            assert_close(got, run_oracle(w.n, w.gates), dtype, w.name)
            alone = run_gpu(w.n, w.gates, dtype, B.SV_ARITH_AUTO)
            assert_close(got, alone, dtype, w.name + " alone vs batched")
    finally:
        for h in handles:
            B.sv_destroy(h)


def test_batch_with_empty_and_swap_only_circuits():
    gl = [C.pack([]), C.pack([C.gate_swap(0, 2)]), C.pack(C.ghz(5))]
    ns = [3, 3, 5]
    hs = B.sv_run_batch(ns, B.SV_C128, gl)
    try:
        for n, g, h in zip(ns, gl, hs):
            assert_close(B.sv_read_amplitudes(h).astype(np.complex128), run_oracle(n, g), B.SV_C128)
    finally:
        for h in hs:
            B.sv_destroy(h)


def wait_all(srv, tickets, timeout_s=120.0):
    res = {}
    t0 = time.time()
    while len(res) < len(tickets):
        assert time.time() - t0 < timeout_s, "server did not finish in time"
        for t in tickets:
            if t in res:
                continue
            done, h = B.sv_poll(srv, t)
            if done:
                res[t] = h
        time.sleep(0.001)
    return res


def test_server_results_match_oracle_under_continuous_admission():
    ws = C.batched_workloads(30, n_lo=4, n_hi=18, d_lo=2, d_hi=8, seed=55)
    srv = B.sv_server_create(64 << 20, 8)  # 64 MiB budget, at most 8 active: forces admission waits
    try:
        tickets = []
        for i, w in enumerate(ws):
            tickets.append(B.sv_submit(srv, w.n, B.SV_C64 if i % 2 else B.SV_C128, w.gates))
            if i % 7 == 0:
                time.sleep(0.002)  # let some requests start before the others arrive
        res = wait_all(srv, tickets)
        for i, (w, t) in enumerate(zip(ws, tickets)):
            dt = B.SV_C64 if i % 2 else B.SV_C128
            got = B.sv_read_amplitudes(res[t]).astype(np.complex128)
            assert_close(got, run_oracle(w.n, w.gates), dt, w.name)
            # the same circuit alone (its own state, no other request on the GPU) gives the same result
            alone = run_gpu(w.n, w.gates, dt, B.SV_ARITH_AUTO)
            assert_close(got, alone, dt, w.name + " in the mix vs alone")
            B.sv_destroy(res[t])
        with pytest.raises(B.SvError) as e:
            B.sv_submit(srv, 30, B.SV_C128, C.pack([]))
        assert e.value.code == B.SV_ERR_OOM
        with pytest.raises(B.SvError) as e:
            B.sv_poll(srv, 10 ** 9)
        assert e.value.code == B.SV_ERR_NOT_FOUND
    finally:
        B.sv_server_destroy(srv)


def test_batch_chunk_sizes_from_a_tuner():
    """sv_run_batch_k: per-circuit chunk sizes (as an autotuner picks them) give the oracle's results; an
    out-of-range size is refused before any work."""
    ws = C.batched_workloads(10, n_lo=6, n_hi=16, d_lo=2, d_hi=5, seed=91)
    ks = [0, 6, 8, 10, 12, 13, 7, 9, 11, 13]
    for dt in (B.SV_C128, B.SV_C64):
        hs = B.sv_run_batch([w.n for w in ws], dt, [w.gates for w in ws], chunk_k=ks)
        try:
            for w, h in zip(ws, hs):
                assert_close(B.sv_read_amplitudes(h).astype(np.complex128), run_oracle(w.n, w.gates), dt, w.name)
        finally:
            for h in hs:
                B.sv_destroy(h)
    with pytest.raises(B.SvError) as e:
        B.sv_run_batch([w.n for w in ws], B.SV_C64, [w.gates for w in ws], chunk_k=[5] * len(ws))
    assert e.value.code == B.SV_ERR_ARG
