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


def test_c128_batch_with_tensor_core_blocks():
    # Circuits from 10 to 18 qubits: those with chunks of 2^12 amplitudes (n >= 12) get dense blocks, run in
    # the batched tensor-core kernel beside the per-gate kernel in the same rounds; the smaller ones and the
    # ones given 2^10-amplitude chunks stay per-gate.  Every result against the oracle and against the same
    # batch without blocks.
    ws = C.batched_workloads(20, n_lo=10, n_hi=18, d_lo=4, d_hi=8, seed=91)
    ns, gl = [w.n for w in ws], [w.gates for w in ws]
    ks = [10 if i % 5 == 0 else 0 for i in range(len(ws))]
    B.sv_batch_set_option(B.SV_OPT_TENSOR_BLOCKS, 3)
    try:
        hs = B.sv_run_batch(ns, B.SV_C128, gl, chunk_k=ks)
        st = B.sv_last_batch_stats()
    finally:
        B.sv_batch_set_option(B.SV_OPT_TENSOR_BLOCKS, 0)
    assert st["tc_rounds"] > 0 and st["tc_rounds"] <= st["rounds"], st
    plain = B.sv_run_batch(ns, B.SV_C128, gl, chunk_k=ks)
    assert B.sv_last_batch_stats()["tc_rounds"] == 0
    try:
        for w, h, h0 in zip(ws, hs, plain):
            got = B.sv_read_amplitudes(h).astype(np.complex128)
            assert_close(got, run_oracle(w.n, w.gates), B.SV_C128, w.name + " tensor-core batch")
            assert_close(got, B.sv_read_amplitudes(h0).astype(np.complex128), B.SV_C128, w.name + " vs per-gate")
    finally:
        for h in hs + plain:
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


# ---- rounds large enough for the FP64 / double-float split kernel ---------------------------------------
# k_fused_batch_mixed runs a complex128 round only when the round has at least four chunks per CTA of the
# grid (152 SMs x 3 CTAs x 4 = 1824 chunks of 2^12 amplitudes on a GB300).  96 circuits of 17 qubits give
# 96 x 32 = 3072 chunks per round.

def bursty_c128_workloads(count=96, n=17):
    return [C.random_workload(n, 3 + i % 3, seed=500 + i) for i in range(count)]


def test_batch_rounds_in_the_split_kernel_match_oracle_and_single_runs():
    ws = bursty_c128_workloads()
    hs = B.sv_run_batch([w.n for w in ws], B.SV_C128, [w.gates for w in ws])
    stats = B.sv_last_batch_stats()
    try:
        assert stats["mixed_rounds"] >= 1 and stats["max_round_chunks"] >= 1824, stats
        for w, h in zip(ws, hs):
            got = B.sv_read_amplitudes(h).astype(np.complex128)
            assert_close(got, run_oracle(w.n, w.gates), B.SV_C128, w.name)
            assert_close(got, run_gpu(w.n, w.gates, B.SV_C128, B.SV_ARITH_AUTO), B.SV_C128, w.name + " alone")
    finally:
        for h in hs:
            B.sv_destroy(h)


def poll_outcome(srv, tickets, timeout_s=180.0):
    """ticket -> state handle, or the SvError code of a failed request."""
    res = {}
    t0 = time.time()
    while len(res) < len(tickets):
        assert time.time() - t0 < timeout_s, "server did not finish in time"
        for t in tickets:
            if t in res:
                continue
            try:
                done, h = B.sv_poll(srv, t)
            except B.SvError as e:
                res[t] = e.code
                continue
            if done:
                res[t] = h
        time.sleep(0.001)
    return res


def test_server_burst_uses_the_split_kernel_and_matches_oracle():
    ws = bursty_c128_workloads()
    srv = B.sv_server_create(64 << 30, 256)
    try:
        B.sv_server_pause(srv, True)  # queue the burst, then admit it at once: one round holds all 96
        tickets = [B.sv_submit(srv, w.n, B.SV_C128, w.gates) for w in ws]
        assert B.sv_server_get_stats(srv)["pending"] == len(ws)
        B.sv_server_pause(srv, False)
        res = poll_outcome(srv, tickets)
        stats = B.sv_server_get_stats(srv)
        assert stats["mixed_rounds"] >= 1 and stats["max_round_chunks"] >= 1824, stats
        assert stats["completed"] == len(ws) and stats["failed"] == 0, stats
        for w, t in zip(ws, tickets):
            got = B.sv_read_amplitudes(res[t]).astype(np.complex128)
            assert_close(got, run_oracle(w.n, w.gates), B.SV_C128, w.name)
            assert_close(got, run_gpu(w.n, w.gates, B.SV_C128, B.SV_ARITH_AUTO), B.SV_C128, w.name + " alone")
            B.sv_destroy(res[t])
        assert B.sv_server_get_stats(srv)["budget_used"] == 0
    finally:
        B.sv_server_destroy(srv)


def test_server_mixed_dtype_burst_each_result_same_alone_and_in_the_mix():
    """complex64 and complex128 requests admitted together advance in rounds of their own dtype, side by side;
    every result equals the oracle's and the same circuit run alone."""
    ws = C.batched_workloads(48, n_lo=8, n_hi=17, d_lo=2, d_hi=6, seed=66)
    dts = [B.SV_C64 if i % 2 else B.SV_C128 for i in range(len(ws))]
    srv = B.sv_server_create(8 << 30, 64)
    try:
        B.sv_server_pause(srv, True)
        tickets = [B.sv_submit(srv, w.n, dt, w.gates) for w, dt in zip(ws, dts)]
        B.sv_server_pause(srv, False)
        res = poll_outcome(srv, tickets)
        for w, dt, t in zip(ws, dts, tickets):
            got = B.sv_read_amplitudes(res[t]).astype(np.complex128)
            assert_close(got, run_oracle(w.n, w.gates), dt, w.name)
            assert_close(got, run_gpu(w.n, w.gates, dt, B.SV_ARITH_AUTO), dt, w.name + " in the mix vs alone")
            B.sv_destroy(res[t])
    finally:
        B.sv_server_destroy(srv)


@pytest.mark.parametrize("hook", ["SV_FAULT_POISON_TICKET", "SV_FAULT_CORRUPT_DESC_TICKET"],
                         ids=["poisoned_queue_entry", "corrupted_pass_descriptor"])
def test_server_isolates_a_bad_request(monkeypatch, hook):
    """A request whose queued gate records were overwritten (poisoned entry) or whose pass descriptor is
    corrupted is refused on the host before any launch; its ticket reports SV_ERR_ARG and every other request
    completes with the oracle's result.  The hooks only touch host memory."""
    monkeypatch.setenv(hook, "3")  # tickets of a new server count from 1
    ws = C.batched_workloads(6, n_lo=6, n_hi=12, d_lo=2, d_hi=4, seed=71)
    srv = B.sv_server_create(1 << 30, 8)
    try:
        tickets = [B.sv_submit(srv, w.n, B.SV_C128, w.gates) for w in ws]
        assert tickets[2] == 3
        res = poll_outcome(srv, tickets)
        for w, t in zip(ws, tickets):
            if t == 3:
                assert res[t] == B.SV_ERR_ARG
                continue
            assert_close(B.sv_read_amplitudes(res[t]).astype(np.complex128), run_oracle(w.n, w.gates), B.SV_C128,
                         w.name)
            B.sv_destroy(res[t])
        stats = B.sv_server_get_stats(srv)
        assert stats["failed"] == 1 and stats["completed"] == len(ws) - 1, stats
        assert stats["budget_used"] == 0
    finally:
        B.sv_server_destroy(srv)
