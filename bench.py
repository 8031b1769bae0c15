#!/usr/bin/env python3
"""Benchmark of the state-vector gate path on GB300.

Workload (one "step"): start from |0...0> on n = 30 qubits, apply the seeded 20-layer random circuit (each
layer: a Haar-random U(2) on every qubit, then CNOTs on a random perfect matching; 900 gates, seed 1002),
then reduce the norm in double precision and read 1024 amplitudes back to the host.  The headline is
complex128 (IEEE double storage, 16 GiB state); complex64 is measured on the same circuit for comparison.

Reported: gates/s (value), effective HBM GB/s (2 * state bytes per gate, i.e. every gate counted as one
unfused read+write sweep), the dominant kernel's roofline (CUDA events around its launches inside the
timed region), the FP64 CPU oracle timed on the host's cores on a bounded sample, an end-to-end number
through the C ABI with host buffers, SM clocks sampled during the timed region.

Timing: W untimed warm-up steps, then K steps bracketed by a barrier and a device synchronize; CUDA events
on the launching (legacy default) stream; the state (16 GiB) is larger than L2, so no flush is needed.
With torchrun (N > 1) every rank runs its own replica (weak scaling, no collective on the data path); the
reported time is the maximum over ranks and the value the total gates of all ranks divided by it.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
RANK = int(os.environ.get("RANK", "0"))
WORLD = int(os.environ.get("WORLD_SIZE", "1"))
LOCAL_RANK = int(os.environ.get("LOCAL_RANK", "0"))
if WORLD > 1:
    # One GPU per process: the library's CUDA runtime sees only this rank's device.
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    devs = vis.split(",") if vis else [str(i) for i in range(64)]
    os.environ["CUDA_VISIBLE_DEVICES"] = devs[LOCAL_RANK]

sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import circuits as C  # noqa: E402

N_QUBITS = 30
DEPTH = 20
SEED = 1002
READ_COUNT = 1024
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=N_QUBITS)
    ap.add_argument("--depth", type=int, default=DEPTH)
    ap.add_argument("--no-f64", action="store_true", help="skip the native-FP64 context measurement")
    ap.add_argument("--no-autotune", action="store_true", help="use the library's default chunk size")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="budget of the CPU-oracle sample")
    ap.add_argument("--workload", choices=["random", "batched", "served", "qft20", "qft33"], default="random",
                    help="random: the headline n=30 circuit; batched: 4096 circuits in one sv_run_batch call; "
                         "served: Poisson request stream through the serving loop; qft20 / qft33: the QFT "
                         "configurations (n = 20; n = 33 followed by 10 random layers)")
    ap.add_argument("--batch-count", type=int, default=4096)
    ap.add_argument("--served-rates", default="10,30,100", help="request rates (per s) to sweep")
    ap.add_argument("--served-count", type=int, default=200, help="requests per rate")
    ap.add_argument("--served-rate", type=float, default=30.0, help="rate of the served sample in the default line")
    ap.add_argument("--served-requests", type=int, default=100, help="requests of the served sample in the default line")
    ap.add_argument("--no-extra", action="store_true", help="skip the served and batched samples of the default line")
    ap.add_argument("--no-n33", action="store_true", help="skip the n = 33 single-gate sweep")
    ap.add_argument("--tensor-blocks", default=None,
                    help="force SV_OPT_TENSOR_BLOCKS instead of the autotuner's choice: one value for both dtypes, "
                         "or 'C128,C64'")
    return ap.parse_args()


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# ---------------------------------------------------------------------------------------------------------
# Clock sampling during the timed region
# ---------------------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0]],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------------------------------------
# CPU oracle (bounded sample): the cpu_baseline leg and the --impl reference arm
# ---------------------------------------------------------------------------------------------------------
def oracle_sample_gates(gates, n):
    """A fixed spread of the circuit's first layer: U(2) on low, middle and high qubits, and CNOTs."""
    picks = [0, n // 2, n - 1, 5, 3 * n // 4, n // 4, n + 2, n + 7, 10, n - 5]
    return [gates[i:i + 1] for i in picks if i < len(gates)]


class OracleRunner:
    def __init__(self, n, gates):
        import oracle
        self.oracle = oracle
        self.threads = os.cpu_count() or 1
        self.psi = oracle.basis_state(n, 0)
        self.sample = oracle_sample_gates(gates, n)
        self.i = 0

    def step(self):
        g = self.sample[self.i % len(self.sample)]
        self.i += 1
        self.oracle.apply_circuit(self.psi, g, threads=self.threads)

    def desc(self, n):
        return (f"single gates of the n={n} circuit's first layer (U(2) on qubits spread from 0 to n-1, and CNOTs), "
                f"FP64 oracle (Algorithm 1 loop, outer loop over {self.threads} OpenMP threads), from |0...0>")


RENORM_PERIOD = 64


def gpu_results_for_accuracy(B, n_acc, depth, opts=None):
    """The GPU's final states for the bench's circuit family at a size the host oracle finishes in seconds:
    complex128 double-float (with the FP64 share), all-FP64, and complex64 without and with periodic
    renormalisation (every RENORM_PERIOD gates, FP64 norm).  `opts` maps a dtype to the options of the timed
    run ({option: value}: chunk size, FP64 share, tensor blocks), applied to the double-float and complex64
    states so that their errors are those of the configuration timed.  Compared in the CPU leg."""
    w = C.random_workload(n_acc, depth, seed=SEED)
    res = {}
    for name, dt, arith, renorm in (("c128_df32", B.SV_C128, B.SV_ARITH_DF32, 0),
                                    ("c128_f64", B.SV_C128, B.SV_ARITH_F64, 0),
                                    ("c64", B.SV_C64, B.SV_ARITH_AUTO, 0),
                                    ("c64_renorm", B.SV_C64, B.SV_ARITH_AUTO, RENORM_PERIOD)):
        h = B.sv_create(n_acc, dt)
        try:
            if dt == B.SV_C128:
                B.sv_set_option(h, B.SV_OPT_ARITH, arith)
            if arith != B.SV_ARITH_F64:
                for opt, val in (opts or {}).get(dt, {}).items():
                    B.sv_set_option(h, opt, val)
            B.sv_set_option(h, B.SV_OPT_RENORM_PERIOD, renorm)
            B.sv_apply_circuit(h, w.gates)
            res[name] = B.sv_read_amplitudes(h).astype(np.complex128)
        finally:
            B.sv_destroy(h)
    return w, res


def cpu_leg_accuracy(n_acc, depth, w, gpu_states):
    """CPU leg, part 2: the full FP64 oracle on the same n_acc-qubit circuit (timed), and the max-abs
    amplitude error and 1 - fidelity of each GPU result against it."""
    import oracle
    t0 = time.perf_counter()
    want = oracle.simulate(n_acc, w.gates, 0, threads=oracle.max_threads())
    dt = time.perf_counter() - t0
    out = {"n": n_acc, "layers": depth, "reference": "FP64 oracle, full state",
           "oracle_seconds": dt, "oracle_gates_per_s": len(w.gates) / dt}
    scale = float(np.max(np.abs(want)))
    for name, got in gpu_states.items():
        fid = abs(np.vdot(want, got)) ** 2 / (np.vdot(want, want).real * np.vdot(got, got).real)
        err = float(np.max(np.abs(got - want)))
        out[name] = {"max_abs_err": err, "max_abs_err_rel": err / scale,
                     "one_minus_fidelity": float(max(0.0, 1.0 - fid)),
                     "norm_deviation": float(abs(np.vdot(got, got).real - 1.0))}
    out["max_abs_psi"] = scale
    out["renorm_period_gates"] = RENORM_PERIOD
    return out


def cpu_baseline(n, gates, budget_s):
    r = OracleRunner(n, gates)
    r.step()  # first touch of the 2^n-amplitude array outside the timing
    t0 = time.perf_counter()
    count = 0
    while True:
        r.step()
        count += 1
        if time.perf_counter() - t0 >= budget_s or count >= 200:
            break
    dt = time.perf_counter() - t0
    return {"value": count / dt, "unit": "gates/s", "cores": r.threads, "kind": "oracle",
            "sample": f"{count} " + r.desc(n) + f"; {dt:.1f} s"}


def run_reference(args):
    if RANK != 0:
        return
    w = C.random_workload(args.n, args.depth, seed=SEED)
    r = OracleRunner(args.n, w.gates)
    for _ in range(max(args.warmup, 1)):
        r.step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        r.step()
    dt = time.perf_counter() - t0
    value = args.steps / dt
    line = {
        "impl": "reference", "metric": f"gates/s, n={args.n} random circuit ({args.depth} layers), complex128",
        "value": value, "unit": "gates/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic", "config": workload_config(args),
        "cpu_baseline": {"value": value, "unit": "gates/s", "cores": r.threads, "kind": "oracle",
                         "sample": f"each step = 1 " + r.desc(args.n)},
        "e2e": {"value": value, "unit": "gates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def workload_config(args):
    return {"workload": f"random circuit, n={args.n} qubits, {args.depth} layers of Haar U(2) on every qubit + "
                        f"CNOTs on a random perfect matching ({args.depth * (args.n + args.n // 2)} gates), "
                        f"from |0...0>, seed {SEED}; then FP64 norm and {READ_COUNT} amplitudes read back",
            "n": args.n, "layers": args.depth, "gates": args.depth * (args.n + args.n // 2),
            "state_bytes_c128": 16 << args.n, "l2": "state larger than L2 (126 MB): no flush needed",
            "parallelism": f"replicas x{args.gpus}"}


# ---------------------------------------------------------------------------------------------------------
# Our arm
# ---------------------------------------------------------------------------------------------------------
def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, v):
    if dist is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(dist, v):
    if dist is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def run_ours(args):
    import torch
    from paper_1801_01037_gb300 import build as sv_build
    dist = None
    if WORLD > 1:
        import torch.distributed as td
        td.init_process_group("gloo")
        dist = td
    sv_build.build()
    from paper_1801_01037_gb300 import _binding as B
    B.load()
    torch.cuda.init()
    w = C.random_workload(args.n, args.depth, seed=SEED)
    gates = w.gates
    G = len(gates)

    def step(h, graph=True):
        B.sv_init_basis(h, 0)
        (B.sv_apply_circuit_graph if graph else B.sv_apply_circuit)(h, gates)
        nrm = B.sv_norm(h)
        amps = B.sv_read_amplitudes(h, 0, READ_COUNT)
        return nrm, amps

    # Chunk size, FP64 share and tensor blocks per dtype from the autotuner, timed on an 8-layer circuit of the
    # same shape (another seed; untimed here).
    chunk_k, tuning, tensor_blocks = {}, {}, {}
    f64_share = B.SV_F64_SHARE_DEFAULT  # share of chunks done on the FP64 pipe unless the autotuner picks one
    if not args.no_autotune:
        from paper_1801_01037_gb300 import autotune
        probe = C.random_workload(args.n, 8, seed=SEED + 7).gates
        for dt, ar in ((B.SV_C128, B.SV_ARITH_DF32), (B.SV_C64, B.SV_ARITH_AUTO)):
            res = autotune.tune(args.n, dt, probe, ar, save=False)
            chunk_k[dt] = res["best"]
            tensor_blocks[dt] = int(res.get("best_tensor_blocks", 0))
            tuning["c128" if dt == B.SV_C128 else "c64"] = res
            if dt == B.SV_C128:
                f64_share = int(res["best_f64_share"])
    if args.tensor_blocks is not None:
        tb = [int(v) for v in str(args.tensor_blocks).split(",")]
        tensor_blocks = {B.SV_C128: tb[0], B.SV_C64: tb[-1]}

    def timed(dtype, arith, steps, warmup, profile=False, sampler=None, renorm=0):
        h = B.sv_create(args.n, dtype)
        try:
            B.sv_set_option(h, B.SV_OPT_RENORM_PERIOD, renorm)
            if dtype == B.SV_C128:
                B.sv_set_option(h, B.SV_OPT_ARITH, arith)
                B.sv_set_option(h, B.SV_OPT_F64_SHARE, f64_share)
            if dtype in chunk_k:
                B.sv_set_option(h, B.SV_OPT_CHUNK_QUBITS, chunk_k[dtype])
            if arith != B.SV_ARITH_F64:
                B.sv_set_option(h, B.SV_OPT_TENSOR_BLOCKS, tensor_blocks.get(dtype, 0))
            B.sv_set_option(h, B.SV_OPT_PROFILE, 1 if profile else 0)
            graph = renorm == 0  # renormalisation runs between launches, so not inside a captured graph
            for _ in range(warmup):
                step(h, graph)
            torch.cuda.synchronize()
            barrier(dist)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            fused_launches, fused_ms = 0, 0.0
            if sampler:
                sampler.start()
            e0.record()
            for _ in range(steps):
                nrm, _ = step(h, graph)
                if profile:
                    l, ms = B.sv_profile_last(h, 0)
                    fused_launches += l
                    fused_ms += ms
            e1.record()
            torch.cuda.synchronize()
            clocks = sampler.stop() if sampler else None
            barrier(dist)
            ms = e0.elapsed_time(e1)
            stats = B.sv_last_plan_stats(h)
            stats.update(B.sv_last_plan_blocks(h))
            return {"ms": ms, "norm": nrm, "fused_launches": fused_launches, "fused_ms": fused_ms, "stats": stats,
                    "clocks": clocks}
        finally:
            B.sv_destroy(h)

    def sweep_roofline(dtype, arith, u, label, peak, n=None):
        """Single-gate sweeps (the unfused path) on targets spread over all qubits, timed per launch."""
        n = n or args.n
        h = B.sv_create(n, dtype)
        try:
            if dtype == B.SV_C128:
                B.sv_set_option(h, B.SV_OPT_ARITH, arith)
            B.sv_set_option(h, B.SV_OPT_PROFILE, 1)
            B.sv_set_option(h, B.SV_OPT_PRODUCT_START, 0)  # every gate is a sweep launch, even on |0...0>
            targets = sorted({0, 1, n // 4, n // 2, 3 * n // 4, n - 2, n - 1})
            for t in targets[:2]:
                B.sv_apply_gate(h, u, t)
            ms_list = []
            for t in targets:
                B.sv_apply_gate(h, u, t)
                _, ms = B.sv_profile_last(h, 1)
                ms_list.append(ms)
            ab = (8 if dtype == B.SV_C64 else 16) << n
            avg = sum(ms_list) / len(ms_list)
            ach = 2 * ab / (avg * 1e-3) / 1e9
            return {"kernel": f"k_sweep ({label}), n={n}", "n": n, "bound": "hbm", "achieved": ach, "peak": peak,
                    "unit": "GB/s",
                    "frac": ach / peak, "avg_launch_ms": avg, "algorithmic_bytes_per_launch": 2 * ab,
                    "targets": targets, "per_target_ms": [round(x, 3) for x in ms_list]}
        finally:
            B.sv_destroy(h)

    sampler = ClockSampler()
    c128 = timed(B.SV_C128, B.SV_ARITH_DF32, args.steps, args.warmup, profile=True, sampler=sampler)
    c64 = timed(B.SV_C64, B.SV_ARITH_AUTO, args.steps, args.warmup)
    f64 = None if args.no_f64 else timed(B.SV_C128, B.SV_ARITH_F64, 1, 1)

    # end to end through the public API with host buffers: gate records uploaded and results read every step
    h = B.sv_create(args.n, B.SV_C128)
    try:
        if B.SV_C128 in chunk_k:
            B.sv_set_option(h, B.SV_OPT_CHUNK_QUBITS, chunk_k[B.SV_C128])
        B.sv_set_option(h, B.SV_OPT_F64_SHARE, f64_share)
        B.sv_set_option(h, B.SV_OPT_TENSOR_BLOCKS, tensor_blocks.get(B.SV_C128, 0))
        for _ in range(max(1, args.warmup)):
            step(h, graph=False)
        torch.cuda.synchronize()
        barrier(dist)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            step(h, graph=False)
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        st = B.sv_last_plan_stats(h)
        st_blk = B.sv_last_plan_blocks(h)
    finally:
        B.sv_destroy(h)
    # bytes of the plan's device blob uploaded per step: one 192-byte record per fused gate (a block's header
    # replaces its gates; the bench circuit has no two-qubit gates), then, 128-byte aligned, 6 digit planes of
    # 2 KiB per complex128 block; sweeps take their record as a kernel parameter
    records = st["fused_gates"] - st_blk["block_gates"] + st_blk["blocks"]
    blob_bytes = ((records * 192 + 127) // 128 * 128 + st_blk["blocks"] * 6 * 2048) if st_blk["blocks"] else records * 192

    t_max = max_over_ranks(dist, c128["ms"]) / 1e3
    total_gates = sum_over_ranks(dist, G * args.steps)
    value = total_gates / t_max
    e2e_max = max_over_ranks(dist, e2e_s)
    e2e_value = total_gates / e2e_max
    c64_t = max_over_ranks(dist, c64["ms"]) / 1e3
    state_bytes = 16 << args.n

    peak, peak_kind = measured_peaks()
    u_dense = C.haar_u2(np.random.Generator(np.random.PCG64(7)))
    sweeps = [sweep_roofline(B.SV_C128, B.SV_ARITH_DF32, u_dense, "c128 dense U(2), double-float", peak),
              sweep_roofline(B.SV_C128, B.SV_ARITH_DF32, C.X, "c128 X, moves", peak),
              sweep_roofline(B.SV_C64, B.SV_ARITH_AUTO, u_dense, "c64 dense U(2)", peak)]
    # the same complex128 sweep on the 128 GiB state of n = 33 (spec range n = 30-33), when it fits
    if args.n == N_QUBITS and not args.no_n33:
        import torch
        free_b, _ = torch.cuda.mem_get_info()
        if free_b >= (16 << 33) + (2 << 30):
            sweeps.append(sweep_roofline(B.SV_C128, B.SV_ARITH_DF32, u_dense, "c128 dense U(2), double-float", peak,
                                         n=33))
    avg_ms = c128["fused_ms"] / max(1, c128["fused_launches"])
    hbm_achieved = 2 * state_bytes / (avg_ms * 1e-3) / 1e9 if c128["fused_launches"] else None
    # FP32-pipe roofline of the fused pass (it is bound by instruction issue, not by HBM).  With `f64_share`
    # percent of the chunks computed on the FP64 pipe, the FP32 pipes carry the rest of the double-float work;
    # the FP64 pipe's own work (8 multiply-adds per amplitude of a dense gate) is reported beside it.
    df_frac = 1.0 - f64_share / 100.0
    # Gates folded into the product-state factors at the start of each step never reach a kernel.
    kernel_gates = gates_after_product_start(gates, args.n)
    ops_step = df32_ops_per_step(kernel_gates, args.n, c128["stats"]["passes"]) * df_frac
    ops_launch = ops_step / max(1, c128["stats"]["passes"])
    sm_hz = (c128["clocks"] or {}).get("sm_mhz") or 2070.0
    alu_peak = 152 * 128 * sm_hz * 1e6 / 1e12
    alu_achieved = ops_launch / (avg_ms * 1e-3) / 1e12 if c128["fused_launches"] else None
    f64_fma_launch = f64_fmas_per_step(kernel_gates, args.n) * (f64_share / 100.0) / max(1, c128["stats"]["passes"])
    f64_peak = 152 * 1.73 * sm_hz * 1e6 / 1e12  # measured FP64 multiply-adds per clock per SM
    f64_achieved = f64_fma_launch / (avg_ms * 1e-3) / 1e12 if c128["fused_launches"] else None
    traffic = committed_traffic(args.n, "k_fused_tc" if c128["stats"]["blocks"] else "k_fused_mixed")
    blocks_on = c128["stats"]["blocks"] > 0
    # init, passes, sweeps, bit-permutation passes, the two norm kernels, and the two product-start kernels
    folded_start = c128["stats"]["absorbed"] > 0
    launches_per_step = (1 + c128["stats"]["passes"] + c128["stats"]["sweep_gates"] + c128["stats"]["remaps"] + 2
                         + (2 if folded_start else 0))
    # The other configurations of the metric, measured after the timed region: a bounded served stream
    # (complex64, 150 GB budget) and a 512-circuit batch per dtype (chunk sizes per size class of n).
    served = batched = qft = None
    if not args.no_extra:
        served = served_measure(B, args.served_rate, args.served_requests)
        ws_b = C.batched_workloads(512, seed=1004)
        batched = {}
        for dt_b, name in ((B.SV_C64, "c64"), (B.SV_C128, "c128")):
            ks, picked = batch_chunk_sizes(B, [w.n for w in ws_b], dt_b, not args.no_autotune)
            batched[name] = {**batched_measure(B, ws_b, dt_b, ks, tensor_blocks.get(B.SV_C128, 0)),
                             "chunk_qubits": picked or "default"}
        batched["workload"] = "512 random circuits, n log-uniform in [10, 22], 10-40 layers, seed 1004"
        qft = {"qft20": qft_measure(B, "qft20", 5, 3, tensor_blocks.get(B.SV_C128, 0))}
        if args.n == N_QUBITS and not args.no_n33:
            import torch
            free_b, _ = torch.cuda.mem_get_info()
            if free_b >= (16 << 33) + (2 << 30):
                qft["qft33"] = qft_measure(B, "qft33", 1, 1, tensor_blocks.get(B.SV_C128, 0))
    # c64 with periodic renormalisation (every RENORM_PERIOD gates), one step, for its cost beside c64 without
    c64_renorm = timed(B.SV_C64, B.SV_ARITH_AUTO, 1, 1, renorm=RENORM_PERIOD)
    cpu = cpu_baseline(args.n, gates, args.cpu_seconds) if RANK == 0 and WORLD == 1 else None
    accuracy = None
    if RANK == 0:
        n_acc = min(args.n, 22)
        opts = {B.SV_C128: {B.SV_OPT_F64_SHARE: f64_share, B.SV_OPT_TENSOR_BLOCKS: tensor_blocks.get(B.SV_C128, 0)},
                B.SV_C64: {B.SV_OPT_TENSOR_BLOCKS: tensor_blocks.get(B.SV_C64, 0)}}
        for dt in (B.SV_C128, B.SV_C64):
            if dt in chunk_k and chunk_k[dt] <= n_acc:
                opts[dt][B.SV_OPT_CHUNK_QUBITS] = chunk_k[dt]
        w_acc, gpu_states = gpu_results_for_accuracy(B, n_acc, args.depth, opts)
        accuracy = cpu_leg_accuracy(n_acc, args.depth, w_acc, gpu_states)
        accuracy["options"] = {"c128_df32": {"f64_share": f64_share, "tensor_blocks": tensor_blocks.get(B.SV_C128, 0),
                                             "chunk_qubits": chunk_k.get(B.SV_C128, "default")},
                               "c64": {"tensor_blocks": tensor_blocks.get(B.SV_C64, 0),
                                       "chunk_qubits": chunk_k.get(B.SV_C64, "default")}}

    if RANK != 0:
        return
    # FP64-equivalent work of the method (16 flops per touched amplitude of a dense 2x2 gate, 6 per touched
    # amplitude of a diagonal one, none for an exchange) per fused launch
    flops_launch = 2.0 * f64_fmas_per_step(kernel_gates, args.n) / max(1, c128["stats"]["passes"])
    line = {
        "metric": f"gates/s, n={args.n} random circuit ({args.depth} layers), complex128",
        "value": value,
        "unit": "gates/s",
        "n_gpus": WORLD,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": t_max * 1e3 / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": f"complex128 storage (IEEE double); arithmetic f32x2 double-float on the FP32 pipes with {f64_share}% "
                 f"of the chunks in native f64 on the FP64 pipe",
        "data": "synthetic (seeded Haar-random U(2) layers and random-matching CNOTs)",
        "config": {**workload_config(args),
                   "chunk_qubits": {"c128": chunk_k.get(B.SV_C128, "default 12"), "c64": chunk_k.get(B.SV_C64, "default 13")},
                   "autotune_ms": tuning},
        "f64_native": None if f64 is None else {"value": G / (f64["ms"] / 1e3), "unit": "gates/s",
                                                 "ms_per_step": f64["ms"],
                                                 "note": "the same step with IEEE FP64 arithmetic throughout "
                                                         "(SV_ARITH_F64), 1 timed step after 1 warm-up"},
        "c64": {"value": total_gates / c64_t, "unit": "gates/s",
                "ms_per_step": c64_t * 1e3 / args.steps,
                "effective_hbm_gbs": G * args.steps / c64_t * 2 * (8 << args.n) / 1e9,
                "with_renormalisation": {"period_gates": RENORM_PERIOD, "ms_per_step": c64_renorm["ms"],
                                         "value": G / (c64_renorm["ms"] / 1e3), "unit": "gates/s",
                                         "note": "1 step, direct launches (renormalisation between launches)"}},
        "effective_hbm_gbs": value * 2 * state_bytes / 1e9 / WORLD,
        "served": served,
        "batched": batched,
        "qft": qft,
        "plan": {"passes_per_step": c128["stats"]["passes"], "sweeps_per_step": c128["stats"]["sweep_gates"],
                 "fused_gates_per_step": c128["stats"]["fused_gates"],
                 "folded_into_product_start": c128["stats"]["absorbed"],
                 "tensor_blocks_per_step": c128["stats"]["blocks"], "gates_in_tensor_blocks": c128["stats"]["block_gates"],
                 "tensor_blocks_option": {"c128": tensor_blocks.get(B.SV_C128, 0), "c64": tensor_blocks.get(B.SV_C64, 0)}},
        # The method's roofline of the dominant kernel (algorithmic bytes: one read and one write of the state
        # per fused pass, against the measured HBM copy bandwidth).  The pass is limited by arithmetic issue, not
        # by HBM: its FP32-pipe and FP64-pipe views follow, and its FP64-equivalent flop rate.
        "roofline": {"kernel": (("k_fused_tc (passes with dense tcgen05 blocks) and " if c128["stats"]["blocks"] else "")
                                + ("k_fused_mixed (c128 fused chunk pass: double-float CTAs + one FP64 CTA per SM)"
                                   if f64_share > 0 else "k_fused<c128, double-float> (fused chunk pass)")),
                     "bound": "hbm", "achieved": hbm_achieved, "peak": peak, "unit": "GB/s",
                     "frac": (hbm_achieved / peak) if hbm_achieved else None, "traffic": traffic,
                     "algorithmic_bytes_per_launch": 2 * state_bytes, "avg_launch_ms": avg_ms,
                     "launches_timed": c128["fused_launches"], "peak_source": f"{peak_kind} hbm_gbs",
                     "limited_by": ("the bf16 tensor-core MMAs of the blocks' exact digit products and the digit "
                                    "conversions around them (see tensor_core_view)" if blocks_on else
                                    "FP32-pipe issue of the double-float arithmetic (see alu_view)"),
                     "fp64_equivalent": {"flops_per_launch": flops_launch,
                                         "achieved_tflops": (flops_launch / (avg_ms * 1e-3) / 1e12) if hbm_achieved else None,
                                         "note": "16 flops per touched amplitude of a dense gate, 6 of a diagonal one"},
                     # the double-float method's operation count describes passes that apply every gate one by one;
                     # with tensor-core blocks most gates never run that way, so the view is left out
                     "alu_view": None if blocks_on else {
                         "achieved": alu_achieved, "peak": alu_peak, "unit": "T FP32-pipe ops/s",
                         "frac": (alu_achieved / alu_peak) if alu_achieved else None,
                         "algorithmic_ops_per_launch": ops_launch,
                         "peak_source": f"152 SMs x 128 lanes x {sm_hz:.0f} MHz (median SM clock sampled under load)",
                         "note": "operations of the double-float method itself (its chosen arithmetic)"},
                     "f64_share_percent": f64_share,
                     "tensor_core_view": tensor_view(c128, args.n, chunk_k.get(B.SV_C128, 12), avg_ms, sm_hz),
                     "fp64_pipe_view": None if blocks_on else {
                         "achieved": f64_achieved, "peak": f64_peak, "unit": "T FP64 FMA/s",
                         "frac": (f64_achieved / f64_peak) if f64_achieved else None,
                         "peak_source": "152 SMs x 1.73 FP64 FMA/clock (probe) x median SM clock"}},
        "sweep_roofline": sweeps,
        "cpu_baseline": cpu,
        "accuracy": accuracy,
        "e2e": {"value": e2e_value, "unit": "gates/s",
                "h2d_bytes_per_step": blob_bytes + st["sweep_gates"] * 192 + (96 * args.n if st["absorbed"] else 0),
                "d2h_bytes_per_step": 8 + READ_COUNT * 16,
                "note": "h2d: the plan's device blob uploaded per step (192-byte gate records, block headers and "
                        "the blocks' 12 KiB of digit planes each; a single-gate sweep takes its record as a kernel "
                        "parameter), plus 96 B per qubit of product-start factors; d2h: the FP64 norm and 1024 "
                        "amplitudes"},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": c128["clocks"],
        "norm_last_step": c128["norm"],
    }
    print(json.dumps(line), flush=True)


def tensor_view(run, n, k, avg_ms, sm_hz):
    """bf16 tensor-core work of the dense complex128 blocks: per block and chunk of 2^k amplitudes, 2^(k-11) tiles
    of 128 rows x 26 digit products of 128 x 32 x 32 multiply-adds (issued as 12 MMAs of N = 64 .. 224 per tile,
    which also multiply one zero plane: 27/26 of this work).  Averaged over the fused launches of the step
    (blocks run in most of them), against the measured bf16 dense peak scaled to the sampled clock."""
    blocks = run["stats"].get("blocks", 0)
    if not blocks or not run["fused_launches"]:
        return None
    flops_step = blocks * 2.0 ** (n - k) * 2 ** (k - 11) * 26 * 2 * (128 * 32 * 16) * 2
    flops_launch = flops_step / max(1, run["stats"]["passes"])
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        peak = float(pk["bf16_tflops_sustained"]) * (sm_hz / float(pk.get("sm_max_mhz", 2070.0)))
        src = "measured bf16_tflops_sustained x sampled / max SM clock"
    except Exception:
        peak, src = 1700.0, "fallback sustained bf16 (1.7 PFLOP/s)"
    ach = flops_launch / (avg_ms * 1e-3) / 1e12
    return {"achieved": ach, "peak": peak, "unit": "TFLOP/s (bf16 MMA)", "frac": ach / peak,
            "flops_per_launch": flops_launch, "blocks_per_step": blocks, "peak_source": src,
            "note": "exact base-256 digit products: 26 bf16 products per block and 128-row tile"}


# FP32-pipe operations of the double-float method per amplitude (integer, float add/sub, FMA and conversion
# instructions each count one): a dense 2x2 update (four 4-term compensated dot products: 6 per term, 7 per
# TwoSum step, 3 for the final Fast2Sum, i.e. 48 per real output), a complex scaling (diagonal / anti-diagonal
# entries, two 2-term dot products), and the double <-> float-pair conversion once per pass at load and store.
DF32_OPS_DENSE = 96
DF32_OPS_SCALE = 44
DF32_OPS_CONVERT = 68


def gates_after_product_start(gates, n):
    """The records left for the kernels when the step starts from a product state (|0...0> or |x>): the library
    folds every uncontrolled single-qubit gate and SWAP on qubits that no earlier remaining record touches into
    the qubits' factors (sv_init_product's rule).  Used only to count the kernels' algorithmic work."""
    touched = [False] * n
    keep, folded = [], 0
    for g in gates:
        kind, t = int(g["kind"]), int(g["target"])
        if kind == C.GATE_U and int(g["ncontrols"]) == 0 and not touched[t]:
            folded += 1
            continue
        if kind == C.GATE_SWAP and not touched[t] and not touched[int(g["target2"])]:
            folded += 1
            continue
        if kind == C.GATE_U4_ROW:
            keep.append(g)
            continue
        touched[t] = True
        if kind in (C.GATE_SWAP, C.GATE_U4):
            touched[int(g["target2"])] = True
        for c in range(int(g["ncontrols"])):
            touched[int(g["controls"][c])] = True
        keep.append(g)
    return keep if (not keep or folded >= max(2, n // 4)) else list(gates)


def df32_ops_per_step(gates, n, passes):
    """Algorithmic FP32-pipe operations of one application of `gates` with `passes` fused passes."""
    ops = float(passes) * DF32_OPS_CONVERT * 2 ** n
    for g in gates:
        if int(g["kind"]) != C.GATE_U:
            continue
        u = C.unpack_u(g)
        touched = 2.0 ** (n - int(g["ncontrols"]))
        if u[0, 1] == 0 and u[1, 0] == 0:
            if u[0, 0] == 1 and u[1, 1] == 1:
                continue
            ops += DF32_OPS_SCALE * touched * (0.5 if u[0, 0] == 1 else 1.0)
        elif u[0, 0] == 0 and u[1, 1] == 0:
            if not (u[0, 1] == 1 and u[1, 0] == 1):
                ops += DF32_OPS_SCALE * touched
        else:
            ops += DF32_OPS_DENSE * touched
    return ops


def f64_fmas_per_step(gates, n):
    """Real multiply-adds of the pair update in FP64 (8 per amplitude of a dense gate, 4 per touched amplitude of
    a diagonal or anti-diagonal one, none for an exchange)."""
    f = 0.0
    for g in gates:
        if int(g["kind"]) != C.GATE_U:
            continue
        u = C.unpack_u(g)
        touched = 2.0 ** (n - int(g["ncontrols"]))
        if u[0, 1] == 0 and u[1, 0] == 0:
            f += 0.0 if (u[0, 0] == 1 and u[1, 1] == 1) else 4 * touched * (0.5 if u[0, 0] == 1 else 1.0)
        elif u[0, 0] == 0 and u[1, 1] == 0:
            f += 0.0 if (u[0, 1] == 1 and u[1, 0] == 1) else 4 * touched
        else:
            f += 8 * touched
    return f


def committed_traffic(n, kernel="k_fused_mixed"):
    """DRAM bytes per launch of a fused c128 pass kernel on n qubits, scaled from the committed ncu capture at
    n = 28 (a pass reads and writes the whole state once, so traffic is proportional to 2^n), if that capture
    still matches the kernel source (null otherwise)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "fused_c128_traffic_n28.txt")
    try:
        kv = dict(line.split("=", 1) for line in open(path).read().split() if "=" in line)
        h = hashlib.sha256()
        for f in ("sv_fused.cu", "sv_arith.cuh"):
            h.update(open(os.path.join(ROOT, "paper_1801_01037_gb300", "csrc", f), "rb").read())
        if kv.get("source_sha256") != h.hexdigest()[:16]:
            return None
        return float(kv[kernel + "_bytes_n28"]) * 2.0 ** (n - 28)
    except Exception:
        return None


def qft_measure(B, which, steps, warmup, tensor_blocks=0):
    """qft20 = QFT on n = 20 from a seeded basis state (seed 1001, 16 MiB state, L2-resident: launch overhead and
    graph replay matter); qft33 = QFT on n = 33 then 10 random layers (seed 1003, 128 GiB state).  complex128,
    library defaults apart from SV_OPT_TENSOR_BLOCKS = `tensor_blocks`; a step = init |x>, graph replay of the
    circuit, FP64 norm, 1024 amplitudes read back."""
    import torch
    w = C.qft_workload(20, seed=1001) if which == "qft20" else C.qft_random_workload(33, 10, seed=1003)
    h = B.sv_create(w.n, B.SV_C128)
    try:
        B.sv_set_option(h, B.SV_OPT_TENSOR_BLOCKS, tensor_blocks)
        def step():
            B.sv_init_basis(h, w.x0)
            B.sv_apply_circuit_graph(h, w.gates)
            B.sv_norm(h)
            B.sv_read_amplitudes(h, 0, READ_COUNT)
        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            step()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        st = B.sv_last_plan_stats(h)
        blk = B.sv_last_plan_blocks(h)
    finally:
        B.sv_destroy(h)
    G = len(w.gates)
    return {"metric": f"gates/s, {w.name}, complex128", "value": G / (ms / 1e3), "unit": "gates/s",
            "ms_per_step": ms, "steps": steps, "warmup": warmup, "gates": G, "n": w.n,
            "effective_hbm_gbs": G / (ms / 1e3) * 2 * (16 << w.n) / 1e9,
            "plan": {"passes": st["passes"], "sweeps": st["sweep_gates"], "relabels": st["relabels"],
                     "tensor_blocks_option": tensor_blocks, "tensor_blocks": blk["blocks"]},
            "step": "init |x>, graph replay of the circuit, FP64 norm, 1024 amplitudes read back"}


def run_single_config(args):
    """The other single-state configurations (see qft_measure), as their own JSON line."""
    from paper_1801_01037_gb300 import build as sv_build
    sv_build.build()
    from paper_1801_01037_gb300 import _binding as B
    B.load()
    tb = int(str(args.tensor_blocks).split(",")[0]) if args.tensor_blocks is not None else 0
    print(json.dumps(qft_measure(B, args.workload, args.steps, args.warmup, tb)), flush=True)


SIZE_CLASSES = ((0, 13), (14, 17), (18, 99))


def batch_chunk_sizes(B, ns, dt, tune):
    """Chunk size per circuit: for each size class of n (up to 13, 14-17, 18 and up) the autotuner times the
    candidate k (and, for complex128, the FP64 share) on a 6-layer random circuit at the class's largest n in
    the batch; every circuit of the class gets that k.  tune=False: the library default (0) for all."""
    if not tune:
        return [0] * len(ns), {}
    from paper_1801_01037_gb300 import autotune
    arith = B.SV_ARITH_DF32 if dt == B.SV_C128 else B.SV_ARITH_AUTO
    ks, picked = [0] * len(ns), {}
    for lo, hi in SIZE_CLASSES:
        members = [i for i, n in enumerate(ns) if lo <= n <= hi]
        if not members:
            continue
        n_rep = max(ns[i] for i in members)
        probe = C.random_workload(n_rep, 6, seed=1004 + 7).gates
        k = int(autotune.tune(n_rep, dt, probe, arith, save=False)["best"])
        picked[f"n{lo}-{min(hi, max(ns))}"] = {"tuned_at_n": n_rep, "k": k}
        for i in members:
            ks[i] = k
    return ks, picked


def batched_measure(B, ws, dt, ks, tensor_blocks=0):
    """One sv_run_batch_k call over all circuits, end to end on the host clock (plan, allocate, upload, the
    captured rounds, synchronise), after a warm-up call on the first 64 circuits; complex128 batches with
    SV_OPT_TENSOR_BLOCKS = `tensor_blocks` (sv_batch_set_option)."""
    import torch
    ns, gl = [w.n for w in ws], [w.gates for w in ws]
    B.sv_batch_set_option(B.SV_OPT_TENSOR_BLOCKS, tensor_blocks if dt == B.SV_C128 else 0)
    for h in B.sv_run_batch(ns[:64], dt, gl[:64], chunk_k=ks[:64]):  # warm-up: kernels, allocator
        B.sv_destroy(h)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hs = B.sv_run_batch(ns, dt, gl, chunk_k=ks)
    dt_s = time.perf_counter() - t0
    st = B.sv_last_batch_stats()
    # a property of every result (unitary circuits keep the norm at 1); parity with the oracle is tested in
    # tests/test_gpu_batch_serve.py
    dev = max(abs(B.sv_norm(h) - 1.0) for h in hs)
    for h in hs:
        B.sv_destroy(h)
    gates_total = sum(len(g) for g in gl)
    B.sv_batch_set_option(B.SV_OPT_TENSOR_BLOCKS, 0)
    return {"circuits": len(ws), "seconds": dt_s, "circuits_per_s": len(ws) / dt_s, "gates_per_s": gates_total / dt_s,
            "rounds": st["rounds"], "mixed_rounds": st["mixed_rounds"], "tensor_core_rounds": st["tc_rounds"],
            "tensor_blocks_option": tensor_blocks if dt == B.SV_C128 else 0,
            "max_round_chunks": st["max_round_chunks"], "max_norm_deviation": dev}


def run_batched(args):
    """4096 independent random circuits (n log-uniform in [10, 22], 10-40 layers, seed 1004) in one
    sv_run_batch_k call per dtype, chunk sizes from the autotuner per size class of n; complex128 with
    tensor-core blocks of >= 3 dense updates (--tensor-blocks overrides; 0 turns them off)."""
    from paper_1801_01037_gb300 import build as sv_build
    sv_build.build()
    from paper_1801_01037_gb300 import _binding as B
    B.load()
    ws = C.batched_workloads(args.batch_count, seed=1004)
    ns = [w.n for w in ws]
    res = {}
    tb = int(str(args.tensor_blocks).split(",")[0]) if args.tensor_blocks is not None else 3
    for dt, name in ((B.SV_C64, "c64"), (B.SV_C128, "c128")):
        ks, picked = batch_chunk_sizes(B, ns, dt, not args.no_autotune)
        res[name] = {**batched_measure(B, ws, dt, ks, tb), "chunk_qubits": picked or "default"}
    print(json.dumps({"metric": "batched random circuits: circuits/s (one sv_run_batch call, end to end)",
                      "workload": f"{len(ws)} circuits, n log-uniform in [10, 22], depth 10-40 layers, seed 1004",
                      "gates": sum(len(w.gates) for w in ws), "amplitudes": sum(2 ** n for n in ns), **res}),
          flush=True)


def served_measure(B, rate, count, budget=150 * 10 ** 9, max_active=512):
    """Poisson arrivals (seed 1005) through the serving loop, complex64: circuits/s over the stream and latency
    percentiles (completion seen by sv_poll minus scheduled arrival)."""
    import threading
    stream = C.served_stream(count, rate, seed=1005)
    srv = B.sv_server_create(budget, max_active)
    tickets, arrival, done_at = [], {}, {}
    lock = threading.Lock()
    finished = threading.Event()

    def poller():
        while not finished.is_set() or len(done_at) < len(stream):
            with lock:
                pending = [t for t in tickets if t not in done_at]
            for t in pending:
                d, h = B.sv_poll(srv, t)
                if d:
                    done_at[t] = time.perf_counter()
                    B.sv_destroy(h)
            if len(done_at) == len(stream):
                break
            time.sleep(0.0002)

    try:
        th = threading.Thread(target=poller)
        th.start()
        t0 = time.perf_counter()
        for at, w in stream:
            now = time.perf_counter() - t0
            if at > now:
                time.sleep(at - now)
            t = B.sv_submit(srv, w.n, B.SV_C64, w.gates)
            with lock:
                tickets.append(t)
                arrival[t] = t0 + at
        finished.set()
        th.join()
        stats = B.sv_server_get_stats(srv)
    finally:
        B.sv_server_destroy(srv)
    t_end = max(done_at.values())
    lat = np.array([(done_at[t] - arrival[t]) * 1e3 for t in tickets])
    return {"rate_per_s": rate, "requests": len(stream), "circuits_per_s": len(stream) / (t_end - t0),
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "rounds": stats["rounds"], "max_round_chunks": stats["max_round_chunks"]}


def run_served(args):
    """Poisson arrivals through the serving loop (150 GB budget), complex64; per rate: circuits/s and
    latency percentiles."""
    import torch
    from paper_1801_01037_gb300 import build as sv_build
    sv_build.build()
    from paper_1801_01037_gb300 import _binding as B
    B.load()
    torch.cuda.init()
    sweep = [served_measure(B, float(x), args.served_count) for x in args.served_rates.split(",")]
    print(json.dumps({"metric": "served circuits/s and p50/p99 latency (complex64, 150 GB budget, continuous batching)",
                      "workload": "Poisson arrivals; each request a random circuit with n log-uniform in [12, 28], "
                                  "10-30 layers, seed 1005", "sweep": sweep}), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "served":
        run_served(args)
    elif args.workload in ("qft20", "qft33"):
        run_single_config(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
