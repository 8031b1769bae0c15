"""Chunk-size autotuner for the fused pass.

The fused pass holds 2^k amplitudes per CTA in shared memory.  A larger k lets a pass take more gates (fewer
passes, fewer HBM sweeps) but leaves fewer CTAs per SM to hide each other's load and barrier latency.  This
module times candidate k on the GPU through the C ABI (``SV_OPT_CHUNK_QUBITS``) for a circuit of the caller's
shape, then (complex128, double-float) the share of chunks given to the FP64 pipe (``SV_OPT_F64_SHARE``) and
whether dense tensor-core blocks pay (``SV_OPT_TENSOR_BLOCKS``),
keeps the fastest per (n, dtype, arithmetic) in a JSON cache, and applies it to a state.

Cache file: ``$SV_AUTOTUNE_CACHE`` or ``~/.cache/gb300_statevec_autotune.json``.
"""
from __future__ import annotations

import json
import os
import time

from . import _binding as B

CANDIDATES = {B.SV_C128: (10, 11, 12, 13), B.SV_C64: (11, 12, 13)}


def cache_path() -> str:
    return os.environ.get("SV_AUTOTUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache",
                                                            "gb300_statevec_autotune.json"))


def _key(n: int, dtype: int, arith: int) -> str:
    return f"n{n}_dt{dtype}_ar{arith}"


def load_cache() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(cache: dict) -> None:
    p = cache_path()
    os.makedirs(os.path.dirname(p), exist_ok=True)
    tmp = p + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, p)


F64_SHARES = (0, 10, 12, 14, 16, 18, 20)
# Tensor-core block options tried per dtype.  complex64 blocks are not tried: they gain a few per cent at
# most, and their FP32 accumulation on the tensor cores shrinks the state's norm by about 3e-7 per block (a
# drift, not random rounding), 40x the per-gate passes' norm drift on the bench circuit; SV_OPT_TENSOR_BLOCKS
# still turns them on by hand.
TENSOR_BLOCKS = {B.SV_C128: (0, 3, 4, 6), B.SV_C64: (0,)}


def time_candidate(n: int, dtype: int, arith: int, gates, k: int, repeats: int = 2, f64_share: int = -1,
                   tensor_blocks: int = 0) -> float:
    """Best device time (ms, summed over the fused-pass launches) of one application of `gates` with 2^k chunks
    (and, for complex128, `f64_share` percent of the chunks in native FP64; `tensor_blocks` as the option
    SV_OPT_TENSOR_BLOCKS)."""
    h = B.sv_create(n, dtype)
    try:
        if dtype == B.SV_C128:
            B.sv_set_option(h, B.SV_OPT_ARITH, arith)
            B.sv_set_option(h, B.SV_OPT_F64_SHARE, f64_share)
        B.sv_set_option(h, B.SV_OPT_CHUNK_QUBITS, k)
        B.sv_set_option(h, B.SV_OPT_TENSOR_BLOCKS, tensor_blocks)
        B.sv_set_option(h, B.SV_OPT_PROFILE, 1)
        best = float("inf")
        for _ in range(repeats + 1):  # the first run captures the graph
            B.sv_init_basis(h, 0)
            t0 = time.perf_counter()
            B.sv_apply_circuit_graph(h, gates)
            B.sv_sync(h)
            wall = (time.perf_counter() - t0) * 1e3
            total = 0.0
            for kind in (0, 1, 2):
                _, ms = B.sv_profile_last(h, kind)
                total += ms
            best = min(best, total if total > 0 else wall)
        return best
    finally:
        B.sv_destroy(h)


def tune(n: int, dtype: int, gates, arith: int = B.SV_ARITH_AUTO, candidates=None, save: bool = True) -> dict:
    """Time every candidate chunk size on `gates` (a circuit of the intended shape), cache and return
    {"best": k, "ms": {k: ms}}."""
    cands = [k for k in (candidates or CANDIDATES[dtype]) if k <= n]
    if not cands:
        cands = [n]
    ms = {k: time_candidate(n, dtype, arith, gates, k) for k in cands}
    best = min(ms, key=ms.get)
    res = {"best": best, "ms": {str(k): v for k, v in ms.items()}}
    share = -1
    if dtype == B.SV_C128 and arith != B.SV_ARITH_F64:
        sh = {s: time_candidate(n, dtype, arith, gates, best, f64_share=s) for s in F64_SHARES}
        share = min(sh, key=sh.get)
        res["best_f64_share"] = share
        res["f64_share_ms"] = {str(s): v for s, v in sh.items()}
    if arith != B.SV_ARITH_F64:
        # dense tensor-core blocks (off, or blocks that replace at least 3, 4 or 6 dense one-qubit updates)
        tb = {t: time_candidate(n, dtype, arith, gates, best, f64_share=share, tensor_blocks=t)
              for t in TENSOR_BLOCKS[dtype]}
        res["best_tensor_blocks"] = min(tb, key=tb.get)
        res["tensor_blocks_ms"] = {str(t): v for t, v in tb.items()}
    if save:
        cache = load_cache()
        cache[_key(n, dtype, arith)] = res
        save_cache(cache)
    return res


def best_chunk_qubits(n: int, dtype: int, arith: int = B.SV_ARITH_AUTO) -> int | None:
    ent = load_cache().get(_key(n, dtype, arith))
    return int(ent["best"]) if ent else None


def apply(h: int, arith: int = B.SV_ARITH_AUTO) -> int | None:
    """Set the cached best chunk size (and FP64 share) on state handle `h` (no-op without a cache entry);
    returns the chunk size."""
    n, dtype, _ = B.sv_get_info(h)
    ent = load_cache().get(_key(n, dtype, arith))
    if not ent:
        return None
    B.sv_set_option(h, B.SV_OPT_CHUNK_QUBITS, int(ent["best"]))
    if "best_f64_share" in ent:
        B.sv_set_option(h, B.SV_OPT_F64_SHARE, int(ent["best_f64_share"]))
    if "best_tensor_blocks" in ent:
        B.sv_set_option(h, B.SV_OPT_TENSOR_BLOCKS, int(ent["best_tensor_blocks"]))
    return int(ent["best"])
