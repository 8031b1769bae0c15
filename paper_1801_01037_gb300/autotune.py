"""Chunk-size autotuner for the fused pass.

The fused pass holds 2^k amplitudes per CTA in shared memory.  A larger k lets a pass take more gates (fewer
passes, fewer HBM sweeps) but leaves fewer CTAs per SM to hide each other's load and barrier latency.  This
module times candidate k on the GPU through the C ABI (``SV_OPT_CHUNK_QUBITS``) for a circuit of the caller's
shape, keeps the fastest per (n, dtype, arithmetic) in a JSON cache, and applies it to a state.

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


def time_candidate(n: int, dtype: int, arith: int, gates, k: int, repeats: int = 2) -> float:
    """Best device time (ms, summed over the fused-pass launches) of one application of `gates` with 2^k chunks."""
    h = B.sv_create(n, dtype)
    try:
        if dtype == B.SV_C128:
            B.sv_set_option(h, B.SV_OPT_ARITH, arith)
        B.sv_set_option(h, B.SV_OPT_CHUNK_QUBITS, k)
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
    if save:
        cache = load_cache()
        cache[_key(n, dtype, arith)] = res
        save_cache(cache)
    return res


def best_chunk_qubits(n: int, dtype: int, arith: int = B.SV_ARITH_AUTO) -> int | None:
    ent = load_cache().get(_key(n, dtype, arith))
    return int(ent["best"]) if ent else None


def apply(h: int, arith: int = B.SV_ARITH_AUTO) -> int | None:
    """Set the cached best chunk size on state handle `h` (no-op without a cache entry); returns it."""
    n, dtype, _ = B.sv_get_info(h)
    k = best_chunk_qubits(n, dtype, arith)
    if k is not None:
        B.sv_set_option(h, B.SV_OPT_CHUNK_QUBITS, k)
    return k
