"""ctypes binding of ``libsv.so`` (argument marshalling only; every step runs in the CUDA library).

Each ``sv_*`` function here has the name and argument order of its C counterpart in ``include/sv.h``;
pointers become numpy arrays / integers, output parameters become return values, and a non-zero status
raises :class:`SvError`.  The library is loaded from this package's directory and never built or replaced by
a fallback at import time: if it is missing, :func:`load` raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsv.so")

SV_OK = 0
SV_ERR_ARG = -1
SV_ERR_OOM = -2
SV_ERR_CUDA = -3
SV_ERR_NOT_UNITARY = -4
SV_ERR_TIMEOUT = -5
SV_ERR_BUSY = -6
SV_ERR_NOT_FOUND = -7
SV_ERR_NO_DEVICE = -8

SV_C64 = 1
SV_C128 = 2
SV_ARITH_AUTO = 0
SV_ARITH_F64 = 1
SV_ARITH_DF32 = 2

SV_OPT_ARITH = 1
SV_OPT_CHUNK_QUBITS = 2
SV_OPT_FUSION = 3
SV_OPT_RENORM_PERIOD = 4
SV_OPT_CANONICAL = 5
SV_OPT_PROFILE = 6
SV_OPT_F64_SHARE = 7
SV_OPT_CUBES = 8
SV_F64_SHARE_DEFAULT = 16
SV_OPT_PRODUCT_START = 9
SV_OPT_TENSOR_BLOCKS = 10

SV_GATE_U = 0
SV_GATE_SWAP = 1
SV_GATE_U4 = 2
SV_GATE_U4_ROW = 3

EXPORTED = [
    "sv_create", "sv_create_from_buffer", "sv_destroy", "sv_init_basis", "sv_init_product", "sv_write_amplitudes", "sv_set_option",
    "sv_get_info", "sv_get_layout", "sv_canonicalize", "sv_apply_gate", "sv_apply_gate2q", "sv_apply_swap", "sv_apply_circuit",
    "sv_apply_circuit_graph", "sv_read_amplitudes", "sv_read_amplitudes_at", "sv_read_probabilities", "sv_sample", "sv_expect_z", "sv_norm", "sv_norm_noalloc",
    "sv_renormalize", "sv_sync", "sv_last_plan_stats", "sv_plan_dry_run", "sv_profile_last", "sv_run_batch", "sv_run_batch_k", "sv_server_create", "sv_server_destroy",
    "sv_submit", "sv_poll", "sv_last_error", "sv_version", "sv_last_batch_stats", "sv_server_pause",
    "sv_server_get_stats", "sv_last_plan_blocks", "sv_batch_set_option", "sv_plan_dry_run_blocks",
]

BATCH_STATS_FIELDS = ["rounds", "mixed_rounds", "max_round_chunks", "total_chunks", "tc_rounds"]
SERVER_STATS_FIELDS = ["submitted", "admitted", "completed", "failed", "rounds", "mixed_rounds", "max_round_chunks",
                       "active", "pending", "budget_used"]


class SvError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"sv error {code}: {msg}")
        self.code = code


_lib = None
P = ctypes.c_void_p
PP = ctypes.POINTER(ctypes.c_void_p)


def load(path: str | None = None):
    """Load ``libsv.so`` (raises ``OSError`` if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise OSError(f"{path} not found: build it with `python -m paper_1801_01037_gb300.build`")
    lib = ctypes.CDLL(path)
    i, u64, sz, d = ctypes.c_int, ctypes.c_uint64, ctypes.c_size_t, ctypes.c_double
    sig = {
        "sv_create": [i, i, P, PP],
        "sv_create_from_buffer": [i, i, P, P, PP],
        "sv_destroy": [P],
        "sv_init_basis": [P, u64],
        "sv_init_product": [P, P],
        "sv_write_amplitudes": [P, u64, u64, P],
        "sv_set_option": [P, i, ctypes.c_int64],
        "sv_get_info": [P, P, P, P],
        "sv_get_layout": [P, P],
        "sv_canonicalize": [P],
        "sv_apply_gate": [P, P, i, P, i],
        "sv_apply_gate2q": [P, P, i, i, P, i],
        "sv_apply_swap": [P, i, i],
        "sv_apply_circuit": [P, P, sz],
        "sv_apply_circuit_graph": [P, P, sz],
        "sv_read_amplitudes": [P, u64, u64, P],
        "sv_read_amplitudes_at": [P, P, u64, P],
        "sv_read_probabilities": [P, u64, u64, P],
        "sv_norm": [P, ctypes.POINTER(d)],
        "sv_sample": [P, P, u64, P],
        "sv_expect_z": [P, u64, ctypes.POINTER(d)],
        "sv_norm_noalloc": [P, i, i, P, P],
        "sv_renormalize": [P],
        "sv_sync": [P],
        "sv_last_plan_stats": [P, P, P, P, P, P, P],
        "sv_plan_dry_run": [i, i, i, P, sz, P, P, P, P, i, P],
        "sv_profile_last": [P, i, ctypes.POINTER(i), ctypes.POINTER(d)],
        "sv_run_batch": [i, P, i, P, P, P, P],
        "sv_run_batch_k": [i, P, i, P, P, P, P, P],
        "sv_server_create": [sz, i, PP],
        "sv_server_destroy": [P],
        "sv_submit": [P, i, i, P, sz, ctypes.POINTER(u64)],
        "sv_poll": [P, u64, ctypes.POINTER(i), PP],
        "sv_last_batch_stats": [P],
        "sv_server_pause": [P, i],
        "sv_server_get_stats": [P, P],
        "sv_last_plan_blocks": [P, P, P],
        "sv_batch_set_option": [i, i],
        "sv_plan_dry_run_blocks": [i, i, i, i, P, sz, P, P, P, P],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.sv_last_error.restype = ctypes.c_char_p
    lib.sv_last_error.argtypes = []
    lib.sv_version.restype = ctypes.c_char_p
    lib.sv_version.argtypes = []
    _lib = lib
    return lib


def _check(rc: int):
    if rc != SV_OK:
        raise SvError(rc, load().sv_last_error().decode())


def _dtype_np(dtype: int):
    return np.complex64 if dtype == SV_C64 else np.complex128


def _stream_ptr(stream) -> int | None:
    """torch.cuda.Stream / int / None -> raw cudaStream_t value."""
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


# ---------------------------------------------------------------------------------------------------------
# One wrapper per C entry point
# ---------------------------------------------------------------------------------------------------------
def sv_create(n: int, dtype: int = SV_C128, stream=None) -> int:
    h = ctypes.c_void_p()
    _check(load().sv_create(n, dtype, _stream_ptr(stream), ctypes.byref(h)))
    return h.value


def sv_create_from_buffer(n: int, dtype: int, dev_ptr: int, stream=None) -> int:
    h = ctypes.c_void_p()
    _check(load().sv_create_from_buffer(n, dtype, dev_ptr, _stream_ptr(stream), ctypes.byref(h)))
    return h.value


def sv_destroy(h: int) -> None:
    _check(load().sv_destroy(h))


def sv_init_basis(h: int, x: int) -> None:
    _check(load().sv_init_basis(h, x))


def sv_init_product(h: int, factors) -> None:
    """Product state: factors[t] = (alpha_t, beta_t), complex, qubit t in alpha_t|0> + beta_t|1>."""
    f = np.ascontiguousarray(np.asarray(factors, dtype=np.complex128).reshape(-1, 2)).view(np.float64).ravel()
    _check(load().sv_init_product(h, f.ctypes.data))


def sv_write_amplitudes(h: int, first: int, values: np.ndarray) -> None:
    v = np.ascontiguousarray(values)
    _check(load().sv_write_amplitudes(h, first, v.size, v.ctypes.data))


def sv_set_option(h: int, option: int, value: int) -> None:
    _check(load().sv_set_option(h, option, value))


def sv_get_info(h: int):
    n, dt, ptr = ctypes.c_int(), ctypes.c_int(), ctypes.c_void_p()
    _check(load().sv_get_info(h, ctypes.byref(n), ctypes.byref(dt), ctypes.byref(ptr)))
    return n.value, dt.value, ptr.value


def sv_get_layout(h: int) -> np.ndarray:
    n = sv_get_info(h)[0]
    perm = np.zeros(n, dtype=np.int32)
    _check(load().sv_get_layout(h, perm.ctypes.data))
    return perm


def sv_canonicalize(h: int) -> None:
    _check(load().sv_canonicalize(h))


def sv_apply_gate(h: int, u, target: int, controls=()) -> None:
    u = np.asarray(u, dtype=np.complex128).reshape(2, 2)
    U = np.ascontiguousarray(np.stack([u.real, u.imag], axis=-1).reshape(8))
    c = np.ascontiguousarray(np.asarray(controls, dtype=np.int32))
    _check(load().sv_apply_gate(h, U.ctypes.data, target, c.ctypes.data if c.size else None, int(c.size)))


def sv_apply_gate2q(h: int, v, q0: int, q1: int, controls=()) -> None:
    """Dense two-qubit gate v (4x4, entry order b0 + 2 b1 with b0 the bit of q0)."""
    v = np.asarray(v, dtype=np.complex128).reshape(4, 4)
    V = np.ascontiguousarray(np.stack([v.real, v.imag], axis=-1).reshape(32))
    c = np.ascontiguousarray(np.asarray(controls, dtype=np.int32))
    _check(load().sv_apply_gate2q(h, V.ctypes.data, q0, q1, c.ctypes.data if c.size else None, int(c.size)))


def sv_apply_swap(h: int, a: int, b: int) -> None:
    _check(load().sv_apply_swap(h, a, b))


def _gate_array(gates: np.ndarray) -> np.ndarray:
    g = np.ascontiguousarray(gates)
    if g.dtype.itemsize != 96:
        raise ValueError("gate records must be 96-byte sv_gate structs")
    return g


def sv_apply_circuit(h: int, gates: np.ndarray) -> None:
    g = _gate_array(gates)
    _check(load().sv_apply_circuit(h, g.ctypes.data if g.size else None, g.size))


def sv_apply_circuit_graph(h: int, gates: np.ndarray) -> None:
    g = _gate_array(gates)
    _check(load().sv_apply_circuit_graph(h, g.ctypes.data if g.size else None, g.size))


def sv_read_amplitudes(h: int, first: int = 0, count: int | None = None, out: np.ndarray | None = None) -> np.ndarray:
    n, dt, _ = sv_get_info(h)
    if count is None:
        count = (1 << n) - first
    if out is None:
        out = np.empty(count, dtype=_dtype_np(dt))
    _check(load().sv_read_amplitudes(h, first, count, out.ctypes.data))
    return out


def sv_read_amplitudes_at(h: int, idx) -> np.ndarray:
    _, dt, _ = sv_get_info(h)
    ix = np.ascontiguousarray(np.asarray(idx, dtype=np.uint64))
    out = np.empty(ix.size, dtype=_dtype_np(dt))
    _check(load().sv_read_amplitudes_at(h, ix.ctypes.data, ix.size, out.ctypes.data))
    return out


def sv_read_probabilities(h: int, first: int = 0, count: int | None = None) -> np.ndarray:
    n = sv_get_info(h)[0]
    if count is None:
        count = (1 << n) - first
    out = np.empty(count, dtype=np.float64)
    _check(load().sv_read_probabilities(h, first, count, out.ctypes.data))
    return out


def sv_sample(h: int, u) -> np.ndarray:
    """Logical outcome indices for the caller's uniform numbers u (each in [0, 1))."""
    uu = np.ascontiguousarray(np.asarray(u, dtype=np.float64))
    out = np.empty(uu.size, dtype=np.uint64)
    _check(load().sv_sample(h, uu.ctypes.data, uu.size, out.ctypes.data))
    return out


def sv_expect_z(h: int, mask: int) -> float:
    v = ctypes.c_double()
    _check(load().sv_expect_z(h, mask, ctypes.byref(v)))
    return v.value


def sv_norm(h: int) -> float:
    v = ctypes.c_double()
    _check(load().sv_norm(h, ctypes.byref(v)))
    return v.value


def sv_norm_noalloc(psi_ptr: int, n: int, dtype: int, d_out_ptr: int, stream=None) -> None:
    """Queue the norm of the 2^n amplitudes at device address psi_ptr into the double at device address
    d_out_ptr, using only the library's fixed scratch array (no allocation)."""
    _check(load().sv_norm_noalloc(psi_ptr, n, dtype, _stream_ptr(stream), d_out_ptr))


def sv_renormalize(h: int) -> None:
    _check(load().sv_renormalize(h))


def sv_sync(h: int) -> None:
    _check(load().sv_sync(h))


def sv_last_plan_stats(h: int) -> dict:
    v = [ctypes.c_int() for _ in range(6)]
    _check(load().sv_last_plan_stats(h, *[ctypes.byref(x) for x in v]))
    return dict(zip(["passes", "fused_gates", "sweep_gates", "relabels", "remaps", "absorbed"], [x.value for x in v]))


def sv_last_plan_blocks(h: int) -> dict:
    b, g = ctypes.c_int(), ctypes.c_int()
    _check(load().sv_last_plan_blocks(h, ctypes.byref(b), ctypes.byref(g)))
    return {"blocks": b.value, "block_gates": g.value}


def sv_profile_last(h: int, kind: int = 0):
    """(launches, summed device ms) of the last apply call's launches of one kind (0 fused pass, 1 single-gate sweep)."""
    n, ms = ctypes.c_int(), ctypes.c_double()
    _check(load().sv_profile_last(h, kind, ctypes.byref(n), ctypes.byref(ms)))
    return n.value, ms.value


def sv_plan_dry_run(n: int, dtype: int, gates: np.ndarray, chunk_k: int = 0) -> dict:
    """Host-only planner dry run: launches, per-gate launch index and execution order, per-launch bit masks."""
    g = _gate_array(gates)
    ns = ctypes.c_int()
    step = np.full(g.size, -1, dtype=np.int32)
    order = np.full(g.size, -1, dtype=np.int32)
    cap = max(1, g.size + 1)
    qm = np.zeros(cap, dtype=np.uint64)
    perm = np.zeros(n, dtype=np.int32)
    _check(load().sv_plan_dry_run(n, dtype, chunk_k, g.ctypes.data if g.size else None, g.size, ctypes.byref(ns),
                                  step.ctypes.data, order.ctypes.data, qm.ctypes.data, cap, perm.ctypes.data))
    return {"nsteps": ns.value, "step_of_gate": step, "order_of_gate": order, "step_qmask": qm[:ns.value],
            "final_perm": perm}


def sv_run_batch(ns, dtype: int, gate_lists, stream=None, chunk_k=None) -> list:
    """Run circuits as one batch; chunk_k: optional per-circuit chunk sizes (0 = default)."""
    count = len(ns)
    arrs = [_gate_array(g) for g in gate_lists]
    n_arr = np.ascontiguousarray(np.asarray(ns, dtype=np.int32))
    ptrs = (ctypes.c_void_p * count)(*[a.ctypes.data if a.size else None for a in arrs])
    ngs = (ctypes.c_size_t * count)(*[a.size for a in arrs])
    out = (ctypes.c_void_p * count)()
    if chunk_k is None:
        _check(load().sv_run_batch(count, n_arr.ctypes.data, dtype, ptrs, ngs, _stream_ptr(stream), out))
    else:
        k_arr = np.ascontiguousarray(np.asarray(chunk_k, dtype=np.int32))
        _check(load().sv_run_batch_k(count, n_arr.ctypes.data, dtype, ptrs, ngs, k_arr.ctypes.data,
                                     _stream_ptr(stream), out))
    return [out[i] for i in range(count)]


def sv_server_create(hbm_budget_bytes: int, max_active: int) -> int:
    h = ctypes.c_void_p()
    _check(load().sv_server_create(hbm_budget_bytes, max_active, ctypes.byref(h)))
    return h.value


def sv_server_destroy(h: int) -> None:
    _check(load().sv_server_destroy(h))


def sv_submit(srv: int, n: int, dtype: int, gates: np.ndarray) -> int:
    g = _gate_array(gates)
    t = ctypes.c_uint64()
    _check(load().sv_submit(srv, n, dtype, g.ctypes.data if g.size else None, g.size, ctypes.byref(t)))
    return t.value


def sv_poll(srv: int, ticket: int):
    """(done, state handle or None)."""
    d, r = ctypes.c_int(), ctypes.c_void_p()
    _check(load().sv_poll(srv, ticket, ctypes.byref(d), ctypes.byref(r)))
    return bool(d.value), r.value


def sv_last_batch_stats() -> dict:
    """Statistics of this thread's last sv_run_batch call (sv_batch_stats)."""
    v = (ctypes.c_uint64 * len(BATCH_STATS_FIELDS))()
    _check(load().sv_last_batch_stats(ctypes.cast(v, ctypes.c_void_p)))
    return dict(zip(BATCH_STATS_FIELDS, list(v)))


def sv_plan_dry_run_blocks(n: int, dtype: int, gates: np.ndarray, tensor_blocks: int, chunk_k: int = 0) -> dict:
    """Host-only dry run of the dense-block planner: {passes, passes_with_blocks, blocks, block_gates}."""
    g = _gate_array(gates)
    out = [ctypes.c_int() for _ in range(4)]
    _check(load().sv_plan_dry_run_blocks(n, dtype, chunk_k, tensor_blocks, g.ctypes.data if g.size else None, g.size,
                                         *[ctypes.byref(v) for v in out]))
    return dict(zip(("passes", "passes_with_blocks", "blocks", "block_gates"), (v.value for v in out)))


def sv_batch_set_option(option: int, value: int) -> None:
    """Set an option (SV_OPT_TENSOR_BLOCKS) for this thread's later sv_run_batch calls."""
    _check(load().sv_batch_set_option(option, value))


def sv_server_pause(srv: int, paused: bool) -> None:
    _check(load().sv_server_pause(srv, 1 if paused else 0))


def sv_server_get_stats(srv: int) -> dict:
    v = (ctypes.c_uint64 * len(SERVER_STATS_FIELDS))()
    _check(load().sv_server_get_stats(srv, ctypes.cast(v, ctypes.c_void_p)))
    return dict(zip(SERVER_STATS_FIELDS, list(v)))


def sv_last_error() -> str:
    return load().sv_last_error().decode()


def sv_version() -> str:
    return load().sv_version().decode()
