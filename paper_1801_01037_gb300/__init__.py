"""GB300 state-vector simulator: Python binding of the C ABI in ``include/sv.h``.

The library stores the 2^n amplitudes of an n-qubit state in HBM and applies (controlled) single-qubit gates
with hand-written sm_103a kernels: the strided pair update of LaRose, arXiv:1801.01037, Sec. V.A, fused over
chunks of 2^k amplitudes, with the paper's qubit relabelling (Sec. VI.B) kept as a layout map.

>>> from paper_1801_01037_gb300 import State, SV_C128
>>> s = State(20, SV_C128)
>>> s.apply_circuit(gates)          # packed 96-byte sv_gate records (see ``circuits``)
>>> amps = s.read_amplitudes(0, 16)
"""
from __future__ import annotations

from ._binding import *  # noqa: F401,F403
from ._binding import (SV_C64, SV_C128, SV_OPT_ARITH, SV_OPT_CANONICAL, SV_OPT_CHUNK_QUBITS, SV_OPT_FUSION,
                       SV_OPT_RENORM_PERIOD, SvError, load)
from . import _binding as _b


class State:
    """Owning wrapper around an ``sv_state`` handle."""

    def __init__(self, n: int, dtype: int = SV_C128, stream=None, handle: int | None = None):
        self.h = handle if handle is not None else _b.sv_create(n, dtype, stream)
        self.n, self.dtype, _ = _b.sv_get_info(self.h)

    @classmethod
    def from_buffer(cls, n: int, dtype: int, dev_ptr: int, stream=None) -> "State":
        return cls(n, dtype, handle=_b.sv_create_from_buffer(n, dtype, dev_ptr, stream))

    def close(self):
        if self.h:
            _b.sv_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # gates
    def init_basis(self, x: int = 0):
        _b.sv_init_basis(self.h, x)

    def apply_gate(self, u, target: int, controls=()):
        _b.sv_apply_gate(self.h, u, target, controls)

    def apply_swap(self, a: int, b: int):
        _b.sv_apply_swap(self.h, a, b)

    def apply_circuit(self, gates, graph: bool = False):
        (_b.sv_apply_circuit_graph if graph else _b.sv_apply_circuit)(self.h, gates)

    def set_option(self, option: int, value: int):
        _b.sv_set_option(self.h, option, value)

    # read-out
    def read_amplitudes(self, first: int = 0, count: int | None = None):
        return _b.sv_read_amplitudes(self.h, first, count)

    def read_amplitudes_at(self, idx):
        return _b.sv_read_amplitudes_at(self.h, idx)

    def read_probabilities(self, first: int = 0, count: int | None = None):
        return _b.sv_read_probabilities(self.h, first, count)

    def write_amplitudes(self, first: int, values):
        _b.sv_write_amplitudes(self.h, first, values)

    def norm(self) -> float:
        return _b.sv_norm(self.h)

    def renormalize(self):
        _b.sv_renormalize(self.h)

    def layout(self):
        return _b.sv_get_layout(self.h)

    def canonicalize(self):
        _b.sv_canonicalize(self.h)

    def sync(self):
        _b.sv_sync(self.h)

    def plan_stats(self) -> dict:
        return _b.sv_last_plan_stats(self.h)
