"""Full-size checks at the benchmark's sizes and launch configuration (default options of sv_apply_circuit),
where the oracle cannot run: properties that hold at any size.

* n = 30, 20 random layers (seed 1002), complex128 and complex64: the circuit followed by its inverse
  returns |0...0>, and the norm stays 1 after the forward circuit.
* n = 30 QFT of a seeded basis state: sampled amplitudes equal the closed form e^{2 pi i x y / 2^n} / 2^{n/2}.
* n = 33 complex128 (128 GiB): QFT of |x>, then 10 random layers and their inverse, equals the QFT closed
  form at sampled indices.
"""
import numpy as np
import pytest

import circuits as C
from gpu_helpers import C128_ABS

pytestmark = pytest.mark.gpu
B = pytest.importorskip("paper_1801_01037_gb300")._binding


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1801_01037_gb300 import build
    build.build()
    B.load()


def free_bytes():
    import torch
    f, _ = torch.cuda.mem_get_info()
    return f


def qft_closed(n, x, y):
    y = np.asarray(y, dtype=np.uint64)
    ph = ((np.uint64(x) * y) & np.uint64(2 ** n - 1)).astype(np.float64) / 2.0 ** n
    return np.exp(2j * np.pi * ph) / 2.0 ** (n / 2)


@pytest.mark.parametrize("dtype", [B.SV_C128, B.SV_C64], ids=["c128", "c64"])
def test_n30_random_circuit_then_inverse_is_identity(dtype):
    w = C.random_workload(30, 20, seed=1002)
    h = B.sv_create(30, dtype)
    try:
        B.sv_apply_circuit(h, w.gates)
        nrm = B.sv_norm(h)
        assert abs(nrm - 1.0) < (1e-12 if dtype == B.SV_C128 else 1e-5)
        B.sv_apply_circuit(h, C.inverse(w.gates))
        head = B.sv_read_amplitudes(h, 0, 1 << 16).astype(np.complex128)
        idx = np.random.default_rng(3).integers(1, 2 ** 30, 1 << 16)
        rest = B.sv_read_amplitudes_at(h, idx).astype(np.complex128)
        tol = C128_ABS if dtype == B.SV_C128 else 1e-4
        assert abs(head[0] - 1.0) <= tol
        assert np.max(np.abs(head[1:])) <= tol and np.max(np.abs(rest)) <= tol
    finally:
        B.sv_destroy(h)


def test_n30_qft_closed_form_sampled():
    w = C.qft_workload(30, seed=1002)
    h = B.sv_create(30, B.SV_C128)
    try:
        B.sv_init_basis(h, w.x0)
        B.sv_apply_circuit(h, w.gates)
        idx = np.concatenate([np.arange(4096), np.random.default_rng(5).integers(0, 2 ** 30, 1 << 16)])
        got = B.sv_read_amplitudes_at(h, idx)
        assert np.max(np.abs(got - qft_closed(30, w.x0, idx))) <= C128_ABS
    finally:
        B.sv_destroy(h)


def test_n33_qft_random_layers_and_inverse():
    if free_bytes() < (16 << 33) + (4 << 30):
        pytest.skip("needs 132 GiB of free device memory")
    rng = np.random.Generator(np.random.PCG64(1003))
    x = int(rng.integers(0, 2 ** 33))
    layers = C.pack(C.random_layers(33, 10, rng))
    h = B.sv_create(33, B.SV_C128)
    try:
        B.sv_init_basis(h, x)
        B.sv_apply_circuit(h, C.pack(C.qft(33)))
        B.sv_apply_circuit(h, layers)
        assert abs(B.sv_norm(h) - 1.0) < 1e-12
        B.sv_apply_circuit(h, C.inverse(layers))
        idx = np.random.default_rng(6).integers(0, 2 ** 33, 1 << 15)
        got = B.sv_read_amplitudes_at(h, idx)
        assert np.max(np.abs(got - qft_closed(33, x, idx))) <= C128_ABS
    finally:
        B.sv_destroy(h)
