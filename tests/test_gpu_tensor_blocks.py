"""Dense gate blocks on the tensor cores (SV_OPT_TENSOR_BLOCKS): runs of gates on at most four chunk bits
composed on the host into one 16 x 16 unitary (Sec. II.B: a multi-qubit gate acts as a matrix on its
qubits' basis states) and applied to every row of the chunk with tcgen05 MMAs.  Every result is compared
element by element with the FP64 oracle at the complex64 tolerance, and with the per-gate path, over
several chunk sizes, circuit families (random layers, QFT with controlled phases, controlled and two-qubit
gates) and ragged cases (chunks of one tile, states just above the chunk size)."""
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


def run(n, gates, dtype, blocks, chunk_k=0, x0=0, graph=False, arith=B.SV_ARITH_AUTO):
    h = B.sv_create(n, dtype)
    try:
        if dtype == B.SV_C128:
            B.sv_set_option(h, B.SV_OPT_ARITH, arith)
        B.sv_set_option(h, B.SV_OPT_TENSOR_BLOCKS, 1 if blocks else 0)
        if chunk_k:
            B.sv_set_option(h, B.SV_OPT_CHUNK_QUBITS, chunk_k)
        if x0:
            B.sv_init_basis(h, x0)
        (B.sv_apply_circuit_graph if graph else B.sv_apply_circuit)(h, gates)
        st = B.sv_last_plan_blocks(h)
        return B.sv_read_amplitudes(h).astype(np.complex128), st
    finally:
        B.sv_destroy(h)


def mixed_circuit(n, rng, layers=3):
    """Haar U(2) layers with CNOTs, controlled U(2) with 1-2 controls, diagonal phases and dense two-qubit
    gates, on qubits spread over the whole register."""
    g = []
    for _ in range(layers):
        for q in range(n):
            g.append(C.gate_u(C.haar_u2(rng), q))
        perm = rng.permutation(n)
        for i in range(0, n - 1, 2):
            g.append(C.cnot(int(perm[i]), int(perm[i + 1])))
        for _ in range(n // 2):
            t, c1, c2 = (int(x) for x in rng.choice(n, 3, replace=False))
            g.append(C.gate_u(C.haar_u2(rng), t, (c1,) if rng.random() < 0.5 else (c1, c2)))
            g.append(C.gate_u(C.phase(rng.uniform(0, 2 * np.pi)), t, (c1,)))
        for _ in range(max(1, n // 4)):
            a, b = (int(x) for x in rng.choice(n, 2, replace=False))
            g.append(C.gate_u4(C.haar_u4(rng), a, b))
    return C.pack(g)


@pytest.mark.parametrize("n,chunk_k", [(11, 11), (12, 11), (12, 12), (13, 12), (14, 13), (17, 12), (20, 13)])
def test_random_layers_on_tensor_cores_match_oracle(n, chunk_k):
    w = C.random_workload(n, 4, seed=300 + n)
    got, st = run(n, w.gates, B.SV_C64, True, chunk_k)
    assert st["blocks"] > 0 and st["block_gates"] >= 2 * st["blocks"], st
    want = run_oracle(n, w.gates)
    assert_close(got, want, B.SV_C64, f"n={n} k={chunk_k} tensor blocks")
    per_gate, st0 = run(n, w.gates, B.SV_C64, False, chunk_k)
    assert st0["blocks"] == 0
    assert_close(got, per_gate, B.SV_C64, "tensor blocks vs per-gate")


@pytest.mark.parametrize("n,chunk_k", [(12, 12), (15, 11), (18, 13)])
def test_mixed_gate_families_on_tensor_cores(n, chunk_k):
    rng = np.random.Generator(np.random.PCG64(77 + n))
    gates = mixed_circuit(n, rng)
    got, st = run(n, gates, B.SV_C64, True, chunk_k)
    assert st["blocks"] > 0, st
    assert_close(got, run_oracle(n, gates), B.SV_C64, f"mixed n={n}")


def test_qft_then_layers_on_tensor_cores():
    w = C.qft_random_workload(16, 3, seed=5)
    got, st = run(16, w.gates, B.SV_C64, True, 12, x0=w.x0)
    assert st["blocks"] > 0, st
    assert_close(got, run_oracle(16, w.gates, x0=w.x0), B.SV_C64, "qft + layers")


def test_tensor_blocks_in_a_captured_graph_and_deep_circuit():
    n = 22
    w = C.random_workload(n, 12, seed=2024)
    got, st = run(n, w.gates, B.SV_C64, True, 13, graph=True)
    assert st["blocks"] > 0, st
    want = run_oracle(n, w.gates)
    assert_close(got, want, B.SV_C64, "graph, 12 layers, n=22")
    again, _ = run(n, w.gates, B.SV_C64, True, 13, graph=False)
    assert np.array_equal(got, again), "blocks are deterministic and the graph replays the same launches"


def test_tensor_blocks_are_ignored_where_they_do_not_apply():
    # chunks of fewer than 2^11 amplitudes (a 128-row tile), complex128 with native FP64 arithmetic, and
    # complex128 chunks of 2^13 amplitudes keep the per-gate path
    w = C.random_workload(10, 3, seed=9)
    got, st = run(10, w.gates, B.SV_C64, True)
    assert st["blocks"] == 0
    assert_close(got, run_oracle(10, w.gates), B.SV_C64, "n=10")
    w = C.random_workload(14, 2, seed=9)
    got, st = run(14, w.gates, B.SV_C128, True, arith=B.SV_ARITH_F64)
    assert st["blocks"] == 0
    assert_close(got, run_oracle(14, w.gates), B.SV_C128, "n=14 FP64")
    got, st = run(14, w.gates, B.SV_C128, True, chunk_k=13)
    assert st["blocks"] == 0


def test_passes_where_blocks_take_little_of_the_work_keep_the_per_gate_path():
    # A pass keeps its blocks only if they take at least 3/4 of its per-gate work.  A CNOT and four dense gates
    # on chunk bits 0-3 form a block (the CNOT first, so that the dense gates are not folded into a product
    # start); twenty gates controlled by a qubit outside the chunk cannot join one, so with them the pass stays
    # per-gate, and without them it runs the block.
    rng = np.random.Generator(np.random.PCG64(23))
    lead = [C.cnot(0, 1)] + [C.gate_u(C.haar_u2(rng), q) for q in range(4)]
    tail = [C.gate_u(C.haar_u2(rng), 4 + i % 8, (15,)) for i in range(20)]
    for dtype in (B.SV_C128, B.SV_C64):
        gates = C.pack(lead + tail)
        got, st = run(16, gates, dtype, True, 12)
        assert st["blocks"] == 0, st
        assert_close(got, run_oracle(16, gates), dtype, "per-gate pass, blocks on")
        gates = C.pack(lead)
        got, st = run(16, gates, dtype, True, 12)
        assert st["blocks"] == 1, st
        assert_close(got, run_oracle(16, gates), dtype, "one block")


# ---- complex128: exact digit products ------------------------------------------------------------------

@pytest.mark.parametrize("n,chunk_k", [(11, 11), (12, 11), (12, 12), (13, 12), (15, 11), (17, 12), (20, 12)])
def test_c128_random_layers_on_tensor_cores_match_oracle(n, chunk_k):
    w = C.random_workload(n, 4, seed=600 + n)
    got, st = run(n, w.gates, B.SV_C128, True, chunk_k)
    assert st["blocks"] > 0 and st["block_gates"] >= 2 * st["blocks"], st
    want = run_oracle(n, w.gates)
    assert_close(got, want, B.SV_C128, f"c128 n={n} k={chunk_k} tensor blocks")
    per_gate, _ = run(n, w.gates, B.SV_C128, False, chunk_k)
    assert_close(got, per_gate, B.SV_C128, "c128 tensor blocks vs double-float per gate")


@pytest.mark.parametrize("n,chunk_k", [(12, 12), (16, 11), (18, 12)])
def test_c128_mixed_gate_families_on_tensor_cores(n, chunk_k):
    rng = np.random.Generator(np.random.PCG64(177 + n))
    gates = mixed_circuit(n, rng)
    got, st = run(n, gates, B.SV_C128, True, chunk_k)
    assert st["blocks"] > 0, st
    assert_close(got, run_oracle(n, gates), B.SV_C128, f"c128 mixed n={n}")


def test_c128_qft_and_deep_circuit_on_tensor_cores():
    w = C.qft_random_workload(16, 3, seed=15)
    got, st = run(16, w.gates, B.SV_C128, True, 12, x0=w.x0)
    assert st["blocks"] > 0, st
    assert_close(got, run_oracle(16, w.gates, x0=w.x0), B.SV_C128, "c128 qft + layers")
    n = 22
    w = C.random_workload(n, 12, seed=2025)
    got, st = run(n, w.gates, B.SV_C128, True, 12, graph=True)
    assert st["blocks"] > 0, st
    assert_close(got, run_oracle(n, w.gates), B.SV_C128, "c128 graph, 12 layers, n=22")
    again, _ = run(n, w.gates, B.SV_C128, True, 12)
    assert np.array_equal(got, again)


def test_c128_tensor_blocks_on_small_and_unnormalised_states():
    # a whole-state chunk (n = k = 11, 2-norm 1) through many blocks, and a state scaled far from norm 1
    n = 11
    w = C.random_workload(n, 30, seed=7)
    got, st = run(n, w.gates, B.SV_C128, True, 11)
    assert st["blocks"] > 20, st
    assert_close(got, run_oracle(n, w.gates), B.SV_C128, "c128 n=11, 30 layers")
    psi0 = C.random_state(12, seed=8) * 2.0 ** -40
    h = B.sv_create(12, B.SV_C128)
    try:
        B.sv_set_option(h, B.SV_OPT_TENSOR_BLOCKS, 1)
        B.sv_write_amplitudes(h, 0, psi0)
        g = C.random_workload(12, 3, seed=10).gates
        B.sv_apply_circuit(h, g)
        got = B.sv_read_amplitudes(h)
    finally:
        B.sv_destroy(h)
    want = run_oracle(12, g, psi0)
    assert np.max(np.abs(got - want)) <= 1e-12 * 2.0 ** -40
    # and scaled up: a chunk norm of 2^110 (the chunk exponent must not stop below it)
    psi1 = C.random_state(12, seed=9) * 2.0 ** 110
    h = B.sv_create(12, B.SV_C128)
    try:
        B.sv_set_option(h, B.SV_OPT_TENSOR_BLOCKS, 1)
        B.sv_write_amplitudes(h, 0, psi1)
        B.sv_apply_circuit(h, g)
        got = B.sv_read_amplitudes(h)
        assert B.sv_last_plan_blocks(h)["blocks"] > 0
    finally:
        B.sv_destroy(h)
    want = run_oracle(12, g, psi1)
    assert np.max(np.abs(got - want)) <= 1e-12 * 2.0 ** 110
