"""Dense two-qubit gates (a 4x4 unitary on two qubits, Sec. II.B's multi-qubit gates) on the GPU against the
FP64 oracle: every arithmetic mode, near and far qubit pairs in both orders, controls inside and outside the
chunk, SWAP relabelling before the gate, the single-call entry point, graphs, the batched path and the
complex64 register cubes next to them."""
import numpy as np
import pytest

import circuits as C
import oracle
from gpu_helpers import MODES, MODE_IDS, assert_close, make_state, run_gpu, run_oracle

pytestmark = pytest.mark.gpu
B = pytest.importorskip("paper_1801_01037_gb300")._binding


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1801_01037_gb300 import build
    build.build()
    B.load()


def two_qubit_circuit(n, rng, layers=3):
    gates = []
    for layer in range(layers):
        for q in range(0, n - 1, 2):
            if layer % 2 == 0:
                a, b = q, q + 1
            else:
                a, b = q + 1, (q + 1 + n // 2) % n
                if a == b:
                    b = (a + 1) % n
            ctl = ()
            if q % 6 == 4:
                c0 = (b + 2) % n
                if c0 not in (a, b):
                    ctl = (c0,)
            gates.append(C.gate_u4(C.haar_u4(rng), a, b, ctl))
        gates.append(C.gate_u(C.haar_u2(rng), layer % n))
        if n > 2:
            gates.append(C.cnot(layer % n, n - 1 - layer % n) if layer % n != n - 1 - layer % n else C.gate_u(C.H, 0))
            gates.append(C.gate_swap(0, n - 2))
    return C.pack(gates)


@pytest.mark.parametrize("mode", MODES, ids=MODE_IDS)
@pytest.mark.parametrize("n,chunk_k", [(2, 0), (5, 0), (12, 0), (16, 0), (16, 8), (19, 0)])
def test_two_qubit_circuits_match_oracle(mode, n, chunk_k):
    _, dtype, arith = mode
    w = two_qubit_circuit(n, np.random.default_rng(500 + n + chunk_k))
    psi0 = C.random_state(n, seed=n + 3)
    if dtype == B.SV_C64:
        psi0 = psi0.astype(np.complex64).astype(np.complex128)
    want = run_oracle(n, w, psi0)
    got = run_gpu(n, w, dtype, arith, psi0=psi0, chunk_k=chunk_k)
    assert_close(got, want, dtype, f"n={n} k={chunk_k}")
    got_graph = run_gpu(n, w, dtype, arith, psi0=psi0, chunk_k=chunk_k, graph=True)
    assert np.array_equal(got_graph, got)


@pytest.mark.parametrize("mode", MODES, ids=MODE_IDS)
def test_single_two_qubit_gate_calls(mode):
    """sv_apply_gate2q (one gate per call, its own pass) on every ordered pair of a few qubits, with and
    without controls; the Kronecker gate A (x) B agrees with B on q0 then A on q1."""
    _, dtype, arith = mode
    n = 14
    rng = np.random.default_rng(8)
    psi0 = C.random_state(n, seed=4)
    if dtype == B.SV_C64:
        psi0 = psi0.astype(np.complex64).astype(np.complex128)
    want = psi0.copy()
    h = make_state(n, dtype, arith, psi0=psi0)
    try:
        B.sv_set_option(h, B.SV_OPT_PRODUCT_START, 0)
        for q0, q1, ctl in [(0, 1, ()), (1, 0, ()), (3, 13, ()), (13, 2, (5,)), (7, 12, (0, 11)), (4, 5, (13,))]:
            v = C.haar_u4(rng)
            B.sv_apply_gate2q(h, v, q0, q1, ctl)
            oracle.apply_gate4(want, v, q0, q1, ctl)
        a, b = C.haar_u2(rng), C.haar_u2(rng)
        B.sv_apply_gate2q(h, np.kron(a, b), 6, 9)
        oracle.apply_gate(oracle.apply_gate(want, b, 6), a, 9)
        assert_close(B.sv_read_amplitudes(h).astype(np.complex128), want, dtype, "single calls")
    finally:
        B.sv_destroy(h)


@pytest.mark.parametrize("mode", [m for m in MODES if m[0] != "c128_df32"], ids=["c128_f64", "c64"])
def test_paper_cnot_matrix_is_an_exact_move(mode):
    """The CNOT matrix of Sec. II.B as a dense two-qubit gate moves amplitudes exactly (FP64 and FP32
    arithmetic: products by 1 and 0), like the controlled X."""
    _, dtype, arith = mode
    v = np.zeros((4, 4))
    v[0, 0] = v[1, 1] = v[2, 3] = v[3, 2] = 1.0  # |b1 b0>: b1 = control (index bit 1 of the gate)
    n = 13
    psi0 = C.random_state(n, seed=21)
    if dtype == B.SV_C64:
        psi0 = psi0.astype(np.complex64).astype(np.complex128)
    w = C.pack([C.gate_u4(v, 3, 11), C.gate_u4(v, 12, 0, (5,))])
    want = run_oracle(n, C.pack([C.cnot(11, 3), C.gate_u(C.X, 12, (0, 5))]), psi0)
    got = run_gpu(n, w, dtype, arith, psi0=psi0)
    assert np.array_equal(got, want)


def test_c64_cubes_identical_with_two_qubit_gates():
    """Two-qubit gates sit outside the complex64 register cubes: results with and without cubes are identical."""
    n = 17
    w = two_qubit_circuit(n, np.random.default_rng(31), layers=4)
    psi0 = C.random_state(n, seed=2).astype(np.complex64).astype(np.complex128)
    outs = []
    for cubes in (0, 1):
        h = make_state(n, B.SV_C64, B.SV_ARITH_AUTO, psi0=psi0)
        try:
            B.sv_set_option(h, B.SV_OPT_CUBES, cubes)
            B.sv_apply_circuit(h, w)
            outs.append(B.sv_read_amplitudes(h))
        finally:
            B.sv_destroy(h)
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("dtype", [B.SV_C128, B.SV_C64], ids=["c128", "c64"])
def test_batch_with_two_qubit_gates(dtype):
    rng = np.random.default_rng(77)
    ns = [3, 9, 14, 6]
    lists = [two_qubit_circuit(n, rng) for n in ns]
    handles = B.sv_run_batch(ns, dtype, lists)
    try:
        for n, w, h in zip(ns, lists, handles):
            got = B.sv_read_amplitudes(h).astype(np.complex128)
            assert_close(got, run_oracle(n, w), dtype, f"batch n={n}")
    finally:
        for h in handles:
            B.sv_destroy(h)


def test_two_qubit_gate_is_never_folded_into_a_product_state():
    n = 8
    rng = np.random.default_rng(5)
    w = C.pack([C.gate_u(C.haar_u2(rng), 0), C.gate_u4(C.haar_u4(rng), 1, 2), C.gate_u(C.haar_u2(rng), 3)])
    h = B.sv_create(n, B.SV_C128)
    try:
        B.sv_apply_circuit(h, w)
        assert B.sv_last_plan_stats(h)["absorbed"] == 2
        assert_close(B.sv_read_amplitudes(h), run_oracle(n, w), B.SV_C128, "product start + two-qubit gate")
    finally:
        B.sv_destroy(h)


@pytest.mark.parametrize("mode", MODES, ids=MODE_IDS)
@pytest.mark.parametrize("n,chunk_k", [(6, 0), (7, 6), (9, 6), (15, 7)])
def test_two_qubit_gates_at_small_chunks_and_four_controls(mode, n, chunk_k):
    """Smallest chunks (k = 6, so the contiguous rows shrink to leave room for both bits), states no larger
    than a chunk, and the maximum of four controls next to the two targets."""
    _, dtype, arith = mode
    rng = np.random.default_rng(40 + n + chunk_k)
    gates = []
    for _ in range(6):
        q = rng.choice(n, 6, replace=False)
        gates.append(C.gate_u4(C.haar_u4(rng), int(q[0]), int(q[1]), tuple(int(c) for c in q[2:6])))
        gates.append(C.gate_u4(C.haar_u4(rng), int(q[1]), int(q[0])))
        gates.append(C.gate_u(C.haar_u2(rng), int(q[2]), (int(q[3]),)))
        gates.append(C.gate_swap(int(q[4]), int(q[5])))
    w = C.pack(gates)
    psi0 = C.random_state(n, seed=3 * n)
    if dtype == B.SV_C64:
        psi0 = psi0.astype(np.complex64).astype(np.complex128)
    want = run_oracle(n, w, psi0)
    assert_close(run_gpu(n, w, dtype, arith, psi0=psi0, chunk_k=chunk_k), want, dtype, f"n={n} k={chunk_k}")


def test_two_qubit_gates_on_a_buffer_state_end_in_logical_order():
    """A caller-owned buffer (always in logical order) after two-qubit gates and SWAP relabels."""
    torch = pytest.importorskip("torch")
    n = 16
    rng = np.random.default_rng(61)
    w = two_qubit_circuit(n, rng)
    psi0 = C.random_state(n, seed=8)
    t = torch.from_numpy(psi0).to("cuda")
    torch.cuda.synchronize()
    h = B.sv_create_from_buffer(n, B.SV_C128, t.data_ptr())
    try:
        B.sv_apply_circuit(h, w)
        B.sv_sync(h)
        assert list(B.sv_get_layout(h)) == list(range(n))
        assert_close(t.cpu().numpy(), run_oracle(n, w, psi0), B.SV_C128, "buffer state")
    finally:
        B.sv_destroy(h)
