"""Product-state start (Sec. V: a state without entanglement is the Kronecker product of one-qubit states).

sv_init_product forms the amplitudes on the GPU; while a state is still a product state, the apply calls fold
leading single-qubit gates and SWAPs into the qubits' factors and run only the rest.  Everything is compared
with the FP64 oracle (oracle.product_state, then the circuit through the pair update)."""
import numpy as np
import pytest

import circuits as C
import oracle
from gpu_helpers import MODES, MODE_IDS, assert_close, make_state, run_oracle

pytestmark = pytest.mark.gpu
B = pytest.importorskip("paper_1801_01037_gb300")._binding


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1801_01037_gb300 import build
    build.build()
    B.load()


def random_factors(n, seed):
    rng = np.random.default_rng(seed)
    return [C.haar_u2(rng)[:, 0] for _ in range(n)]


def expected(dtype, psi):
    return psi.astype(np.complex64).astype(np.complex128) if dtype == B.SV_C64 else psi


@pytest.mark.parametrize("mode", MODES, ids=MODE_IDS)
@pytest.mark.parametrize("n", [1, 2, 7, 16, 21])
def test_init_product_matches_oracle(mode, n):
    _, dtype, arith = mode
    f = random_factors(n, 40 + n)
    h = make_state(n, dtype, arith)
    try:
        B.sv_init_product(h, f)
        got = B.sv_read_amplitudes(h).astype(np.complex128)
        assert_close(got, oracle.product_state(f), dtype, "product state")
        assert abs(B.sv_norm(h) - 1.0) < (1e-13 if dtype == B.SV_C128 else 1e-5)
    finally:
        B.sv_destroy(h)


@pytest.mark.parametrize("mode", MODES, ids=MODE_IDS)
@pytest.mark.parametrize("graph", [False, True], ids=["direct", "graph"])
def test_leading_gates_fold_into_the_product_start(mode, graph):
    """Random layers from a product state: the first layer's n single-qubit gates are folded into the factors
    (not planned), the rest runs on the GPU; the result matches the oracle applying every gate in order."""
    _, dtype, arith = mode
    n = 18
    f = random_factors(n, 7)
    w = C.random_workload(n, 3, seed=70).gates
    want = run_oracle(n, w, oracle.product_state(f))
    h = make_state(n, dtype, arith)
    try:
        for rep in range(2):
            B.sv_init_product(h, f)
            (B.sv_apply_circuit_graph if graph else B.sv_apply_circuit)(h, w)
            st = B.sv_last_plan_stats(h)
            assert st["absorbed"] == n
            assert st["fused_gates"] + st["sweep_gates"] == len(w) - n
            assert_close(B.sv_read_amplitudes(h).astype(np.complex128), want, dtype, f"rep {rep}")
    finally:
        B.sv_destroy(h)


@pytest.mark.parametrize("mode", MODES, ids=MODE_IDS)
def test_product_start_ends_at_the_first_entangling_gate(mode):
    """Calls in sequence: single-qubit gates and a SWAP are folded while no gate has entangled the qubits;
    after a CNOT the state is general and later single-qubit gates run as kernels."""
    _, dtype, arith = mode
    n = 12
    rng = np.random.default_rng(3)
    u = [C.haar_u2(rng) for _ in range(4)]
    calls = [
        [C.gate_u(u[0], 0), C.gate_swap(0, 5), C.gate_u(u[1], 5)],   # all folded
        [C.gate_u(u[2], 3), C.gate_u(u[3], 4), C.cnot(3, 7), C.gate_u(u[3], 9), C.gate_u(u[2], 3)],
        # U(3), U(4), U(9) fold (3 >= n/4); the CNOT and the U(3) after it remain
        [C.gate_u(u[1], 9), C.gate_u(u[0], 2)],                      # general state now: nothing folded
    ]
    folded = [3, 3, 0]
    psi = oracle.basis_state(n, 0b100000000001)
    h = make_state(n, dtype, arith, x0=0b100000000001)
    try:
        for call, nf in zip(calls, folded):
            w = C.pack(call)
            B.sv_apply_circuit(h, w)
            assert B.sv_last_plan_stats(h)["absorbed"] == nf
            psi = oracle.apply_circuit(psi, w)
            assert_close(B.sv_read_amplitudes(h).astype(np.complex128), psi, dtype, str(call))
    finally:
        B.sv_destroy(h)


def test_product_start_of_a_single_gate_and_of_controls():
    """sv_apply_gate on a fresh state folds; a controlled gate on untouched qubits is not folded; a call whose
    foldable gates are too few to pay for re-forming the state (1 < max(2, n/4)) runs them all as kernels."""
    n = 9
    h = B.sv_create(n, B.SV_C128)
    try:
        B.sv_apply_gate(h, C.H, 4)
        assert B.sv_last_plan_stats(h)["absorbed"] == 1
        B.sv_apply_gate(h, C.X, 2, [4])
        assert B.sv_last_plan_stats(h)["absorbed"] == 0
        want = run_oracle(n, C.pack([C.gate_u(C.H, 4), C.cnot(4, 2)]))
        assert_close(B.sv_read_amplitudes(h), want, B.SV_C128, "H then CNOT")
        w = C.pack([C.gate_u(C.H, 0), C.cnot(0, 1)])
        B.sv_init_basis(h, 3)
        B.sv_apply_circuit(h, w)
        assert B.sv_last_plan_stats(h)["absorbed"] == 0
        assert_close(B.sv_read_amplitudes(h), run_oracle(n, w, x0=3), B.SV_C128, "H(0) CNOT from |3>")
        B.sv_init_basis(h, 3)
        B.sv_set_option(h, B.SV_OPT_PRODUCT_START, 0)
        B.sv_apply_gate(h, C.H, 4)
        assert B.sv_last_plan_stats(h)["absorbed"] == 0
    finally:
        B.sv_destroy(h)


def test_init_product_rejects_bad_factors():
    h = B.sv_create(3, B.SV_C128)
    try:
        with pytest.raises(B.SvError) as e:
            B.sv_init_product(h, [(1, 0), (0.6, 0.6), (0, 1)])
        assert e.value.code == B.SV_ERR_ARG and "normalised" in str(e.value)
        with pytest.raises(B.SvError) as e:
            B.sv_init_product(h, [(1, 0), (np.nan, 0), (0, 1)])
        assert e.value.code == B.SV_ERR_ARG
        # the state is untouched (still |0>)
        assert B.sv_read_amplitudes(h)[0] == 1
    finally:
        B.sv_destroy(h)
