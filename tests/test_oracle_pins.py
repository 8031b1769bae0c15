"""Pins for the FP64 CPU oracle against facts fixed by the paper and by the mathematics, not by the oracle.

* Brute force: the dense 2^n x 2^n operator of Sec. II.A (Kronecker product of the per-qubit gates,
  Eq. tensor-product-gates) and of Sec. V.A (I x .. x Q_i x .. x I), built with numpy's ``kron`` and
  multiplied onto the state, for n <= 7, every target and random control sets.
* The paper's worked examples (fixtures under tests/golden/, each citing its passage).
* Closed forms: QFT of a basis state, uniform state from H on every qubit, GHZ, circuit x inverse.
"""
import math

import numpy as np
import pytest

import circuits as C
import oracle
from conftest import golden_lines

RNG = np.random.Generator(np.random.PCG64(20240601))


# ----------------------------------------------------------------------------------------------------------------
# Dense Kronecker operator (the "direct approach" of Sec. IV applied to one gate): built independently of the
# pair loop.  Little-endian reading: the leftmost Kronecker factor belongs to the highest qubit.
# ----------------------------------------------------------------------------------------------------------------
P0 = np.array([[1, 0], [0, 0]], dtype=np.complex128)
P1 = np.array([[0, 0], [0, 1]], dtype=np.complex128)


def kron_chain(factors_by_qubit):
    """factors_by_qubit[q] is the 2x2 factor on qubit q; returns kron(f[n-1], ..., f[0])."""
    out = np.array([[1.0 + 0j]])
    for f in reversed(factors_by_qubit):
        out = np.kron(out, f)
    return out


def dense_gate(n, u, target, controls=()):
    """I - P_ctl (x) I_t + P_ctl (x) Q_t, with P_ctl the projector onto 'every control bit is 1'."""
    ident = [C.I2] * n
    full = kron_chain(ident)
    if controls:
        proj = [P1 if q in controls else C.I2 for q in range(n)]
        proj_u = [P1 if q in controls else (u if q == target else C.I2) for q in range(n)]
        return full - kron_chain(proj) + kron_chain(proj_u)
    return kron_chain([u if q == target else C.I2 for q in range(n)])


def dense_swap(n, a, b):
    """SWAP = CNOT(a->b) CNOT(b->a) CNOT(a->b), each as a dense operator."""
    c_ab = dense_gate(n, C.X, b, (a,))
    c_ba = dense_gate(n, C.X, a, (b,))
    return c_ab @ c_ba @ c_ab


def dense_gate4(n, v, q0, q1, controls=()):
    """The 2^n x 2^n operator of a (controlled) two-qubit gate written out element by element from its
    definition (Sec. II.B: a 4x4 matrix on the four basis states of its qubits): <i|O|j> = v[r(i), r(j)] with
    r(k) = b0 + 2 b1 the gate's bits of k, when i and j agree outside q0 and q1 and every control bit of j is 1;
    the identity on the other columns."""
    dim = 2 ** n
    m = (1 << q0) | (1 << q1)
    cm = sum(1 << c for c in controls)
    sub = lambda k: ((k >> q0) & 1) + 2 * ((k >> q1) & 1)
    op = np.zeros((dim, dim), dtype=np.complex128)
    for j in range(dim):
        if (j & cm) != cm:
            op[j, j] = 1.0
            continue
        for i in range(dim):
            if (i & ~m) == (j & ~m):
                op[i, j] = v[sub(i), sub(j)]
    return op


def rand_state(n):
    v = RNG.standard_normal(2 ** n) + 1j * RNG.standard_normal(2 ** n)
    return v / np.linalg.norm(v)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 7])
def test_uncontrolled_gate_matches_kronecker_operator(n):
    for t in range(n):
        u = C.haar_u2(RNG)
        psi = rand_state(n)
        want = dense_gate(n, u, t) @ psi
        got = oracle.apply_gate(psi.copy(), u, t)
        assert np.max(np.abs(got - want)) < 1e-14


@pytest.mark.parametrize("n", [2, 3, 5, 7])
def test_controlled_gate_matches_kronecker_operator(n):
    for _ in range(12):
        t = int(RNG.integers(n))
        others = [q for q in range(n) if q != t]
        m = int(RNG.integers(1, min(4, n - 1) + 1))
        ctl = tuple(int(c) for c in RNG.choice(others, size=m, replace=False))
        u = C.haar_u2(RNG)
        psi = rand_state(n)
        want = dense_gate(n, u, t, ctl) @ psi
        got = oracle.apply_gate(psi.copy(), u, t, ctl)
        assert np.max(np.abs(got - want)) < 1e-14, (t, ctl)


@pytest.mark.parametrize("n", [2, 3, 6])
def test_swap_matches_three_cnots(n):
    for a in range(n):
        for b in range(n):
            if a == b:
                continue
            psi = rand_state(n)
            want = dense_swap(n, a, b) @ psi
            got = oracle.apply_swap(psi.copy(), a, b)
            assert np.array_equal(got, want)  # pure moves: bit-exact


def test_circuit_is_product_of_gate_operators():
    """A circuit is its gates applied in order (Sec. II.B): compare with the product of dense operators."""
    n = 5
    gates = C.random_layers(n, 3, RNG) + [C.gate_swap(0, 3), C.gate_u(C.haar_u2(RNG), 2, (0, 4))]
    psi = rand_state(n)
    want = psi.copy()
    for g in gates:
        op = dense_swap(n, g.target, g.target2) if g.kind == C.GATE_SWAP else dense_gate(n, g.u, g.target, g.controls)
        want = op @ want
    got = oracle.apply_circuit(psi.copy(), C.pack(gates))
    assert np.max(np.abs(got - want)) < 1e-13


# ----------------------------------------------------------------------------------------------------------------
# The paper's worked examples
# ----------------------------------------------------------------------------------------------------------------
def test_pauli_x_and_hadamard_actions():
    s = C.SQRT1_2
    val = {"0": 0.0, "1": 1.0, "s": s, "-s": -s}
    for gate, x, *amps in golden_lines("pauli_x_hadamard.txt"):
        u = C.X if gate == "X" else C.H
        got = oracle.apply_gate(oracle.basis_state(1, int(x)), u, 0)
        want = np.array([val[amps[0]] + 1j * val[amps[1]], val[amps[2]] + 1j * val[amps[3]]])
        assert np.array_equal(got, want)


def test_cnot_truth_table():
    for ket_in, ket_out in golden_lines("cnot_truth_table.txt"):
        x_in, x_out = int(ket_in, 2), int(ket_out, 2)
        got = oracle.apply_gate(oracle.basis_state(2, x_in), C.X, 0, (1,))
        assert np.array_equal(got, oracle.basis_state(2, x_out))


def test_pair_strides_n3():
    """X on qubit i sends |k> to its partner: the pairs of Fig. 'statevector' (stride 2^i)."""
    for row in golden_lines("pair_strides_n3.txt"):
        q = int(row[0].rstrip(":"))
        for pair in row[1:]:
            a, b = (int(v) for v in pair.split("-"))
            assert np.array_equal(oracle.apply_gate(oracle.basis_state(3, a), C.X, q), oracle.basis_state(3, b))
            assert np.array_equal(oracle.apply_gate(oracle.basis_state(3, b), C.X, q), oracle.basis_state(3, a))


def test_tensor_product_two_qubits():
    """Preparing qubit 1 in psi0 and qubit 0 in psi1 gives Eq. tensor-product-2qubit-example."""
    u0, u1 = C.haar_u2(RNG), C.haar_u2(RNG)
    a0, b0 = u0[:, 0]
    a1, b1 = u1[:, 0]
    f = {"a0": a0, "b0": b0, "a1": a1, "b1": b1}
    psi = oracle.basis_state(2, 0)
    oracle.apply_gate(psi, u0, 1)
    oracle.apply_gate(psi, u1, 0)
    for idx, left, right in golden_lines("tensor_product_2q.txt"):
        assert abs(psi[int(idx)] - f[left] * f[right]) < 1e-15


def test_product_state_matches_paper_two_qubit_example():
    """oracle.product_state against the same worked example: qubit 1 in (a0, b0), qubit 0 in (a1, b1)."""
    u0, u1 = C.haar_u2(RNG), C.haar_u2(RNG)
    a0, b0 = u0[:, 0]
    a1, b1 = u1[:, 0]
    f = {"a0": a0, "b0": b0, "a1": a1, "b1": b1}
    psi = oracle.product_state([(a1, b1), (a0, b0)])
    for idx, left, right in golden_lines("tensor_product_2q.txt"):
        assert abs(psi[int(idx)] - f[left] * f[right]) < 1e-15


@pytest.mark.parametrize("n", [1, 3, 6, 9])
def test_product_state_equals_one_qubit_preparations(n):
    """Sec. V: the product state equals |0...0> after a one-qubit preparation unitary on each qubit (the pair
    update of Algorithm 1, an independent route), and its norm is the product of the factors' norms (1)."""
    us = [C.haar_u2(RNG) for _ in range(n)]
    want = oracle.basis_state(n, 0)
    for t, u in enumerate(us):
        oracle.apply_gate(want, u, t)
    got = oracle.product_state([u[:, 0] for u in us])
    assert np.max(np.abs(got - want)) < 1e-14
    assert abs(oracle.norm2(got) - 1.0) < 1e-14
    # amplitude k is the product of the per-qubit entries selected by the bits of k (qubit 0 = bit 0)
    for k in RNG.integers(0, 2 ** n, 8):
        p = 1.0 + 0j
        for t in range(n):
            p *= us[t][(int(k) >> t) & 1, 0]
        assert abs(got[int(k)] - p) < 1e-15


@pytest.mark.parametrize("n,x", [(1, 1), (4, 0b1010), (7, 77)])
def test_product_state_closed_forms(n, x):
    """Basis factors give |x> exactly; |+> on every qubit gives the uniform state 2^(-n/2)."""
    basis = oracle.product_state([(0, 1) if (x >> t) & 1 else (1, 0) for t in range(n)])
    assert np.array_equal(basis, oracle.basis_state(n, x))
    h = 1 / math.sqrt(2)
    plus = oracle.product_state([(h, h)] * n)
    assert np.max(np.abs(plus - 2.0 ** (-n / 2))) < 1e-15


@pytest.mark.parametrize("n", [2, 3, 5])
def test_two_qubit_gate_matches_its_operator(n):
    """Every ordered pair of qubits, with and without controls, against the element-wise operator."""
    for q0 in range(n):
        for q1 in range(n):
            if q0 == q1:
                continue
            rest = [q for q in range(n) if q not in (q0, q1)]
            for ctl in ([()] + ([tuple(rest[:1])] if rest else []) + ([tuple(rest[:2])] if len(rest) > 1 else [])):
                v = C.haar_u4(RNG)
                psi = rand_state(n)
                want = dense_gate4(n, v, q0, q1, ctl) @ psi
                got = oracle.apply_gate4(psi.copy(), v, q0, q1, ctl)
                assert np.max(np.abs(got - want)) < 1e-14


def test_two_qubit_kronecker_gate_is_two_one_qubit_gates():
    """Eq. tensor-product-gates: (A (x) B) on (q0, q1) = B on q0 then A on q1 (the pair update)."""
    n = 5
    for q0, q1 in [(0, 1), (3, 1), (4, 0)]:
        a, b = C.haar_u2(RNG), C.haar_u2(RNG)
        psi = rand_state(n)
        want = oracle.apply_gate(oracle.apply_gate(psi.copy(), b, q0), a, q1)
        got = oracle.apply_gate4(psi.copy(), np.kron(a, b), q0, q1)
        assert np.max(np.abs(got - want)) < 1e-15


def test_paper_cnot_matrix_as_two_qubit_gate():
    """The CNOT matrix of Sec. II.B (its truth table in tests/golden/cnot_truth_table.txt: the first ket symbol
    is the control, index bit 1) as a dense gate with q1 = control equals the controlled X, exactly."""
    v = np.zeros((4, 4))
    for inp, out in golden_lines("cnot_truth_table.txt"):
        v[int(out, 2), int(inp, 2)] = 1.0
    n = 4
    for control, target in [(1, 0), (0, 3), (3, 2)]:
        psi = rand_state(n)
        want = oracle.apply_gate(psi.copy(), C.X, target, (control,))
        got = oracle.apply_gate4(psi.copy(), v, target, control)
        assert np.array_equal(got, want)
    # the same through packed records (four per gate) and the circuit entry point
    psi = rand_state(n)
    w = C.pack([C.gate_u4(v, 0, 1), C.gate_u(C.H, 2), C.gate_u4(C.haar_u4(RNG), 2, 3, (0,))])
    step = oracle.apply_gate(oracle.apply_gate4(psi.copy(), v, 0, 1), C.H, 2)
    g = C.unpack(w)[2]
    step = oracle.apply_gate4(step, g.u, 2, 3, (0,))
    assert np.array_equal(oracle.apply_circuit(psi.copy(), w), step)


def test_non_sequential_storage_example():
    """Sec. VI.B: interchanging index bits 1 and 2 of an n = 3 vector stores alpha_0,1,4,5,2,3,6,7."""
    order = [int(v) for v in golden_lines("nonsequential_order_n3.txt")[0]]
    psi = np.arange(8, dtype=np.complex128) * (1 + 0.5j)
    got = oracle.apply_swap(psi.copy(), 1, 2)
    assert np.array_equal(got, psi[order])


# ----------------------------------------------------------------------------------------------------------------
# Closed forms and invariants
# ----------------------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 10])
def test_qft_closed_form(n):
    gates = C.pack(C.qft(n))
    assert len(gates) == n + n * (n - 1) // 2 + n // 2
    ys = np.arange(2 ** n)
    for x in sorted({0, 1, 2 ** n - 1, int(RNG.integers(2 ** n))}):
        got = oracle.simulate(n, gates, x)
        want = np.exp(2j * np.pi * ((x * ys) % 2 ** n) / 2 ** n) / math.sqrt(2 ** n)
        assert np.max(np.abs(got - want)) < 1e-13


@pytest.mark.parametrize("n", [1, 4, 11])
def test_hadamard_on_every_qubit_gives_uniform_state(n):
    got = oracle.simulate(n, C.pack(C.hadamard_all(n)))
    assert np.max(np.abs(got - 2.0 ** (-n / 2))) < 1e-15
    assert np.all(got.imag == 0)


@pytest.mark.parametrize("n", [2, 3, 9])
def test_ghz_exact(n):
    got = oracle.simulate(n, C.pack(C.ghz(n)))
    want = np.zeros(2 ** n, dtype=np.complex128)
    want[0] = want[-1] = C.SQRT1_2
    assert np.array_equal(got, want)  # H|0> = (s, s) exactly, the CNOTs only move amplitudes


def test_circuit_followed_by_inverse_is_identity():
    n = 8
    g = C.pack(C.random_layers(n, 10, RNG) + C.qft(n))
    psi = oracle.simulate(n, np.concatenate([g, C.inverse(g)]))
    assert abs(psi[0] - 1) < 1e-13
    assert np.max(np.abs(psi[1:])) < 1e-13


def test_norm_is_preserved():
    n = 10
    psi = oracle.simulate(n, C.random_workload(n, 5, seed=7).gates)
    assert abs(oracle.norm2(psi) - 1.0) < 1e-13
    assert abs(np.sum(oracle.probabilities(psi)) - 1.0) < 1e-13


def test_thread_count_does_not_change_result():
    n = 12
    w = C.random_workload(n, 3, seed=11)
    a = oracle.simulate(n, w.gates, threads=1)
    b = oracle.simulate(n, w.gates, threads=4)
    assert np.array_equal(a, b)
    # the collapse(2) split of both loops (used for the large parity comparisons) changes only which thread
    # updates a pair, so it too is bit-identical, for gates on every qubit including the highest
    c = oracle.simulate(n, w.gates, threads=4, collapse=True)
    assert np.array_equal(a, c)


def test_rejects_malformed_gates():
    psi = oracle.basis_state(3)
    with pytest.raises(ValueError):
        oracle.apply_gate(psi, C.X, 3)
    with pytest.raises(ValueError):
        oracle.apply_gate(psi, C.X, 1, (1,))
    with pytest.raises(ValueError):
        oracle.apply_gate(psi, C.X, 1, (0, 0))
    with pytest.raises(ValueError):
        oracle.apply_swap(psi, 2, 2)
