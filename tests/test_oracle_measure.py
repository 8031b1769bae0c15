"""Pins for the oracle's measurement read-outs (the probability interpretation |alpha_k|^2 of Sec. II.A):
sampling by inverse cumulative probability and Pauli-Z expectations, against closed forms."""
import math

import numpy as np
import pytest

import circuits as C
import oracle


def test_basis_state_always_gives_its_index():
    psi = oracle.basis_state(6, 37)
    u = np.random.default_rng(1).random(200)
    assert np.all(oracle.sample(psi, u) == 37)


@pytest.mark.parametrize("n", [1, 3, 8])
def test_uniform_state_gives_floor_of_u_times_dim(n):
    psi = oracle.simulate(n, C.pack(C.hadamard_all(n)))
    # stay clear of the interval ends, where the rounding of the cumulative sum decides
    u = (np.arange(2 ** n) + 0.5) / 2 ** n
    assert np.array_equal(oracle.sample(psi, u), np.arange(2 ** n, dtype=np.uint64))


def test_ghz_gives_all_zeros_or_all_ones():
    n = 7
    psi = oracle.simulate(n, C.pack(C.ghz(n)))
    assert list(oracle.sample(psi, [0.1, 0.49, 0.51, 0.9])) == [0, 0, 2 ** n - 1, 2 ** n - 1]


def test_expect_z_of_basis_states_is_a_parity():
    for x in (0, 5, 13, 31):
        psi = oracle.basis_state(5, x)
        for mask in (0, 1, 6, 31):
            assert oracle.expect_z(psi, mask) == (-1) ** bin(x & mask).count("1")


def test_expect_z_of_a_product_state_is_a_product_of_cosines():
    n = 5
    th = np.random.default_rng(2).uniform(0, np.pi, n)
    psi = oracle.simulate(n, C.pack([C.gate_u(C.ry(th[q]), q) for q in range(n)]))
    for mask in (1, 2, 5, 22, 31):
        want = math.prod(math.cos(th[q]) for q in range(n) if mask >> q & 1)
        assert abs(oracle.expect_z(psi, mask) - want) < 1e-14
