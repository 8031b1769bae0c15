"""Measurement read-outs on the GPU against the oracle: sampling (the caller's uniform numbers mapped through
the cumulative probabilities in logical order) and Pauli-Z expectations, including states whose qubits are
relabelled (non-identity layout after SWAPs)."""
import numpy as np
import pytest

import circuits as C
import oracle
from gpu_helpers import MODES, MODE_IDS, make_state

pytestmark = pytest.mark.gpu
B = pytest.importorskip("paper_1801_01037_gb300")._binding


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1801_01037_gb300 import build
    build.build()
    B.load()


@pytest.mark.parametrize("mode", MODES, ids=MODE_IDS)
@pytest.mark.parametrize("n", [3, 12, 17])
def test_sampling_and_expectations_match_oracle(mode, n):
    _, dtype, arith = mode
    w = C.qft_random_workload(n, 2, seed=60 + n)  # QFT SWAPs relabel the qubits
    want = oracle.simulate(n, w.gates, w.x0)
    if dtype == B.SV_C64:
        want_cmp = want.astype(np.complex64).astype(np.complex128)
    else:
        want_cmp = want
    h = make_state(n, dtype, arith, x0=w.x0)
    try:
        B.sv_apply_circuit(h, w.gates)
        assert list(B.sv_get_layout(h)) != list(range(n)) or n < 2
        u = np.random.default_rng(n).random(4000)
        got = B.sv_sample(h, u).astype(np.int64)
        # the chosen index's cumulative interval (from the oracle's probabilities) must contain u * total
        c = np.cumsum(oracle.probabilities(want_cmp))
        lo = np.concatenate([[0.0], c])[got]
        hi = c[got]
        t = u * c[-1]
        slack = 1e-12 if dtype == B.SV_C128 else 1e-5
        assert np.all(lo <= t + slack) and np.all(t <= hi + slack)
        same = np.mean(got == oracle.sample(want_cmp, u).astype(np.int64))
        assert same > 0.99
        for mask in (1, 1 << (n - 1), (1 << n) - 1, 0b101 & ((1 << n) - 1)):
            ez = B.sv_expect_z(h, mask)
            assert abs(ez - oracle.expect_z(want, mask)) < (1e-12 if dtype == B.SV_C128 else 1e-5)
    finally:
        B.sv_destroy(h)


def test_sampling_rejects_out_of_range_numbers():
    h = B.sv_create(4, B.SV_C128)
    try:
        with pytest.raises(B.SvError) as e:
            B.sv_sample(h, [0.2, 1.0])
        assert e.value.code == B.SV_ERR_ARG
    finally:
        B.sv_destroy(h)
