"""Input generators: record layout, unitarity of the seeded gates, determinism from the seed, config shapes."""
import numpy as np

import circuits as C


def test_record_layout_is_96_bytes():
    assert C.GATE_DTYPE.itemsize == 96
    assert C.GATE_DTYPE.fields["kind"][1] == 64
    assert C.GATE_DTYPE.fields["controls"][1] == 80


def test_haar_u2_is_unitary():
    rng = np.random.Generator(np.random.PCG64(1))
    for _ in range(100):
        u = C.haar_u2(rng)
        assert np.max(np.abs(u.conj().T @ u - np.eye(2))) < 1e-14


def test_generators_are_deterministic_and_shaped():
    a = C.random_workload(12, 4, seed=3)
    b = C.random_workload(12, 4, seed=3)
    assert np.array_equal(a.gates, b.gates)
    assert len(a.gates) == 4 * (12 + 6)
    q = C.qft_workload(20, seed=1001)
    assert len(q.gates) == 20 + 190 + 10 and 0 <= q.x0 < 2 ** 20
    r = C.random_workload(30, 20, seed=1002)
    assert len(r.gates) == 900


def test_inverse_round_trip_of_records():
    w = C.random_workload(6, 2, seed=9)
    inv2 = C.inverse(C.inverse(w.gates))
    assert np.array_equal(inv2, w.gates)


def test_batched_sizes_within_bounds():
    ws = C.batched_workloads(64, seed=1004)
    assert all(10 <= w.n <= 22 for w in ws)
