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


def test_bulk_layers_have_the_layer_structure():
    rng = np.random.Generator(np.random.PCG64(5))
    n, depth = 7, 4
    g = C.random_layers_packed(n, depth, rng)
    assert len(g) == depth * (n + n // 2)
    per = n + n // 2
    for L in range(depth):
        ones = g[L * per:L * per + n]
        assert list(ones["target"]) == list(range(n)) and np.all(ones["ncontrols"] == 0)
        for r in ones:
            u = C.unpack_u(r)
            assert np.max(np.abs(u.conj().T @ u - np.eye(2))) < 1e-14
        cn = g[L * per + n:(L + 1) * per]
        qubits = list(cn["target"]) + list(cn["controls"][:, 0])
        assert len(set(qubits)) == 2 * (n // 2) and np.all(cn["ncontrols"] == 1)
        assert all(np.array_equal(C.unpack_u(r), C.X) for r in cn)
