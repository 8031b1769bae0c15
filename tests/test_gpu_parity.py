"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle, element by element, on seeded inputs.

Sizes run from n = 1 (one pair) through n = 18 (64 chunks of 2^12), so the fused pass is exercised with a
single chunk, with exactly one chunk, with many chunks, and the single-gate sweep with ragged tails (fewer
items than one tile).  Tolerances are in ``gpu_helpers``."""
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


def class_matrices(rng):
    u = C.haar_u2(rng)
    ph = np.exp(1j * rng.uniform(0, 2 * np.pi, 2))
    return {
        "general": u,
        "diag": np.diag(ph),
        "phase": np.diag([1, ph[0]]),
        "antidiag": np.array([[0, ph[0]], [ph[1], 0]]),
        "x": C.X,
        "identity": np.eye(2),
        "h": C.H,
    }


@pytest.mark.parametrize("mode", MODES, ids=MODE_IDS)
@pytest.mark.parametrize("n", [1, 2, 5, 11, 14])
def test_single_gate_every_class_target_and_control_pattern(mode, n):
    _, dtype, arith = mode
    rng = np.random.default_rng(100 + n)
    psi0 = C.random_state(n, seed=n)
    h = make_state(n, dtype, arith, psi0)
    want = psi0.copy()
    try:
        for t in range(n):
            others = [q for q in range(n) if q != t]
            ctl_sets = [()] + [tuple(rng.choice(others, size=m, replace=False)) for m in (1, 2, 3) if m <= len(others)]
            for ctl in ctl_sets:
                for name, u in class_matrices(rng).items():
                    B.sv_apply_gate(h, u, t, ctl)
                    oracle.apply_gate(want, u, t, ctl)
        got = B.sv_read_amplitudes(h).astype(np.complex128)
    finally:
        B.sv_destroy(h)
    assert_close(got, want, dtype, f"n={n}")


def mixed_circuit(n, rng):
    gates = []
    for _ in range(3):
        gates += C.random_layers(n, 1, rng)
        if n >= 3:
            a, b, c = (int(x) for x in rng.choice(n, 3, replace=False))
            gates.append(C.gate_swap(a, b))
            gates.append(C.gate_u(C.X, c, (a, b)))                       # Toffoli
            gates.append(C.gate_u(C.phase(rng.uniform(0, 6)), a, (c,)))   # controlled phase
            gates.append(C.gate_u(np.diag(np.exp(1j * rng.uniform(0, 6, 2))), b))
            gates.append(C.gate_u(C.haar_u2(rng), c, tuple(q for q in (a, b) if q != c)))
    return C.pack(gates)


@pytest.mark.parametrize("mode", MODES, ids=MODE_IDS)
@pytest.mark.parametrize("n", [3, 8, 12, 13, 16, 18])
@pytest.mark.parametrize("chunk_k", [0, 6, 8])
def test_fused_circuits_match_oracle(mode, n, chunk_k):
    _, dtype, arith = mode
    rng = np.random.default_rng(7 * n + chunk_k)
    gates = np.concatenate([mixed_circuit(n, rng), C.pack(C.qft(n))])
    psi0 = C.random_state(n, seed=1000 + n)
    want = run_oracle(n, gates, psi0)
    got = run_gpu(n, gates, dtype, arith, psi0, chunk_k=chunk_k)
    assert_close(got, want, dtype, f"n={n} k={chunk_k}")


def controlled_circuit(n, rng, count=60):
    """Gates of every class with 1-4 controls on random qubits, between Haar layers (so that the fused
    passes see controls inside and outside the chunk, and targets of diagonal gates outside it)."""
    gates = C.random_layers(n, 1, rng)
    for i in range(count):
        t = int(rng.integers(n))
        others = [q for q in range(n) if q != t]
        ctl = tuple(int(q) for q in rng.choice(others, size=int(rng.integers(1, 5)), replace=False))
        u = list(class_matrices(rng).values())[i % 7]
        gates.append(C.gate_u(u, t, ctl))
        if i % 15 == 14:
            gates += C.random_layers(n, 1, rng)
    return C.pack(gates)


@pytest.mark.parametrize("mode", MODES, ids=MODE_IDS)
@pytest.mark.parametrize("n,chunk_k", [(9, 0), (12, 0), (14, 0), (14, 8), (16, 6)])
def test_fused_controlled_gates_every_class_and_control_count(mode, n, chunk_k):
    """Controlled gates visit only the amplitudes whose local control bits are 1 (the enumerated index with
    the control and target bits inserted): every class, 1-4 controls, against the oracle."""
    _, dtype, arith = mode
    rng = np.random.default_rng(31 * n + chunk_k)
    gates = controlled_circuit(n, rng)
    psi0 = C.random_state(n, seed=77 + n)
    want = run_oracle(n, gates, psi0)
    got = run_gpu(n, gates, dtype, arith, psi0, chunk_k=chunk_k)
    assert_close(got, want, dtype, f"n={n} k={chunk_k}")


@pytest.mark.parametrize("mode", MODES, ids=MODE_IDS)
def test_unfused_sweeps_match_oracle(mode):
    _, dtype, arith = mode
    n = 15
    gates = mixed_circuit(n, np.random.default_rng(3))
    psi0 = C.random_state(n, seed=5)
    assert_close(run_gpu(n, gates, dtype, arith, psi0, fusion=0), run_oracle(n, gates, psi0), dtype)


@pytest.mark.parametrize("mode", MODES, ids=MODE_IDS)
def test_qft_n20_from_seeded_basis_state(mode):
    """The QFT workload (n = 20, |x> from seed 1001): oracle and closed form e^{2 pi i x y / 2^n} / 2^{n/2}."""
    _, dtype, arith = mode
    w = C.qft_workload(20, seed=1001)
    got = run_gpu(w.n, w.gates, dtype, arith, x0=w.x0)
    want = run_oracle(w.n, w.gates, x0=w.x0)
    assert_close(got, want, dtype, "qft20 vs oracle")
    y = np.arange(2 ** w.n)
    closed = np.exp(2j * np.pi * ((w.x0 * y) % 2 ** w.n) / 2 ** w.n) / 2 ** (w.n / 2)
    assert_close(got, closed, dtype, "qft20 vs closed form")


@pytest.mark.parametrize("mode", MODES, ids=MODE_IDS)
def test_permutation_circuits_are_bit_exact(mode):
    """X, CNOT, Toffoli and SWAP only move amplitudes: the result equals the oracle's bit for bit."""
    _, dtype, arith = mode
    n = 14
    rng = np.random.default_rng(11)
    gates = []
    for _ in range(40):
        a, b, c = (int(x) for x in rng.choice(n, 3, replace=False))
        gates += [C.gate_u(C.X, a), C.cnot(a, b), C.gate_u(C.X, c, (a, b)), C.gate_swap(b, c)]
    gates = C.pack(gates)
    psi0 = C.random_state(n, seed=2)
    if dtype == B.SV_C64:
        psi0 = psi0.astype(np.complex64).astype(np.complex128)
    want = run_oracle(n, gates, psi0)
    for fusion in (0, 1):
        got = run_gpu(n, gates, dtype, arith, psi0, fusion=fusion)
        assert np.array_equal(got, want)


def test_ghz_exact_in_f64_mode():
    n = 16
    g = C.pack(C.ghz(n))
    got = run_gpu(n, g, B.SV_C128, B.SV_ARITH_F64)
    want = np.zeros(2 ** n, dtype=np.complex128)
    want[0] = want[-1] = C.SQRT1_2
    assert np.array_equal(got, want)
    # double-float: one dense update of (1, 0) carries an error of a few 2^-46 of the pair's largest component
    got = run_gpu(n, g, B.SV_C128, B.SV_ARITH_DF32)
    assert np.count_nonzero(got) == 2 and abs(got[0] - C.SQRT1_2) < 2e-14 and got[0] == got[-1]


@pytest.mark.parametrize("n", [2, 4, 7])
def test_deep_small_circuit_stays_within_c128_tolerance(n):
    """Large amplitudes and many gates: the worst case for the double-float error, which scales with the
    magnitude of each pair.  1500+ gates on n <= 7 qubits (amplitudes of order 0.1-1)."""
    gates = C.pack(C.random_layers(n, 1500 // (n + n // 2) + 1, np.random.default_rng(n)))
    psi0 = C.random_state(n, seed=77)
    for arith in (B.SV_ARITH_DF32, B.SV_ARITH_F64):
        got = run_gpu(n, gates, B.SV_C128, arith, psi0)
        assert_close(got, run_oracle(n, gates, psi0), B.SV_C128, f"n={n} arith={arith}")


@pytest.mark.parametrize("mode", MODES, ids=MODE_IDS)
def test_graph_replay_and_determinism(mode):
    _, dtype, arith = mode
    n = 17
    gates = C.random_workload(n, 4, seed=21).gates
    a = run_gpu(n, gates, dtype, arith)
    b = run_gpu(n, gates, dtype, arith)
    assert np.array_equal(a, b)
    h = make_state(n, dtype, arith)
    try:
        for rep in range(3):
            B.sv_init_basis(h, 0)
            B.sv_apply_circuit_graph(h, gates)
            assert np.array_equal(B.sv_read_amplitudes(h).astype(np.complex128), a)
    finally:
        B.sv_destroy(h)


def fsum_norm2(v):
    """sum |v_k|^2: the squares in FP64, added with math.fsum (correctly rounded)."""
    import math
    return math.fsum(np.concatenate([v.real * v.real, v.imag * v.imag]).tolist())


@pytest.mark.parametrize("mode", MODES, ids=MODE_IDS)
def test_norm_probabilities_and_readout(mode):
    _, dtype, arith = mode
    n = 19
    w = C.qft_random_workload(n, 2, seed=4)
    want = run_oracle(n, w.gates, x0=w.x0)
    h = make_state(n, dtype, arith, x0=w.x0)
    try:
        B.sv_apply_circuit(h, w.gates)
        nrm = B.sv_norm(h)
        assert abs(nrm - oracle.norm2(want)) < (1e-13 if dtype == B.SV_C128 else 1e-5)
        # The reduction itself accumulates in FP64: against the correctly rounded sum (math.fsum) of the squares
        # of the GPU's own amplitudes it agrees to 1e-15 relative in every mode, and with native FP64 gates (the
        # same state as the oracle's up to FMA rounding) also against the oracle state's correctly rounded norm.
        # (The oracle's own norm2 adds in index order, with an error that grows like 2^n ulps in the worst case.)
        mine = B.sv_read_amplitudes(h).astype(np.complex128)
        assert abs(nrm - fsum_norm2(mine)) <= 1e-15 * nrm
        if arith == B.SV_ARITH_F64:
            assert abs(nrm - fsum_norm2(want)) <= 1e-15 * nrm
        p = B.sv_read_probabilities(h, 5, 1000)
        tol = 1e-13 if dtype == B.SV_C128 else 1e-6 * np.max(oracle.probabilities(want))
        assert np.max(np.abs(p - oracle.probabilities(want)[5:1005])) <= tol
        idx = np.random.default_rng(1).integers(0, 2 ** n, 5000)
        assert_close(B.sv_read_amplitudes_at(h, idx).astype(np.complex128), want[idx], dtype, "gather")
        part = B.sv_read_amplitudes(h, 777, 3333).astype(np.complex128)
        assert_close(part, want[777:777 + 3333], dtype, "range read")
        layout = B.sv_get_layout(h)
        B.sv_canonicalize(h)
        assert list(B.sv_get_layout(h)) == list(range(n))
        assert_close(B.sv_read_amplitudes(h).astype(np.complex128), want, dtype, f"canonical (layout was {layout})")
        # renormalisation divides by the norm
        B.sv_renormalize(h)
        assert abs(B.sv_norm(h) - 1.0) < (1e-13 if dtype == B.SV_C128 else 1e-5)
    finally:
        B.sv_destroy(h)


def fsum_signed(v, mask):
    """sum_k (-1)^popcount(k & mask) |v_k|^2 with the squares in FP64, added with math.fsum."""
    import math
    k = np.arange(v.size, dtype=np.uint64)
    par = np.zeros(v.size, dtype=np.int64)
    m = k & np.uint64(mask)
    while np.any(m):
        par ^= (m & np.uint64(1)).astype(np.int64)
        m >>= np.uint64(1)
    sg = 1.0 - 2.0 * par
    return math.fsum(np.concatenate([sg * v.real * v.real, sg * v.imag * v.imag]).tolist())


@pytest.mark.parametrize("dtype", [B.SV_C128, B.SV_C64], ids=["c128", "c64"])
@pytest.mark.parametrize("n", [21, 22])
def test_norm_expectation_and_renormalisation_past_the_vector_span(dtype, n):
    """From n = 21 on most of the reduction runs in the norm kernel's vector loop (four 16-byte loads per thread
    and iteration) and the rest in its tail: the FP64 norm and Pauli-Z expectations against the correctly
    rounded sums of the GPU's own amplitudes, and the renormalised amplitudes against an FP64 rescale of the
    amplitudes read before it (a state written with norm 1.7^2, so the factor is far from 1)."""
    rng = np.random.default_rng(40 + n)
    v = rng.standard_normal(2 ** n) + 1j * rng.standard_normal(2 ** n)
    v *= 1.7 / np.linalg.norm(v)
    h = B.sv_create(n, dtype)
    try:
        B.sv_write_amplitudes(h, 0, v.astype(np.complex128 if dtype == B.SV_C128 else np.complex64))
        mine = B.sv_read_amplitudes(h).astype(np.complex128)
        nrm = B.sv_norm(h)
        assert abs(nrm - fsum_norm2(mine)) <= 1e-15 * nrm
        for mask in (1, (1 << (n - 1)) | 6, (1 << n) - 1):
            ez = B.sv_expect_z(h, mask)
            assert abs(ez - fsum_signed(mine, mask)) <= 1e-15 * nrm, mask
        B.sv_renormalize(h)
        after = B.sv_read_amplitudes(h).astype(np.complex128)
        want = mine / np.sqrt(nrm)
        if dtype == B.SV_C128:
            np.testing.assert_allclose(after, want, rtol=2 ** -50, atol=0)
            assert abs(B.sv_norm(h) - 1.0) < 1e-14
        else:
            # within one float ulp of the FP64 rescale, componentwise
            for got, ref in ((after.real, want.real), (after.imag, want.imag)):
                ulp = np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)
                assert np.all(np.abs(got - ref) <= ulp)
            assert abs(B.sv_norm(h) - 1.0) < 1e-6
    finally:
        B.sv_destroy(h)


def test_buffer_state_over_torch_tensor_stays_in_logical_order():
    torch = pytest.importorskip("torch")
    n = 15
    psi0 = C.random_state(n, seed=9)
    t = torch.from_numpy(psi0).to("cuda")
    torch.cuda.synchronize()
    h = B.sv_create_from_buffer(n, B.SV_C128, t.data_ptr())
    try:
        w = C.pack(C.qft(n))
        B.sv_apply_circuit(h, w)
        B.sv_sync(h)
        want = run_oracle(n, w, psi0)
        assert_close(t.cpu().numpy(), want, B.SV_C128, "tensor contents")
    finally:
        B.sv_destroy(h)


@pytest.mark.parametrize("mode", MODES, ids=MODE_IDS)
@pytest.mark.parametrize("n", [3, 14, 19])
def test_composed_one_qubit_runs_match_oracle(mode, n):
    """Runs of one-qubit gates on one qubit are composed into one matrix (FP64, host) before planning; the
    oracle applies them one by one.  Identity products (X X, S S^dagger) are dropped."""
    _, dtype, arith = mode
    rng = np.random.default_rng(90 + n)
    gates = []
    for layer in range(4):
        for q in range(n):
            gates += [C.gate_u(C.rz(rng.uniform(0, 6.3)), q), C.gate_u(C.ry(rng.uniform(0, 6.3)), q),
                      C.gate_u(C.haar_u2(rng), q)]
        for q in range(0, n - 1, 2):
            gates.append(C.cnot(q, q + 1) if layer % 2 == 0 else C.cnot(q + 1, (q + 2) % n))
    gates += [C.gate_u(C.X, 0), C.gate_u(C.X, 0), C.gate_u(C.S, n - 1), C.gate_u(C.S.conj().T, n - 1)]
    w = C.pack(gates)
    psi0 = C.random_state(n, seed=n)
    if dtype == B.SV_C64:
        psi0 = psi0.astype(np.complex64).astype(np.complex128)
    want = run_oracle(n, w, psi0)
    assert_close(run_gpu(n, w, dtype, arith, psi0=psi0), want, dtype, "composed runs")
    assert_close(run_gpu(n, w, dtype, arith, psi0=psi0, fusion=0), want, dtype, "composed runs, sweeps")


@pytest.mark.parametrize("n,chunk_k", [(8, 8), (13, 0), (17, 0), (17, 9), (20, 12)])
def test_c64_register_cubes_identical_to_per_gate_passes(n, chunk_k):
    """Complex64 passes apply runs of gates on at most four chunk bits from registers (SV_OPT_CUBES).  The
    same arithmetic in the same order as the per-gate shared-memory loop: results are bit-identical, and
    within the complex64 tolerance of the oracle.  Circuits mix every gate class, in-cube and out-of-cube
    controls, and diagonal gates on bits outside the cube and outside the chunk."""
    rng = np.random.default_rng(700 + n)
    gates = []
    for layer in range(6):
        for q in range(n):
            r = rng.integers(0, 6)
            if r == 0:
                gates.append(C.gate_u(C.haar_u2(rng), q))
            elif r == 1:
                gates.append(C.gate_u(np.diag(np.exp(1j * rng.uniform(0, 6.3, 2))), q, [int((q + 3) % n)]))
            elif r == 2:
                gates.append(C.gate_u(C.phase(rng.uniform(0, 6.3)), q, [int((q + n // 2) % n)]))
            elif r == 3:
                gates.append(C.cnot(int(rng.integers(0, n - 1) + q + 1) % n, q))
            elif r == 4:
                ph = np.exp(1j * rng.uniform(0, 6.3, 2))
                gates.append(C.gate_u(np.array([[0, ph[0]], [ph[1], 0]]), q))
            else:
                gates.append(C.gate_u(C.haar_u2(rng), q, [int((q + 1) % n), int((q + 5) % n)]))
    w = C.pack(gates)
    psi0 = C.random_state(n, seed=n + 1)
    outs = []
    for cubes in (0, 1):
        h = make_state(n, B.SV_C64, B.SV_ARITH_AUTO, psi0=psi0, chunk_k=chunk_k)
        try:
            B.sv_set_option(h, B.SV_OPT_CUBES, cubes)
            B.sv_apply_circuit(h, w)
            outs.append(B.sv_read_amplitudes(h))
        finally:
            B.sv_destroy(h)
    assert np.array_equal(outs[0], outs[1])
    want = run_oracle(n, w, psi0.astype(np.complex64).astype(np.complex128))
    assert_close(outs[1].astype(np.complex128), want, B.SV_C64, "register cubes")


@pytest.mark.parametrize("mode", MODES, ids=MODE_IDS)
@pytest.mark.parametrize("n,chunk_k", [(2, 0), (5, 0), (13, 0), (16, 0), (21, 0), (21, 6), (22, 9)])
def test_canonicalize_random_layouts_is_bit_exact(mode, n, chunk_k):
    """SWAPs only relabel qubits (Sec. VI.B); sv_canonicalize then moves the data back into logical order with
    bit-permutation passes.  Pure data movement: the result equals the oracle's exactly, in every mode, for
    random layouts that mix the low (row) bits with high ones and need several passes."""
    _, dtype, arith = mode
    rng = np.random.default_rng(100 + n + chunk_k)
    psi0 = C.random_state(n, seed=n)
    if dtype == B.SV_C64:
        psi0 = psi0.astype(np.complex64).astype(np.complex128)
    swaps = C.pack([C.gate_swap(*rng.choice(n, 2, replace=False)) for _ in range(3 * n)]) if n > 1 else C.pack([])
    want = run_oracle(n, swaps, psi0)
    h = make_state(n, dtype, arith, psi0=psi0, chunk_k=chunk_k)
    try:
        B.sv_apply_circuit(h, swaps)
        layout = list(B.sv_get_layout(h))
        assert np.array_equal(B.sv_read_amplitudes(h).astype(np.complex128), want)
        B.sv_canonicalize(h)
        assert list(B.sv_get_layout(h)) == list(range(n))
        got = B.sv_read_amplitudes(h).astype(np.complex128)
        assert np.array_equal(got, want), f"layout was {layout}"
    finally:
        B.sv_destroy(h)


@pytest.mark.parametrize("dtype", [B.SV_C128, B.SV_C64], ids=["c128", "c64"])
def test_buffer_state_graph_replay_stays_in_logical_order(dtype):
    """A buffer state (caller-owned memory, always in logical order) through the captured-graph path: the
    graph ends with the bit-permutation passes that undo the QFT's SWAP relabelling."""
    torch = pytest.importorskip("torch")
    n = 18
    psi0 = C.random_state(n, seed=19)
    tdt = torch.complex64 if dtype == B.SV_C64 else torch.complex128
    t = torch.from_numpy(psi0).to(tdt).to("cuda")
    torch.cuda.synchronize()
    start = t.clone()
    w = C.pack(C.qft(n))
    want = run_oracle(n, w, t.cpu().numpy().astype(np.complex128))
    h = B.sv_create_from_buffer(n, dtype, t.data_ptr())
    try:
        for rep in range(2):
            t.copy_(start)
            torch.cuda.synchronize()
            B.sv_apply_circuit_graph(h, w)
            B.sv_sync(h)
            assert list(B.sv_get_layout(h)) == list(range(n))
            assert_close(t.cpu().numpy().astype(np.complex128), want, dtype, f"graph replay {rep}")
    finally:
        B.sv_destroy(h)


def test_host_validation_leaves_state_untouched():
    n = 6
    h = make_state(n, B.SV_C128, B.SV_ARITH_DF32, x0=5)
    try:
        before = B.sv_read_amplitudes(h)
        bad = C.pack([C.gate_u(C.H, 0), C.gate_u(C.X, 9)])
        with pytest.raises(B.SvError) as e:
            B.sv_apply_circuit(h, bad)
        assert e.value.code == B.SV_ERR_ARG and "gate 1" in str(e.value)
        with pytest.raises(B.SvError) as e:
            B.sv_apply_gate(h, np.array([[1, 1], [0, 1]]), 0)
        assert e.value.code == B.SV_ERR_NOT_UNITARY
        assert np.array_equal(B.sv_read_amplitudes(h), before)
    finally:
        B.sv_destroy(h)


def test_oversized_state_is_refused():
    with pytest.raises(B.SvError) as e:
        B.sv_create(36, B.SV_C128)
    assert e.value.code == B.SV_ERR_OOM


@pytest.mark.parametrize("share", [0, 20, 50])
def test_fp64_share_of_double_float_pass(share):
    """Complex128 double-float passes with part of the chunks done in native FP64 (SV_OPT_F64_SHARE): the result
    matches the oracle, and which chunks use FP64 depends only on their index (bit-identical reruns)."""
    import os as _os
    n = 23  # enough chunks (2^11 of 2^12 amplitudes) for the split to be used
    w = C.random_workload(n, 3, seed=31)
    want = oracle.apply_circuit(oracle.basis_state(n, 0), w.gates, threads=_os.cpu_count() or 1)
    outs = []
    for rep in range(2):
        h = make_state(n, B.SV_C128, B.SV_ARITH_DF32)
        try:
            B.sv_set_option(h, B.SV_OPT_F64_SHARE, share)
            B.sv_apply_circuit(h, w.gates)
            outs.append(B.sv_read_amplitudes(h).astype(np.complex128))
        finally:
            B.sv_destroy(h)
    assert np.array_equal(outs[0], outs[1])
    assert_close(outs[0], want, B.SV_C128, f"share={share}")
