"""C-ABI checks that need no GPU: the library loads, exports every entry point declared in include/sv.h,
rejects bad arguments on the host before any device work, and its planner (host logic) produces schedules
that are valid reorderings of the circuit.  The planner check replays the planned execution order through
the FP64 oracle and compares with the original order."""
import os
import re

import numpy as np
import pytest

import circuits as C
import oracle
from conftest import ROOT

pkg = pytest.importorskip("paper_1801_01037_gb300")
B = pkg._binding


@pytest.fixture(scope="module")
def lib():
    from paper_1801_01037_gb300 import build
    build.build()
    return B.load()


def header_functions():
    src = open(os.path.join(ROOT, "include", "sv.h")).read()
    return sorted(set(re.findall(r"^\s*(?:sv_status|const char \*)\s*(sv_\w+)\s*\(", src, re.M)))


def test_every_declared_entry_point_is_exported(lib):
    names = header_functions()
    assert len(names) >= 25
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(B.EXPORTED) == names


def test_binding_constants_match_header():
    """Every integer #define of include/sv.h that the Python binding also names has the same value there."""
    src = open(os.path.join(ROOT, "include", "sv.h")).read()
    defs = dict(re.findall(r"^#define\s+(SV_\w+)\s+(-?\d+)\b", src, re.M))
    shared = [k for k in defs if hasattr(B, k)]
    assert len(shared) >= 10
    for k in shared:
        assert getattr(B, k) == int(defs[k]), k
    enums = dict(re.findall(r"\b(SV_\w+)\s*=\s*(-?\d+)\s*[,}]", src))
    for k, v in enums.items():
        if hasattr(B, k):
            assert getattr(B, k) == int(v), k


def test_gate_record_matches_header(lib):
    src = open(os.path.join(ROOT, "include", "sv.h")).read()
    assert "double U[8];" in src and C.GATE_DTYPE.itemsize == 96


def test_null_and_range_errors_without_device(lib):
    import ctypes
    assert lib.sv_destroy(None) == B.SV_OK
    assert lib.sv_apply_gate(None, None, 0, None, 0) == B.SV_ERR_ARG
    out = ctypes.c_void_p()
    assert lib.sv_create(0, B.SV_C128, None, ctypes.byref(out)) == B.SV_ERR_ARG
    assert lib.sv_create(37, B.SV_C128, None, ctypes.byref(out)) == B.SV_ERR_ARG
    assert lib.sv_create(4, 7, None, ctypes.byref(out)) == B.SV_ERR_ARG
    assert lib.sv_norm(None, None) == B.SV_ERR_ARG
    assert lib.sv_init_product(None, None) == B.SV_ERR_ARG
    assert lib.sv_last_plan_stats(None, None, None, None, None, None, None) == B.SV_ERR_ARG
    assert lib.sv_poll(None, 1, None, None) == B.SV_ERR_ARG
    assert b"NULL" in lib.sv_last_error()


def test_batch_option_checks_without_device(lib):
    from paper_1801_01037_gb300 import _binding as B
    with pytest.raises(B.SvError):
        B.sv_batch_set_option(B.SV_OPT_CHUNK_QUBITS, 12)
    with pytest.raises(B.SvError):
        B.sv_batch_set_option(B.SV_OPT_TENSOR_BLOCKS, 65)
    B.sv_batch_set_option(B.SV_OPT_TENSOR_BLOCKS, 3)
    B.sv_batch_set_option(B.SV_OPT_TENSOR_BLOCKS, 0)


def test_block_planner_dry_run(lib):
    """The dense-block planner through the C ABI, on the host: random layers form blocks on chunks of 2^11 and
    2^12 amplitudes (and 2^13 for complex64), each block replacing at least two gates; nothing forms without the
    option, with chunks below one 128-row tile, or for complex128 chunks of 2^13; the QFT's passes of controlled
    phases stay per-gate (blocks would take less than 3/4 of a pass's work); a pass whose dense gates all sit on
    four chunk bits forms exactly one block unless twenty gates with a control outside the chunk follow them."""
    from paper_1801_01037_gb300 import _binding as B
    w = C.random_workload(16, 6, seed=12)
    for dtype, k in ((B.SV_C128, 11), (B.SV_C128, 12), (B.SV_C64, 12), (B.SV_C64, 13)):
        r = B.sv_plan_dry_run_blocks(16, dtype, w.gates, 3, chunk_k=k)
        assert r["blocks"] > 0 and r["block_gates"] >= 2 * r["blocks"], (dtype, k, r)
        assert 0 < r["passes_with_blocks"] <= r["passes"]
        assert B.sv_plan_dry_run_blocks(16, dtype, w.gates, 0, chunk_k=k)["blocks"] == 0
    assert B.sv_plan_dry_run_blocks(16, B.SV_C128, w.gates, 3, chunk_k=13)["blocks"] == 0
    assert B.sv_plan_dry_run_blocks(16, B.SV_C64, w.gates, 3, chunk_k=10)["blocks"] == 0
    assert B.sv_plan_dry_run_blocks(10, B.SV_C64, C.random_workload(10, 4, seed=3).gates, 1)["blocks"] == 0
    q = C.qft_workload(20, seed=1001)
    assert B.sv_plan_dry_run_blocks(20, B.SV_C128, q.gates, 3)["blocks"] == 0
    rng = np.random.Generator(np.random.PCG64(23))
    lead = [C.cnot(0, 1)] + [C.gate_u(C.haar_u2(rng), t) for t in range(4)]
    tail = [C.gate_u(C.haar_u2(rng), 4 + i % 8, (15,)) for i in range(20)]
    r = B.sv_plan_dry_run_blocks(16, B.SV_C128, C.pack(lead), 1, chunk_k=12)
    assert (r["blocks"], r["block_gates"]) == (1, 5), r
    assert B.sv_plan_dry_run_blocks(16, B.SV_C128, C.pack(lead + tail), 1, chunk_k=12)["blocks"] == 0
    # a block replaces gates only up to its minimum size: 5 gates worth 4.125 dense updates
    assert B.sv_plan_dry_run_blocks(16, B.SV_C128, C.pack(lead), 5, chunk_k=12)["blocks"] == 0
    with pytest.raises(B.SvError):
        B.sv_plan_dry_run_blocks(16, B.SV_C128, w.gates, 65)


def test_no_device_is_reported_not_hidden(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import ctypes
    out = ctypes.c_void_p()
    assert lib.sv_create(4, B.SV_C128, None, ctypes.byref(out)) == B.SV_ERR_NO_DEVICE


def test_validation_rejects_bad_gates(lib):
    bad = [
        C.pack([C.gate_u(C.X, 5)]),                   # target out of range
        C.pack([C.gate_u(C.X, 1, (1,))]),             # control == target
        C.pack([C.gate_u(C.X, 1, (0, 0))]),           # repeated control
        C.pack([C.gate_swap(2, 2)]),                  # SWAP of one qubit
    ]
    for g in bad:
        with pytest.raises(B.SvError) as e:
            B.sv_plan_dry_run(4, B.SV_C128, g)
        assert e.value.code == B.SV_ERR_ARG
    nonunitary = C.pack([C.gate_u(np.array([[1, 0], [0, 1.001]]), 0)])
    with pytest.raises(B.SvError) as e:
        B.sv_plan_dry_run(4, B.SV_C128, nonunitary)
    assert e.value.code == B.SV_ERR_NOT_UNITARY


def test_validation_of_two_qubit_records(lib):
    v = C.haar_u4(np.random.default_rng(4))
    good = C.pack([C.gate_u4(v, 0, 2, (1,))])
    B.sv_plan_dry_run(4, B.SV_C128, good)
    bad = []
    bad.append(good[:3].copy())                                     # a row record missing
    bad.append(good[1:].copy())                                     # rows without their first record
    x = good.copy(); x[2]["target2"] = 3; bad.append(x)             # rows name other qubits
    x = good.copy(); x[0]["target2"] = 0; x[1:]["target2"] = 0; bad.append(x)  # both qubits the same
    x = good.copy(); x[0]["controls"][0] = 2; bad.append(x)         # control equal to a target
    x = good.copy(); x[0]["target"] = 7; x[1:]["target"] = 7; bad.append(x)    # qubit out of range
    for g in bad:
        with pytest.raises(B.SvError) as e:
            B.sv_plan_dry_run(4, B.SV_C128, g)
        assert e.value.code == B.SV_ERR_ARG
    x = good.copy(); x[3]["U"][0] += 1e-6                           # not unitary
    with pytest.raises(B.SvError) as e:
        B.sv_plan_dry_run(4, B.SV_C128, x)
    assert e.value.code == B.SV_ERR_NOT_UNITARY


def replay_in_plan_order(n, gates, plan):
    """The circuit's gates in the planner's execution order."""
    order = plan["order_of_gate"]
    assert sorted(order) == list(range(len(gates)))
    return gates[np.argsort(order)]


PLAN_CASES = [
    ("random", lambda: C.random_workload(14, 6, seed=5).gates, 14),
    ("qft", lambda: C.pack(C.qft(13)), 13),
    ("qft_random", lambda: C.qft_random_workload(15, 3, seed=8).gates, 15),
    ("mixed", lambda: C.pack(C.ghz(12) + [C.gate_swap(0, 11), C.gate_u(C.haar_u2(np.random.default_rng(1)), 11, (0, 3, 7))]
                             + C.random_layers(12, 2, np.random.default_rng(2))), 12),
    ("two_qubit", lambda: C.pack(two_qubit_circuit(14, np.random.default_rng(9))), 14),
]


def two_qubit_circuit(n, rng):
    """Dense two-qubit gates on near and far qubit pairs (some controlled, one identity), mixed with one-qubit
    gates, CNOTs and SWAPs."""
    gates = []
    for layer in range(3):
        for q in range(0, n - 1, 2):
            a, b = (q, q + 1) if layer % 2 == 0 else (q + 1, (q + 7) % n)
            ctl = () if q % 4 else ((b + 2) % n,) if (b + 2) % n not in (a, b) else ()
            gates.append(C.gate_u4(C.haar_u4(rng), a, b, ctl))
        gates.append(C.gate_u(C.haar_u2(rng), layer))
        gates.append(C.cnot(layer, n - 1 - layer))
        gates.append(C.gate_swap(layer, n - 2))
    gates.append(C.gate_u4(np.eye(4), 2, 9))
    return gates


@pytest.mark.parametrize("name,make,n", PLAN_CASES, ids=[c[0] for c in PLAN_CASES])
@pytest.mark.parametrize("dtype,chunk_k", [(B.SV_C128, 0), (B.SV_C64, 0), (B.SV_C128, 8)])
def test_planner_schedule_is_a_valid_reordering(lib, name, make, n, dtype, chunk_k):
    gates = make()
    plan = B.sv_plan_dry_run(n, dtype, gates, chunk_k)
    # 1. gates sharing a qubit keep their relative order
    order = plan["order_of_gate"]
    last = {}
    for i, g in enumerate(gates):
        kind = int(g["kind"])
        if kind == C.GATE_U4_ROW:
            assert order[i] == order[i - 1] + 1  # a two-qubit gate's records stay together
            continue
        qs = [int(g["target"])] + ([int(g["target2"])] if kind in (C.GATE_SWAP, C.GATE_U4) else [])
        if kind != C.GATE_SWAP:
            qs += [int(c) for c in g["controls"][:g["ncontrols"]]]
        for q in qs:
            if q in last:
                assert order[i] > order[last[q]]
            last[q] = i
    # 2. the reordered circuit gives the same state (FP64 oracle)
    want = oracle.simulate(n, gates, 3)
    got = oracle.simulate(n, replay_in_plan_order(n, gates, plan), 3)
    assert np.max(np.abs(got - want)) < 1e-12
    # 3. launches apply gates in order, and every pairing gate's physical target lies in its launch's chunk bits
    steps = plan["step_of_gate"]
    perm = list(range(n))
    for i in np.argsort(order):
        g = gates[i]
        if g["kind"] == C.GATE_SWAP:
            a, b = int(g["target"]), int(g["target2"])
            perm[a], perm[b] = perm[b], perm[a]
            assert steps[i] == -1
            continue
        if g["kind"] == C.GATE_U4_ROW:
            assert steps[i] == steps[i - 1]
            continue
        if g["kind"] == C.GATE_U4:
            v = C.unpack_u4(gates[i:i + 4])
            if np.array_equal(v, np.eye(4)):
                assert steps[i] == -1
                continue
            assert steps[i] >= 0
            for t in (int(g["target"]), int(g["target2"])):
                assert plan["step_qmask"][steps[i]] >> np.uint64(perm[t]) & np.uint64(1)
            continue
        u = C.unpack_u(g)
        if np.array_equal(u, np.eye(2)):
            assert steps[i] == -1
            continue
        assert steps[i] >= 0
        diagonal = u[0, 1] == 0 and u[1, 0] == 0
        if not diagonal:
            assert plan["step_qmask"][steps[i]] >> np.uint64(perm[int(g["target"])]) & np.uint64(1)
    assert list(plan["final_perm"]) == perm
    # steps are visited in non-decreasing order along the execution order
    seq = [steps[i] for i in np.argsort(order) if steps[i] >= 0]
    assert seq == sorted(seq)


def rotation_runs_circuit(n, rng):
    """Runs of one-qubit rotations on each qubit (Rz Ry Rz) between CNOT layers, then an X X pair and an
    S S^dagger pair (exact identities) after the last CNOT layer."""
    gates = []
    for layer in range(3):
        for q in range(n):
            gates += [C.gate_u(C.rz(rng.uniform(0, 6.3)), q), C.gate_u(C.ry(rng.uniform(0, 6.3)), q),
                      C.gate_u(C.rz(rng.uniform(0, 6.3)), q)]
        for q in range(0, n - 1, 2):
            gates.append(C.cnot(q, q + 1) if layer % 2 == 0 else C.cnot(q + 1, (q + 2) % n))
    gates += [C.gate_u(C.X, 0), C.gate_u(C.X, 0), C.gate_u(C.S, 3), C.gate_u(C.S.conj().T, 3)]
    return C.pack(gates)


@pytest.mark.parametrize("dtype", [B.SV_C128, B.SV_C64])
def test_one_qubit_runs_are_composed(lib, dtype):
    """Runs of one-qubit gates on one qubit become one gate (their product, FP64): the schedule keeps the
    circuit's meaning (replayed through the oracle in plan order) and launches fewer gate applications."""
    n = 14
    gates = rotation_runs_circuit(n, np.random.default_rng(12))
    plan = B.sv_plan_dry_run(n, dtype, gates)
    order = plan["order_of_gate"]
    assert sorted(order) == list(range(len(gates)))
    want = oracle.simulate(n, gates, 5)
    got = oracle.simulate(n, replay_in_plan_order(n, gates, plan), 5)
    assert np.max(np.abs(got - want)) < 1e-12
    steps = plan["step_of_gate"]
    # the three rotations of a run share one step; X X and S S^dagger compose to the identity and are dropped
    for i in range(0, 3 * n, 3):
        assert steps[i] == steps[i + 1] == steps[i + 2] >= 0
        assert order[i + 1] == order[i] + 1 and order[i + 2] == order[i] + 2
    assert all(steps[len(gates) - 4 + j] == -1 for j in range(4))


def test_fusion_reduces_launches(lib):
    w = C.random_workload(30, 20, seed=1002)
    plan = B.sv_plan_dry_run(30, B.SV_C128, w.gates)
    assert plan["nsteps"] < len(w.gates) // 5


def test_swaps_fold_into_layout(lib):
    """The QFT's closing SWAPs never become launches: they relabel qubits (Sec. VI.B)."""
    n = 10
    plan = B.sv_plan_dry_run(n, B.SV_C128, C.pack(C.qft(n)))
    assert list(plan["final_perm"]) == list(range(n))[::-1]


def _struct_fields(src, name):
    body = re.search(r"typedef struct " + name + r" \{(.*?)\} " + name + ";", src, re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        assert decl.startswith("uint64_t "), decl
        fields += [f.strip() for f in decl[len("uint64_t "):].split(",")]
    return fields


def test_stats_structs_match_binding():
    """The binding reads sv_batch_stats and sv_server_stats as arrays of uint64 in declaration order."""
    src = open(os.path.join(ROOT, "include", "sv.h")).read()
    assert _struct_fields(src, "sv_batch_stats") == B.BATCH_STATS_FIELDS
    assert _struct_fields(src, "sv_server_stats") == B.SERVER_STATS_FIELDS
