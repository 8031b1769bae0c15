"""Element-wise parity with the FP64 oracle at the benchmark's own configuration.

The bench times the 20-layer random circuit (Haar U(2) on every qubit, then CNOTs on a random perfect
matching; seed 1002) on n = 30 qubits from |0...0>, with the library's launch configuration: chunks of 2^12
(complex128) / 2^13 (complex64) amplitudes, 16 percent of the complex128 chunks in native FP64 beside the
double-float CTAs (or dense tensor-core blocks, which the autotuner may choose), the product-state start and
graph replay.  Here the same circuit runs the same way and
every amplitude is compared with the oracle's state vector (Algorithm 1 of Sec. V.B applied gate by gate in
FP64 on the host).  The oracle needs 16 GiB of host memory at n = 30 and a few minutes on the host cores
(collapse(2) threading); on a host with less memory the test runs n = 28 with the same options.

Bound (written here): complex128 max-abs <= 1e-12 and 1 - F <= 1e-12 in both arithmetic modes; complex64
max-abs <= 1e-4 max|psi| and 1 - F <= 1e-8.  The measured errors (absolute and relative to max|psi|) are
printed for the record.
"""
import os

import numpy as np
import pytest

import circuits as C
import oracle

pytestmark = pytest.mark.gpu
B = pytest.importorskip("paper_1801_01037_gb300")._binding

SEED = 1002
DEPTH = 20
SLICE = 1 << 24  # amplitudes compared per read-back slice


def host_available_bytes():
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) * 1024
    except OSError:
        pass
    return 0


def bench_n():
    # oracle state (16 B x 2^n) plus slices and numpy temporaries; n = 30 wants about 24 GiB free
    return 30 if host_available_bytes() >= (24 << 30) else 28


@pytest.fixture(scope="module")
def reference():
    from paper_1801_01037_gb300 import build
    build.build()
    B.load()
    n = bench_n()
    w = C.random_workload(n, DEPTH, seed=SEED)
    psi = oracle.simulate(n, w.gates, 0, threads=os.cpu_count() or 1, collapse=True)
    return n, w, psi


# (name, dtype, arithmetic, chunk qubits, SV_OPT_TENSOR_BLOCKS): the autotuner picks between the per-gate
# passes and dense tensor-core blocks of at least 4 dense gate updates, so both are checked
CASES = [
    ("c128_df32_share16", B.SV_C128, B.SV_ARITH_DF32, 12, 0),
    ("c128_df32_tensor_blocks", B.SV_C128, B.SV_ARITH_DF32, 12, 4),
    ("c128_f64", B.SV_C128, B.SV_ARITH_F64, 12, 0),
    ("c64", B.SV_C64, B.SV_ARITH_AUTO, 13, 0),
    ("c64_tensor_blocks", B.SV_C64, B.SV_ARITH_AUTO, 13, 4),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_bench_circuit_matches_oracle_elementwise(reference, case):
    name, dtype, arith, k, tensor_blocks = case
    n, w, want = reference
    h = B.sv_create(n, dtype)
    try:
        if dtype == B.SV_C128:
            B.sv_set_option(h, B.SV_OPT_ARITH, arith)
            B.sv_set_option(h, B.SV_OPT_F64_SHARE, 16)
        B.sv_set_option(h, B.SV_OPT_CHUNK_QUBITS, k)
        B.sv_set_option(h, B.SV_OPT_TENSOR_BLOCKS, tensor_blocks)
        B.sv_init_basis(h, 0)
        B.sv_apply_circuit_graph(h, w.gates)
        stats = B.sv_last_plan_stats(h)
        assert stats["absorbed"] > 0, "the bench's product-state start should fold the first layer"
        blocks = B.sv_last_plan_blocks(h)["blocks"]
        assert (blocks > 0) == (tensor_blocks > 0), blocks
        max_err, max_ref, dot, n_got, n_want = 0.0, 0.0, 0j, 0.0, 0.0
        for first in range(0, 1 << n, SLICE):
            got = B.sv_read_amplitudes(h, first, SLICE).astype(np.complex128)
            ref = want[first:first + SLICE]
            max_err = max(max_err, float(np.max(np.abs(got - ref))))
            max_ref = max(max_ref, float(np.max(np.abs(ref))))
            dot += np.vdot(ref, got)
            n_got += float(np.vdot(got, got).real)
            n_want += float(np.vdot(ref, ref).real)
        infid = max(0.0, 1.0 - abs(dot) ** 2 / (n_got * n_want))
        print(f"\n[bench parity] n={n} {name}: max-abs {max_err:.3e}, max-abs / max|psi| {max_err / max_ref:.3e}, "
              f"1-F {infid:.3e}, passes {stats['passes']}, folded {stats['absorbed']}, tensor blocks {blocks}")
        if dtype == B.SV_C128:
            assert max_err <= 1e-12 and infid <= 1e-12, (max_err, infid)
        else:
            assert max_err <= 1e-4 * max_ref and infid <= 1e-8, (max_err, max_ref, infid)
    finally:
        B.sv_destroy(h)
