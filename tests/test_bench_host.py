"""Host-side arithmetic of bench.py (no GPU): the pair count behind the metric,
the algorithmic-bytes model behind the roofline, and the consistency of the
ncu tables it reads."""
import importlib.util
import os

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("n", [1, 2, 5, 8])
def test_pairs_per_iteration_counts_distinct_outputs(n):
    # the metric's unit: (input, distinct output) pairs, summed over every input
    # by the oracle's own distinct-subsequence counts
    bench = _bench()
    total = 0
    for x in range(1 << n):
        N, _, _ = oracle.subseq_stats(n, x)
        total += int(np.sum(N))
    assert bench.pairs_per_iteration(n) == total


def test_stage_bytes_model():
    bench = _bench()
    n, E = 24, 4
    full = bench.stage_bytes(n, 11, 13, E, False)
    half = bench.stage_bytes(n, 11, 13, E, True)
    for k in full:
        assert half[k] * 2 == full[k]
    N = (1 << n) // 2
    # a stepped FP32 iteration: forward rows, combine, adjoint rows, the one-pass boundary
    it = sum(half[k] for k in ("rows_fwd", "combine", "rows_adj", "cols_step"))
    assert it == 19 * N * E
    assert half["cols_step"] == 201326592  # the bench line's algorithmic_bytes at n = 24


def test_measured_tables_are_consistent():
    bench = _bench()
    for table in (bench.MEASURED_TRAFFIC, bench.MEASURED_SMEM_WAVEFRONTS):
        for (stage, n, n1, n2, w), v in table.items():
            assert n1 + n2 == n and w in (1, 2, 4, 8, 16, 32) and v > 0
            assert stage in bench.stage_bytes(n, n1, n2, 4, True)
    for (stage, n, n1, n2, w), v in bench.MEASURED_TRAFFIC.items():
        # DRAM bytes of one launch stay within a factor of the algorithmic bytes
        # (below them where L2 keeps part of the input, above them for re-reads)
        alg = bench.stage_bytes(n, n1, n2, 4, True)[stage]
        assert 0.5 * alg <= v <= 1.5 * alg
