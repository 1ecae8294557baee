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


def test_counter_file_is_consistent():
    # the ncu counters the bench reports come from a summary file that names
    # the kernel source it was captured from; its entries are keyed by valid
    # schedules and their DRAM bytes stay within a factor of the algorithmic
    # bytes (below them where L2 keeps part of the input, above for re-reads)
    import json
    bench = _bench()
    if not os.path.exists(bench.COUNTERS):
        pytest.skip("no counter file")
    j = json.load(open(bench.COUNTERS))
    assert len(j["source_sha"]) == 16 and j["launches"]
    for r in j["launches"]:
        assert r["n1"] + r["n2"] == r["n"] and r["width"] in (1, 2, 4, 8, 16, 32)
        alg = bench.stage_bytes(r["n"], r["n1"], r["n2"], 4, True)[r["stage"]]
        if r.get("dram_bytes") is not None:
            assert 0.5 * alg <= r["dram_bytes"] <= 1.5 * alg
    # a changed kernel source makes the counters unavailable
    sched = {k: j["launches"][0][k] for k in ("n1", "n2", "width")}
    real = bench.kernel_source_hash
    try:
        bench.kernel_source_hash = lambda: "0" * 16
        assert bench.measured_counters(j["launches"][0]["stage"], j["launches"][0]["n"], sched)[0] == {}
    finally:
        bench.kernel_source_hash = real
    # with the current source, every record carries the L1 data-pipe total,
    # which includes the shared-memory wavefronts
    if j["source_sha"] == bench.kernel_source_hash():
        for r in j["launches"]:
            got, _ = bench.measured_counters(r["stage"], r["n"], {k: r[k] for k in ("n1", "n2", "width")})
            assert got["lsu_wavefronts"] >= got["smem_wavefronts"] > 0
