"""GPU parity of the enumeration kernels against the oracle (bit-exact counts).

Calls through the C ABI: bdc_subseq_counts (warp-cooperative subsequence
enumeration) and the engine's d-free precompute (bdc_bind ->
bdc_get_rep_stats).  Counts are integers and must match exactly.  S_k, the
sum of count*log2(count), is accumulated exactly on the GPU (an integer part
plus a 62-bit fraction), while the oracle sums its N_k terms one by one in
FP64; so S_k must match to 1e-12 relative plus the oracle's own recursive
summation bound (N_k + 4) u S_k (u = 2^-53).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2604_05867_b300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _bdc():
    import paper_2604_05867_b300 as bdc
    return bdc


def _check_S(S_gpu, S_ref, N):
    u = 2.0 ** -53
    tol = (1e-12 + (np.asarray(N, dtype=np.float64) + 4) * u) * np.abs(S_ref)
    assert np.all(np.abs(S_gpu - S_ref) <= tol)


@pytest.mark.parametrize("n", [1, 2, 3, 7, 10])
def test_counts_exhaustive(n):
    bdc = _bdc()
    xs = torch.arange(1 << n, dtype=torch.int64, device="cuda")
    N, S, _ = bdc.subseq_counts(n, xs)
    N = N.cpu().numpy()
    S = S.cpu().numpy()
    for x in range(1 << n):
        Nr, Sr, sc = oracle.subseq_stats(n, x)
        assert np.array_equal(N[x].astype(np.uint64), Nr), (n, x)
        _check_S(S[x], Sr, Nr)


@pytest.mark.parametrize("n", [1, 4, 8])
def test_embedding_counts_every_code(n):
    bdc = _bdc()
    for x in range(1 << n):
        _, _, E = bdc.subseq_counts(n, torch.tensor([x], dtype=torch.int64, device="cuda"), emb=True)
        cnt, _ = oracle.channel_row_bruteforce(n, x, 0.5)
        assert np.array_equal(E.cpu().numpy().astype(np.uint64), cnt), (n, x)


@pytest.mark.parametrize("n", [16, 20, 24, 26])
def test_counts_sampled_large(n):
    bdc = _bdc()
    xs = inputs.random_inputs(n, 6, seed=n)
    alt = int("".join("01"[i % 2] for i in range(n)), 2)
    xs = np.concatenate([xs, [0, (1 << n) - 1, alt]])
    N, S, _ = bdc.subseq_counts(n, torch.tensor(xs, device="cuda"))
    N = N.cpu().numpy()
    S = S.cpu().numpy()
    for i, x in enumerate(xs):
        Nr, Sr, sc = oracle.subseq_stats(n, int(x))
        assert np.array_equal(N[i].astype(np.uint64), Nr)
        _check_S(S[i], Sr, Nr)
    # the alternating string attains F_{n+3}-1 distinct subsequences
    a, b = 0, 1
    for _ in range(n + 3):
        a, b = b, a + b
    assert int(N[-1].sum()) == a - 1


@pytest.mark.parametrize("n", [5, 10, 14])
def test_engine_precompute_reps(n):
    bdc = _bdc()
    eng = bdc.Engine(n, [0.5], options=bdc.default_options(enable_literal=0))
    want = (2 ** n + 2 ** ((n + 1) // 2) + (2 ** (n // 2) if n % 2 == 0 else 0)) // 4
    assert eng.num_reps == want
    rng = np.random.default_rng(n)
    prev = -1
    idx = sorted(set(rng.integers(0, eng.num_reps, size=40).tolist()) | {0, eng.num_reps - 1})
    for r in idx:
        x, o, N, S = eng.rep_stats(r)
        rr, oo = oracle.orbit_rep(x, n)
        assert rr == x and o == oo and x > prev
        prev = x
        Nr, Sr, _ = oracle.subseq_stats(n, x)
        assert np.array_equal(N, Nr)
        _check_S(S, Sr, Nr)
    # output classes: class of every code is the class of its representative
    cls = eng.output_classes()
    ocls, reps, sizes = oracle.output_classes(min(n, 8)) if n <= 8 else (None, None, None)
    if ocls is not None:
        assert np.array_equal(cls[1:], ocls[1:])
    assert eng.num_output_classes == sum(
        ((2 ** k + 2 ** ((k + 1) // 2) + (2 ** (k // 2) if k % 2 == 0 else 0)) // 4) if k else 1
        for k in range(n + 1))
    eng.close()
