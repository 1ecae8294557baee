"""Pins for the oracle's channel and enumeration code (CPU only).

Each test checks the oracle against something other than itself: the
brute-force definition of BDC_d (all 2^n deletion patterns), binomial closed
forms, the paper's Lemma num_superseq (Sec. 5), the bijection theorems of
Sec. 4.2 and Sec. 5.2, itertools' combination order, and the classical
extremes of the number of distinct subsequences.
"""
import itertools
import math

import numpy as np
import pytest

import oracle


def bits(s, L):
    return [(s >> (L - 1 - i)) & 1 for i in range(L)]


def is_subseq(y, k, x, n):
    """Greedy subsequence test on explicit symbol lists."""
    ys, xs = bits(y, k), bits(x, n)
    j = 0
    for b in xs:
        if j < k and ys[j] == b:
            j += 1
    return j == k


@pytest.mark.parametrize("n", [1, 2, 3, 5, 7])
def test_embed_count_matches_bruteforce_patterns(n):
    # DP count == number of deletion patterns producing y (definition, Sec. 2.2)
    for x in range(1 << n):
        cnt, _ = oracle.channel_row_bruteforce(n, x, 0.5)
        for c in range(1, 1 << (n + 1)):
            k = c.bit_length() - 1
            assert oracle.embed_count(n, x, k, c ^ (1 << k)) == int(cnt[c])


@pytest.mark.parametrize("n", [1, 4, 8, 10])
def test_pattern_counts_sum_to_binomial(n):
    # each length-k keep set is one pattern: sum_{|y|=k} Count(y,x) = C(n,k)
    rng = np.random.default_rng(0)
    for x in rng.integers(0, 1 << n, size=8):
        cnt, W = oracle.channel_row_bruteforce(n, int(x), 0.3)
        per_k = np.zeros(n + 1, np.int64)
        for c in range(1, 1 << (n + 1)):
            per_k[c.bit_length() - 1] += int(cnt[c])
        assert [int(v) for v in per_k] == [math.comb(n, k) for k in range(n + 1)]
        # rows of the channel sum to one
        assert abs(W.sum() - 1.0) < 1e-13


@pytest.mark.parametrize("n", [1, 3, 6, 9])
def test_subseq_stats_match_bruteforce(n):
    for x in range(1 << n):
        cnt, _ = oracle.channel_row_bruteforce(n, x, 0.5)
        N, S, sc = oracle.subseq_stats(n, x)
        for k in range(n + 1):
            codes = range(1 << k, 1 << (k + 1))
            nz = [int(cnt[c]) for c in codes if cnt[c] > 0]
            assert int(N[k]) == len(nz)
            assert int(sc[k]) == math.comb(n, k)
            assert abs(S[k] - sum(v * math.log2(v) for v in nz)) <= 1e-9 * max(1.0, S[k])


@pytest.mark.parametrize("n", [1, 2, 5, 8, 11])
def test_total_distinct_subsequences_closed_form(n):
    # sum_x sum_k N_{x,k} = sum_y #supersequences(y) = sum_k 2^k sum_{i<=n-k} C(n,i)
    # (Lemma num_superseq, Sec. 5), which equals 2*3^n - 2^n.
    tot = 0
    for x in range(1 << n):
        N, _, _ = oracle.subseq_stats(n, x)
        tot += int(N.sum())
    lemma = sum((1 << k) * sum(math.comb(n, i) for i in range(n - k + 1)) for k in range(n + 1))
    assert tot == lemma == 2 * 3 ** n - 2 ** n


def fib(m):
    a, b = 0, 1
    for _ in range(m):
        a, b = b, a + b
    return a


@pytest.mark.parametrize("n", [1, 2, 3, 6, 10, 14])
def test_distinct_subsequence_extremes(n):
    # constant strings have n+1 distinct subsequences (the minimum); the
    # alternating string has F_{n+3}-1 (the maximum).
    alt = int("".join("01"[i % 2] for i in range(n)), 2)
    assert int(oracle.subseq_stats(n, 0)[0].sum()) == n + 1
    assert int(oracle.subseq_stats(n, alt)[0].sum()) == fib(n + 3) - 1
    if n <= 10:
        vals = [int(oracle.subseq_stats(n, x)[0].sum()) for x in range(1 << n)]
        assert min(vals) == n + 1 and max(vals) == fib(n + 3) - 1


@pytest.mark.parametrize("n", [1, 4, 7, 9])
def test_unrank_is_lexicographic_bijection(n):
    # Sec. 4.2 theorem: j -> unrank(x,k,j) is a bijection onto the distinct
    # length-k subsequences; the order is lexicographic.
    for x in range(1 << n):
        _, cnt = oracle.nextpos_cnt(n, x, n)
        for k in range(1, n + 1):
            truth = sorted(y for y in range(1 << k) if is_subseq(y, k, x, n))
            assert int(cnt[0, k]) == len(truth)
            got = [oracle.unrank(n, x, k, j) for j in range(len(truth))]
            assert got == truth
            assert oracle.unrank(n, x, k, len(truth)) is None


def test_nextpos_definition():
    n, x = 9, 0b011010011
    np_, _ = oracle.nextpos_cnt(n, x, 3)
    xs = bits(x, n)
    for i in range(n + 1):
        for b in (0, 1):
            want = next((p for p in range(i, n) if xs[p] == b), n)
            assert np_[i, b] == want


@pytest.mark.parametrize("n", [1, 3, 6, 9])
def test_subset_unrank_order(n):
    # Sec. 5.1 Alg. subsetUnrank over the 0-based ground set enumerates the
    # w-subsets in lexicographic order of their sorted element lists, which is
    # exactly itertools.combinations' order.
    for w in range(n + 1):
        combos = list(itertools.combinations(range(n), w))
        assert [tuple(oracle.subset_unrank(n, w, j)) for j in range(len(combos))] == combos


@pytest.mark.parametrize("n", [1, 2, 4, 6, 8])
def test_num_superseq_and_recsuperseq_bijection(n):
    # Lemma num_superseq, and the Sec. 5.2 theorem with the fixed reading of
    # the unmatched tail (positions after y is exhausted repeat y_{k-1}).
    for k in range(1, n + 1):
        total = sum(math.comb(n, i) for i in range(n - k + 1))
        for y in range(1 << k):
            sup = {x for x in range(1 << n) if is_subseq(y, k, x, n)}
            assert len(sup) == total
            got = [oracle.recsuperseq(i, n, k, y, fixed=True) for i in range(total)]
            assert len(set(got)) == total and set(got) == sup


def test_recsuperseq_as_printed_is_not_injective():
    # With the tail filled by 0 as printed, n=2, y="1" maps i=0 and i=2 to the
    # same string "10" and never produces "11".
    got = [oracle.recsuperseq(i, 2, 1, 1, fixed=False) for i in range(3)]
    assert got[0] == got[2] == 0b10 and 0b11 not in got


@pytest.mark.parametrize("L", [1, 2, 5, 8])
def test_orbits(L):
    # reps are the smallest member; orbit sizes add up to 2^L; the number of
    # reps matches Burnside's count (2^L + 2^ceil(L/2) + [L even] 2^(L/2)) / 4
    reps = {}
    for s in range(1 << L):
        r, o = oracle.orbit_rep(s, L)
        mask = (1 << L) - 1
        rv = int("".join(str(b) for b in reversed(bits(s, L))), 2)
        members = {s, s ^ mask, rv, rv ^ mask}
        assert r == min(members) and o == len(members)
        reps[r] = o
    assert sum(reps.values()) == 1 << L
    burnside = ((1 << L) + (1 << ((L + 1) // 2)) + ((1 << (L // 2)) if L % 2 == 0 else 0)) // 4
    assert len(reps) == burnside


@pytest.mark.parametrize("n,d", [(4, 0.3), (6, 0.7), (8, 0.5)])
def test_q_and_D_definitions_agree(n, d):
    rng = np.random.default_rng(1)
    p = rng.dirichlet(np.ones(1 << n))
    rows = oracle.bdc_rows(n, d)
    rowptr, col, val = rows
    # q: scatter over pairs == point sums over all inputs == sparse matvec
    qf = oracle.q_full(n, d, p)
    qd = np.zeros(1 << (n + 1))
    for x in range(1 << n):
        for e in range(rowptr[x], rowptr[x + 1]):
            qd[col[e]] += p[x] * val[e]
    assert np.allclose(qf, qd, rtol=1e-13, atol=0)
    for c in rng.integers(1, 1 << (n + 1), size=20):
        assert abs(oracle.q_point(n, d, p, int(c)) - qf[c]) <= 1e-13 * max(qf[c], 1e-300)
    # D from the walk == D from brute-force rows
    Df = oracle.D_full(n, d, qf)
    for x in range(1 << n):
        s = 0.0
        for e in range(rowptr[x], rowptr[x + 1]):
            s += val[e] * math.log2(val[e] / qf[col[e]])
        assert abs(Df[x] - s) <= 1e-12 * max(1.0, abs(s))
