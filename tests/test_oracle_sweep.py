"""Pins for the oracle's factorised sweep (O2): the output marginal, the
transposed pass and the Blahut-Arimoto run built on them must agree with the
oracle's plain definitions (q_full: the scatter over every (x, y) pair;
D_full: the divergence summed term by term; ba_bdc: BA on the channel rows
built from all 2^n deletion patterns), with the textbook embedding DP
(embed_count) for the counting form, and with the closed form
sum_y W(y|x) = 1 (Sec. 2.2: each x yields exactly one output)."""
import math

import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("n", [1, 2, 5, 8, 10])
@pytest.mark.parametrize("d", [0.0, 0.25, 0.7, 1.0])
def test_sweep_q_matches_definition(n, d):
    rng = np.random.default_rng(n)
    p = rng.dirichlet(np.ones(1 << n))
    q_ref = oracle.q_full(n, d, p)
    q = oracle.sweep_q(n, d, p)
    assert q[0] == 0.0
    assert np.all(np.abs(q - q_ref) <= 1e-13 * np.maximum(q_ref, 1e-300))
    assert abs(q.sum() - 1.0) < 1e-13


def test_sweep_counts_match_embedding_dp():
    n = 7
    for x in range(1 << n):
        e = np.zeros(1 << n)
        e[x] = 1.0
        c = oracle.sweep_q(n, 0.0, e, counts=True)
        for code in range(1, 2 << n):
            k = code.bit_length() - 1
            assert c[code] == oracle.embed_count(n, x, k, code ^ (1 << k))


@pytest.mark.parametrize("n,d", [(6, 0.3), (9, 0.5), (10, 0.85)])
def test_sweep_adjoint_is_the_transpose(n, d):
    # G = W L row by row: rows of W sum to one, and against the brute-force rows
    G1 = oracle.sweep_G(n, d, np.ones(2 << n))
    assert np.all(np.abs(G1 - 1.0) < 1e-13)
    rng = np.random.default_rng(n + 1)
    L = rng.normal(size=2 << n)
    G = oracle.sweep_G(n, d, L)
    for x in rng.integers(0, 1 << n, size=8):
        _, W = oracle.channel_row_bruteforce(n, int(x), d)
        assert abs(G[x] - np.dot(W[1:], L[1:])) <= 1e-12 * (1.0 + np.abs(L).max())


@pytest.mark.parametrize("n,d", [(3, 0.5), (8, 0.2), (10, 0.65)])
def test_sweep_D_matches_definition(n, d):
    rng = np.random.default_rng(2 * n)
    p = rng.dirichlet(np.ones(1 << n))
    q = oracle.q_full(n, d, p)
    S = oracle.subseq_S_all(n)
    D = oracle.D_sweep(n, d, q, S)
    D_ref = oracle.D_full(n, d, q)
    assert np.all(np.abs(D - D_ref) <= 1e-12 * np.maximum(1.0, np.abs(D_ref)))


def test_subseq_S_all_matches_per_input_walk():
    # S is walked on the orbit representative and copied to the orbit (the
    # symmetry theorem of Appendix A); a member's own walk sums the same terms
    # in another order
    n = 9
    S = oracle.subseq_S_all(n)
    for x in range(1 << n):
        _, Sx, _ = oracle.subseq_stats(n, x)
        assert np.all(np.abs(S[x] - Sx) <= 1e-13 * np.maximum(1.0, Sx))


@pytest.mark.parametrize("n", [4, 7, 10, 13])
def test_orbit_reps_burnside(n):
    reps, idx = oracle.orbit_reps(n)
    burnside = ((1 << n) + (1 << ((n + 1) // 2)) + ((1 << (n // 2)) if n % 2 == 0 else 0)) // 4
    assert len(reps) == burnside
    assert np.array_equal(reps[idx[reps]], reps)


@pytest.mark.parametrize("n,d", [(5, 0.5), (8, 0.3)])
def test_ba_sweep_matches_ba_on_brute_force_rows(n, d):
    T = 30
    ref = oracle.ba_bdc(n, d, T)
    r = oracle.ba_sweep(n, d, T)
    assert np.all(np.abs(r["lower"] - ref["lower"]) <= 1e-12)
    assert np.all(np.abs(r["upper"] - ref["upper"]) <= 1e-12)
    assert np.all(np.abs(r["p"] - ref["p"]) <= 1e-10 * ref["p"])


def test_neg_entropy_rows_closed_forms():
    # d = 0: W(x|x) = 1, no entropy; d = 1: only the empty output
    n = 6
    S = oracle.subseq_S_all(n)
    assert np.all(oracle.neg_entropy_rows(n, 0.0, S) == 0.0)
    assert np.all(oracle.neg_entropy_rows(n, 1.0, S) == 0.0)
    # the constant string: every length-k output is 0^k with C(n,k) embeddings,
    # so the output length is Binomial(n, 1-d) and H = h(Binomial)
    d = 0.4
    b = np.array([math.comb(n, k) * d ** (n - k) * (1 - d) ** k for k in range(n + 1)])
    h = -np.sum(b * np.log2(b))
    assert abs(-oracle.neg_entropy_rows(n, d, S)[0] - h) < 1e-13
