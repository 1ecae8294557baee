"""Pins for the oracle's Blahut-Arimoto, certificate and dual-bound code.

Anchors: closed forms C_1(d) = 1-d (Sec. 1), C_n(0) = n, C_n(1) = 0; the exact
channel values C_{n,1} = 1 and C_{n,n} = n printed in the paper's tables;
Arimoto's monotone convergence (Sec. 2.3 theorem); Lemma prob-vs-exact
(Sec. 2.2); subadditivity of C_n (Sec. 1); the symmetry theorem and the
orbit-reduced output formula (Appendix A); an independent scipy maximisation
of the mutual information; and central finite differences of the oracle's
own smoothed bound.
"""
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def mutual_info_bits(p, rows, ny):
    rowptr, col, val = rows
    q = np.zeros(ny)
    for x in range(len(rowptr) - 1):
        np.add.at(q, col[rowptr[x]:rowptr[x + 1]], p[x] * val[rowptr[x]:rowptr[x + 1]])
    I = 0.0
    for x in range(len(rowptr) - 1):
        v = val[rowptr[x]:rowptr[x + 1]]
        c = col[rowptr[x]:rowptr[x + 1]]
        m = v > 0
        I += p[x] * np.sum(v[m] * np.log2(v[m] / q[c[m]]))
    return I


@pytest.mark.parametrize("d", [0.1, 0.5, 0.9])
def test_bec_closed_form_n1(d):
    r = oracle.ba_bdc(1, d, 50)
    assert abs(r["lower"][-1] - (1 - d)) < 1e-14
    assert abs(r["upper"][-1] - (1 - d)) < 1e-14


@pytest.mark.parametrize("n", [1, 3, 6])
def test_noiseless_and_erased(n):
    r0 = oracle.ba_bdc(n, 0.0, 3)
    assert abs(r0["lower"][0] - n) < 1e-12 and abs(r0["upper"][0] - n) < 1e-12
    r1 = oracle.ba_bdc(n, 1.0, 3)
    assert abs(r1["lower"][0]) < 1e-12 and abs(r1["upper"][0]) < 1e-12


@pytest.mark.parametrize("n,d", [(4, 0.5), (6, 0.2), (8, 0.8)])
def test_ba_monotone_bracket_and_stop_statistic(n, d):
    r = oracle.ba_bdc(n, d, 200)
    lo, up, st = r["lower"], r["upper"], r["stat"]
    assert np.all(np.diff(lo) >= -1e-13)           # Arimoto: monotone
    assert np.all(lo <= up + 1e-13)                 # lower <= C <= upper
    # the paper's stopping statistic max_x log2(X^{t+1}/X^t) equals upper - lower
    assert np.allclose(st, up - lo, atol=1e-12)
    assert up[-1] - lo[-1] < up[0] - lo[0]


@pytest.mark.parametrize("n,d", [(2, 0.5), (3, 0.5), (3, 0.25)])
def test_ba_matches_scipy_maximisation(n, d):
    scipy_opt = pytest.importorskip("scipy.optimize")
    rows = oracle.bdc_rows(n, d)
    ny = 1 << (n + 1)

    def negI(t):
        e = np.exp(t - t.max())
        return -mutual_info_bits(e / e.sum(), rows, ny)

    best = None
    rng = np.random.default_rng(0)
    for _ in range(4):
        res = scipy_opt.minimize(negI, rng.normal(size=1 << n), method="Nelder-Mead",
                                 options=dict(maxiter=20000, xatol=1e-10, fatol=1e-14))
        res = scipy_opt.minimize(negI, res.x, method="BFGS", options=dict(gtol=1e-11))
        best = -res.fun if best is None else max(best, -res.fun)
    r = oracle.ba_bdc(n, d, 20000, tol=1e-12)
    assert r["lower"][-1] <= best + 1e-9 <= r["upper"][-1] + 2e-9
    assert abs(r["lower"][-1] - best) < 1e-7


def test_exact_channel_table_entries():
    # The paper's tables print C_{n,1} = 1 and C_{n,n} = n (n = 29, 31); these
    # are the closed forms for every n.  Fixture: tests/golden/paper_tables.txt
    fixtures = {}
    with open(os.path.join(GOLDEN, "paper_tables.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                n, k, v = line.split()
                fixtures[(int(n), int(k))] = float(v)
    assert fixtures[(29, 1)] == 1.0 and fixtures[(31, 1)] == 1.0
    assert fixtures[(29, 29)] == 29.0 and fixtures[(31, 31)] == 31.0
    for n in (3, 5, 7):
        for k in (1, n):
            rows = oracle.exact_rows(n, k)
            r = oracle.ba_sparse(rows, 1 << k, np.full(1 << n, 1.0 / (1 << n)), 3000, tol=1e-11)
            want = 1.0 if k == 1 else float(n)
            assert abs(r["lower"][-1] - want) < 1e-6 and r["upper"][-1] >= want - 1e-12


@pytest.mark.parametrize("n,d", [(4, 0.5), (5, 0.3)])
def test_prob_vs_exact_lemma(n, d):
    # Lemma prob-vs-exact: C_n(d) <= sum_k C(n,k) d^(n-k) (1-d)^k C_{n,k}
    lower_bdc = oracle.ba_bdc(n, d, 3000, tol=1e-10)["lower"][-1]
    rhs = 0.0
    for k in range(1, n + 1):
        rows = oracle.exact_rows(n, k)
        up = oracle.ba_sparse(rows, 1 << k, np.full(1 << n, 1.0 / (1 << n)), 3000, tol=1e-10)["upper"][-1]
        rhs += math.comb(n, k) * d ** (n - k) * (1 - d) ** k * up
    assert lower_bdc <= rhs + 1e-12


def test_subadditivity():
    # C_{a+b}(d) <= C_a(d) + C_b(d) (Sec. 1)
    d = 0.4
    lo5 = oracle.ba_bdc(5, d, 3000, tol=1e-10)["lower"][-1]
    up2 = oracle.ba_bdc(2, d, 3000, tol=1e-12)["upper"][-1]
    up3 = oracle.ba_bdc(3, d, 3000, tol=1e-12)["upper"][-1]
    assert lo5 <= up2 + up3 + 1e-12


def test_symmetry_theorem_and_orbit_formula():
    # Appendix A: from uniform X^(0), X^(t) and Y^(t) are invariant under
    # complement and reversal; Y(r) = sum_{x in R_n} X(x) |O_x|/|O_r| sum_{y in O_r} P(y|x)
    n, d = 7, 0.6
    r = oracle.ba_bdc(n, d, 25)
    p = r["p"]
    mask = (1 << n) - 1
    rev = lambda s, L: int(format(s, "0%db" % L)[::-1], 2) if L else 0
    for x in range(1 << n):
        for g in (x ^ mask, rev(x, n), rev(x, n) ^ mask):
            assert abs(p[g] - p[x]) <= 1e-13 * p[x]
    q = oracle.q_full(n, d, p)
    rowptr, col, val = oracle.bdc_rows(n, d)
    for c in range(2, 1 << (n + 1)):
        k = c.bit_length() - 1
        y = c ^ (1 << k)
        m = (1 << k) - 1
        for g in (y ^ m, rev(y, k), rev(y, k) ^ m):
            assert abs(q[(1 << k) | g] - q[c]) <= 1e-13 * q[c]
    # orbit-reduced formula, on output reps of length k = 4
    k = 4
    W = {}
    for x in range(1 << n):
        for e in range(rowptr[x], rowptr[x + 1]):
            W[(x, int(col[e]))] = val[e]
    in_reps = {}
    for x in range(1 << n):
        rx, ox = oracle.orbit_rep(x, n)
        in_reps[rx] = ox
    for y in range(1 << k):
        ry, oy = oracle.orbit_rep(y, k)
        if ry != y:
            continue
        orbit_y = {y, y ^ 15, rev(y, k), rev(y, k) ^ 15}
        s = 0.0
        for x, ox in in_reps.items():
            s += p[x] * ox / oy * sum(W.get((x, (1 << k) | yy), 0.0) for yy in orbit_y)
        assert abs(s - q[(1 << k) | y]) <= 1e-12 * q[(1 << k) | y]


@pytest.mark.parametrize("n,d", [(5, 0.5), (7, 0.75)])
def test_certify_is_valid_and_tight(n, d):
    r = oracle.ba_bdc(n, d, 400)
    q = oracle.q_full(n, d, r["p"])
    U, _ = oracle.certify(n, d, q)
    # for the q of X^(final), the dual value is the BA upper bound of that X
    r2 = oracle.ba_bdc(n, d, 1, p0=r["p"])
    assert abs(U - r2["upper"][0]) < 1e-12
    assert U >= r["lower"][-1] - 1e-13
    # scale invariance: certify(2q) = certify(q)
    U2, _ = oracle.certify(n, d, 2 * q)
    assert abs(U2 - U) < 1e-12
    # any positive q is valid: a uniform-over-codes q is a (loose) upper bound
    qu = np.ones(1 << (n + 1))
    qu[0] = 0
    Uu, _ = oracle.certify(n, d, qu)
    assert Uu >= r["lower"][-1]


@pytest.mark.parametrize("n,d", [(3, 0.6), (4, 0.8)])
def test_dual_bound_gradient_vs_central_differences(n, d):
    cls, reps, sizes = oracle.output_classes(n)
    rng = np.random.default_rng(0)
    theta = rng.normal(scale=0.5, size=len(reps))
    tau = 0.05
    F, g, gd = oracle.dual_bound(n, d, tau, theta, cls)
    h = 1e-6
    for i in range(len(reps)):
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (oracle.dual_bound(n, d, tau, tp, cls, grad=False)[0]
              - oracle.dual_bound(n, d, tau, tm, cls, grad=False)[0]) / (2 * h)
        assert abs(fd - g[i]) < 1e-6 * max(1.0, abs(g[i]))
    fdd = (oracle.dual_bound(n, d + h, tau, theta, cls, grad=False)[0]
           - oracle.dual_bound(n, d - h, tau, theta, cls, grad=False)[0]) / (2 * h)
    assert abs(fdd - gd) < 1e-5 * max(1.0, abs(gd))
    # tau-LSE brackets the max: max D <= F <= max D + tau*n
    q = np.exp(theta[cls] - theta.max())
    q[0] = 0
    q /= q.sum()
    Dmax = oracle.D_full(n, d, q).max()
    assert Dmax - 1e-12 <= F <= Dmax + tau * n + 1e-12
