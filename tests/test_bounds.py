"""Bound post-processing (Sec. 2.2 Lemma prob-vs-exact; Sec. 6 Lemma
worse-UB and Lemma convex), host routines of the library, no GPU.

Pins: the paper's own tables -- its C(d) table is Lemma prob-vs-exact
applied to its printed C_{29,k} / C_{31,k} tables, its C_{31,k} entries for
19 <= k <= 29 are Lemma worse-UB with s = 2 applied to the C_{29,k} table,
and its high-noise constant 0.3578 is Lemma convex applied to its C(0.64)
entry (tests/golden/paper_table_*.txt); closed forms (C_{n,n} = n,
C_{n,1} = 1, C_{n,0} = 0, C_1(d) = 1 - d); and the inequalities themselves on
capacities the oracle computes by BA at small n."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2604_05867_b300 import bounds

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _table(name):
    rows = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.split("#")[0].split()
        if len(line) == 2:
            rows[int(line[0])] = float(line[1])
    return rows


def _cd_table():
    rows, ratio = [], None
    for line in open(os.path.join(GOLDEN, "paper_table_Cd.txt")):
        f = line.split("#")[0].split()
        if len(f) == 3 and f[0] == "ratio":
            ratio = (float(f[1]), float(f[2]))
        elif len(f) == 3:
            rows.append((float(f[0]), float(f[1]), int(f[2])))
    return rows, ratio


def _vec(n, table):
    v = np.zeros(n + 1)
    for k, c in table.items():
        v[k] = c
    return v


def test_cd_table_is_prob_vs_exact_of_the_ck_tables():
    C = {29: _vec(29, _table("paper_table_C29k.txt")), 31: _vec(31, _table("paper_table_C31k.txt"))}
    rows, _ = _cd_table()
    assert len(rows) == 19
    for d, printed, n in rows:
        v = bounds.prob_vs_exact(n, d, C[n]) / n
        assert bounds.ceil4(v) == pytest.approx(printed, abs=1e-12), (d, v, printed)
    # and the printed choice of n is the better of the two for every d
    best = bounds.cd_table([r[0] for r in rows], C)
    for (d, printed, n), (_, v, nb) in zip(rows, best):
        assert nb == n and bounds.ceil4(v) == pytest.approx(printed, abs=1e-12)


def test_c31_tail_is_worse_ub_of_the_c29_table():
    C29 = _vec(29, _table("paper_table_C29k.txt"))
    C31 = _table("paper_table_C31k.txt")
    C2 = [0.0, 1.0, 2.0]
    for k in range(19, 30):
        v = bounds.split_bound(31, k, 2, C2, C29)
        # the paper applied the lemma to its unrounded C_{29,k} values: the
        # printed entry is within one unit of the last decimal
        assert abs(v - C31[k]) <= 1.5e-4, (k, v, C31[k])


def test_high_noise_constant():
    _, (d_prime, printed) = _cd_table()
    C = {r[0]: r[1] for r in _cd_table()[0]}
    _, ratio = bounds.high_noise(d_prime, C[d_prime])
    assert bounds.ceil4(ratio) == printed
    cd, _ = bounds.high_noise(d_prime, C[d_prime], 0.9)
    assert cd == pytest.approx(ratio * 0.1, rel=1e-15)
    cd1, _ = bounds.high_noise(d_prime, C[d_prime], 1.0)
    assert cd1 == 0.0


@pytest.mark.parametrize("n,s", [(5, 1), (8, 3), (29, 2)])
def test_split_bound_closed_forms(n, s):
    # exact values C_{m,0} = 0, C_{m,1} = 1, C_{m,m} = m (m >= 1) reproduce
    # C_{n,n} = n and C_{n,1} = 1 with equality
    Cs = np.zeros(s + 1)
    Cns = np.zeros(n - s + 1)
    Cs[1], Cs[s] = 1.0, float(s)
    Cns[1], Cns[n - s] = 1.0, float(n - s)
    assert bounds.split_bound(n, n, s, Cs, Cns) == pytest.approx(n, rel=1e-15)
    assert bounds.split_bound(n, 1, s, Cs, Cns) == pytest.approx(1.0, rel=1e-15)
    assert bounds.split_bound(n, 0, s, Cs, Cns) == 0.0


@pytest.mark.parametrize("d", [0.0, 0.2, 0.5, 0.93, 1.0])
def test_prob_vs_exact_closed_forms(d):
    # n = 1: C_1(d) <= (1 - d) C_{1,1} = 1 - d; the trivial bounds C_{n,k} <= k
    # give n (1 - d), the mean number of kept symbols
    assert bounds.prob_vs_exact(1, d, [0.0, 1.0]) == pytest.approx(1 - d, abs=1e-16)
    n = 12
    assert bounds.prob_vs_exact(n, d, np.arange(n + 1, dtype=float)) == pytest.approx(n * (1 - d), rel=1e-14,
                                                                                      abs=1e-15)


def _exact_capacity(n, k, T=3000):
    r = oracle.ba_sparse(oracle.exact_rows(n, k), 1 << k, np.full(1 << n, 1.0 / (1 << n)), T, tol=1e-11)
    return r["lower"][-1], r["upper"][-1]


def test_lemmas_hold_on_oracle_capacities():
    # exact-channel capacities of small n by the oracle's BA (lower, upper
    # bracket the capacity): Lemma worse-UB and Lemma prob-vs-exact hold
    caps = {}
    for m in range(1, 7):
        for k in range(0, m + 1):
            caps[(m, k)] = (0.0, 0.0) if k == 0 else _exact_capacity(m, k)
    assert caps[(6, 1)][1] == pytest.approx(1.0, abs=1e-9) and caps[(6, 6)][0] == pytest.approx(6.0, abs=1e-9)
    n = 6
    for s in (1, 2, 3):
        Cs = [caps[(s, i)][1] for i in range(s + 1)]
        Cns = [caps[(n - s, j)][1] for j in range(n - s + 1)]
        for k in range(n + 1):
            assert caps[(n, k)][0] <= bounds.split_bound(n, k, s, Cs, Cns) + 1e-9
    Cnk = [caps[(n, k)][1] for k in range(n + 1)]
    for d in (0.1, 0.5, 0.8):
        lower_bdc = oracle.ba_bdc(n, d, 3000, tol=1e-11)["lower"][-1]
        assert lower_bdc <= bounds.prob_vs_exact(n, d, Cnk) + 1e-9


def test_ck_table_format():
    t = bounds.ck_table(4, {1: 1.0, 2: 1.23451, 4: 4.0})
    assert t.splitlines()[1:] == ["1 & 1.0000 \\\\", "2 & 1.2346 \\\\", "4 & 4.0000 \\\\"]
