"""Exact deletion channels BDC_{n,k} (Sec. 2.2) on the GPU: length-mixture
instances (bdc_create_lengths) with a one-hot length distribution.

Against the oracle: BA on the channel rows P_{n,k}(y|x) = Count(y,x)/C(n,k)
built by the textbook embedding DP (exact_rows + ba_sparse), per iteration
(bounds 1e-11) and per element of p (1e-9), for every k at n <= 8; the
certified bound against the dual value of the same input computed from those
rows (U in [U_oracle - 1e-12, U_oracle + 1e-6]); the closed forms
C_{n,0} = 0, C_{n,1} = 1, C_{n,n} = n; Lemma prob-vs-exact against the
direct BDC_d engine (sum_k b_k U_{n,k} >= the BDC_d lower bound); and a
length mixture with BDC_d's own weights reproduces BDC_d."""
from math import comb

import numpy as np
import pytest

import oracle
from paper_2604_05867_b300 import bounds

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _bdc():
    import paper_2604_05867_b300 as bdc
    return bdc


def _exact_engine(n, ks, **kw):
    bdc = _bdc()
    return bdc.Engine(n, lengths=bounds.exact_lengths(n, ks), options=bdc.default_options(**kw))


def _oracle_rows_dual(n, k, p):
    """max_x D(P(.|x) || q/sum q) with q = P^T p, from the oracle's rows."""
    rowptr, col, val = oracle.exact_rows(n, k)
    q = np.zeros(1 << k)
    for x in range(1 << n):
        np.add.at(q, col[rowptr[x]:rowptr[x + 1]], p[x] * val[rowptr[x]:rowptr[x + 1]])
    best = -np.inf
    for x in range(1 << n):
        v = val[rowptr[x]:rowptr[x + 1]]
        c = col[rowptr[x]:rowptr[x + 1]]
        best = max(best, float(np.sum(v * np.log2(v / q[c]))))
    return best + np.log2(q.sum())


@pytest.mark.parametrize("n", [3, 6, 8])
@pytest.mark.parametrize("impl", ["sweep", "literal"])
def test_exact_channel_ba_matches_oracle(n, impl):
    T = 40
    ks = list(range(0, n + 1))
    eng = _exact_engine(n, ks)
    eng.iterate(T, -1.0, "fp64", impl)
    P = eng.get_p()
    for z, k in enumerate(ks):
        ref = oracle.ba_sparse(oracle.exact_rows(n, k), 1 << k, np.full(1 << n, 1.0 / (1 << n)), T)
        lo, up = eng.history(z)
        assert np.all(np.abs(lo - ref["lower"]) <= 1e-11), (k, lo[:3], ref["lower"][:3])
        assert np.all(np.abs(up - ref["upper"]) <= 1e-11)
        assert np.all(np.abs(P[z] - ref["p"]) <= 1e-9 * ref["p"])
    eng.close()


@pytest.mark.parametrize("n,ks", [(9, [2, 5, 8]), (10, [1, 4, 7, 10])])
def test_exact_channel_certificate_matches_oracle(n, ks):
    eng = _exact_engine(n, ks)
    eng.iterate(60, -1.0, "fp32", "sweep")
    c = eng.certify()
    P = eng.get_p()
    eps = 2.0 ** -30
    for z, k in enumerate(ks):
        pt = (1 - eps) * P[z] + eps / (1 << n)
        U_ref = _oracle_rows_dual(n, k, pt)
        assert U_ref - 1e-12 <= c["upper"][z] <= U_ref + 1e-6, (k, c["upper"][z], U_ref)
        assert 0 < c["margin"][z] < 1e-6
    eng.close()


@pytest.mark.parametrize("n", [10, 16])
def test_exact_channel_closed_forms(n):
    # C_{n,0} = 0 (one output), C_{n,1} = 1 (one random symbol), C_{n,n} = n
    res = bounds.exact_capacities(n, [0, 1, n], iters=300, tol=1e-7, precision="fp64")
    assert 0.0 <= res[0]["upper"] < 1e-9
    assert 1.0 - 1e-9 <= res[1]["upper"] < 1.0 + 1e-6
    assert n - 1e-9 <= res[n]["upper"] < n + 1e-6


def test_prob_vs_exact_against_direct_engine():
    bdc = _bdc()
    n = 12
    res = bounds.exact_capacities(n, iters=400, tol=1e-6)
    Cnk = np.zeros(n + 1)
    for k, r in res.items():
        Cnk[k] = r["upper"]
        assert r["lower"] <= r["upper"]
    for d in (0.2, 0.5, 0.8):
        eng = bdc.Engine(n, [d], options=bdc.default_options(enable_literal=0))
        lo, up, _ = eng.iterate(400, 1e-6, "fp32", "sweep")
        cert = eng.certify()
        eng.close()
        composed = bounds.prob_vs_exact(n, d, Cnk)
        assert composed >= lo[0]
        # the lemma's bound is never below the capacity, which the direct
        # certificate brackets from above to within its own gap
        assert composed >= cert["lower"][0]


def test_length_mixture_with_bdc_weights_is_bdc():
    bdc = _bdc()
    n, d, T = 11, 0.35, 25
    b = np.array([[comb(n, k) * d ** (n - k) * (1 - d) ** k for k in range(n + 1)]])
    a = bdc.Engine(n, lengths=b, options=bdc.default_options(enable_literal=0))
    r = bdc.Engine(n, [d], options=bdc.default_options(enable_literal=0))
    a.iterate(T, -1.0, "fp64", "sweep")
    r.iterate(T, -1.0, "fp64", "sweep")
    la, ua = a.history(0)
    lr, ur = r.history(0)
    assert np.all(np.abs(la - lr) <= 1e-12) and np.all(np.abs(ua - ur) <= 1e-12)
    assert np.all(np.abs(a.get_p() - r.get_p()) <= 1e-11 * r.get_p())
    ca, cr = a.certify(), r.certify()
    assert abs(ca["upper"][0] - cr["upper"][0]) <= 1e-9
    a.close()
    r.close()


def test_exact_channel_fp32_stepped_matches_fp64():
    # n = 18, 11 + 7 split, 4 columns: the stepped register-resident column
    # kernels on exact channels (weights zero at every length but k)
    bdc = _bdc()
    n, ks, T = 18, [5, 9, 14], 4
    kw = dict(sched_n2_fp32=7, sched_w_fp32=4, enable_literal=0)
    a = _exact_engine(n, ks, **kw)
    assert a.schedule("fp32") == {"n1": 11, "n2": 7, "width": 4}
    b = _exact_engine(n, ks, use_regsteps=0, fuse_update=0, use_half=0, enable_literal=0)
    a.iterate(T, -1.0, "fp32", "sweep")
    b.iterate(T, -1.0, "fp64", "sweep")
    for z in range(len(ks)):
        la, ua = a.history(z)
        lb, ub = b.history(z)
        assert np.all(np.abs(la - lb) <= 2e-5 * np.abs(lb)) and np.all(np.abs(ua - ub) <= 2e-5 * np.abs(ub))
    assert np.all(np.abs(a.get_p() - b.get_p()) <= 2e-3 * b.get_p())
    a.close()
    b.close()


def test_dual_gradient_in_d_is_rejected_for_length_mixtures():
    bdc = _bdc()
    eng = _exact_engine(8, [4])
    th = torch.zeros(eng.num_output_classes, dtype=torch.float64, device="cuda")
    F, mD, g, gd = eng.dual_bound(0, th, 0.05, "fp64", grad=False)
    assert np.isfinite(F)
    with pytest.raises(bdc.BdcError):
        eng.dual_bound(0, th, 0.05, "fp64", grad=True)
    eng.close()
