"""GPU parity against the oracle on the code paths the kernels take at full
size: the split (columns, rows, combine) schedules, the stepped FP32
iteration boundary in the headline configuration's column kernel, the
literal enumeration path at sizes with many work items per class, the
smoothed dual bound on a split FP64 schedule, and the certificate's two forms
(complement half mode for a complement-invariant input, all inputs otherwise).

Bars (Sec. 2.3 quantities): certified bound U in [U_oracle - 1e-12,
U_oracle + 1e-6] bits and U >= the oracle's BA lower bound; FP64 q 1e-12
relative, D and bounds 1e-11; FP32 p per element within 2e-3 relative after
five iterations (each FP32 iteration moves log2 p by D, whose FP32 error is
at most 2e-5 (1 + |D|) ~ 2.2e-4 bits at n = 19, i.e. 1.5e-4 relative in p:
five iterations stay below 1e-3), FP32 D within 2e-5 (1 + |D|).

Oracle values come from the definitions (q_full, D_full, certify,
dual_bound) and, for full BA runs at n >= 16, from the oracle's factorised
sweep (O2), which the -m "not gpu" tests pin against the definitions.
"""
import numpy as np
import pytest

import oracle
from paper_2604_05867_b300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS_CERT = 2.0 ** -30  # weight of the uniform input mixed in before certification (default option)


def _bdc():
    import paper_2604_05867_b300 as bdc
    return bdc


def _engine(n, ds, **kw):
    bdc = _bdc()
    return bdc.Engine(n, ds, options=bdc.default_options(**kw))


# ---------------------------------------------------------------------------
# (a) certificate on split FP64 schedules
# ---------------------------------------------------------------------------
CERT_CASES = [(10, 0.5, 6), (11, 0.7, 7), (12, 0.3, 7), (12, 0.85, 6), (14, 0.6, 0), (16, 0.8, 0)]


@pytest.mark.parametrize("n,d,n2", CERT_CASES)
def test_certified_bound_split_schedule(n, d, n2):
    T = 40
    kw = dict(enable_literal=0)
    if n2:
        kw.update(sched_n2_fp64=n2, sched_w_fp64=2)
    eng = _engine(n, [d], **kw)
    s = eng.schedule("fp64")
    assert s["n2"] > 0, s  # the split schedule, not the single-CTA pass
    eng.iterate(T, -1.0, "fp32", "sweep")
    c = eng.certify()
    p = eng.get_p()[0]
    pt = (1 - EPS_CERT) * p + EPS_CERT / (1 << n)
    U_ref, _ = oracle.certify(n, d, oracle.q_full(n, d, pt))
    lower_ref = oracle.ba_sweep(n, d, T)["lower"][-1]
    U = c["upper"][0]
    assert U_ref - 1e-12 <= U <= U_ref + 1e-6, (U, U_ref)
    assert U >= lower_ref
    assert 0 < c["margin"][0] < 1e-6
    # the FP64 Blahut lower bound of the certified input, to FP32-iterate precision
    assert abs(c["lower"][0] - lower_ref) < 1e-3
    eng.close()


@pytest.mark.parametrize("n,d,n2", [(12, 0.6, 7), (14, 0.45, 0), (16, 0.7, 0)])
def test_certify_given_q_split_schedule(n, d, n2):
    rng = np.random.default_rng(n)
    qh = rng.uniform(0.1, 1.0, size=2 << n)
    qh[0] = 0.0
    qh /= qh.sum()
    kw = dict(enable_literal=0)
    if n2:
        kw.update(sched_n2_fp64=n2, sched_w_fp64=4)
    eng = _engine(n, [d], **kw)
    assert eng.schedule("fp64")["n2"] > 0
    c = eng.certify(torch.tensor(qh[None, :], device="cuda"))
    U_ref, _ = oracle.certify(n, d, qh)
    assert U_ref - 1e-12 <= c["upper"][0] <= U_ref + 1e-6
    assert np.isnan(c["lower"][0])
    eng.close()


def test_certified_bound_two_instances_split():
    # two instances in one engine: the certificate's partial-sum layout with
    # many column blocks per instance
    n, ds, T = 14, [0.35, 0.9], 25
    eng = _engine(n, ds, enable_literal=0, sched_n2_fp64=8, sched_w_fp64=1)
    assert eng.schedule("fp64")["n2"] == 8
    eng.iterate(T, -1.0, "fp32", "sweep")
    c = eng.certify()
    P = eng.get_p()
    for z, d in enumerate(ds):
        pt = (1 - EPS_CERT) * P[z] + EPS_CERT / (1 << n)
        U_ref, _ = oracle.certify(n, d, oracle.q_full(n, d, pt))
        assert U_ref - 1e-12 <= c["upper"][z] <= U_ref + 1e-6
    eng.close()


# ---------------------------------------------------------------------------
# (b) the stepped FP32 iteration boundary, per element
# ---------------------------------------------------------------------------
def test_stepped_fp32_bench_column_kernel_per_element():
    # n = 19 split 11 + 8 with 4 columns: the column tile (2^12 rows x 4) is
    # the headline configuration's (n = 24, 11 + 13, 4 columns), so BA
    # iterations run its stepped, register-resident, complement-half column
    # kernel; every element of p and every D_x against the oracle
    n, d, T = 19, 0.5, 5
    eng = _engine(n, [d], enable_literal=0, sched_n2_fp32=8, sched_w_fp32=4)
    assert eng.schedule("fp32") == {"n1": 11, "n2": 8, "width": 4}
    eng.iterate(T, -1.0, "fp32", "sweep")
    S = oracle.subseq_S_all(n)
    ref = oracle.ba_sweep(n, d, T, S=S)
    lo, up = eng.history(0)
    assert np.all(np.abs(lo - ref["lower"]) <= 2e-5 * np.abs(ref["lower"]))
    assert np.all(np.abs(up - ref["upper"]) <= 2e-5 * np.abs(ref["upper"]))
    p = eng.get_p()[0]
    assert np.all(np.abs(p - ref["p"]) <= 2e-3 * ref["p"])
    # D of the engine's current p, FP32 kernels, against the oracle's D of the same p
    D32 = eng.divergence(precision="fp32").cpu().numpy()[0]
    q_ref = oracle.sweep_q(n, d, p)
    D_ref = oracle.D_sweep(n, d, q_ref, S)
    assert np.all(np.abs(D32 - D_ref) <= 2e-5 * (1.0 + np.abs(D_ref)))
    for x in inputs.random_inputs(n, 6, seed=19):
        r = oracle.D_point(n, d, q_ref, int(x))
        assert abs(D32[x] - r) <= 2e-5 * (1.0 + abs(r))
    eng.close()


def test_bench_configuration_fp32_p_per_element():
    # n = 24 in the headline configuration (11 + 13, 4 columns, stepped FP32)
    # against the FP64 engine on the unstepped full-mode kernels, every
    # element of p after 3 iterations (the FP64 kernels at this size are
    # checked against the oracle in test_full_size_bench_configuration)
    n, d, T = 24, 0.5, 3
    sched = dict(sched_n2_fp32=13, sched_w_fp32=4, sched_n2_fp64=13, sched_w_fp64=4, enable_literal=0)
    a = _engine(n, [d], **sched)
    assert a.schedule("fp32") == {"n1": 11, "n2": 13, "width": 4}
    a.iterate(T, -1.0, "fp32", "sweep")
    pa = a.get_p()[0]
    la, ua = a.history(0)
    a.close()
    b = _engine(n, [d], use_regsteps=0, fuse_update=0, use_half=0, **sched)
    b.iterate(T, -1.0, "fp64", "sweep")
    pb = b.get_p()[0]
    lb, ub = b.history(0)
    b.close()
    assert np.all(np.abs(la - lb) <= 2e-5 * np.abs(lb)) and np.all(np.abs(ua - ub) <= 2e-5 * np.abs(ub))
    assert np.all(np.abs(pa - pb) <= 2e-3 * pb)


# ---------------------------------------------------------------------------
# (c) the literal enumeration path at n = 14 and 16
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n,d", [(14, 0.6), (16, 0.4)])
def test_literal_path_per_element(n, d):
    T = 2
    eng = _engine(n, [d])
    eng.iterate(T, -1.0, "fp64", "literal")
    lo, up = eng.history(0)
    S = oracle.subseq_S_all(n)
    ref = oracle.ba_sweep(n, d, T, S=S)
    assert np.all(np.abs(lo - ref["lower"]) <= 1e-11) and np.all(np.abs(up - ref["upper"]) <= 1e-11)
    p = eng.get_p()[0]
    assert np.all(np.abs(p - ref["p"]) <= 1e-9 * ref["p"])
    # the supersequence walk's output marginal, every code, against the definition
    q_lit = eng.get_q_literal()[0]
    q_ref = oracle.q_full(n, d, p)
    assert q_lit[0] == 0.0
    assert np.all(np.abs(q_lit[1:] - q_ref[1:]) <= 1e-12 * q_ref[1:])
    # (the per-input walk's D_x is checked element by element through p: the
    # last update is p_T = p_{T-1} 2^{D_x} / Z, matched above to 1e-9)
    eng.close()


# ---------------------------------------------------------------------------
# (d) the smoothed dual bound and its adjoint on a split FP64 schedule
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n,d,tau,n2", [(10, 0.7, 0.05, 6), (11, 0.4, 0.02, 7), (12, 0.8, 0.01, 7)])
def test_dual_bound_split_schedule(n, d, tau, n2):
    eng = _engine(n, [d], enable_literal=0, sched_n2_fp64=n2, sched_w_fp64=2)
    assert eng.schedule("fp64")["n2"] == n2
    ocls, _, _ = oracle.output_classes(n)
    rng = np.random.default_rng(100 + n)
    theta = rng.normal(scale=0.7, size=eng.num_output_classes)
    F_ref, g_ref, gd_ref = oracle.dual_bound(n, d, tau, theta, ocls)
    th = torch.tensor(theta, dtype=torch.float64, device="cuda")
    F, mD, g, gd = eng.dual_bound(0, th, tau, "fp64", grad=True)
    assert abs(F - F_ref) <= 1e-10 * max(1.0, abs(F_ref))
    g = g.cpu().numpy()
    assert np.all(np.abs(g - g_ref) <= 1e-9 * np.maximum(1.0, np.abs(g_ref)))
    assert abs(gd - gd_ref) <= 1e-9 * max(1.0, abs(gd_ref))
    assert mD <= F <= mD + tau * n + 1e-12
    eng.close()


# ---------------------------------------------------------------------------
# (e) the certificate's two forms on split schedules: a complement-invariant
# input is certified in the complement half mode (checked bitwise on the
# device), any other input over all inputs
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n,d,n2", [(12, 0.6, 7), (14, 0.45, 0), (16, 0.8, 0)])
def test_certificate_half_mode_matches_full_mode(n, d, n2):
    kw = dict(enable_literal=0)
    if n2:
        kw.update(sched_n2_fp64=n2, sched_w_fp64=2)
    a = _engine(n, [d], **kw)
    assert a.schedule("fp64")["n2"] > 0
    a.iterate(15, -1.0, "fp64", "sweep")
    ca = a.certify()
    p = a.get_p()
    assert np.array_equal(p[0], p[0][::-1])  # complement-invariant: p(x) = p(2^n - 1 - x)
    a.close()
    b = _engine(n, [d], use_half=0, **kw)  # the same input, certified over all inputs
    b.set_p(p)
    cb = b.certify()
    b.close()
    assert abs(ca["upper"][0] - cb["upper"][0]) <= 1e-11, (ca, cb)
    assert abs(ca["lower"][0] - cb["lower"][0]) <= 1e-11
    pt = (1 - EPS_CERT) * p[0] / p[0].sum() + EPS_CERT / (1 << n)
    U_ref, _ = oracle.certify(n, d, oracle.q_full(n, d, pt))
    assert U_ref - 1e-12 <= ca["upper"][0] <= U_ref + 1e-6


@pytest.mark.parametrize("n,d,n2", [(12, 0.7, 7), (14, 0.3, 0)])
def test_certificate_asymmetric_input_split_schedule(n, d, n2):
    rng = np.random.default_rng(7 + n)
    p = rng.uniform(0.2, 1.0, size=(1, 1 << n))
    kw = dict(enable_literal=0)
    if n2:
        kw.update(sched_n2_fp64=n2, sched_w_fp64=2)
    eng = _engine(n, [d], **kw)
    assert eng.schedule("fp64")["n2"] > 0
    eng.set_p(p)
    c = eng.certify()
    eng.close()
    pt = (1 - EPS_CERT) * p[0] / p[0].sum() + EPS_CERT / (1 << n)
    U_ref, _ = oracle.certify(n, d, oracle.q_full(n, d, pt))
    assert U_ref - 1e-12 <= c["upper"][0] <= U_ref + 1e-6, (c, U_ref)
    assert 0 < c["margin"][0] < 1e-6
