"""GPU parity of full Blahut-Arimoto iterations and of the certified bound.

Sweep path (FP64 and FP32) and literal enumeration path (FP64) against the
oracle's BA (Sec. 2.3) iteration by iteration; certified upper bound against
the oracle's exact dual value (|U - U_oracle| <= 1e-6 bits, U >= the oracle's
lower bound, margin > 0); closed forms C_1(d) = 1 - d, C_n(0) = n, C_n(1) = 0;
stopping rule; checkpoint resume is bit-identical.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2604_05867_b300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _bdc():
    import paper_2604_05867_b300 as bdc
    return bdc


def _engine(n, ds, **kw):
    bdc = _bdc()
    return bdc.Engine(n, ds, options=bdc.default_options(**kw))


@pytest.mark.parametrize("impl,prec,tol", [("sweep", "fp64", 1e-11), ("literal", "fp64", 1e-11),
                                           ("sweep", "fp32", 2e-5)])
@pytest.mark.parametrize("n,d", [(4, 0.5), (7, 0.3), (10, 0.8)])
def test_ba_iterations_match_oracle(impl, prec, tol, n, d):
    T = 60
    ref = oracle.ba_bdc(n, d, T)
    eng = _engine(n, [d])
    lo, up, it = eng.iterate(T, -1.0, prec, impl)
    assert it[0] == T
    hlo, hup = eng.history(0)
    assert len(hlo) == T
    assert np.all(np.abs(hlo - ref["lower"]) <= tol * np.maximum(1.0, np.abs(ref["lower"])))
    assert np.all(np.abs(hup - ref["upper"]) <= tol * np.maximum(1.0, np.abs(ref["upper"])))
    p = eng.get_p()[0]
    ptol = 1e-9 if prec == "fp64" else 2e-3
    assert np.all(np.abs(p - ref["p"]) <= ptol * ref["p"] + 1e-300)
    eng.close()


@pytest.mark.parametrize("d", [0.1, 0.5, 0.9])
def test_bec_closed_form(d):
    eng = _engine(1, [d])
    lo, up, _ = eng.iterate(20, -1.0, "fp64", "sweep")
    assert abs(lo[0] - (1 - d)) < 1e-13 and abs(up[0] - (1 - d)) < 1e-13
    c = eng.certify()
    assert c["upper"][0] >= 1 - d and c["upper"][0] - (1 - d) < 1e-9
    eng.close()


def test_noiseless_and_erased_channels():
    n = 9
    eng = _engine(n, [0.0, 1.0])
    lo, up, _ = eng.iterate(2, -1.0, "fp64", "sweep")
    assert abs(lo[0] - n) < 1e-12 and abs(up[0] - n) < 1e-12
    assert abs(lo[1]) < 1e-12 and abs(up[1]) < 1e-12
    eng.close()


def test_stopping_rule_and_monotone_lower():
    n, d, tol = 8, 0.5, 1e-3
    ref = oracle.ba_bdc(n, d, 5000, tol=tol)
    eng = _engine(n, [d], chunk=4)
    lo, up, it = eng.iterate(5000, tol, "fp64", "sweep")
    assert it[0] == ref["iters"]
    hlo, hup = eng.history(0)
    assert np.all(np.diff(hlo) >= -1e-12)
    assert hup[-1] - hlo[-1] < tol
    eng.close()


@pytest.mark.parametrize("n,d", [(6, 0.5), (10, 0.5), (12, 0.7)])
def test_certified_bound(n, d):
    T = 150
    eng = _engine(n, [d])
    eng.iterate(T, -1.0, "fp32", "sweep")
    c = eng.certify()
    # oracle: exact dual value of the same certified input p~ = (1-eps)p + eps u
    p = eng.get_p()[0]
    eps = 2.0 ** -30
    pt = (1 - eps) * p + eps / (1 << n)
    q = oracle.q_full(n, d, pt)
    U_ref, _ = oracle.certify(n, d, q)
    lower_ref = oracle.ba_bdc(n, d, T)["lower"][-1]
    assert c["upper"][0] >= U_ref - 1e-12
    assert c["upper"][0] - U_ref <= 1e-6
    assert c["upper"][0] >= lower_ref
    assert 0 < c["margin"][0] < 1e-6
    assert abs(c["lower"][0] - lower_ref) < 1e-3
    eng.close()


def test_certify_given_q():
    n, d = 8, 0.6
    rng = np.random.default_rng(0)
    qh = rng.uniform(0.1, 1.0, size=2 << n)
    qh[0] = 0.0
    qh /= qh.sum()
    eng = _engine(n, [d])
    c = eng.certify(torch.tensor(qh[None, :], device="cuda"))
    U_ref, _ = oracle.certify(n, d, qh)
    assert U_ref - 1e-12 <= c["upper"][0] <= U_ref + 1e-6
    assert np.isnan(c["lower"][0])
    eng.close()


def test_orbit_invariance_and_symmetrize():
    n, d = 11, 0.4
    eng = _engine(n, [d])
    eng.iterate(40, -1.0, "fp32", "sweep")
    p = eng.get_p()[0]
    x = np.arange(1 << n)
    full = (1 << n) - 1
    rx = np.array([int(format(v, "0%db" % n)[::-1], 2) for v in x])
    assert np.array_equal(p, p[x ^ full]) and np.array_equal(p, p[rx])
    eng.close()


def test_checkpoint_resume_is_bit_identical(tmp_path):
    n, d = 9, 0.5
    a = _engine(n, [d])
    a.iterate(20, -1.0, "fp64", "sweep")
    path = str(tmp_path / "ck.bin")
    a.save(path)
    a.iterate(15, -1.0, "fp64", "sweep")
    pa = a.get_p()
    b = _engine(n, [d])
    b.load(path)
    b.iterate(15, -1.0, "fp64", "sweep")
    pb = b.get_p()
    assert np.array_equal(pa, pb)
    a.close()
    b.close()


def test_precision_switch_and_literal_agree():
    n, d = 10, 0.5
    ref = oracle.ba_bdc(n, d, 30)
    eng = _engine(n, [d])
    eng.iterate(10, -1.0, "fp64", "sweep")
    eng.iterate(10, -1.0, "fp64", "literal")
    eng.iterate(10, -1.0, "fp64", "sweep")
    hlo, hup = eng.history(0)
    assert np.all(np.abs(hlo - ref["lower"]) <= 1e-11)
    assert np.all(np.abs(hup - ref["upper"]) <= 1e-11)
    eng.close()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("fp32", 2e-5)])
def test_half_mode_iterations_match_oracle(prec, tol):
    # a forced split schedule at n = 10 runs the complement half mode
    n, d, T = 10, 0.6, 40
    ref = oracle.ba_bdc(n, d, T)
    eng = _engine(n, [d], sched_n2_fp32=6, sched_w_fp32=4, sched_n2_fp64=7, sched_w_fp64=2)
    eng.iterate(T, -1.0, prec, "sweep")
    hlo, hup = eng.history(0)
    assert np.all(np.abs(hlo - ref["lower"]) <= tol * np.maximum(1.0, np.abs(ref["lower"])))
    assert np.all(np.abs(hup - ref["upper"]) <= tol * np.maximum(1.0, np.abs(ref["upper"])))
    p = eng.get_p()[0]
    assert np.all(np.abs(p - ref["p"]) <= (1e-9 if prec == "fp64" else 2e-3) * ref["p"])
    eng.close()


def test_half_and_full_mode_agree():
    import paper_2604_05867_b300 as bdc
    n, d, T = 16, 0.55, 30
    a = _engine(n, [d, 0.8])
    b = bdc.Engine(n, [d, 0.8], options=bdc.default_options(use_half=0))
    a.iterate(T, -1.0, "fp64", "sweep")
    b.iterate(T, -1.0, "fp64", "sweep")
    for z in range(2):
        la, ua = a.history(z)
        lb, ub = b.history(z)
        assert np.all(np.abs(la - lb) <= 1e-11) and np.all(np.abs(ua - ub) <= 1e-11)
    pa, pb = a.get_p(), b.get_p()
    assert np.all(np.abs(pa - pb) <= 1e-11 * pb)
    a.close()
    b.close()


def test_asymmetric_p_switches_off_symmetry_shortcuts():
    n, d, T = 10, 0.45, 20
    rng = np.random.default_rng(7)
    p0 = rng.dirichlet(np.ones(1 << n))
    ref = oracle.ba_bdc(n, d, T, p0=p0)
    eng = _engine(n, [d], sched_n2_fp64=7, sched_w_fp64=2)
    eng.set_p(p0)
    eng.iterate(T, -1.0, "fp64", "sweep")
    hlo, hup = eng.history(0)
    assert np.all(np.abs(hlo - ref["lower"]) <= 1e-11) and np.all(np.abs(hup - ref["upper"]) <= 1e-11)
    import paper_2604_05867_b300 as bdc
    with pytest.raises(bdc.BdcError):
        eng.iterate(1, -1.0, "fp64", "literal")
    eng.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_half_mode_keeps_p_exactly_orbit_invariant(prec):
    # half-mode iterations average D over each orbit inside the forward pass;
    # the resulting p must be bit-identical across every orbit, and the run must
    # match the full-mode run (separate orbit-mean pass)
    import paper_2604_05867_b300 as bdc
    n, d, T = 12, 0.35, 25
    kw = dict(sched_n2_fp32=6, sched_w_fp32=4, sched_n2_fp64=7, sched_w_fp64=2)
    a = bdc.Engine(n, [d], options=bdc.default_options(**kw))
    b = bdc.Engine(n, [d], options=bdc.default_options(use_half=0, **kw))
    a.iterate(T, -1.0, prec, "sweep")
    b.iterate(T, -1.0, prec, "sweep")
    pa = a.get_p()[0]
    x = np.arange(1 << n)
    full = (1 << n) - 1
    rx = np.array([int(format(v, "0%db" % n)[::-1], 2) for v in x])
    assert np.array_equal(pa, pa[x ^ full]) and np.array_equal(pa, pa[rx])
    pb = b.get_p()[0]
    ptol, htol = (1e-11, 1e-11) if prec == "fp64" else (2e-3, 2e-5 * n)
    assert np.all(np.abs(pa - pb) <= ptol * pb)
    la, ua = a.history(0)
    lb, ub = b.history(0)
    assert np.all(np.abs(la - lb) <= htol) and np.all(np.abs(ua - ub) <= htol)
    a.close()
    b.close()


def _nl(sched, prec):
    # which kernels run register-resident steps (use_regsteps = 15): columns
    # when a column tile holds 512 << NL inputs (3 <= NL <= 5 in FP32, 4 in
    # FP64); forward rows when n2 - NLmax is in [7, 9]; adjoint rows when
    # 3 <= n2 - 9 <= NLmax
    nmax = 5 if prec == "fp32" else 4
    w = sched["width"].bit_length() - 1
    nlc = sched["n1"] + w - 9
    return {"cols": 3 <= nlc <= nmax and nlc <= sched["n1"], "rows_fwd": 7 <= sched["n2"] - nmax <= 9,
            "rows_adj": 3 <= sched["n2"] - 9 <= nmax}


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_register_steps_agree_with_shared_memory_steps(prec):
    import paper_2604_05867_b300 as bdc
    n, T = 20, 6
    kw = dict(sched_n2_fp32=12, sched_w_fp32=32, sched_n2_fp64=12, sched_w_fp64=32)
    a = bdc.Engine(n, [0.3, 0.7], options=bdc.default_options(use_regsteps=15, **kw))
    b = bdc.Engine(n, [0.3, 0.7], options=bdc.default_options(use_regsteps=0, **kw))
    assert all(_nl(a.schedule(prec), prec).values())
    a.iterate(T, -1.0, prec, "sweep")
    b.iterate(T, -1.0, prec, "sweep")
    tol = 1e-12 if prec == "fp64" else 2e-6
    for z in range(2):
        la, ua = a.history(z)
        lb, ub = b.history(z)
        assert np.all(np.abs(la - lb) <= tol * np.abs(lb)) and np.all(np.abs(ua - ub) <= tol * np.abs(ub))
    pa, pb = a.get_p(), b.get_p()
    assert np.all(np.abs(pa - pb) <= (1e-11 if prec == "fp64" else 1e-4) * pb)
    a.close()
    b.close()


def test_register_steps_match_oracle():
    # n = 17 with a forced split (n1 = 7, n2 = 10, 32 columns): the column
    # kernels run register-resident steps, in the complement half mode with
    # the fused orbit mean (second iteration); the row kernels are covered in
    # the sweep tests
    import paper_2604_05867_b300 as bdc
    n, d, T = 17, 0.6, 2
    eng = bdc.Engine(n, [d], options=bdc.default_options(sched_n2_fp64=10, sched_w_fp64=32, use_regsteps=15))
    assert _nl(eng.schedule("fp64"), "fp64")["cols"]
    eng.iterate(T, -1.0, "fp64", "sweep")
    # oracle BA from its matrix-free q and D (the sparse-row BA is too large here)
    pr = np.full(1 << n, 1.0 / (1 << n))
    lo_ref, up_ref = [], []
    for _ in range(T):
        D = oracle.D_full(n, d, oracle.q_full(n, d, pr))
        lo_ref.append(np.log2(np.sum(pr * np.exp2(D))))
        up_ref.append(D.max())
        pr = pr * np.exp2(D)
        pr /= pr.sum()
    lo, up = eng.history(0)
    assert np.all(np.abs(lo - lo_ref) <= 1e-11) and np.all(np.abs(up - up_ref) <= 1e-11)
    p = eng.get_p()[0]
    assert np.all(np.abs(p - pr) <= 1e-9 * pr)
    eng.close()


def test_prepared_graph_matches_stream_launches():
    # bdc_prepare builds the replayed graph ahead of time; replaying it gives
    # the same iterations, bit for bit, as launching every kernel on the stream
    import paper_2604_05867_b300 as bdc
    n, d, T = 16, 0.5, 16
    a = bdc.Engine(n, [d], options=bdc.default_options(chunk=8))
    b = bdc.Engine(n, [d], options=bdc.default_options(chunk=8, use_graph=0))
    a.prepare("fp32", "sweep")
    launches = a.launch_count()
    a.iterate(T, -1.0, "fp32", "sweep")
    b.iterate(T, -1.0, "fp32", "sweep")
    la, ua = a.history(0)
    lb, ub = b.history(0)
    assert np.array_equal(la, lb) and np.array_equal(ua, ub)
    assert np.array_equal(a.get_p(), b.get_p())
    a.close()
    b.close()


def _stepped_engine(n, ds, **kw):
    # n1 = n - 10, 32 columns: the register-step column kernels apply, so BA
    # iterations run stepped (update and next forward columns pass in one kernel)
    import paper_2604_05867_b300 as bdc
    opts = dict(sched_n2_fp32=10, sched_w_fp32=32, sched_n2_fp64=10, sched_w_fp64=32)
    opts.update(kw)
    eng = bdc.Engine(n, ds, options=bdc.default_options(**opts))
    assert _nl(eng.schedule("fp64"), "fp64")["cols"]
    return eng


def test_stepped_iterations_stop_at_the_first_small_gap():
    # the stopping rule on the stepped path: an instance stops after the first
    # iteration whose gap is below tol, and its iterations up to there are the
    # same, bit for bit, as those of a run without a tolerance (graph replays
    # of 3 iterations, so the stop falls inside a chunk)
    n, d = 18, 0.5
    ref = _stepped_engine(n, [d], chunk=3)
    ref.iterate(40, -1.0, "fp64", "sweep")
    lo_r, up_r = ref.history(0)
    gaps = up_r - lo_r
    tol = float(gaps[11]) * (1 + 1e-9)
    stop = int(np.argmax(gaps < tol)) + 1  # first iteration with a gap below tol (at most 12)
    eng = _stepped_engine(n, [d], chunk=3)
    lo, up, it = eng.iterate(40, tol, "fp64", "sweep")
    assert it[0] == stop
    la, ua = eng.history(0)
    assert np.array_equal(la, lo_r[:stop]) and np.array_equal(ua, up_r[:stop])
    ref.close()
    eng.close()


def test_stepped_instances_are_independent():
    n = 18
    ds = [0.3, 0.8]
    both = _stepped_engine(n, ds)
    both.iterate(6, -1.0, "fp32", "sweep")
    for z, d in enumerate(ds):
        one = _stepped_engine(n, [d])
        one.iterate(6, -1.0, "fp32", "sweep")
        lb, ub = both.history(z)
        lo, uo = one.history(0)
        assert np.array_equal(lb, lo) and np.array_equal(ub, uo)
        assert np.array_equal(both.get_p()[z], one.get_p()[0])
        one.close()
    both.close()


def test_stepped_checkpoint_resume_is_bit_identical(tmp_path):
    n, d = 18, 0.6
    a = _stepped_engine(n, [d])
    a.iterate(7, -1.0, "fp32", "sweep")
    path = str(tmp_path / "ck_stepped.bin")
    a.save(path)
    a.iterate(9, -1.0, "fp32", "sweep")
    b = _stepped_engine(n, [d])
    b.load(path)
    b.iterate(9, -1.0, "fp32", "sweep")
    assert np.array_equal(a.get_p(), b.get_p())
    la, ua = a.history(0)
    lb, ub = b.history(0)
    assert np.array_equal(la[-9:], lb[-9:]) and np.array_equal(ua[-9:], ub[-9:])
    a.close()
    b.close()


def test_stepped_instances_stop_independently():
    # two instances with very different gaps: the first stops early inside a
    # graph chunk while the second keeps iterating; each matches its own
    # single-instance run bit for bit (iterations, history, final p)
    n = 18
    ds = [0.05, 0.6]
    ref = [_stepped_engine(n, [d], chunk=4) for d in ds]
    hist = []
    for e in ref:
        e.iterate(30, -1.0, "fp64", "sweep")
        lo, up = e.history(0)
        hist.append((lo, up))
    gaps0 = hist[0][1] - hist[0][0]
    tol = float(gaps0[5]) * (1 + 1e-9)
    stop0 = int(np.argmax(gaps0 < tol)) + 1
    gaps1 = hist[1][1] - hist[1][0]
    stop1 = int(np.argmax(gaps1 < tol)) + 1 if np.any(gaps1 < tol) else 30
    assert stop0 < stop1
    both = _stepped_engine(n, ds, chunk=4)
    lo, up, it = both.iterate(30, tol, "fp64", "sweep")
    assert list(it) == [stop0, stop1]
    for z, (stop, (lr, ur)) in enumerate(zip([stop0, stop1], hist)):
        la, ua = both.history(z)
        assert np.array_equal(la, lr[:stop]) and np.array_equal(ua, ur[:stop])
    for z, (stop, e) in enumerate(zip([stop0, stop1], ref)):
        one = _stepped_engine(n, [ds[z]], chunk=4)
        one.iterate(stop, -1.0, "fp64", "sweep")
        assert np.array_equal(both.get_p()[z], one.get_p()[0])
        one.close()
    for e in ref:
        e.close()
    both.close()


@pytest.mark.parametrize("n,n2,ds", [(18, 8, [0.3, 0.7]), (19, 10, [0.5])])
def test_tma_tile_load_is_bit_identical(n, n2, ds):
    # the one-pass iteration boundary with its Gb tile loaded by TMA (FP32,
    # complement half mode, 4 columns, n1 = n - n2 >= 9; two instances: the
    # tensor map spans both) against the same kernels with per-thread loads:
    # the same values reach the same arithmetic, so bounds and p agree bit for bit
    import paper_2604_05867_b300 as bdc
    T = 6
    kw = dict(sched_n2_fp32=n2, sched_w_fp32=4, enable_literal=0, chunk=3)
    a = bdc.Engine(n, ds, options=bdc.default_options(use_tma=1, **kw))
    b = bdc.Engine(n, ds, options=bdc.default_options(use_tma=0, **kw))
    assert a.schedule("fp32") == {"n1": n - n2, "n2": n2, "width": 4}
    a.iterate(T, -1.0, "fp32", "sweep")
    b.iterate(T, -1.0, "fp32", "sweep")
    for z in range(len(ds)):
        la, ua = a.history(z)
        lb, ub = b.history(z)
        assert len(la) == T and np.array_equal(la, lb) and np.array_equal(ua, ub)
    assert np.array_equal(a.get_p(), b.get_p())
    a.close()
    b.close()


def test_tma_bench_configuration_matches_oracle_bounds():
    # n = 24 in the headline bench's configuration (split 11 + 13, 4 columns,
    # FP32, stepped, TMA tile loads): bit-identical to per-thread loads, and
    # within FP32 rounding of the FP64 sweep's bounds (the FP64 sweep at this
    # size is checked against the oracle in test_full_size_bench_configuration)
    import paper_2604_05867_b300 as bdc
    n, d, T = 24, 0.5, 3
    kw = dict(sched_n2_fp32=13, sched_w_fp32=4, sched_n2_fp64=13, sched_w_fp64=4, enable_literal=0)
    a = bdc.Engine(n, [d], options=bdc.default_options(use_tma=1, **kw))
    b = bdc.Engine(n, [d], options=bdc.default_options(use_tma=0, **kw))
    a.iterate(T, -1.0, "fp32", "sweep")
    b.iterate(T, -1.0, "fp32", "sweep")
    la, ua = a.history(0)
    lb, ub = b.history(0)
    assert np.array_equal(la, lb) and np.array_equal(ua, ub)
    assert np.array_equal(a.get_p(), b.get_p())
    b.close()
    c = bdc.Engine(n, [d], options=bdc.default_options(**kw))
    c.iterate(T, -1.0, "fp64", "sweep")
    lc, uc = c.history(0)
    assert np.all(np.abs(la - lc) <= 2e-5 * np.abs(lc)) and np.all(np.abs(ua - uc) <= 2e-5 * np.abs(uc))
    a.close()
    c.close()


@pytest.mark.parametrize("n2", [9, 10, 11])
def test_combine_split_boundaries_fp32(n2):
    # the combine's split of an output code into u1 u2 at every length of the
    # second part around the CTA width (1024 codes): FP32 stepped half-mode
    # iterations at n = 19 against the all-shared-memory, unstepped, full-mode
    # FP64 kernels (a mistake at one split length moves the bounds far beyond
    # FP32 rounding)
    import paper_2604_05867_b300 as bdc
    n, d, T = 19, 0.6, 3
    a = bdc.Engine(n, [d], options=bdc.default_options(sched_n2_fp32=n2, sched_w_fp32=4, enable_literal=0))
    assert a.schedule("fp32")["n2"] == n2
    a.iterate(T, -1.0, "fp32", "sweep")
    b = bdc.Engine(n, [d], options=bdc.default_options(sched_n2_fp64=n2, sched_w_fp64=4, enable_literal=0,
                                                       use_regsteps=0, fuse_update=0, use_half=0))
    b.iterate(T, -1.0, "fp64", "sweep")
    la, ua = a.history(0)
    lb, ub = b.history(0)
    assert np.all(np.abs(la - lb) <= 2e-5 * np.abs(lb)) and np.all(np.abs(ua - ub) <= 2e-5 * np.abs(ub))
    a.close()
    b.close()


def test_short_calls_replay_the_one_iteration_graph():
    # calls of fewer iterations than a graph chunk replay a one-iteration graph;
    # any mix of call lengths gives the same iterations, bit for bit, as
    # launching every kernel on the stream
    import paper_2604_05867_b300 as bdc
    n, d = 16, 0.5
    a = bdc.Engine(n, [d], options=bdc.default_options(chunk=4))
    b = bdc.Engine(n, [d], options=bdc.default_options(chunk=4, use_graph=0))
    a.prepare("fp32", "sweep")
    for c in (1, 3, 4, 1, 6, 2):
        a.iterate(c, -1.0, "fp32", "sweep")
    b.iterate(17, -1.0, "fp32", "sweep")
    la, ua = a.history(0)
    lb, ub = b.history(0)
    assert len(la) == 17 and np.array_equal(la, lb) and np.array_equal(ua, ub)
    assert np.array_equal(a.get_p(), b.get_p())
    a.close()
    b.close()


@pytest.mark.parametrize("n,n2,w", [(20, 8, 4), (21, 10, 8)])
def test_column_step_with_1024_threads_fp32(n, n2, w):
    # column tiles of 128 KB (n1 + log2 w = 14) run the column kernels with
    # 1024 threads, one CTA per SM (the 8-column layout the bench's autotuner
    # may choose at n = 24): FP32 stepped half-mode iterations against the
    # all-shared-memory, unstepped, full-mode FP64 kernels
    import paper_2604_05867_b300 as bdc
    d, T = 0.55, 3
    a = bdc.Engine(n, [d], options=bdc.default_options(sched_n2_fp32=n2, sched_w_fp32=w, enable_literal=0))
    s = a.schedule("fp32")
    assert (s["n2"], s["width"]) == (n2, w) and (2 << s["n1"]) * w * 4 > 112 * 1024
    a.iterate(T, -1.0, "fp32", "sweep")
    b = bdc.Engine(n, [d], options=bdc.default_options(sched_n2_fp64=n2, sched_w_fp64=w, enable_literal=0,
                                                       use_regsteps=0, fuse_update=0, use_half=0))
    b.iterate(T, -1.0, "fp64", "sweep")
    la, ua = a.history(0)
    lb, ub = b.history(0)
    assert np.all(np.abs(la - lb) <= 2e-5 * np.abs(lb)) and np.all(np.abs(ua - ub) <= 2e-5 * np.abs(ub))
    a.close()
    b.close()
