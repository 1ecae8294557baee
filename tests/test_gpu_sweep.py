"""GPU parity of the output marginal q and the divergence D_x (Sec. 2.3)
against the oracle's plain definitions, through the C ABI.

FP64 results must match to 1e-12 relative (q) and 1e-12 absolute-or-relative
(D).  FP32 results are checked to the rounding that an FP32 sum of at most
2n+1 terms and an FP32 log2 allow: 4e-6 relative on q, and on D an absolute
2e-5 * (1 + |D|).  Schedules are forced to exercise the single-CTA pass, the
two-pass split with several tile widths and the transposed short-code store.
"""
import numpy as np
import pytest

import oracle
from paper_2604_05867_b300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _bdc():
    import paper_2604_05867_b300 as bdc
    return bdc


def _engine(n, ds, **kw):
    bdc = _bdc()
    return bdc.Engine(n, ds, options=bdc.default_options(**kw))


SCHEDS = [dict(), dict(sched_n2_fp32=5, sched_w_fp32=1, sched_n2_fp64=5, sched_w_fp64=1),
          dict(sched_n2_fp32=6, sched_w_fp32=4, sched_n2_fp64=7, sched_w_fp64=2)]


@pytest.mark.parametrize("n,d", [(1, 0.3), (3, 0.5), (8, 0.7), (11, 0.25), (13, 0.9)])
@pytest.mark.parametrize("sched", range(len(SCHEDS)))
def test_q_and_D_match_definition(n, d, sched):
    kw = dict(SCHEDS[sched])
    if n < 7 and kw:
        pytest.skip("split schedules need n >= 7")
    p = inputs.orbit_invariant_dirichlet(n, seed=n)
    eng = _engine(n, [d], enable_literal=0, **kw)
    eng.set_p(p)
    q_ref = oracle.q_full(n, d, p[0])
    D_ref = oracle.D_full(n, d, q_ref)
    q64 = eng.get_q("fp64")[0]
    nz = q_ref > 0
    assert np.all(np.abs(q64[nz] - q_ref[nz]) <= 1e-12 * q_ref[nz])
    assert np.all(q64[~nz] == 0)
    D64 = eng.divergence(precision="fp64").cpu().numpy()[0]
    assert np.all(np.abs(D64 - D_ref) <= 1e-12 * np.maximum(1.0, np.abs(D_ref)))
    q32 = eng.get_q("fp32")[0]
    assert np.all(np.abs(q32[nz] - q_ref[nz]) <= 4e-6 * q_ref[nz])
    D32 = eng.divergence(precision="fp32").cpu().numpy()[0]
    assert np.all(np.abs(D32 - D_ref) <= 2e-5 * (1.0 + np.abs(D_ref)))
    eng.close()


@pytest.mark.parametrize("n,d", [(9, 0.5), (12, 0.8)])
def test_divergence_of_given_q(n, d):
    # any positive q: D uses q / sum q
    rng = np.random.default_rng(3)
    qh = rng.uniform(0.5, 2.0, size=2 << n)
    qh[0] = 0.0
    eng = _engine(n, [d], enable_literal=0)
    D = eng.divergence(torch.tensor(qh[None, :], device="cuda"), precision="fp64").cpu().numpy()[0]
    D_ref = oracle.D_full(n, d, qh / qh[1:].sum())
    assert np.all(np.abs(D - D_ref) <= 1e-12 * np.maximum(1.0, np.abs(D_ref)))
    eng.close()


@pytest.mark.parametrize("n,d", [(18, 0.7), (20, 0.5)])
def test_sampled_points_large(n, d):
    # full size: sampled outputs and inputs, each computed by the oracle one
    # by one from its definition
    p = inputs.orbit_invariant_dirichlet(n, seed=1)
    eng = _engine(n, [d], enable_literal=0)
    eng.set_p(p)
    q64 = eng.get_q("fp64")[0]
    for c in inputs.random_codes(n, 12, seed=2):
        ref = oracle.q_point(n, d, p[0], int(c))
        assert abs(q64[c] - ref) <= 1e-12 * ref
    D64 = eng.divergence(precision="fp64").cpu().numpy()[0]
    for x in inputs.random_inputs(n, 12, seed=3):
        ref = oracle.D_point(n, d, q64, int(x))
        assert abs(D64[x] - ref) <= 1e-11 * max(1.0, abs(ref))
    eng.close()


@pytest.mark.parametrize("prec,tq,tD", [("fp64", 1e-12, 1e-11), ("fp32", 4e-6, 2e-5)])
def test_sampled_points_register_steps(prec, tq, tD):
    # n = 18 split as n1 = 6, n2 = 12: both row kernels run register-resident
    # steps (forward: 2^5 or 2^4 inputs a thread; adjoint: the last 3 steps)
    n, d = 18, 0.45
    p = inputs.orbit_invariant_dirichlet(n, seed=5)
    eng = _engine(n, [d], enable_literal=0, use_regsteps=15, sched_n2_fp32=12, sched_w_fp32=32,
                  sched_n2_fp64=12, sched_w_fp64=32)
    s = eng.schedule(prec)
    assert (s["n1"], s["n2"]) == (6, 12)
    eng.set_p(p)
    q = eng.get_q(prec)[0]
    for c in inputs.random_codes(n, 12, seed=6):
        ref = oracle.q_point(n, d, p[0], int(c))
        assert abs(q[c] - ref) <= tq * ref
    D = eng.divergence(precision=prec).cpu().numpy()[0]
    q64 = eng.get_q("fp64")[0]
    for x in inputs.random_inputs(n, 12, seed=7):
        ref = oracle.D_point(n, d, q64, int(x))
        assert abs(D[x] - ref) <= tD * max(1.0, abs(ref))
    eng.close()


def test_batched_instances_are_independent():
    n = 10
    ds = [0.0, 0.2, 0.5, 0.95, 1.0]
    p = inputs.orbit_invariant_dirichlet(n, seed=5, nd=len(ds))
    eng = _engine(n, ds)
    eng.set_p(p)
    q = eng.get_q("fp64")
    D = eng.divergence(precision="fp64").cpu().numpy()
    for z, d in enumerate(ds):
        q_ref = oracle.q_full(n, d, p[z])
        nz = q_ref > 0
        assert np.all(np.abs(q[z][nz] - q_ref[nz]) <= 1e-12 * q_ref[nz])
        D_ref = oracle.D_full(n, d, q_ref)
        fin = np.isfinite(D_ref)
        assert np.all(np.abs(D[z][fin] - D_ref[fin]) <= 1e-12 * np.maximum(1.0, np.abs(D_ref[fin])))
    eng.close()


def test_full_size_bench_configuration():
    # n = 24 in the headline bench's launch configuration (split 11 + 13, 4
    # columns, half mode, register-resident and stepped iterations) against the
    # unstepped, all-shared-memory, full-mode kernels; then sampled outputs and
    # inputs of the resulting q and D against the oracle, one by one
    n, d = 24, 0.5
    sched = dict(sched_n2_fp32=13, sched_w_fp32=4, sched_n2_fp64=13, sched_w_fp64=4)
    eng = _engine(n, [d], enable_literal=0, **sched)
    assert (eng.schedule("fp32")["n1"], eng.schedule("fp32")["n2"]) == (11, 13)
    eng.iterate(3, -1.0, "fp64", "sweep")
    ref = _engine(n, [d], enable_literal=0, use_regsteps=0, fuse_update=0, use_half=0, **sched)
    ref.iterate(3, -1.0, "fp64", "sweep")
    la, ua = eng.history(0)
    lb, ub = ref.history(0)
    assert np.all(np.abs(la - lb) <= 1e-12 * np.abs(lb)) and np.all(np.abs(ua - ub) <= 1e-12 * np.abs(ub))
    ref.close()
    p = eng.get_p()[0]
    q = eng.get_q("fp64")[0]
    for c in [int((1 << 5) | 0b01101), int(inputs.random_codes(n, 1, seed=11)[0])]:
        r = oracle.q_point(n, d, p, c)
        assert abs(q[c] - r) <= 1e-12 * r
    D = eng.divergence(precision="fp64").cpu().numpy()[0]
    for x in inputs.random_inputs(n, 8, seed=12):
        r = oracle.D_point(n, d, q, int(x))
        assert abs(D[x] - r) <= 1e-11 * max(1.0, abs(r))
    eng.close()


def test_large_sweep_size_n26():
    # n = 26, the large sweep's size, in its launch configuration (FP32 stepped
    # iterations on the default schedule); then the FP64 q and D of the result
    # at sampled outputs and inputs against the oracle, each computed one by
    # one from its definition
    n, d = 26, 0.8
    eng = _engine(n, [d], enable_literal=0)
    eng.iterate(2, -1.0, "fp32", "sweep")
    lo, up = eng.history(0)
    assert len(lo) == 2 and np.all(lo <= up)
    p = eng.get_p()[0]
    q = eng.get_q("fp64")[0]
    for c in [int((1 << 7) | 0b1011001), int(inputs.random_codes(n, 1, seed=21)[0])]:
        r = oracle.q_point(n, d, p, c)
        assert abs(q[c] - r) <= 1e-12 * r
    D = eng.divergence(precision="fp64").cpu().numpy()[0]
    for x in inputs.random_inputs(n, 6, seed=22):
        r = oracle.D_point(n, d, q, int(x))
        assert abs(D[x] - r) <= 1e-11 * max(1.0, abs(r))
    eng.close()
