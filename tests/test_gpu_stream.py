"""The streaming schedule (one global-memory pass per input symbol), the one
FP64 runs at n >= 27 where no shared-memory tile split exists, forced here at
sizes the oracle covers: q and D against the definitions (Sec. 2.3), BA
iterations against the oracle's BA, the certificate against the oracle's
exact dual value, the smoothed dual bound and its gradients against the
oracle's, and agreement with the tiled schedules at n = 16."""
import numpy as np
import pytest

import oracle
from paper_2604_05867_b300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

STREAM = dict(sched_n2_fp64=-1, sched_n2_fp32=-1)


def _engine(n, ds, **kw):
    import paper_2604_05867_b300 as bdc
    return bdc.Engine(n, ds, options=bdc.default_options(**kw))


@pytest.mark.parametrize("n,d", [(3, 0.4), (8, 0.7), (11, 0.25), (13, 0.55)])
def test_stream_q_and_D_match_definition(n, d):
    eng = _engine(n, [d], enable_literal=0, **STREAM)
    assert eng.schedule("fp64")["n2"] == -1 and eng.schedule("fp32")["n2"] == -1
    p = inputs.orbit_invariant_dirichlet(n, seed=n + 1)
    eng.set_p(p)
    q_ref = oracle.q_full(n, d, p[0])
    D_ref = oracle.D_full(n, d, q_ref)
    q = eng.get_q("fp64")[0]
    assert np.all(np.abs(q[1:] - q_ref[1:]) <= 1e-12 * q_ref[1:])
    D = eng.divergence(precision="fp64").cpu().numpy()[0]
    assert np.all(np.abs(D - D_ref) <= 1e-12 * np.maximum(1.0, np.abs(D_ref)))
    q32 = eng.get_q("fp32")[0]
    assert np.all(np.abs(q32[1:] - q_ref[1:]) <= 4e-6 * q_ref[1:])
    D32 = eng.divergence(precision="fp32").cpu().numpy()[0]
    assert np.all(np.abs(D32 - D_ref) <= 2e-5 * (1.0 + np.abs(D_ref)))
    eng.close()


@pytest.mark.parametrize("n,d", [(7, 0.3), (10, 0.8)])
def test_stream_ba_iterations_match_oracle(n, d):
    T = 40
    ref = oracle.ba_bdc(n, d, T)
    eng = _engine(n, [d, 0.5], enable_literal=0, **STREAM)
    eng.iterate(T, -1.0, "fp64", "sweep")
    lo, up = eng.history(0)
    assert np.all(np.abs(lo - ref["lower"]) <= 1e-11) and np.all(np.abs(up - ref["upper"]) <= 1e-11)
    assert np.all(np.abs(eng.get_p()[0] - ref["p"]) <= 1e-9 * ref["p"])
    eng.close()


@pytest.mark.parametrize("n,d", [(10, 0.5), (12, 0.7)])
def test_stream_certificate_matches_oracle(n, d):
    eng = _engine(n, [d], enable_literal=0, **STREAM)
    eng.iterate(60, -1.0, "fp32", "sweep")
    c = eng.certify()
    p = eng.get_p()[0]
    eps = 2.0 ** -30
    U_ref, _ = oracle.certify(n, d, oracle.q_full(n, d, (1 - eps) * p + eps / (1 << n)))
    assert U_ref - 1e-12 <= c["upper"][0] <= U_ref + 1e-6
    assert 0 < c["margin"][0] < 1e-6
    rng = np.random.default_rng(n)
    qh = rng.uniform(0.1, 1.0, size=2 << n)
    qh[0] = 0.0
    cg = eng.certify(torch.tensor(qh[None, :], device="cuda"))
    Ug, _ = oracle.certify(n, d, qh)
    assert Ug - 1e-12 <= cg["upper"][0] <= Ug + 1e-6
    eng.close()


def test_stream_dual_bound_matches_oracle():
    n, d, tau = 8, 0.65, 0.05
    eng = _engine(n, [d], enable_literal=0, **STREAM)
    ocls, _, _ = oracle.output_classes(n)
    theta = np.random.default_rng(3).normal(scale=0.6, size=eng.num_output_classes)
    F_ref, g_ref, gd_ref = oracle.dual_bound(n, d, tau, theta, ocls)
    F, mD, g, gd = eng.dual_bound(0, torch.tensor(theta, dtype=torch.float64, device="cuda"), tau, "fp64")
    assert abs(F - F_ref) <= 1e-10 * max(1.0, abs(F_ref))
    assert np.all(np.abs(g.cpu().numpy() - g_ref) <= 1e-9 * np.maximum(1.0, np.abs(g_ref)))
    assert abs(gd - gd_ref) <= 1e-9 * max(1.0, abs(gd_ref))
    eng.close()


def test_stream_agrees_with_tiled_schedule():
    n, ds = 16, [0.3, 0.75]
    p = inputs.orbit_invariant_dirichlet(n, seed=9, nd=2)
    a = _engine(n, ds, enable_literal=0, sched_n2_fp64=-1)
    b = _engine(n, ds, enable_literal=0)
    assert b.schedule("fp64")["n2"] > 0
    a.set_p(p)
    b.set_p(p)
    qa, qb = a.get_q("fp64"), b.get_q("fp64")
    assert np.all(np.abs(qa[:, 1:] - qb[:, 1:]) <= 1e-13 * qb[:, 1:])
    Da = a.divergence(precision="fp64").cpu().numpy()
    Db = b.divergence(precision="fp64").cpu().numpy()
    assert np.all(np.abs(Da - Db) <= 1e-12 * np.maximum(1.0, np.abs(Db)))
    ca, cb = a.certify(), b.certify()
    assert np.all(np.abs(ca["upper"] - cb["upper"]) <= 1e-11)
    a.iterate(5, -1.0, "fp64", "sweep")
    b.iterate(5, -1.0, "fp64", "sweep")
    for z in range(2):
        la, ua = a.history(z)
        lb, ub = b.history(z)
        assert np.all(np.abs(la - lb) <= 1e-11) and np.all(np.abs(ua - ub) <= 1e-11)
    a.close()
    b.close()
