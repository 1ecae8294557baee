"""GPU parity of the smoothed dual bound and its adjoint (value, dF/dtheta,
dF/dd) against the oracle, central finite differences of the GPU's own FP64
value (h = 1e-6) on seeded random coordinates, and direct optimisation of q
tightening the certified bound."""
import numpy as np
import pytest

import oracle
from paper_2604_05867_b300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _bdc():
    import paper_2604_05867_b300 as bdc
    return bdc


@pytest.mark.parametrize("n,d,tau", [(4, 0.6, 0.05), (7, 0.8, 0.02), (9, 0.35, 0.1)])
def test_dual_bound_matches_oracle(n, d, tau):
    bdc = _bdc()
    eng = bdc.Engine(n, [d], options=bdc.default_options(enable_literal=0))
    cls = eng.output_classes()
    ocls, _, _ = oracle.output_classes(n)
    assert np.array_equal(cls[1:], ocls[1:])
    rng = np.random.default_rng(n)
    theta = rng.normal(scale=0.7, size=eng.num_output_classes)
    F_ref, g_ref, gd_ref = oracle.dual_bound(n, d, tau, theta, ocls)
    th = torch.tensor(theta, dtype=torch.float64, device="cuda")
    F, mD, g, gd = eng.dual_bound(0, th, tau, "fp64", grad=True)
    assert abs(F - F_ref) <= 1e-10 * max(1.0, abs(F_ref))
    g = g.cpu().numpy()
    assert np.all(np.abs(g - g_ref) <= 1e-9 * np.maximum(1.0, np.abs(g_ref)))
    assert abs(gd - gd_ref) <= 1e-9 * max(1.0, abs(gd_ref))
    # FP32 path: same quantities to FP32 rounding
    F32, _, g32, gd32 = eng.dual_bound(0, th.float(), tau, "fp32", grad=True)
    assert abs(F32 - F_ref) <= 2e-4 * max(1.0, abs(F_ref))
    assert np.all(np.abs(g32.cpu().numpy() - g_ref) <= 2e-3 * np.maximum(1.0, np.abs(g_ref)))
    eng.close()


def test_gradient_central_differences():
    # h = 1e-6, FP64, on seeded random coordinates of theta and on d
    bdc = _bdc()
    n, d, tau, h = 12, 0.8, 1e-2, 1e-6
    eng = bdc.Engine(n, [d], options=bdc.default_options(enable_literal=0))
    eng.iterate(30, -1.0, "fp32", "sweep")
    from paper_2604_05867_b300 import dual
    theta = dual.theta_from_q(eng, eng.get_q("fp64")[0])
    th = torch.tensor(theta, dtype=torch.float64, device="cuda")
    F, _, g, gd = eng.dual_bound(0, th, tau, "fp64", grad=True)
    g = g.cpu().numpy()
    for i in inputs.fd_coordinates(len(theta), 32, seed=0):
        tp, tm = th.clone(), th.clone()
        tp[i] += h
        tm[i] -= h
        fd = (eng.dual_bound(0, tp, tau, "fp64", grad=False)[0] - eng.dual_bound(0, tm, tau, "fp64", grad=False)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-5 * max(1e-3, abs(g[i])) + 1e-8, (i, fd, g[i])
    ep = bdc.Engine(n, [d + h], options=bdc.default_options(enable_literal=0))
    em = bdc.Engine(n, [d - h], options=bdc.default_options(enable_literal=0))
    fdd = (ep.dual_bound(0, th, tau, "fp64", grad=False)[0] - em.dual_bound(0, th, tau, "fp64", grad=False)[0]) / (2 * h)
    assert abs(fdd - gd) <= 1e-5 * max(1.0, abs(gd))
    for e in (eng, ep, em):
        e.close()


def test_autograd_and_direct_optimisation_tightens_bound():
    bdc = _bdc()
    from paper_2604_05867_b300 import dual
    n, d = 12, 0.8
    eng = bdc.Engine(n, [d], options=bdc.default_options(enable_literal=0))
    # autograd wrapper gives the same gradient as the direct call
    th = torch.zeros(eng.num_output_classes, dtype=torch.float64, device="cuda", requires_grad=True)
    F = dual.DualBound.apply(th, eng, 0, 0.05, "fp64")
    F.backward()
    _, _, g, _ = eng.dual_bound(0, th.detach(), 0.05, "fp64", grad=True)
    assert torch.allclose(th.grad, g, rtol=1e-12, atol=1e-15)
    res = dual.optimize_dual(eng, 0, tau=1e-3, steps=60, lr=1e-2, ba_iters=20, precision="fp32")
    assert res["certified_final"] <= res["certified_initial"] + 1e-9
    # a certified bound is never below the capacity's BA lower bound
    lo = oracle.ba_bdc(n, d, 1, p0=None)["lower"][0] if n <= 12 else 0.0
    assert res["certified_final"] >= lo
    eng.close()


@pytest.mark.parametrize("n,d,tau", [(8, 0.7, 0.05), (9, 0.45, 0.02)])
def test_autograd_d_gradient_matches_oracle(n, d, tau):
    # d enters the autograd Function as a 0-d tensor: backward gives dF/dd
    # (theta fixed) beside dF/dtheta, both against the oracle's gradient
    bdc = _bdc()
    from paper_2604_05867_b300 import dual
    eng = bdc.Engine(n, [d], options=bdc.default_options(enable_literal=0))
    ocls, _, _ = oracle.output_classes(n)
    rng = np.random.default_rng(7 + n)
    theta = rng.normal(scale=0.5, size=eng.num_output_classes)
    F_ref, g_ref, gd_ref = oracle.dual_bound(n, d, tau, theta, ocls)
    th = torch.tensor(theta, dtype=torch.float64, device="cuda", requires_grad=True)
    dt = torch.tensor(d, dtype=torch.float64, device="cuda", requires_grad=True)
    F = dual.DualBound.apply(th, eng, 0, tau, "fp64", d=dt)
    (2.0 * F).backward()
    assert abs(F.item() - F_ref) <= 1e-10 * max(1.0, abs(F_ref))
    assert abs(dt.grad.item() - 2.0 * gd_ref) <= 1e-9 * max(1.0, abs(gd_ref))
    assert np.all(np.abs(th.grad.cpu().numpy() - 2.0 * g_ref) <= 1e-9 * np.maximum(1.0, np.abs(g_ref)))
    with pytest.raises(ValueError):
        dual.DualBound.apply(th, eng, 0, tau, "fp64", d=torch.tensor(d + 0.1, dtype=torch.float64, device="cuda"))
    eng.close()


def test_class_logits_invert_the_softmax():
    bdc = _bdc()
    from paper_2604_05867_b300 import dual
    n, d = 10, 0.6
    eng = bdc.Engine(n, [d], options=bdc.default_options(enable_literal=0))
    eng.iterate(5, -1.0, "fp64", "sweep")
    q = eng.get_q("fp64")[0]
    theta = dual.theta_from_q(eng, q)
    cls = eng.output_classes()
    # the logits are ln q at each class's codes
    assert np.allclose(theta[cls[1:]], np.log(q[1:]), rtol=0, atol=1e-12)
    q2 = eng.softmax_classes(0, torch.tensor(theta, dtype=torch.float64, device="cuda")).cpu().numpy()
    assert np.all(np.abs(q2[1:] - q[1:]) <= 1e-12 * q[1:])
    eng.close()
