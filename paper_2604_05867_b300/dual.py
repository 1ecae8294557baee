"""Smoothed dual bound as a torch.autograd.Function, and direct optimisation
of the output distribution q.

F(theta) = tau log2 sum_x 2^{D_x(q)/tau} with q = softmax(theta) over output
orbit classes; max_x D_x(q) <= F <= max_x D_x(q) + tau n, and max_x D_x(q)
is an upper bound on C_n(d) for every q (minimax form of the capacity).  The
value and both gradients (theta, and d at fixed theta) come from the
library's sweep kernels (bdc_dual_bound); torch only carries the tensors and
runs the optimiser the caller chooses.
"""
from __future__ import annotations

import numpy as np


def _torch():
    import torch
    return torch


class DualBound:
    """``DualBound.apply(theta, engine, inst, tau, precision, d=None) -> F``
    (a 0-d tensor on theta's device).  ``d`` is an optional 0-d tensor
    holding the instance's deletion probability (it must equal the engine's
    d: the channel is fixed when the engine is built); when it requires
    grad, backward writes dF/dd (at fixed theta) into d.grad beside
    theta.grad.  The last call's F, max_x D_x and dF/dd are kept in
    ``DualBound.last``."""

    last = {}
    _fn = None

    @classmethod
    def apply(cls, theta, engine, inst: int = 0, tau: float = 1e-3, precision: str = "fp64", d=None):
        torch = _torch()
        if cls._fn is None:
            class _F(torch.autograd.Function):
                @staticmethod
                def forward(ctx, th, dd, eng, i, t, prec):
                    if float(dd) != eng.ds[i]:
                        raise ValueError("d must equal the engine's deletion probability of instance %d" % i)
                    want_d = bool(ctx.needs_input_grad[1])
                    F, mD, g, gd = eng.dual_bound(i, th.detach().contiguous(), t, prec, grad=True, grad_d=want_d)
                    ctx.save_for_backward(g, th.new_tensor(gd if want_d else 0.0, dtype=torch.float64))
                    ctx.d_dtype = dd.dtype
                    DualBound.last = {"F": F, "max_D": mD, "grad_d": gd}
                    return th.new_tensor(F)

                @staticmethod
                def backward(ctx, gF):
                    g, gd = ctx.saved_tensors
                    gdd = (gF.to(gd.dtype) * gd).to(ctx.d_dtype) if ctx.needs_input_grad[1] else None
                    return gF * g, gdd, None, None, None, None

            cls._fn = _F
        if d is None:
            d = torch.tensor(engine.ds[inst], dtype=torch.float64, device=theta.device)
        return cls._fn.apply(theta, d, engine, inst, tau, precision)


def class_representatives(engine) -> np.ndarray:
    """Representative code of every output class (class index order)."""
    cls = engine.output_classes()
    reps = np.full(engine.num_output_classes, -1, np.int64)
    codes = np.arange(len(cls))
    for c in codes[1:][::-1]:
        reps[cls[c]] = c
    return reps


def theta_from_q(engine, q, floor: float = 1e-300) -> np.ndarray:
    """Logits whose softmax over classes is q (q orbit-invariant, by code),
    computed by the library (bdc_class_logits)."""
    return engine.class_logits(q, "fp64", floor).cpu().numpy()


def optimize_dual(engine, inst: int = 0, tau: float = 1e-3, steps: int = 200, lr: float = 1e-2,
                  ba_iters: int = 50, precision: str = "fp32", theta0=None):
    """Initialise q from `ba_iters` BA iterations (FP32 sweep), take `steps`
    Adam steps on theta against the smoothed bound, then certify max_x D_x in
    FP64 for the final q.  Returns a dict with the history and the bounds."""
    torch = _torch()
    if theta0 is None:
        if ba_iters > 0:
            engine.iterate(ba_iters, -1.0, "fp32", "sweep")
        q0 = engine.get_q("fp64")[inst]
        theta0 = theta_from_q(engine, q0)
    dtype = torch.float32 if precision == "fp32" else torch.float64
    theta = torch.tensor(theta0, dtype=dtype, device=engine.device, requires_grad=True)
    q_init = engine.softmax_classes(inst, theta.detach().to(torch.float64).contiguous(), "fp64")
    cert0 = engine.certify(q_init.repeat(engine.nd, 1).contiguous())
    opt = torch.optim.Adam([theta], lr=lr, betas=(0.9, 0.999))
    hist = []
    for _ in range(steps):
        opt.zero_grad()
        F = DualBound.apply(theta, engine, inst, tau, precision)
        F.backward()
        opt.step()
        hist.append((float(F.item()), DualBound.last["max_D"]))
    q_fin = engine.softmax_classes(inst, theta.detach().to(torch.float64).contiguous(), "fp64")
    cert = engine.certify(q_fin.repeat(engine.nd, 1).contiguous())
    return {"theta": theta.detach(), "history": hist, "certified_initial": float(cert0["upper"][inst]),
            "certified_final": float(cert["upper"][inst]), "margin": float(cert["margin"][inst])}
