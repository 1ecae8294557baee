"""Workload of test_gpu_checked.py, run in a child process: a set of engine
calls covering every kernel family (single-pass, split, stepped, streaming
sweeps; literal walks; exact channels; certificate; divergence; dual bound;
counts; the allocation-free marginal), printed as JSON.  The library is the
release build, or the checked build when BDC_CHECKED=1."""
import ctypes
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def main():
    import torch

    import paper_2604_05867_b300 as bdc
    from paper_2604_05867_b300 import bounds, inputs

    out = {"lib": bdc.LIB_PATH}

    def run(name, n, ds, prec, impl="sweep", T=6, **kw):
        e = bdc.Engine(n, ds, options=bdc.default_options(**kw))
        e.iterate(T, -1.0, prec, impl)
        rec = {"hist": [list(map(float, e.history(z)[0])) + list(map(float, e.history(z)[1])) for z in range(e.nd)],
               "p": float(np.sum(e.get_p() * np.arange(1, (1 << n) + 1))),
               "cert": list(map(float, e.certify()["upper"]))}
        if impl == "sweep":
            rec["q64"] = float(np.sum(e.get_q("fp64")))
            rec["D64"] = float(e.divergence(precision="fp64").sum().item())
        out[name] = rec
        e.close()

    run("single", 10, [0.4], "fp64")
    run("split", 14, [0.3, 0.7], "fp64", sched_n2_fp64=8, sched_w_fp64=2)
    run("stepped", 19, [0.5], "fp32", sched_n2_fp32=8, sched_w_fp32=4, enable_literal=0)
    run("stream", 11, [0.6], "fp64", sched_n2_fp64=-1, enable_literal=0)
    run("literal", 12, [0.55], "fp64", impl="literal")
    e = bdc.Engine(8, lengths=bounds.exact_lengths(8, [2, 5]))
    e.iterate(8, -1.0, "fp64", "sweep")
    out["exact"] = list(map(float, e.certify()["upper"]))
    e.close()
    d = bdc.Engine(8, [0.7])
    th = torch.tensor(np.random.default_rng(0).normal(size=d.num_output_classes), device="cuda")
    F, mD, g, gd = d.dual_bound(0, th, 0.05, "fp64")
    out["dual"] = [F, mD, float(g.sum().item()), gd]
    d.close()
    xs = torch.tensor(inputs.random_inputs(16, 64, seed=1), device="cuda")
    N, S, _ = bdc.subseq_counts(16, xs)
    out["counts"] = [int(N.sum().item()), float(S.sum().item())]
    f = bdc.lib().bdc_output_marginal_static
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    p = torch.tensor(inputs.orbit_invariant_dirichlet(14, seed=3)[0], device="cuda")
    q = torch.zeros(2 << 14, dtype=torch.float64, device="cuda")
    assert f(14, 0.45, ctypes.c_void_p(p.data_ptr()), ctypes.c_void_p(q.data_ptr()), None) == 0
    torch.cuda.synchronize()
    out["static"] = float(q.sum().item())
    print(json.dumps(out))


if __name__ == "__main__":
    main()
