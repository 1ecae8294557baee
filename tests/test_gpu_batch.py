"""Batched form: several engines (different n, several d each) iterated by one
CUDA graph must give the same bounds as the oracle's BA for every instance,
and the same bits as iterating each engine alone."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_batch_matches_oracle_and_single_engines():
    import paper_2604_05867_b300 as bdc
    stream = torch.cuda.Stream()
    spec = {8: [0.3, 0.7], 10: [0.5, 0.6, 0.9], 15: [0.8]}
    opts = bdc.default_options(enable_literal=0)
    engs = [bdc.Engine(n, ds, options=opts, stream=stream) for n, ds in spec.items()]
    batch = bdc.Batch(engs, chunk=8)
    ran = batch.iterate(24, -1.0, "fp64")
    assert ran == 24
    for eng, (n, ds) in zip(engs, spec.items()):
        for z, d in enumerate(ds):
            lo, up = eng.history(z)
            assert len(lo) == 24
            if n <= 10:
                ref = oracle.ba_bdc(n, d, 24)
                assert np.all(np.abs(lo - ref["lower"]) <= 1e-11)
                assert np.all(np.abs(up - ref["upper"]) <= 1e-11)
        # the same engine alone, same number of iterations: identical bits
        alone = bdc.Engine(n, ds, options=opts, stream=stream)
        alone.iterate(24, -1.0, "fp64", "sweep")
        assert np.array_equal(alone.get_p(), eng.get_p())
        alone.close()
    # FP32 batch keeps going from the FP64 state, with a stopping tolerance
    ran = batch.iterate(64, 1e-3, "fp32")
    assert ran >= 8
    batch.close()
    for e in engs:
        e.close()


def test_autotune_keeps_results_and_caches(tmp_path):
    import paper_2604_05867_b300 as bdc
    n, d = 17, 0.6
    eng = bdc.Engine(n, [d], options=bdc.default_options(enable_literal=0))
    eng.iterate(5, -1.0, "fp64", "sweep")
    q_before = eng.get_q("fp64")
    cache = str(tmp_path / "sched.json")
    s = eng.autotune("fp64", reps=1, cache=cache)
    assert not s["cached"] and 8 <= s["n2"] <= 13
    # schedules change the summation grouping only: q within FP64 rounding
    q_after = eng.get_q("fp64")
    nz = q_before > 0
    assert np.all(np.abs(q_after[nz] - q_before[nz]) <= 1e-12 * q_before[nz])
    eng.iterate(3, -1.0, "fp64", "sweep")
    other = bdc.Engine(n, [d], options=bdc.default_options(enable_literal=0))
    s2 = other.autotune("fp64", cache=cache)
    assert s2["cached"] and s2["n2"] == s["n2"] and s2["width"] == s["width"]
    assert other.schedule("fp64")["n2"] == s["n2"]
    eng.close()
    other.close()
