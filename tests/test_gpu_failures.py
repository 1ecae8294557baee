"""Failure paths reported as status codes, without any GPU fault.

- BDC_ENONFINITE: an input distribution with zero mass on every input but
  one leaves outputs with q(y) = 0 that other inputs reach, so (with the
  floor under q switched off) D_x = +Inf reaches the bounds' reductions; a NaN placed by the host into a given q
  reaches the certificate.  The instance stops, the call returns the status,
  and the engine and the CUDA context stay usable.
- BDC_EINVAL from the device check of a given q that is not positive.
- BDC_ETIMEOUT: the TMA tile wait of the column kernel is given no poll at
  all (tma_wait_polls < 0), so it gives up at once; each CTA records the
  status, waits (bounded) for its copies in flight and returns; the next
  kernels skip the stopped instance; the host reads the status.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _bdc():
    import paper_2604_05867_b300 as bdc
    return bdc


def test_zero_mass_input_gives_nonfinite_status_and_engine_recovers():
    bdc = _bdc()
    n, d = 10, 0.5
    # q_floor = 0: no floor under the output marginal before its log
    eng = bdc.Engine(n, [d, 0.3], options=bdc.default_options(enable_literal=0, q_floor=0.0))
    p = np.full((2, 1 << n), 1.0 / (1 << n))
    p[0] = 0.0
    p[0, 0] = 1.0  # all mass on 0^n: outputs containing a 1 get q = 0
    eng.set_p(p)
    with pytest.raises(bdc.BdcError) as ei:
        eng.iterate(3, -1.0, "fp64", "sweep")
    assert ei.value.status == -5
    # the other instance iterated normally
    lo, up = eng.history(1)
    assert len(lo) == 3 and np.all(np.isfinite(lo)) and np.all(lo <= up + 1e-12)
    # the engine and the context stay usable
    eng.set_p(np.full((2, 1 << n), 1.0 / (1 << n)))
    lo, up, it = eng.iterate(4, -1.0, "fp64", "sweep")
    assert list(it) == [4, 4] and np.all(np.isfinite(lo))
    torch.cuda.synchronize()
    eng.close()


@pytest.mark.parametrize("n,sched", [(8, {}), (14, dict(sched_n2_fp64=8, sched_w_fp64=2))])
def test_given_q_with_nan_or_zero(n, sched):
    bdc = _bdc()
    d = 0.6
    eng = bdc.Engine(n, [d, d], options=bdc.default_options(enable_literal=0, **sched))
    rng = np.random.default_rng(n)
    q = rng.uniform(0.1, 1.0, size=(2, 2 << n))
    q[:, 0] = 0.0
    q[0, 5] = np.nan
    with pytest.raises(bdc.BdcError) as ei:
        eng.certify(torch.tensor(q, device="cuda"))
    assert ei.value.status == -5
    q[0, 5] = 0.0
    with pytest.raises(bdc.BdcError) as ei:
        eng.certify(torch.tensor(q, device="cuda"))
    assert ei.value.status == -1
    q[0, 5] = 0.5
    c = eng.certify(torch.tensor(q, device="cuda"))
    assert np.all(np.isfinite(c["upper"]))
    eng.close()


def test_tma_wait_timeout_status():
    bdc = _bdc()
    n, d = 18, 0.5
    kw = dict(sched_n2_fp32=8, sched_w_fp32=4, enable_literal=0, use_tma=1)
    eng = bdc.Engine(n, [d], options=bdc.default_options(tma_wait_polls=-1, **kw))
    assert eng.schedule("fp32") == {"n1": 10, "n2": 8, "width": 4}
    with pytest.raises(bdc.BdcError) as ei:
        eng.iterate(3, -1.0, "fp32", "sweep")
    assert ei.value.status == -4
    torch.cuda.synchronize()
    eng.close()
    # the same configuration with the default bound runs normally afterwards
    ok = bdc.Engine(n, [d], options=bdc.default_options(**kw))
    lo, up, it = ok.iterate(3, -1.0, "fp32", "sweep")
    assert it[0] == 3 and np.isfinite(lo[0]) and lo[0] <= up[0]
    ok.close()
