"""The allocation-free output marginal, bdc_output_marginal_static.

Some callers cannot allocate device memory (inside another component's CUDA
graph capture, under a host framework that owns every allocation, or under
strict memory accounting).  This entry point keeps its scratch in a fixed
array inside the library instead.  Here it is called through the C ABI and
compared with the engine's output marginal (bdc_get_q), to the 1e-12
relative tolerance of the other FP64 marginal tests, on two calls in a row;
calls of different sizes share the same scratch; sizes beyond the fixed
array are rejected with a clear error."""
import ctypes

import numpy as np
import pytest

from paper_2604_05867_b300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _fn():
    import paper_2604_05867_b300 as bdc
    f = bdc.lib().bdc_output_marginal_static
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    return bdc, f


def _engine_q(bdc, n, d, p):
    eng = bdc.Engine(n, [d], options=bdc.default_options(enable_literal=0))
    eng.set_p(p)
    q = eng.get_q("fp64")[0]
    eng.close()
    return q


def _static_q(bdc, f, n, d, p):
    p_dev = torch.tensor(p[0], dtype=torch.float64, device="cuda")
    q_dev = torch.full((2 << n,), float("nan"), dtype=torch.float64, device="cuda")
    s = torch.cuda.current_stream()
    st = f(n, d, ctypes.c_void_p(p_dev.data_ptr()), ctypes.c_void_p(q_dev.data_ptr()), ctypes.c_void_p(s.cuda_stream))
    assert st == 0, bdc.lib().bdc_last_error()
    torch.cuda.synchronize()
    return q_dev.cpu().numpy()


@pytest.mark.parametrize("n,d", [(16, 0.7), (11, 0.35)])
def test_static_marginal_matches_engine_on_two_calls(n, d):
    bdc, f = _fn()
    p = inputs.orbit_invariant_dirichlet(n, seed=n)
    q_ref = _engine_q(bdc, n, d, p)
    for _ in range(2):
        q = _static_q(bdc, f, n, d, p)
        assert q[0] == 0.0
        assert np.all(np.abs(q[1:] - q_ref[1:]) <= 1e-12 * q_ref[1:])


def test_static_marginal_shared_scratch_and_limit():
    bdc, f = _fn()
    pa = inputs.orbit_invariant_dirichlet(18, seed=1)
    pb = inputs.orbit_invariant_dirichlet(14, seed=2)
    qa_ref = _engine_q(bdc, 18, 0.5, pa)
    qb_ref = _engine_q(bdc, 14, 0.9, pb)
    qa = _static_q(bdc, f, 18, 0.5, pa)
    qb = _static_q(bdc, f, 14, 0.9, pb)
    assert np.all(np.abs(qa[1:] - qa_ref[1:]) <= 1e-12 * qa_ref[1:])
    assert np.all(np.abs(qb[1:] - qb_ref[1:]) <= 1e-12 * qb_ref[1:])
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    st = f(19, 0.5, ctypes.c_void_p(dummy.data_ptr()), ctypes.c_void_p(dummy.data_ptr()), None)
    assert st == -1 and b"18" in bdc.lib().bdc_last_error()
