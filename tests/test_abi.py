"""The C-ABI library loads on a CPU-only host and exports every function
declared in include/bdc.h (no compute calls without a GPU); argument
validation that needs no device works; the build compiles for sm_103a."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bdc.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(bdc_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("bdc_create", "bdc_workspace_bytes", "bdc_bind", "bdc_destroy", "bdc_ba_iterate",
                     "bdc_divergence", "bdc_certify_upper", "bdc_get_p", "bdc_set_p", "bdc_get_q",
                     "bdc_subseq_counts", "bdc_last_error", "bdc_dual_bound", "bdc_save", "bdc_load"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2604_05867_b300 import build
    build.build()
    L = ctypes.CDLL(build.LIB)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_create_validates_without_gpu():
    import paper_2604_05867_b300 as bdc
    L = bdc.lib()
    h = ctypes.c_void_p()
    d = (ctypes.c_double * 1)(0.5)
    assert L.bdc_create(0, ctypes.cast(d, ctypes.c_void_p), 1, None, ctypes.byref(h)) == -1
    assert L.bdc_create(29, ctypes.cast(d, ctypes.c_void_p), 1, None, ctypes.byref(h)) == -1
    bad = (ctypes.c_double * 1)(1.5)
    assert L.bdc_create(10, ctypes.cast(bad, ctypes.c_void_p), 1, None, ctypes.byref(h)) == -1
    assert b"[0, 1]" in L.bdc_last_error()
    assert L.bdc_create(20, ctypes.cast(d, ctypes.c_void_p), 1, None, ctypes.byref(h)) == 0
    ws = L.bdc_workspace_bytes(h)
    assert ws > (1 << 20) * 4 * 6  # at least the FP32 p, D, Hb and q, L arrays
    # no workspace bound yet: iteration is refused, not run
    lo = (ctypes.c_double * 1)()
    assert L.bdc_ba_iterate(h, 1, -1.0, 0, 0, ctypes.cast(lo, ctypes.c_void_p), None, None) == -6
    L.bdc_destroy(h)


def test_sched_and_workspace_scale():
    import paper_2604_05867_b300 as bdc
    L = bdc.lib()
    d = (ctypes.c_double * 1)(0.5)
    sizes = []
    for n in (10, 16, 22):
        h = ctypes.c_void_p()
        assert L.bdc_create(n, ctypes.cast(d, ctypes.c_void_p), 1, None, ctypes.byref(h)) == 0
        sizes.append(L.bdc_workspace_bytes(h))
        L.bdc_destroy(h)
    assert sizes[0] < sizes[1] < sizes[2]


@pytest.mark.parametrize("n", [26, 27, 28])
def test_schedules_up_to_n28(n):
    # FP32 splits n into shared-memory column and row tiles up to n = 28; FP64
    # (half the elements per tile) only up to n = 26, and streams beyond; the
    # workspace of one instance stays within the device's memory
    import paper_2604_05867_b300 as bdc
    L = bdc.lib()
    d = (ctypes.c_double * 1)(0.5)
    opt = bdc.default_options(enable_literal=0)
    h = ctypes.c_void_p()
    assert L.bdc_create(n, ctypes.cast(d, ctypes.c_void_p), 1, ctypes.byref(opt), ctypes.byref(h)) == 0
    n1, n2, w = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    assert L.bdc_get_schedule(h, 0, ctypes.byref(n1), ctypes.byref(n2), ctypes.byref(w)) == 0
    assert n2.value > 0 and n1.value + n2.value == n
    assert (2 << n1.value) * w.value <= 32768 and (2 << n2.value) <= 32768
    assert L.bdc_get_schedule(h, 1, ctypes.byref(n1), ctypes.byref(n2), ctypes.byref(w)) == 0
    if n <= 26:
        assert n2.value > 0 and (2 << n1.value) * w.value <= 16384 and (2 << n2.value) <= 16384
    else:
        assert n2.value == -1
    assert L.bdc_workspace_bytes(h) < 200e9
    L.bdc_destroy(h)


def test_checked_build_exports_every_declared_symbol():
    from paper_2604_05867_b300 import build
    if not os.path.exists(build.LIB_CHECKS):
        pytest.skip("checked build not compiled")
    L = ctypes.CDLL(build.LIB_CHECKS)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing
