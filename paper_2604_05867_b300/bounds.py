"""Bounds on the deletion-channel capacity C(d) from certified finite-length
results (Sec. 2.2 and Sec. 6).

- ``exact_capacities``: certified upper bounds on the exact-channel
  capacities C_{n,k} (BDC_{n,k}: a uniformly random length-k subsequence of
  x), all k in one engine of length-mixture instances, iterated and
  certified by the library's kernels.
- ``prob_vs_exact``, ``split_bound``, ``high_noise``: Lemma prob-vs-exact,
  Lemma worse-UB and Lemma convex (Rahmati and Duman), evaluated by the
  library's host routines (bdc_bound_*).
- ``ck_table`` / ``cd_table``: the results in the layout of the paper's
  tables of C_{n,k} and of C(d), values rounded up to 4 decimals (they are
  upper bounds).
"""
from __future__ import annotations

import ctypes
import math
from typing import Dict, Optional, Sequence

import numpy as np


def _lib():
    import paper_2604_05867_b300 as bdc
    L = bdc.lib()
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    for name, args in (("bdc_bound_prob_vs_exact", [I, D, P, P]), ("bdc_bound_split", [I, I, I, P, P, P]),
                       ("bdc_bound_high_noise", [D, D, D, P, P])):
        f = getattr(L, name)
        f.restype = I
        f.argtypes = args
    return bdc, L


def exact_lengths(n: int, ks: Sequence[int]) -> np.ndarray:
    """Length distributions of the exact channels BDC_{n,k}: one-hot rows."""
    b = np.zeros((len(ks), n + 1))
    for r, k in enumerate(ks):
        b[r, int(k)] = 1.0
    return b


def prob_vs_exact(n: int, d: float, Cnk: Sequence[float]) -> float:
    """sum_{k=1}^n C(n,k) d^(n-k) (1-d)^k Cnk[k] >= C_n(d) (Cnk[0] unused)."""
    bdc, L = _lib()
    c = np.ascontiguousarray(Cnk, np.float64)
    if len(c) != n + 1:
        raise ValueError("Cnk needs n+1 entries")
    out = ctypes.c_double(0)
    bdc._check(L.bdc_bound_prob_vs_exact(int(n), float(d), c.ctypes.data_as(ctypes.c_void_p), ctypes.byref(out)))
    return out.value


def split_bound(n: int, k: int, s: int, Cs: Sequence[float], Cns: Sequence[float]) -> float:
    """Lemma worse-UB: a bound on C_{n,k} from bounds on C_{s,i} (Cs[i]) and
    C_{n-s,j} (Cns[j])."""
    bdc, L = _lib()
    a = np.ascontiguousarray(Cs, np.float64)
    b = np.ascontiguousarray(Cns, np.float64)
    if len(a) != s + 1 or len(b) != n - s + 1:
        raise ValueError("Cs needs s+1 and Cns n-s+1 entries")
    out = ctypes.c_double(0)
    bdc._check(L.bdc_bound_split(int(n), int(k), int(s), a.ctypes.data_as(ctypes.c_void_p),
                                 b.ctypes.data_as(ctypes.c_void_p), ctypes.byref(out)))
    return out.value


def high_noise(d_prime: float, C_dprime: float, d: Optional[float] = None):
    """Lemma convex: (bound on C(d) for d in [d', 1] or None, bound on
    C(d')/(1-d'))."""
    bdc, L = _lib()
    cd = ctypes.c_double(0)
    r = ctypes.c_double(0)
    dd = float(d_prime if d is None else d)
    bdc._check(L.bdc_bound_high_noise(float(d_prime), float(C_dprime), dd, ctypes.byref(cd), ctypes.byref(r)))
    return (None if d is None else cd.value), r.value


def ceil4(v: float) -> float:
    """Round an upper bound up to 4 decimals (the tables' precision)."""
    return math.ceil(v * 1e4 - 1e-9) / 1e4


def exact_capacities(n: int, ks: Optional[Sequence[int]] = None, iters: int = 2000, tol: float = 1e-4,
                     precision: str = "fp32", options=None, stream=None) -> Dict[int, dict]:
    """Certified upper bounds on C_{n,k} for every k in ks (default 1..n):
    one engine of exact-channel instances (bdc_create_lengths), BA
    iterations until each gap is below tol bits or `iters` iterations, then
    the FP64 certificate (Sec. 2.3 minimax bound, rounding margin included).
    Returns {k: dict(upper, lower, margin, iters)}."""
    import paper_2604_05867_b300 as bdc
    ks = list(range(1, n + 1)) if ks is None else [int(k) for k in ks]
    eng = bdc.Engine(n, lengths=exact_lengths(n, ks), options=options, stream=stream)
    try:
        lo, up, it = eng.iterate(iters, tol, precision, "sweep")
        c = eng.certify()
        out = {}
        for r, k in enumerate(ks):
            out[k] = {"upper": float(c["upper"][r]), "lower": float(c["lower"][r]), "margin": float(c["margin"][r]),
                      "iters": int(it[r]), "ba_lower": float(lo[r]), "ba_upper": float(up[r])}
        return out
    finally:
        eng.close()


def ck_table(n: int, Ck: Dict[int, float]) -> str:
    """'k & bound' rows like the paper's table of C_{n,k} (4 decimals, up)."""
    rows = ["k & Upper bound on C_{%d,k} \\\\" % n]
    for k in sorted(Ck):
        rows.append("%d & %.4f \\\\" % (k, ceil4(Ck[k])))
    return "\n".join(rows)


def cd_table(ds: Sequence[float], by_n: Dict[int, Sequence[float]]) -> list:
    """C(d) <= min over n of (1/n) prob_vs_exact(n, d, Cnk): rows (d, bound,
    best n), like the paper's table of C(d).  by_n maps n to its bounds
    Cnk[0..n]."""
    rows = []
    for d in ds:
        best = None
        for n, Cnk in by_n.items():
            v = prob_vs_exact(n, d, Cnk) / n
            if best is None or v < best[0]:
                best = (v, n)
        rows.append((float(d), best[0], best[1]))
    return rows
