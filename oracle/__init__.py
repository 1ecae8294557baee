"""FP64 CPU oracle for Blahut-Arimoto on the binary deletion channel BDC_d.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA library (``paper_2604_05867_b300``)
and never imports it.

Everything here is the paper's definitions written out plainly (Sec. 2.2
channel rule, Sec. 2.3 Blahut-Arimoto, Sec. 4 unranking, Sec. 5 supersequence
enumeration, Appendix A orbits), in ``bdc_oracle.c`` compiled with gcc, plus
thin numpy wrappers.  Parity status of each function is stated in its
docstring; all are pinned by ``-m "not gpu"`` tests (tests/test_oracle_*.py).

Encoding: a string s of length L is the integer with s_0 as its most
significant bit; an output y of length k has code ``(1 << k) | y``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bdc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_u64 = ctypes.c_uint64
_i64 = ctypes.c_int64
_int = ctypes.c_int
_dbl = ctypes.c_double
_P = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile bdc_oracle.c into liboracle.so with gcc (OpenMP on)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            sig = {
                "orc_embed_count": (_u64, [_int, _u64, _int, _u64]),
                "orc_channel_row_bruteforce": (None, [_int, _u64, _dbl, _P, _P]),
                "orc_subseq_stats": (None, [_int, _u64, _P, _P, _P]),
                "orc_subseq_list": (_i64, [_int, _u64, _P, _P]),
                "orc_q_full": (None, [_int, _dbl, _P, _P]),
                "orc_q_point": (_dbl, [_int, _dbl, _P, _u64]),
                "orc_D_point": (_dbl, [_int, _dbl, _P, _u64]),
                "orc_D_full": (None, [_int, _dbl, _P, _P]),
                "orc_certify": (_dbl, [_int, _dbl, _P, _P]),
                "orc_ba_sparse": (_int, [_i64, _i64, _P, _P, _P, _P, _int, _dbl, _P, _P, _P]),
                "orc_bdc_rows": (_i64, [_int, _dbl, _P, _P, _P]),
                "orc_exact_rows": (_i64, [_int, _int, _P, _P, _P]),
                "orc_nextpos_cnt": (None, [_int, _u64, _int, _P, _P]),
                "orc_unrank": (_int, [_int, _u64, _int, _u64, _P]),
                "orc_subset_unrank": (_int, [_int, _int, _u64, _P]),
                "orc_recsuperseq": (_u64, [_u64, _int, _int, _u64, _int]),
                "orc_orbit_rep": (_u64, [_u64, _int, _P]),
                "orc_dual_bound": (_dbl, [_int, _dbl, _dbl, _P, _P, _i64, _P, _P]),
                "orc_D_list": (None, [_int, _dbl, _P, _P, _i64, _P]),
                "orc_pairs_list": (_i64, [_int, _P, _i64]),
                "orc_set_threads": (_int, [_int]),
                "orc_sweep_forward": (None, [_int, _dbl, _dbl, _P, _P]),
                "orc_sweep_adjoint": (None, [_int, _dbl, _dbl, _P, _P]),
                "orc_subseq_S_list": (None, [_int, _P, _i64, _P]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# --------------------------------------------------------------------------
# Channel (Sec. 2.2)
# --------------------------------------------------------------------------
def embed_count(n: int, x: int, k: int, y: int) -> int:
    """#times y (length k) appears as a subsequence of x (length n); DP."""
    return int(lib().orc_embed_count(n, x, k, y))


def channel_row_bruteforce(n: int, x: int, d: float):
    """(counts, W) over all 2^(n+1) codes, by enumerating all 2^n deletion
    patterns of x (the definition of BDC_d, Sec. 1 / Sec. 2.2)."""
    cnt = np.zeros(1 << (n + 1), np.uint64)
    W = np.zeros(1 << (n + 1), np.float64)
    lib().orc_channel_row_bruteforce(n, x, float(d), _ptr(cnt), _ptr(W))
    return cnt, W


def subseq_stats(n: int, x: int):
    """Per length k=0..n: N_k (#distinct subsequences, Sec. 4.1's N_{x,k}),
    S_k = sum count*log2(count), and sum of counts (= C(n,k))."""
    N = np.zeros(n + 1, np.uint64)
    S = np.zeros(n + 1, np.float64)
    sc = np.zeros(n + 1, np.uint64)
    lib().orc_subseq_stats(n, x, _ptr(N), _ptr(S), _ptr(sc))
    return N, S, sc


def subseq_list(n: int, x: int):
    """All nonempty distinct subsequences of x as (codes, counts)."""
    m = lib().orc_subseq_list(n, x, None, None)
    codes = np.zeros(m, np.uint64)
    counts = np.zeros(m, np.uint64)
    lib().orc_subseq_list(n, x, _ptr(codes), _ptr(counts))
    return codes, counts


# --------------------------------------------------------------------------
# Output marginal, divergence, dual bound (Sec. 2.3)
# --------------------------------------------------------------------------
def q_full(n: int, d: float, p: np.ndarray) -> np.ndarray:
    """q(y) = sum_x p(x) W(y|x) over all codes (slot 0 = 0)."""
    p = np.ascontiguousarray(p, np.float64)
    q = np.zeros(1 << (n + 1), np.float64)
    lib().orc_q_full(n, float(d), _ptr(p), _ptr(q))
    return q


def q_point(n: int, d: float, p: np.ndarray, code: int) -> float:
    """q at one output code, summing over all 2^n inputs."""
    p = np.ascontiguousarray(p, np.float64)
    return float(lib().orc_q_point(n, float(d), _ptr(p), int(code)))


def D_point(n: int, d: float, q: np.ndarray, x: int) -> float:
    """D_x = sum_y W(y|x) log2(W(y|x)/q(y)) for q indexed by code."""
    q = np.ascontiguousarray(q, np.float64)
    return float(lib().orc_D_point(n, float(d), _ptr(q), int(x)))


def D_full(n: int, d: float, q: np.ndarray) -> np.ndarray:
    q = np.ascontiguousarray(q, np.float64)
    D = np.zeros(1 << n, np.float64)
    lib().orc_D_full(n, float(d), _ptr(q), _ptr(D))
    return D


def D_list(n: int, d: float, q: np.ndarray, xs: np.ndarray) -> np.ndarray:
    """D_x for the given inputs (OpenMP over the list)."""
    q = np.ascontiguousarray(q, np.float64)
    xs = np.ascontiguousarray(xs, np.uint64)
    D = np.zeros(len(xs), np.float64)
    lib().orc_D_list(n, float(d), _ptr(q), _ptr(xs), len(xs), _ptr(D))
    return D


def pairs_list(n: int, xs: np.ndarray) -> int:
    """Number of (x, distinct y) pairs, the empty output included, that the
    divergence walk over these inputs enumerates."""
    xs = np.ascontiguousarray(xs, np.uint64)
    return int(lib().orc_pairs_list(n, _ptr(xs), len(xs)))


def set_threads(t: int) -> int:
    """Threads of the oracle's OpenMP loops (t <= 0 keeps the current
    setting); returns the number in use."""
    return int(lib().orc_set_threads(int(t)))


def certify(n: int, d: float, q: np.ndarray):
    """max_x D(W_x || q/sum q) for any positive q, and the argmax input."""
    q = np.ascontiguousarray(q, np.float64)
    arg = np.zeros(1, np.int64)
    U = float(lib().orc_certify(n, float(d), _ptr(q), _ptr(arg)))
    return U, int(arg[0])


# --------------------------------------------------------------------------
# Blahut-Arimoto (Sec. 2.3)
# --------------------------------------------------------------------------
def bdc_rows(n: int, d: float):
    """Sparse rows (rowptr, col=code, val=W) of BDC_d by brute force."""
    L = lib()
    nnz = L.orc_bdc_rows(n, float(d), None, None, None)
    rowptr = np.zeros((1 << n) + 1, np.int64)
    col = np.zeros(nnz, np.int64)
    val = np.zeros(nnz, np.float64)
    L.orc_bdc_rows(n, float(d), _ptr(rowptr), _ptr(col), _ptr(val))
    return rowptr, col, val


def exact_rows(n: int, k: int):
    """Sparse rows of the exact deletion channel BDC_{n,k} (col = y)."""
    L = lib()
    nnz = L.orc_exact_rows(n, k, None, None, None)
    rowptr = np.zeros((1 << n) + 1, np.int64)
    col = np.zeros(nnz, np.int64)
    val = np.zeros(nnz, np.float64)
    L.orc_exact_rows(n, k, _ptr(rowptr), _ptr(col), _ptr(val))
    return rowptr, col, val


def ba_sparse(rows, ny: int, p0: np.ndarray, max_iters: int, tol: float = -1.0):
    """Generic BA on sparse rows.  Returns dict(p, lower, upper, stat, iters):
    per iteration t, lower/upper/stat use X^(t) and Y^(t); p is the final X."""
    rowptr, col, val = rows
    nx = len(rowptr) - 1
    p = np.array(p0, np.float64, copy=True)
    lo = np.zeros(max_iters)
    up = np.zeros(max_iters)
    st = np.zeros(max_iters)
    it = lib().orc_ba_sparse(nx, ny, _ptr(rowptr), _ptr(col), _ptr(val), _ptr(p), int(max_iters),
                             float(tol), _ptr(lo), _ptr(up), _ptr(st))
    return dict(p=p, lower=lo[:it], upper=up[:it], stat=st[:it], iters=it)


def ba_bdc(n: int, d: float, max_iters: int, tol: float = -1.0, p0=None):
    """BA on BDC_d with uniform X^(0) (unless p0 is given)."""
    if p0 is None:
        p0 = np.full(1 << n, 1.0 / (1 << n))
    return ba_sparse(bdc_rows(n, d), 1 << (n + 1), p0, max_iters, tol)


# --------------------------------------------------------------------------
# Paper algorithms (Sec. 4, Sec. 5) and orbits (Appendix A)
# --------------------------------------------------------------------------
def nextpos_cnt(n: int, x: int, kmax: int):
    np_ = np.zeros((n + 1, 2), np.int32)
    cnt = np.zeros((n + 1, kmax + 1), np.uint64)
    lib().orc_nextpos_cnt(n, x, kmax, _ptr(np_), _ptr(cnt))
    return np_, cnt


def unrank(n: int, x: int, k: int, j: int):
    y = np.zeros(1, np.uint64)
    r = lib().orc_unrank(n, x, k, j, _ptr(y))
    return None if r != 0 else int(y[0])


def subset_unrank(n: int, w: int, j: int):
    s = np.zeros(max(w, 1), np.int32)
    m = lib().orc_subset_unrank(n, w, j, _ptr(s))
    return [int(v) for v in s[:m]]


def recsuperseq(i: int, n: int, k: int, y: int, fixed: bool = True) -> int:
    return int(lib().orc_recsuperseq(i, n, k, y, 1 if fixed else 0))


def orbit_rep(s: int, L: int):
    o = np.zeros(1, np.int32)
    r = lib().orc_orbit_rep(s, L, _ptr(o))
    return int(r), int(o[0])


def output_classes(n: int):
    """Class index of every code (orbit of its string under cpl/rev), classes
    numbered by increasing representative code.  Returns (cls, rep_codes,
    sizes)."""
    nout = 1 << (n + 1)
    repc = np.zeros(nout, np.int64)
    size = np.zeros(nout, np.int64)
    for c in range(1, nout):
        k = c.bit_length() - 1
        r, o = orbit_rep(c ^ (1 << k), k) if k > 0 else (0, 1)
        repc[c] = (1 << k) | r
        size[c] = o
    reps = np.unique(repc[1:])
    idx = {int(r): i for i, r in enumerate(reps)}
    cls = np.zeros(nout, np.int64)
    for c in range(1, nout):
        cls[c] = idx[int(repc[c])]
    return cls, reps, np.array([size[int(r)] for r in reps], np.int64)


def dual_bound(n: int, d: float, tau: float, theta: np.ndarray, cls: np.ndarray, grad: bool = True):
    """F = tau log2 sum_x 2^{D_x(q)/tau} with q = softmax over classes of
    theta; returns (F, dF/dtheta, dF/dd)."""
    theta = np.ascontiguousarray(theta, np.float64)
    cls = np.ascontiguousarray(cls, np.int64)
    g = np.zeros(len(theta), np.float64)
    gd = np.zeros(1, np.float64)
    F = lib().orc_dual_bound(n, float(d), float(tau), _ptr(theta), _ptr(cls), len(theta),
                             _ptr(g) if grad else None, _ptr(gd))
    return float(F), g, float(gd[0])


# --------------------------------------------------------------------------
# O2: factorised sweep (plain FP64; pinned against the definitions above)
# --------------------------------------------------------------------------
def sweep_q(n: int, d: float, p: np.ndarray, counts: bool = False) -> np.ndarray:
    """q(y) = sum_x p(x) W(y|x) by the prefix recursion (O2).  counts=True
    uses the embedding counts instead of W: sum_x p(x) Count(y, x)."""
    p = np.ascontiguousarray(p, np.float64)
    q = np.zeros(1 << (n + 1), np.float64)
    a, c = (1.0, 1.0) if counts else (float(d), 1.0 - float(d))
    lib().orc_sweep_forward(n, a, c, _ptr(p), _ptr(q))
    return q


def sweep_G(n: int, d: float, L: np.ndarray, counts: bool = False) -> np.ndarray:
    """G(x) = sum_y W(y|x) L(y) (or sum_y Count(y,x) L(y) with counts=True)
    by the transposed recursion (O2)."""
    L = np.ascontiguousarray(L, np.float64)
    G = np.zeros(1 << n, np.float64)
    a, c = (1.0, 1.0) if counts else (float(d), 1.0 - float(d))
    lib().orc_sweep_adjoint(n, a, c, _ptr(L), _ptr(G))
    return G


def orbit_reps(n: int):
    """(reps, rep_index): the orbit representatives of {0,1}^n under
    complement and reversal (the smallest member, Appendix A) in increasing
    order, and for every x the index of its orbit's representative."""
    x = np.arange(1 << n, dtype=np.int64)
    r = np.zeros_like(x)
    for i in range(n):
        r |= ((x >> i) & 1) << (n - 1 - i)
    full = (1 << n) - 1
    rep = np.minimum(np.minimum(x, x ^ full), np.minimum(r, r ^ full))
    reps = np.unique(rep)
    return reps, np.searchsorted(reps, rep)


def subseq_S_all(n: int) -> np.ndarray:
    """S_k(x) = sum_{|y|=k} Count log2 Count for every x, [2^n][n+1]: the
    trie walk on orbit representatives (OpenMP), copied to every member of
    the orbit (Count is preserved by complement and reversal)."""
    reps, idx = orbit_reps(n)
    xs = np.ascontiguousarray(reps, np.uint64)
    S = np.zeros((len(xs), n + 1), np.float64)
    lib().orc_subseq_S_list(n, _ptr(xs), len(xs), _ptr(S))
    return S[idx]


def keep_weights(n: int, d: float) -> np.ndarray:
    """omega_k = d^(n-k) (1-d)^k, the probability of one keep pattern of
    weight k (0^0 = 1)."""
    k = np.arange(n + 1, dtype=np.float64)
    return np.power(float(d), n - k) * np.power(1.0 - float(d), k)


def neg_entropy_rows(n: int, d: float, S: np.ndarray) -> np.ndarray:
    """sum_y W(y|x) log2 W(y|x) for every x from S (rows of S per x):
    sum_k omega_k (S_k(x) + C(n,k) log2 omega_k), terms with omega_k = 0
    dropped (0 log 0 = 0)."""
    from math import comb
    w = keep_weights(n, d)
    out = np.zeros(S.shape[0], np.float64)
    for k in range(n + 1):
        if w[k] > 0.0:
            out += w[k] * (S[:, k] + comb(n, k) * np.log2(w[k]))
    return out


def D_sweep(n: int, d: float, q: np.ndarray, S: np.ndarray) -> np.ndarray:
    """D_x = sum_y W log2 W - sum_y W log2 q(y) for every x (O2): the first
    term from S, the second by the transposed recursion."""
    with np.errstate(divide="ignore"):
        L = np.where(q > 0.0, np.log2(np.where(q > 0.0, q, 1.0)), 0.0)
    L[0] = 0.0
    return neg_entropy_rows(n, d, S) - sweep_G(n, d, L)


def ba_sweep(n: int, d: float, T: int, p0=None, S=None):
    """T Blahut-Arimoto iterations (Sec. 2.3) with q and D from O2; per
    iteration t the bounds of X^(t) (lower = log2 sum p 2^D, upper = max D);
    p is the final X.  S: subseq_S_all(n), computed if not given."""
    if S is None:
        S = subseq_S_all(n)
    p = np.full(1 << n, 1.0 / (1 << n)) if p0 is None else np.array(p0, np.float64, copy=True)
    lo, up = [], []
    for _ in range(T):
        D = D_sweep(n, d, sweep_q(n, d, p), S)
        Z = float(np.sum(p * np.exp2(D)))
        lo.append(np.log2(Z))
        up.append(float(D.max()))
        p = p * np.exp2(D) / Z
    return dict(p=p, lower=np.array(lo), upper=np.array(up), iters=T)
