"""B300 Blahut-Arimoto engine for the finite-length binary deletion channel.

Thin ctypes binding over ``libbdc.so`` (the C ABI declared in
``include/bdc.h``).  Every step of the computation runs in the library's CUDA
kernels; this module only marshals arguments and owns the device workspace
(a torch uint8 tensor) and the stream.  There is no CPU fallback: if the
shared library is missing, importing :func:`lib` raises.

Encoding: x in {0,1}^n is the integer with x_0 as its most significant bit;
an output y of length k has the code ``(1 << k) | y``.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# BDC_CHECKED=1 loads the checked build (device-side index checks, BDC_ECHECK)
LIB_PATH = os.path.join(_HERE, "libbdc_checks.so" if os.environ.get("BDC_CHECKED") == "1" else "libbdc.so")

FP32, FP64 = 0, 1
SWEEP, LITERAL = 0, 1
_PREC = {"fp32": FP32, "fp64": FP64, FP32: FP32, FP64: FP64}
_IMPL = {"sweep": SWEEP, "literal": LITERAL, SWEEP: SWEEP, LITERAL: LITERAL}

STATUS = {0: "BDC_OK", -1: "BDC_EINVAL", -2: "BDC_ENOMEM", -3: "BDC_ECUDA", -4: "BDC_ETIMEOUT",
          -5: "BDC_ENONFINITE", -6: "BDC_ENOTBOUND", -7: "BDC_ECHECK"}


class BdcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s (%d): %s" % (STATUS.get(status, "?"), status, msg))
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [("symmetrize", ctypes.c_int), ("use_graph", ctypes.c_int), ("chunk", ctypes.c_int),
                ("q_floor", ctypes.c_double), ("certify_mix", ctypes.c_double),
                ("sched_n2_fp32", ctypes.c_int), ("sched_w_fp32", ctypes.c_int),
                ("sched_n2_fp64", ctypes.c_int), ("sched_w_fp64", ctypes.c_int),
                ("enable_literal", ctypes.c_int), ("use_half", ctypes.c_int),
                ("use_regsteps", ctypes.c_int), ("fuse_update", ctypes.c_int),
                ("use_tma", ctypes.c_int), ("tma_wait_polls", ctypes.c_int)]


_lib = None


def lib():
    """Load libbdc.so (built by ``paper_2604_05867_b300.build``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libbdc.so is not built; run `python -m paper_2604_05867_b300.build` "
                              "(there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        P, I, D, I64, SZ = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64, ctypes.c_size_t
        sig = {
            "bdc_default_options": (None, [P]),
            "bdc_create": (I, [I, P, I, P, P]),
            "bdc_create_lengths": (I, [I, P, I, P, P]),
            "bdc_workspace_bytes": (SZ, [P]),
            "bdc_bind": (I, [P, P, SZ, P]),
            "bdc_destroy": (None, [P]),
            "bdc_ba_iterate": (I, [P, I, D, I, I, P, P, P]),
            "bdc_prepare": (I, [P, I, I]),
            "bdc_get_history": (I, [P, I, P, P, I, P]),
            "bdc_divergence": (I, [P, P, I, P]),
            "bdc_certify_upper": (I, [P, P, P, P, P]),
            "bdc_get_p": (I, [P, P]),
            "bdc_set_p": (I, [P, P]),
            "bdc_get_q": (I, [P, I, P]),
            "bdc_get_q_literal": (I, [P, P]),
            "bdc_get_rep_stats": (I, [P, I64, P, P, P, P]),
            "bdc_num_reps": (I64, [P]),
            "bdc_save": (I, [P, ctypes.c_char_p]),
            "bdc_load": (I, [P, ctypes.c_char_p]),
            "bdc_num_output_classes": (I64, [P]),
            "bdc_output_classes": (I, [P, P]),
            "bdc_dual_bound": (I, [P, I, P, D, I, P, P, P, P]),
            "bdc_subseq_counts": (I, [I, P, I64, P, P, P, P]),
            "bdc_launch_count": (I64, [P]),
            "bdc_softmax_classes": (I, [P, I, P, I, P]),
            "bdc_class_logits": (I, [P, P, D, I, P]),
            "bdc_batch_create": (I, [P, I, I, P]),
            "bdc_get_schedule": (I, [P, I, P, P, P]),
            "bdc_autotune": (I, [P, I, I, I, I, P]),
            "bdc_batch_iterate": (I, [P, I, D, I, P]),
            "bdc_batch_destroy": (None, [P]),
            "bdc_profile_iteration": (I, [P, I, I, I, P, ctypes.c_char_p, I, P]),
            "bdc_measure_peaks": (I, [P, SZ, P, P]),
            "bdc_last_error": (ctypes.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status: int):
    if status != 0:
        raise BdcError(status, lib().bdc_last_error().decode(errors="replace"))


def _np_ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def default_options(**kw) -> Options:
    o = Options()
    lib().bdc_default_options(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream), stream


class Engine:
    """One (n, d[0..nd)) problem family on one GPU.

    The workspace is a torch uint8 CUDA tensor owned by this object; the
    engine runs all its kernels on ``stream`` (default: the current stream at
    construction).  ``bdc_bind`` runs the d-free precompute synchronously.

    ``lengths`` (an array [nb, n+1], instead of ``ds``) makes a
    length-mixture channel per row (bdc_create_lengths): a one-hot row at k
    is the exact deletion channel BDC_{n,k}.
    """

    def __init__(self, n: int, ds: Sequence[float] = (), options: Optional[Options] = None, device=None,
                 stream=None, lengths=None):
        import torch
        self.n = int(n)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        L = lib()
        h = ctypes.c_void_p()
        opt = ctypes.byref(options) if options is not None else None
        if lengths is not None:
            b = np.ascontiguousarray(np.atleast_2d(lengths), np.float64)
            if b.shape[1] != self.n + 1:
                raise ValueError("lengths must have n+1 columns")
            self.lengths = b
            self.ds = [float("nan")] * b.shape[0]
            self.nd = b.shape[0]
            _check(L.bdc_create_lengths(self.n, _np_ptr(b), self.nd, opt, ctypes.byref(h)))
        else:
            self.lengths = None
            self.ds = [float(v) for v in ds]
            self.nd = len(self.ds)
            darr = (ctypes.c_double * self.nd)(*self.ds)
            _check(L.bdc_create(self.n, ctypes.cast(darr, ctypes.c_void_p), self.nd, opt, ctypes.byref(h)))
        self._h = h
        self.ws_bytes = int(L.bdc_workspace_bytes(h))
        with torch.cuda.device(self.device):
            self._ws = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device=self.device)
            self._sh, self.stream = _stream_handle(stream)
        base = self._ws.data_ptr()
        aligned = (base + 255) & ~255
        _check(L.bdc_bind(h, ctypes.c_void_p(aligned), self.ws_bytes, self._sh))
        self.num_reps = int(L.bdc_num_reps(h))
        self.num_output_classes = int(L.bdc_num_output_classes(h))

    def close(self):
        if getattr(self, "_h", None):
            lib().bdc_destroy(self._h)
            self._h = None
            self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- iteration ---------------------------------------------------------
    def iterate(self, max_iters: int, tol: float = -1.0, precision="fp32", impl="sweep"):
        lo = np.zeros(self.nd)
        up = np.zeros(self.nd)
        it = np.zeros(self.nd, np.int32)
        _check(lib().bdc_ba_iterate(self._h, int(max_iters), float(tol), _PREC[precision], _IMPL[impl],
                                    _np_ptr(lo), _np_ptr(up), _np_ptr(it)))
        return lo, up, it

    def prepare(self, precision="fp32", impl="sweep"):
        """Build the CUDA graph `iterate` replays (bdc_prepare), outside any timed region."""
        _check(lib().bdc_prepare(self._h, _PREC[precision], _IMPL[impl]))

    def history(self, inst: int = 0, length: int = 8192):
        lo = np.zeros(length)
        up = np.zeros(length)
        cnt = ctypes.c_int(0)
        _check(lib().bdc_get_history(self._h, inst, _np_ptr(lo), _np_ptr(up), length, ctypes.byref(cnt)))
        return lo[:cnt.value], up[:cnt.value]

    def schedule(self, precision="fp32"):
        n1, n2, w = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib().bdc_get_schedule(self._h, _PREC[precision], ctypes.byref(n1), ctypes.byref(n2), ctypes.byref(w)))
        return {"n1": n1.value, "n2": n2.value, "width": w.value}

    def set_schedule(self, precision="fp32", n2: int = 13, width: int = 4):
        """Use the sweep schedule (n1 = n - n2, n2, column tile width) instead of
        searching (bdc_autotune with n2 > 0); raises on a schedule outside the
        reserved buffers."""
        ms = ctypes.c_double(0)
        _check(lib().bdc_autotune(self._h, _PREC[precision], 1, int(n2), int(width), ctypes.byref(ms)))
        return self.schedule(precision)

    def autotune(self, precision="fp32", reps: int = 3, cache: Optional[str] = None):
        """Pick the fastest sweep schedule for this engine (bdc_autotune).  With
        `cache` (a JSON file path) a result stored for this GPU model, n and
        precision is reused, and a new result is stored."""
        import json
        import torch
        key = "%s|n=%d|%s" % (torch.cuda.get_device_name(self.device), self.n, precision)
        table = {}
        if cache and os.path.exists(cache):
            with open(cache) as f:
                table = json.load(f)
        ms = ctypes.c_double(0)
        if key in table:
            s = table[key]
            _check(lib().bdc_autotune(self._h, _PREC[precision], 1, int(s["n2"]), int(s["width"]), ctypes.byref(ms)))
            return dict(s, cached=True)
        _check(lib().bdc_autotune(self._h, _PREC[precision], int(reps), 0, 0, ctypes.byref(ms)))
        s = self.schedule(precision)
        s["ms_per_sweep_pair"] = ms.value
        if cache:
            table[key] = s
            tmp = cache + ".tmp%d" % os.getpid()
            with open(tmp, "w") as f:
                json.dump(table, f, indent=1, sort_keys=True)
            os.replace(tmp, cache)
        return dict(s, cached=False)

    def launch_count(self) -> int:
        return int(lib().bdc_launch_count(self._h))

    def profile(self, precision="fp32", impl="sweep", reps: int = 3):
        """Mean ms per stage of `reps` real iterations run without graphs,
        timed with CUDA events on the engine stream: dict name -> ms."""
        ms = np.zeros(32)
        names = ctypes.create_string_buffer(1024)
        ns = ctypes.c_int(0)
        _check(lib().bdc_profile_iteration(self._h, _PREC[precision], _IMPL[impl], int(reps), _np_ptr(ms), names,
                                           1024, ctypes.byref(ns)))
        keys = names.value.decode().split(",") if ns.value else []
        out = {}
        for i, k in enumerate(keys):
            out[k] = out.get(k, 0.0) + float(ms[i])
        return out

    # -- divergence / certification ------------------------------------------
    def divergence(self, q=None, precision="fp64"):
        """D_x for every instance and input, as a float64 CUDA tensor [nd, 2^n].
        q: None (output marginal of the current p) or a CUDA tensor [nd, 2^(n+1)]
        of float32 (precision fp32) or float64 (fp64)."""
        import torch
        out = torch.empty((self.nd, 1 << self.n), dtype=torch.float64, device=self.device)
        qp = None
        if q is not None:
            want = torch.float32 if _PREC[precision] == FP32 else torch.float64
            assert q.dtype == want and q.is_cuda and q.is_contiguous() and q.numel() == self.nd << (self.n + 1)
            qp = ctypes.c_void_p(q.data_ptr())
        _check(lib().bdc_divergence(self._h, qp, _PREC[precision], ctypes.c_void_p(out.data_ptr())))
        return out

    def certify(self, q=None):
        """Certified FP64 upper bound on C_n(d) per instance: dict(upper, margin, lower)."""
        up = np.zeros(self.nd)
        mg = np.zeros(self.nd)
        lo = np.zeros(self.nd)
        qp = None
        if q is not None:
            import torch
            assert q.dtype == torch.float64 and q.is_cuda and q.is_contiguous()
            qp = ctypes.c_void_p(q.data_ptr())
        _check(lib().bdc_certify_upper(self._h, qp, _np_ptr(up), _np_ptr(mg), _np_ptr(lo)))
        return dict(upper=up, margin=mg, lower=lo)

    # -- state -----------------------------------------------------------------
    def get_p(self) -> np.ndarray:
        p = np.zeros((self.nd, 1 << self.n))
        _check(lib().bdc_get_p(self._h, _np_ptr(p)))
        return p

    def set_p(self, p: np.ndarray):
        p = np.ascontiguousarray(np.broadcast_to(p, (self.nd, 1 << self.n)), np.float64)
        _check(lib().bdc_set_p(self._h, _np_ptr(p)))

    def get_q(self, precision="fp64") -> np.ndarray:
        q = np.zeros((self.nd, 2 << self.n))
        _check(lib().bdc_get_q(self._h, _PREC[precision], _np_ptr(q)))
        return q

    def get_q_literal(self) -> np.ndarray:
        """Output marginal of the current p by the literal (supersequence
        enumeration) path, FP64, host [nd, 2^(n+1)] by code."""
        q = np.zeros((self.nd, 2 << self.n))
        _check(lib().bdc_get_q_literal(self._h, _np_ptr(q)))
        return q

    def rep_stats(self, r: int):
        x = ctypes.c_uint64(0)
        o = ctypes.c_int(0)
        N = np.zeros(self.n + 1, np.uint64)
        S = np.zeros(self.n + 1, np.float64)
        _check(lib().bdc_get_rep_stats(self._h, int(r), ctypes.byref(x), ctypes.byref(o), _np_ptr(N), _np_ptr(S)))
        return int(x.value), int(o.value), N, S

    def output_classes(self) -> np.ndarray:
        c = np.zeros(2 << self.n, np.int64)
        _check(lib().bdc_output_classes(self._h, _np_ptr(c)))
        return c

    def save(self, path: str):
        _check(lib().bdc_save(self._h, path.encode()))

    def load(self, path: str):
        _check(lib().bdc_load(self._h, path.encode()))

    # -- smoothed dual bound -------------------------------------------------------
    def dual_bound(self, inst: int, theta, tau: float, precision="fp64", grad: bool = True,
                   grad_d: Optional[bool] = None):
        """(F, max_D, grad_theta tensor or None, dF/dd or None) for instance inst.
        grad_d defaults to grad (dF/dd exists for BDC_d instances only)."""
        import torch
        want = torch.float32 if _PREC[precision] == FP32 else torch.float64
        assert theta.dtype == want and theta.is_cuda and theta.is_contiguous()
        assert theta.numel() == self.num_output_classes
        if grad_d is None:
            grad_d = grad
        F = ctypes.c_double(0)
        mD = ctypes.c_double(0)
        gd = ctypes.c_double(0)
        g = torch.empty_like(theta) if grad else None
        _check(lib().bdc_dual_bound(self._h, int(inst), ctypes.c_void_p(theta.data_ptr()), float(tau),
                                    _PREC[precision], ctypes.byref(F), ctypes.byref(mD),
                                    ctypes.c_void_p(g.data_ptr()) if grad else None,
                                    ctypes.byref(gd) if grad_d else None))
        return F.value, mD.value, g, (gd.value if grad_d else None)

    def class_logits(self, q, precision="fp64", floor: float = 1e-300):
        """Logits over output classes whose softmax is q (bdc_class_logits);
        q: host array or CUDA tensor of 2^(n+1) doubles by code."""
        import torch
        qd = torch.as_tensor(np.asarray(q) if not torch.is_tensor(q) else q, dtype=torch.float64,
                             device=self.device).contiguous()
        assert qd.numel() == 2 << self.n
        want = torch.float32 if _PREC[precision] == FP32 else torch.float64
        th = torch.empty(self.num_output_classes, dtype=want, device=self.device)
        with torch.cuda.device(self.device):
            torch.cuda.current_stream().synchronize()
        _check(lib().bdc_class_logits(self._h, ctypes.c_void_p(qd.data_ptr()), float(floor), _PREC[precision],
                                      ctypes.c_void_p(th.data_ptr())))
        return th


    def softmax_classes(self, inst: int, theta, precision="fp64"):
        """q over every code (float64 CUDA tensor [2^(n+1)]) = softmax of theta over classes."""
        import torch
        q = torch.empty(2 << self.n, dtype=torch.float64, device=self.device)
        _check(lib().bdc_softmax_classes(self._h, int(inst), ctypes.c_void_p(theta.data_ptr()), _PREC[precision],
                                         ctypes.c_void_p(q.data_ptr())))
        return q


class Batch:
    """Several engines iterated by one CUDA graph (bdc_batch_*).  The engines
    must have been created on the same stream."""

    def __init__(self, engines, chunk: int = 8):
        self.engines = list(engines)
        arr = (ctypes.c_void_p * len(self.engines))(*[e._h.value for e in self.engines])
        h = ctypes.c_void_p()
        _check(lib().bdc_batch_create(ctypes.cast(arr, ctypes.c_void_p), len(self.engines), int(chunk),
                                      ctypes.byref(h)))
        self._h = h

    def iterate(self, max_iters: int, tol: float = -1.0, precision="fp32") -> int:
        n = ctypes.c_int(0)
        _check(lib().bdc_batch_iterate(self._h, int(max_iters), float(tol), _PREC[precision], ctypes.byref(n)))
        return n.value

    def close(self):
        if getattr(self, "_h", None):
            lib().bdc_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def subseq_counts(n: int, xs, emb: bool = False, stream=None):
    """Per input x (CUDA int64 tensor of inputs of length n): N_k (#distinct
    subsequences of each length) and S_k = sum count*log2 count, computed on
    the device by the library's warp-cooperative enumeration.  With emb=True
    and one input, also the embedding count of every output code."""
    import torch
    xs = xs.to(torch.int64).contiguous()
    nx = xs.numel()
    N = torch.zeros((nx, n + 1), dtype=torch.int64, device=xs.device)
    S = torch.zeros((nx, n + 1), dtype=torch.float64, device=xs.device)
    E = torch.zeros(2 << n, dtype=torch.int64, device=xs.device) if emb else None
    sh, _ = _stream_handle(stream)
    _check(lib().bdc_subseq_counts(n, ctypes.c_void_p(xs.data_ptr()), nx, ctypes.c_void_p(N.data_ptr()),
                                   ctypes.c_void_p(S.data_ptr()), ctypes.c_void_p(E.data_ptr()) if emb else None,
                                   sh))
    return N, S, E


def measure_peaks(stream=None) -> dict:
    """Device microbenchmarks (bdc_measure_peaks): FP32 / FP64 FMA-or-add
    instruction rates (1e12/s), L2 read GB/s, shared-memory TB/s, SM count."""
    import torch
    buf = torch.empty(64 << 20, dtype=torch.uint8, device="cuda")
    out = np.zeros(5)
    sh, _ = _stream_handle(stream)
    _check(lib().bdc_measure_peaks(ctypes.c_void_p(buf.data_ptr()), buf.numel(), sh, _np_ptr(out)))
    return {"fp32_tops": float(out[0]), "fp64_tops": float(out[1]), "l2_read_gbs": float(out[2]),
            "smem_tbs": float(out[3]), "sms": int(out[4])}
