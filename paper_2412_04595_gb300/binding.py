"""Python binding of the C ABI in include/sog.h (argument marshalling only).

Every computation runs in ``libsog.so``; this module converts PyTorch
tensors to device pointers and streams and calls the entry points of the
same names.  It raises if the library is missing: there is no CPU path.
"""
from __future__ import annotations

import ctypes
import os

from . import _build

SOG_PREC_FP64, SOG_PREC_MIXED = 0, 1
SOG_WIN_ES, SOG_WIN_GAUSS, SOG_WIN_KB = 0, 1, 2
_WIN_NAMES = {SOG_WIN_ES: "es", SOG_WIN_GAUSS: "gauss", SOG_WIN_KB: "kb"}

STATUS = {0: "SOG_OK", 1: "SOG_ERR_ARG", 2: "SOG_ERR_NONNEUTRAL", 3: "SOG_ERR_OUT_OF_BOX",
          4: "SOG_ERR_NOMEM", 5: "SOG_ERR_CUDA", 6: "SOG_ERR_PARAMS", 7: "SOG_ERR_TIMEOUT"}


class SogParams(ctypes.Structure):
    """Mirror of ``sog_params`` (include/sog.h)."""
    _fields_ = [("L", ctypes.c_double * 3), ("b", ctypes.c_double), ("r0", ctypes.c_double),
                ("omega", ctypes.c_double), ("sigma", ctypes.c_double), ("rc", ctypes.c_double),
                ("M", ctypes.c_int32), ("m", ctypes.c_int32), ("I", ctypes.c_int32 * 3),
                ("hz", ctypes.c_double), ("P_win", ctypes.c_int32), ("shape", ctypes.c_double),
                ("I_long", ctypes.c_int32 * 2), ("P_long", ctypes.c_int32),
                ("shape_long", ctypes.c_double), ("P_cheb", ctypes.c_int32),
                ("window", ctypes.c_int32), ("long_direct", ctypes.c_int32),
                ("win_poly", ctypes.c_int32)]

    def to_dict(self):
        return dict(L=tuple(self.L), b=self.b, r0=self.r0, omega=self.omega, sigma=self.sigma,
                    rc=self.rc, M=self.M, m=self.m, I=tuple(self.I), hz=self.hz,
                    P_win=self.P_win, shape=self.shape, I_long=tuple(self.I_long),
                    P_long=self.P_long, shape_long=self.shape_long, P_cheb=self.P_cheb,
                    window=_WIN_NAMES[self.window],
                    long_direct=bool(self.long_direct), win_poly=int(self.win_poly))

    @classmethod
    def from_dict(cls, d):
        p = cls()
        p.L[:] = list(d["L"])
        for k in ("b", "r0", "omega", "sigma", "rc", "hz", "shape", "shape_long"):
            setattr(p, k, float(d[k]))
        for k in ("M", "m", "P_win", "P_long", "P_cheb"):
            setattr(p, k, int(d[k]))
        p.I[:] = list(d["I"])
        p.I_long[:] = list(d["I_long"])
        p.window = {v: k for k, v in _WIN_NAMES.items()}[d.get("window", "es")]
        p.long_direct = 1 if d.get("long_direct", False) else 0
        p.win_poly = int(d.get("win_poly", 0))
        return p


class SogOpts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("window", ctypes.c_int32),
                ("n_nb", ctypes.c_double), ("manual", ctypes.POINTER(SogParams)),
                ("win_poly", ctypes.c_int32)]


_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libsog.so (built by ``_build.build()``).  Raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        if not build_if_missing:
            raise RuntimeError("libsog.so is not built: run __graft_entry__.build() "
                               "(there is no CPU fallback)")
        _build.build()
    L = ctypes.CDLL(_build.LIB)
    vp, i64, d, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int32
    L.sog_select_params.argtypes = [i64, d, d, d, d, ctypes.POINTER(SogOpts), ctypes.POINTER(SogParams)]
    L.sog_plan_create.argtypes = [ctypes.POINTER(vp), i64, d, d, d, d, ctypes.POINTER(SogOpts)]
    L.sog_plan_get_params.argtypes = [vp, ctypes.POINTER(SogParams)]
    L.sog_plan_precision.argtypes = [vp]
    L.sog_plan_precision.restype = i32
    L.sog_plan_device_bytes.argtypes = [vp]
    L.sog_plan_device_bytes.restype = i64
    L.sog_eval.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    L.sog_eval_components.argtypes = [vp, vp, vp, vp, vp, vp]
    L.sog_eval_host.argtypes = [vp, vp, vp, vp, vp, vp]
    L.sog_plan_check.argtypes = [vp]
    L.sog_plan_destroy.argtypes = [vp]
    L.sog_plan_destroy.restype = None
    L.sog_plan_set_timing.argtypes = [vp, i32]
    L.sog_plan_get_timing.argtypes = [vp, ctypes.POINTER(ctypes.c_float)]
    L.sog_plan_launches.argtypes = [vp]
    L.sog_plan_launches.restype = i64
    L.sog_measure_fma_peak.argtypes = [i32, ctypes.POINTER(d)]
    L.sog_plan_autotune.argtypes = [vp, vp, vp, i32, vp]
    L.sog_plan_tiles.argtypes = [vp, ctypes.POINTER(i32)]
    L.sog_tune_cutoff.argtypes = [i64, d, d, d, d, ctypes.POINTER(SogOpts), vp, vp,
                                  ctypes.POINTER(d), i32, i32, ctypes.POINTER(d),
                                  ctypes.POINTER(ctypes.c_float), vp]
    L.sog_md_create.argtypes = [ctypes.POINTER(vp), vp]
    L.sog_md_step.argtypes = [vp, vp, vp, vp, vp, vp, d, i32, i32, vp, vp, vp]
    L.sog_md_destroy.argtypes = [vp]
    L.sog_md_destroy.restype = None
    L.sog_status_str.argtypes = [ctypes.c_int]
    L.sog_status_str.restype = ctypes.c_char_p
    L.sog_assemble_noalloc.argtypes = [i64, i32, ctypes.POINTER(SogParams), vp, vp, vp, vp, vp,
                                       vp, vp]
    pa = ctypes.POINTER(vp)
    L.sog_batch_create.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(i64),
                                   ctypes.POINTER(d), ctypes.POINTER(d), ctypes.POINTER(SogOpts)]
    L.sog_batch_eval.argtypes = [vp, pa, pa, pa, vp, pa, vp]
    L.sog_batch_check.argtypes = [vp, ctypes.POINTER(i32)]
    L.sog_batch_size.argtypes = [vp]
    L.sog_batch_size.restype = i32
    L.sog_batch_plan.argtypes = [vp, i32]
    L.sog_batch_plan.restype = vp
    L.sog_batch_launches.argtypes = [vp]
    L.sog_batch_launches.restype = i64
    L.sog_batch_destroy.argtypes = [vp]
    L.sog_batch_destroy.restype = None
    u64 = ctypes.c_uint64
    L.sog_mlp_create.argtypes = [ctypes.POINTER(vp), i32, i32, u64]
    L.sog_mlp_num_params.argtypes = [vp]
    L.sog_mlp_num_params.restype = i64
    L.sog_mlp_get_params.argtypes = [vp, vp, i64]
    L.sog_mlp_set_params.argtypes = [vp, vp, i64]
    L.sog_mlp_forward.argtypes = [vp, vp, i32, vp, vp]
    L.sog_mlp_loss_grad.argtypes = [vp, vp, vp, i32, vp, vp, vp]
    L.sog_mlp_train.argtypes = [vp, vp, vp, i32, i32, ctypes.c_float,
                                ctypes.POINTER(ctypes.c_float), vp]
    L.sog_mlp_destroy.argtypes = [vp]
    L.sog_mlp_destroy.restype = None
    L.sog_features.argtypes = [i64, d, d, d, d, vp, i32, ctypes.POINTER(ctypes.c_float)]
    for f in ("sog_select_params", "sog_plan_create", "sog_plan_get_params", "sog_eval",
              "sog_eval_components", "sog_eval_host", "sog_plan_check", "sog_plan_set_timing",
              "sog_plan_get_timing", "sog_assemble_noalloc", "sog_batch_create", "sog_batch_eval",
              "sog_batch_check", "sog_mlp_create", "sog_mlp_get_params", "sog_mlp_set_params",
              "sog_mlp_forward", "sog_mlp_loss_grad", "sog_mlp_train", "sog_features"):
        getattr(L, f).restype = ctypes.c_int
    _lib = L
    return L


class SogError(RuntimeError):
    def __init__(self, code, where):
        msg = load().sog_status_str(code).decode()
        super().__init__("%s: %s (%s)" % (where, STATUS.get(code, code), msg))
        self.code = code


def _check(code, where):
    if code != 0:
        raise SogError(code, where)


def _opts(precision, window, n_nb, manual, win_poly=0):
    o = SogOpts()
    o.precision = precision
    o.window = window
    o.n_nb = float(n_nb) if n_nb else 0.0
    o.win_poly = int(win_poly)
    if manual is not None:
        mp = manual if isinstance(manual, SogParams) else SogParams.from_dict(manual)
        o._manual_ref = mp
        o.manual = ctypes.pointer(mp)
    return o


def sog_select_params(N, Lx, Ly, Lz, tol, window=SOG_WIN_ES, n_nb=None, win_poly=0) -> dict:
    out = SogParams()
    o = _opts(SOG_PREC_MIXED, window, n_nb, None, win_poly)
    _check(load().sog_select_params(int(N), Lx, Ly, Lz, tol, ctypes.byref(o), ctypes.byref(out)),
           "sog_select_params")
    return out.to_dict()


def _require(*specs, cuda=True):
    """Check tensor arguments before their pointers reach the C ABI.  Each
    spec is (tensor or None, name, dtype, numel[, at_least]): dtype, element
    count (exact, or at least ``numel``) and contiguity of every tensor are
    checked first, then (``cuda``) that all are on a CUDA device.  A tensor
    of the wrong size would otherwise be read or written out of bounds by the
    library."""
    for spec in specs:
        t, name, dtype, numel = spec[:4]
        at_least = len(spec) > 4 and spec[4]
        if t is None:
            continue
        if t.dtype != dtype:
            raise ValueError("%s must be %s, got %s" % (name, dtype, t.dtype))
        n = t.numel()
        if (n < numel) if at_least else (n != numel):
            raise ValueError("%s must have %s%d elements, got %d"
                             % (name, "at least " if at_least else "", numel, n))
        if not t.is_contiguous():
            raise ValueError("%s must be contiguous" % name)
    if cuda:
        for spec in specs:
            if spec[0] is not None and not spec[0].is_cuda:
                raise ValueError("%s must be a CUDA tensor" % spec[1])


def sog_tune_cutoff(N, L, tol, q, r, n_nb, reps=3, precision=SOG_PREC_MIXED, window=SOG_WIN_ES,
                    win_poly=0, stream=None):
    """sog_tune_cutoff: the candidate neighbour count (cutoff) of least
    measured evaluation time on (q, r); returns (best n_nb, {n_nb: ms})
    (ms -1: infeasible candidate)."""
    import torch
    N = int(N)
    dt = torch.float64 if precision == SOG_PREC_FP64 else torch.float32
    _require((q, "q", dt, N), (r, "r", dt, 3 * N))
    cands = [float(x) for x in n_nb]
    if not 1 <= len(cands) <= 32:
        raise ValueError("1 to 32 candidates")
    L_ = tuple(map(float, L))
    o = _opts(precision, window, None, None, win_poly)
    arr = (ctypes.c_double * len(cands))(*cands)
    ms = (ctypes.c_float * len(cands))()
    best = ctypes.c_double(0.0)
    _check(load().sog_tune_cutoff(N, L_[0], L_[1], L_[2], float(tol), ctypes.byref(o), _ptr(q),
                                  _ptr(r), arr, len(cands), int(reps), ctypes.byref(best), ms,
                                  _stream_ptr(stream)), "sog_tune_cutoff")
    return best.value, {c: float(m) for c, m in zip(cands, ms)}


def sog_assemble_noalloc(params, q, phi_parts, grad_parts=None, phi=None, E=None, F=None,
                         stream=None):
    """sog_assemble_noalloc: Phi, U and F from the four parts of
    ``Plan.eval_components`` without a plan or any device allocation.
    ``params`` is a dict or SogParams; q, phi, F are contiguous CUDA tensors of
    one dtype (float64: FP64, float32: mixed) with N, N and 3N elements; the
    parts are float64 with 4N and 12N elements; E float64 with at least one."""
    import torch
    prec = {torch.float64: SOG_PREC_FP64, torch.float32: SOG_PREC_MIXED}.get(q.dtype)
    if prec is None:
        raise ValueError("q must be float32 or float64")
    N = q.numel()
    if phi_parts is None:
        raise ValueError("phi_parts is required")
    if F is not None and grad_parts is None:
        raise ValueError("grad_parts is required for F")
    _require((q, "q", q.dtype, N), (phi_parts, "phi_parts", torch.float64, 4 * N),
             (grad_parts, "grad_parts", torch.float64, 12 * N), (phi, "phi", q.dtype, N),
             (F, "F", q.dtype, 3 * N), (E, "E", torch.float64, 1, True))
    prm = params if isinstance(params, SogParams) else SogParams.from_dict(params)
    _check(load().sog_assemble_noalloc(int(q.numel()), prec, ctypes.byref(prm), _ptr(q),
                                       _ptr(phi_parts), _ptr(grad_parts), _ptr(phi), _ptr(E),
                                       _ptr(F), _stream_ptr(stream)), "sog_assemble_noalloc")


def sog_measure_fma_peak(precision=SOG_PREC_MIXED) -> float:
    """Measured FMA rate of the current device in TFLOP/s (FP32 for
    SOG_PREC_MIXED, FP64 for SOG_PREC_FP64)."""
    out = ctypes.c_double()
    _check(load().sog_measure_fma_peak(int(precision), ctypes.byref(out)), "sog_measure_fma_peak")
    return float(out.value)


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


class Plan:
    """Owns one ``sog_plan``.  Tensors passed to ``eval`` must be contiguous
    CUDA tensors of the plan's dtype (float64 for FP64, float32 for mixed)."""

    def __init__(self, N, L, tol, precision=SOG_PREC_MIXED, window=SOG_WIN_ES, n_nb=None,
                 manual=None, win_poly=0):
        L_ = tuple(map(float, L))
        self.N = int(N)
        self._lib = load()
        self._opts = _opts(precision, window, n_nb, manual, win_poly)
        h = ctypes.c_void_p()
        _check(self._lib.sog_plan_create(ctypes.byref(h), self.N, L_[0], L_[1], L_[2], float(tol),
                                         ctypes.byref(self._opts)), "sog_plan_create")
        self._h = h
        self.precision = precision
        out = SogParams()
        _check(self._lib.sog_plan_get_params(h, ctypes.byref(out)), "sog_plan_get_params")
        self.params = out.to_dict()

    @property
    def dtype(self):
        import torch
        return torch.float64 if self.precision == SOG_PREC_FP64 else torch.float32

    def device_bytes(self) -> int:
        return int(self._lib.sog_plan_device_bytes(self._h))

    def _io_specs(self, q, r, phi=None, E=None, F=None):
        import torch
        if q is None or r is None:
            raise ValueError("q and r are required")
        N, dt = self.N, self.dtype
        return [(q, "q", dt, N), (r, "r", dt, 3 * N), (phi, "phi", dt, N), (F, "F", dt, 3 * N),
                (E, "E", torch.float64, 1, True)]

    def _check_io(self, q, r, phi=None, E=None, F=None, cuda=True):
        _require(*self._io_specs(q, r, phi, E, F), cuda=cuda)

    def eval(self, q, r, phi=None, E=None, F=None, stream=None):
        """sog_eval: enqueue the evaluation; outputs are written in place.
        q, phi: N elements; r, F: 3N (N x 3); E: float64, at least one."""
        self._check_io(q, r, phi, E, F)
        _check(self._lib.sog_eval(self._h, _ptr(q), _ptr(r), _ptr(phi), _ptr(E), _ptr(F),
                                  _stream_ptr(stream)), "sog_eval")

    def eval_components(self, q, r, phi_parts, grad_parts, stream=None):
        """sog_eval_components: phi_parts float64 with 4N elements, grad_parts
        float64 with 12N (either may be None)."""
        import torch
        _require(*self._io_specs(q, r), (phi_parts, "phi_parts", torch.float64, 4 * self.N),
                 (grad_parts, "grad_parts", torch.float64, 12 * self.N))
        _check(self._lib.sog_eval_components(self._h, _ptr(q), _ptr(r), _ptr(phi_parts),
                                             _ptr(grad_parts), _stream_ptr(stream)),
               "sog_eval_components")

    def eval_host(self, q, r, phi=None, E=None, F=None):
        """sog_eval_host on CPU tensors (pinned for speed) or numpy arrays of
        the plan's dtype, with the sizes of ``eval``."""
        import numpy as np
        import torch

        def ten(a):
            if a is None:
                return None
            return a if hasattr(a, "data_ptr") else torch.from_numpy(np.asarray(a))

        q, r, phi, E, F = map(ten, (q, r, phi, E, F))
        self._check_io(q, r, phi, E, F, cuda=False)
        for name, t in (("q", q), ("r", r), ("phi", phi), ("E", E), ("F", F)):
            if t is not None and t.is_cuda:
                raise ValueError("%s must be a host tensor or array" % name)

        def hp(a):
            return None if a is None else ctypes.c_void_p(a.data_ptr())
        return self._lib.sog_eval_host(self._h, hp(q), hp(r), hp(phi), hp(E), hp(F))

    STAGES = ("binning", "near", "mid_spread", "mid_fft", "mid_gather", "long_spread",
              "long_fft", "long_gather", "k0", "assemble")
    # long range by direct sums (Algorithm 3): moments, coefficients, evaluation
    STAGES_DIRECT = STAGES[:5] + ("long_moments", "long_coeffs", "long_eval") + STAGES[8:]

    def set_timing(self, enable):
        """False/0: off; True/1: stage events in the concurrent evaluation;
        2: stages run one after another on the caller's stream (isolated
        durations)."""
        _check(self._lib.sog_plan_set_timing(self._h, int(enable)), "sog_plan_set_timing")

    def timing(self) -> dict:
        """Device milliseconds of each stage of the last evaluation."""
        buf = (ctypes.c_float * len(self.STAGES))()
        _check(self._lib.sog_plan_get_timing(self._h, buf), "sog_plan_get_timing")
        names = self.STAGES_DIRECT if self.params.get("long_direct") else self.STAGES
        return dict(zip(names, [float(x) for x in buf]))

    def launches(self) -> int:
        return int(self._lib.sog_plan_launches(self._h))

    def autotune(self, q, r, reps=3, stream=None):
        """sog_plan_autotune on (q, r); returns the chosen tiles."""
        self._check_io(q, r)
        _check(self._lib.sog_plan_autotune(self._h, _ptr(q), _ptr(r), int(reps),
                                           _stream_ptr(stream)), "sog_plan_autotune")
        return self.tiles()

    def tiles(self) -> dict:
        out = (ctypes.c_int32 * 4)()
        _check(self._lib.sog_plan_tiles(self._h, out), "sog_plan_tiles")
        return {"mid_tile": out[0], "mid_ctas_per_tile": out[1], "long_tile": out[2],
                "long_ctas_per_tile": out[3]}

    def check(self) -> int:
        return int(self._lib.sog_plan_check(self._h))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.sog_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Owns one ``sog_batch``: independent systems evaluated by one graph
    launch.  ``systems`` is a list of (N, (Lx, Ly, Lz)); ``tol`` a float or a
    list.  Tensors are contiguous CUDA tensors of the batch's dtype."""

    def __init__(self, systems, tol, precision=SOG_PREC_MIXED, window=SOG_WIN_ES, n_nb=None):
        self._lib = load()
        n = len(systems)
        tols = list(tol) if hasattr(tol, "__len__") else [float(tol)] * n
        Ns = (ctypes.c_int64 * n)(*[int(s[0]) for s in systems])
        Ls = (ctypes.c_double * (3 * n))(*[float(x) for s in systems for x in s[1]])
        Ts = (ctypes.c_double * n)(*tols)
        o = _opts(precision, window, n_nb, None)
        h = ctypes.c_void_p()
        _check(self._lib.sog_batch_create(ctypes.byref(h), n, Ns, Ls, Ts, ctypes.byref(o)),
               "sog_batch_create")
        self._h = h
        self.size = n
        self.precision = precision
        self.params = []
        for i in range(n):
            out = SogParams()
            _check(self._lib.sog_plan_get_params(self._lib.sog_batch_plan(h, i), ctypes.byref(out)),
                   "sog_plan_get_params")
            self.params.append(out.to_dict())
        self.sizes = [int(sy[0]) for sy in systems]

    @property
    def dtype(self):
        import torch
        return torch.float64 if self.precision == SOG_PREC_FP64 else torch.float32

    def eval(self, q, r, phi=None, E=None, F=None, stream=None):
        """sog_batch_eval: q, r, phi, F are lists of per-system tensors; E one
        float64 CUDA tensor of size nsys (or None)."""
        import torch
        n = self.size

        def arr(ts, name, per):
            if ts is None:
                return None
            if len(ts) != n:
                raise ValueError("%s must hold %d tensors" % (name, n))
            _require(*[(t, "%s[%d]" % (name, i), self.dtype, per * self.sizes[i])
                       for i, t in enumerate(ts)])
            return (ctypes.c_void_p * n)(*[t.data_ptr() if t is not None else None for t in ts])

        if q is None or r is None:
            raise ValueError("q and r are required")
        qa, ra, pa, fa = arr(q, "q", 1), arr(r, "r", 3), arr(phi, "phi", 1), arr(F, "F", 3)
        if any(t is None for t in q) or any(t is None for t in r):
            raise ValueError("every system needs q and r")
        _require((E, "E", torch.float64, n, True))
        _check(self._lib.sog_batch_eval(self._h, qa, ra, pa, _ptr(E), fa, _stream_ptr(stream)),
               "sog_batch_eval")

    def check(self):
        bad = ctypes.c_int32(-1)
        st = int(self._lib.sog_batch_check(self._h, ctypes.byref(bad)))
        return st, int(bad.value)

    def launches(self) -> int:
        return int(self._lib.sog_batch_launches(self._h))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.sog_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


N_FEATURES = 8


def sog_features(N, L, tol, r):
    """sog_features: the proposer's eight features of a system (host list);
    r is the N x 3 CUDA tensor of positions (float32 or float64)."""
    import torch
    prec = SOG_PREC_FP64 if r.dtype == torch.float64 else SOG_PREC_MIXED
    if not r.is_cuda or not r.is_contiguous():
        raise ValueError("r must be a contiguous CUDA tensor")
    out = (ctypes.c_float * N_FEATURES)()
    _check(load().sog_features(int(N), float(L[0]), float(L[1]), float(L[2]), float(tol), _ptr(r),
                               prec, out), "sog_features")
    return [float(v) for v in out]


class MLP:
    """Owns one ``sog_mlp`` (FP32 parameters on the device)."""

    def __init__(self, n_in=N_FEATURES, n_hidden=32, seed=0):
        self._lib = load()
        h = ctypes.c_void_p()
        _check(self._lib.sog_mlp_create(ctypes.byref(h), int(n_in), int(n_hidden), int(seed)),
               "sog_mlp_create")
        self._h = h
        self.n_in, self.n_hidden = int(n_in), int(n_hidden)
        self.num_params = int(self._lib.sog_mlp_num_params(h))

    def get_params(self):
        import numpy as np
        out = np.empty(self.num_params, dtype=np.float32)
        _check(self._lib.sog_mlp_get_params(self._h, ctypes.c_void_p(out.ctypes.data),
                                            self.num_params), "sog_mlp_get_params")
        return out

    def set_params(self, p):
        import numpy as np
        a = np.ascontiguousarray(p, dtype=np.float32)
        _check(self._lib.sog_mlp_set_params(self._h, ctypes.c_void_p(a.ctypes.data), a.size),
               "sog_mlp_set_params")

    def forward(self, X, Y=None, stream=None):
        import torch
        if Y is None:
            Y = torch.empty(X.shape[0], dtype=torch.float32, device=X.device)
        _check(self._lib.sog_mlp_forward(self._h, _ptr(X), int(X.shape[0]), _ptr(Y),
                                         _stream_ptr(stream)), "sog_mlp_forward")
        return Y

    def loss_grad(self, X, T, stream=None):
        import torch
        g = torch.empty(self.num_params, dtype=torch.float32, device=X.device)
        loss = torch.empty(1, dtype=torch.float32, device=X.device)
        _check(self._lib.sog_mlp_loss_grad(self._h, _ptr(X), _ptr(T), int(X.shape[0]), _ptr(g),
                                           _ptr(loss), _stream_ptr(stream)), "sog_mlp_loss_grad")
        return loss, g

    def train(self, X, T, iters, lr=1e-2, stream=None):
        out = ctypes.c_float()
        _check(self._lib.sog_mlp_train(self._h, _ptr(X), _ptr(T), int(X.shape[0]), int(iters),
                                       float(lr), ctypes.byref(out), _stream_ptr(stream)),
               "sog_mlp_train")
        return float(out.value)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.sog_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MD:
    """Owns one ``sog_md``: velocity-Verlet steps with a plan's forces
    (sog_md_step).  Tensors are contiguous CUDA tensors of the plan's dtype:
    q [N], r, v, F [N, 3], inv_mass [N] or None; order int32 [N] or None."""

    def __init__(self, plan):
        self._lib = load()
        self.plan = plan
        h = ctypes.c_void_p()
        _check(self._lib.sog_md_create(ctypes.byref(h), plan._h), "sog_md_create")
        self._h = h

    def step(self, q, r, v, F, dt, nsteps=1, inv_mass=None, E=None, sort_every=0, order=None,
             stream=None):
        import torch
        N, dt_ = self.plan.N, self.plan.dtype
        if sort_every > 0 and order is None:
            raise ValueError("order is required when sort_every > 0")
        _require((q, "q", dt_, N), (r, "r", dt_, 3 * N), (v, "v", dt_, 3 * N),
                 (F, "F", dt_, 3 * N), (inv_mass, "inv_mass", dt_, N),
                 (E, "E", torch.float64, 1, True), (order, "order", torch.int32, N))
        _check(self._lib.sog_md_step(self._h, _ptr(q), _ptr(r), _ptr(v), _ptr(F), _ptr(inv_mass),
                                     float(dt), int(nsteps), int(sort_every), _ptr(E),
                                     _ptr(order), _stream_ptr(stream)), "sog_md_step")

    def close(self):
        if getattr(self, "_h", None):
            self._lib.sog_md_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
