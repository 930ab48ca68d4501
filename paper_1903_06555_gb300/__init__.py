"""GB300-native w-stacking w-projection measurement operator (arXiv 1903.06555).

A thin ctypes binding over libphi.so, whose C ABI is declared in
include/phi.h.  This module only marshals arguments: every step of the
operator (fold, k-means w-stacks, sort, image-domain chirp, FFT, on-the-fly
w-kernel quadrature, degridding and gridding) runs in the library's CUDA
kernels.  PyTorch supplies device memory and the current CUDA stream.

    import paper_1903_06555_gb300 as phi
    plan = phi.Plan(uvw, image_n=2048, fov_rad=math.radians(25), n_stacks=8,
                    conj_fold=True)
    y = plan.degrid(x)      # y = Phi x
    d = plan.grid(y)        # d = Re(Phi^H y)

There is no CPU fallback: without the compiled library or a CUDA device the
calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import _build

HERE = os.path.dirname(os.path.abspath(__file__))

PHI_OK, PHI_ERR_ARG, PHI_ERR_OOM, PHI_ERR_CUDA, PHI_ERR_HORIZON, PHI_ERR_SUPPORT, \
    PHI_ERR_TIMEOUT, PHI_ERR_STATE = range(8)
PHI_F32, PHI_F64 = 0, 1
PHI_SUPPORT_STACK, PHI_SUPPORT_VIS = 0, 1
PHI_KERNEL_QUADRATURE, PHI_KERNEL_TABLE, PHI_KERNEL_RADIAL = 0, 1, 2
STAGES = ("prep", "fft", "degrid", "grid", "finish", "clear")
NUM_STAGES = len(STAGES)


class PlanDesc(ctypes.Structure):
    """Mirror of phi_plan_desc (include/phi.h)."""
    _fields_ = [
        ("image_n", ctypes.c_int32),
        ("support", ctypes.c_int32),
        ("n_stacks", ctypes.c_int32),
        ("kmeans_max_iter", ctypes.c_int32),
        ("conj_fold", ctypes.c_int32),
        ("max_support", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("support_rule", ctypes.c_int32),
        ("max_refine", ctypes.c_int32),
        ("tile", ctypes.c_int32),
        ("max_grid_mib", ctypes.c_int32),
        ("kernel_mode", ctypes.c_int32),
        ("grid_staging", ctypes.c_int32),
        ("grid_deterministic", ctypes.c_int32),
        ("oversample", ctypes.c_double),
        ("fov_rad", ctypes.c_double),
        ("kmeans_tol", ctypes.c_double),
        ("alpha", ctypes.c_double),
        ("quad_rel_tol", ctypes.c_double),
        ("quad_abs_tol", ctypes.c_double),
        ("kb_beta", ctypes.c_double),
        ("cycles_per_panel", ctypes.c_double),
        ("table_tol", ctypes.c_double),
    ]


class PlanSummary(ctypes.Structure):
    """Mirror of phi_plan_summary (include/phi.h)."""
    _fields_ = [
        ("n_vis", ctypes.c_int64),
        ("n_kept", ctypes.c_int64),
        ("n_dropped", ctypes.c_int64),
        ("device_bytes", ctypes.c_int64),
        ("image_n", ctypes.c_int32),
        ("npad", ctypes.c_int32),
        ("n_stacks", ctypes.c_int32),
        ("kmeans_sweeps", ctypes.c_int32),
        ("max_jw", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("du", ctypes.c_double),
        ("dl", ctypes.c_double),
        ("beta", ctypes.c_double),
        ("window_radius", ctypes.c_double),
        ("support_coeff", ctypes.c_double),
        ("kernel_mode", ctypes.c_int32),
        ("group", ctypes.c_int32),
        ("table_n_rho", ctypes.c_int64),
        ("table_n_w", ctypes.c_int64),
        ("table_h_rho", ctypes.c_double),
        ("table_h_w", ctypes.c_double),
    ]


class WKernelParams(ctypes.Structure):
    """Mirror of phi_wkernel_params (include/phi.h)."""
    _fields_ = [
        ("du", ctypes.c_double),
        ("window_radius", ctypes.c_double),
        ("kb_beta", ctypes.c_double),
        ("quad_rel_tol", ctypes.c_double),
        ("quad_abs_tol", ctypes.c_double),
        ("cycles_per_panel", ctypes.c_double),
        ("support", ctypes.c_int32),
        ("max_refine", ctypes.c_int32),
        ("max_panels", ctypes.c_int32),
        ("precision", ctypes.c_int32),
    ]


WKERNEL_NOALLOC_MAX_PANELS = 32

_LIB = None
_LOCK = threading.Lock()
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64


def lib_path() -> str:
    return _build.LIB


def lib():
    """Load libphi.so (building it first if its sources are newer)."""
    global _LIB
    with _LOCK:
        if _LIB is None:
            if _build.stale():
                _build.build()
            L = ctypes.CDLL(_build.LIB)
            L.phi_plan_desc_default.argtypes = [ctypes.POINTER(PlanDesc)]
            L.phi_plan_create.argtypes = [ctypes.POINTER(_vp), ctypes.POINTER(PlanDesc), _vp, _vp,
                                          _i64, _vp]
            L.phi_plan_create_fixed.argtypes = [ctypes.POINTER(_vp), ctypes.POINTER(PlanDesc), _vp,
                                                _vp, _i64, ctypes.POINTER(ctypes.c_double),
                                                ctypes.POINTER(ctypes.c_int32), _vp]
            L.phi_plan_destroy.argtypes = [_vp]
            L.phi_plan_destroy.restype = None
            L.phi_plan_info.argtypes = [_vp, ctypes.POINTER(PlanSummary), _vp, _vp, _vp]
            L.phi_plan_stats.argtypes = [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64),
                                         ctypes.POINTER(_i64), ctypes.c_int, _vp]
            L.phi_plan_set_timing.argtypes = [_vp, ctypes.c_int]
            L.phi_plan_timings.argtypes = [_vp, ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(_i64), ctypes.c_int, _vp]
            L.phi_degrid.argtypes = [_vp, _vp, _vp, _vp]
            L.phi_grid.argtypes = [_vp, _vp, _vp, _vp]
            L.phi_degrid_dde.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_int32, _vp, _vp]
            L.phi_grid_dde.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_int32, _vp, _vp]
            L.phi_wkernel.argtypes = [_vp, _vp, _vp, _i64, _vp, ctypes.POINTER(_i64), _vp]
            L.phi_wkernel_noalloc.argtypes = [ctypes.POINTER(WKernelParams), _vp, _vp, _i64, _vp,
                                              ctypes.POINTER(_i64), _vp]
            L.phi_error_string.argtypes = [ctypes.c_int]
            L.phi_error_string.restype = ctypes.c_char_p
            _LIB = L
    return _LIB


class PhiError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {lib().phi_error_string(status).decode()} (status {status})")


def _check(status: int, what: str):
    if status != PHI_OK:
        raise PhiError(status, what)


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def default_desc(**kw) -> PlanDesc:
    d = PlanDesc()
    _check(lib().phi_plan_desc_default(ctypes.byref(d)), "phi_plan_desc_default")
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = {"f32": PHI_F32, "f64": PHI_F64}[v]
        if k == "support_rule" and isinstance(v, str):
            v = {"stack": PHI_SUPPORT_STACK, "vis": PHI_SUPPORT_VIS}[v]
        if k == "kernel_mode" and isinstance(v, str):
            v = {"quadrature": PHI_KERNEL_QUADRATURE, "table": PHI_KERNEL_TABLE,
                 "radial": PHI_KERNEL_RADIAL}[v]
        if not hasattr(d, k):
            raise TypeError(f"unknown descriptor field {k}")
        setattr(d, k, type(getattr(d, k))(v))
    return d


class Plan:
    """A resident operator plan: sorted visibility records, stack centres,
    per-pixel factors, one padded grid and a cuFFT plan, all on the device.

    uvw: (M, 3) float64 tensor of baselines in wavelengths (any device; it is
    copied to the current CUDA device).  weights: optional (M,) float64.
    Keyword arguments are phi_plan_desc fields (image_n, fov_rad,
    oversample, support, n_stacks, conj_fold, precision='f32'|'f64',
    support_rule='stack'|'vis', quad_rel_tol, ...).
    """

    def __init__(self, uvw, weights=None, stream=None, centres=None, stack_jw=None, **desc):
        self.desc = default_desc(**desc)
        dev = torch.device("cuda", torch.cuda.current_device())
        uvw = torch.as_tensor(uvw, dtype=torch.float64).to(dev).contiguous()
        if uvw.ndim != 2 or uvw.shape[1] != 3:
            raise ValueError("uvw must be (M, 3)")
        self.n_vis = int(uvw.shape[0])
        w = None
        if weights is not None:
            w = torch.as_tensor(weights, dtype=torch.float64).to(dev).contiguous()
            if w.shape != (self.n_vis,):
                raise ValueError("weights must be (M,)")
        self.device = dev
        self.real_dtype = torch.float64 if self.desc.precision == PHI_F64 else torch.float32
        self.complex_dtype = torch.complex128 if self.desc.precision == PHI_F64 else torch.complex64
        h = ctypes.c_void_p()
        wptr = ctypes.c_void_p(w.data_ptr() if w is not None else 0)
        if centres is None:
            if stack_jw is not None:
                raise ValueError("stack_jw needs centres")
            _check(lib().phi_plan_create(ctypes.byref(h), ctypes.byref(self.desc),
                                         ctypes.c_void_p(uvw.data_ptr()), wptr, self.n_vis,
                                         _stream(stream)), "phi_plan_create")
        else:
            K = int(self.desc.n_stacks)
            c = (ctypes.c_double * K)(*[float(v) for v in centres])
            j = None if stack_jw is None else (ctypes.c_int32 * K)(*[int(v) for v in stack_jw])
            _check(lib().phi_plan_create_fixed(ctypes.byref(h), ctypes.byref(self.desc),
                                               ctypes.c_void_p(uvw.data_ptr()), wptr, self.n_vis,
                                               c, j, _stream(stream)), "phi_plan_create_fixed")
        self._h = h
        self.image_n = int(self.desc.image_n)

    # -- lifetime ---------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            torch.cuda.synchronize(self.device)
            lib().phi_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def handle(self):
        return self._h

    # -- operator -----------------------------------------------------------
    def _image(self, x):
        n = self.image_n
        if x.shape != (n, n) or x.dtype != self.real_dtype or x.device != self.device:
            raise ValueError(f"image must be ({n}, {n}) {self.real_dtype} on {self.device}")
        return x.contiguous()

    def _vis(self, y):
        if y.shape != (self.n_vis,) or y.dtype != self.complex_dtype or y.device != self.device:
            raise ValueError(f"visibilities must be ({self.n_vis},) {self.complex_dtype} on {self.device}")
        return y.contiguous()

    def degrid(self, x, out=None, stream=None):
        """y = Phi x (complex, caller visibility order)."""
        x = self._image(x)
        y = torch.empty(self.n_vis, dtype=self.complex_dtype, device=self.device) if out is None \
            else self._vis(out)
        _check(lib().phi_degrid(self._h, ctypes.c_void_p(x.data_ptr()),
                                ctypes.c_void_p(y.data_ptr()), _stream(stream)), "phi_degrid")
        return y

    def grid(self, y, out=None, stream=None):
        """x = Re(Phi^H y) (real image)."""
        y = self._vis(y)
        n = self.image_n
        x = torch.empty((n, n), dtype=self.real_dtype, device=self.device) if out is None \
            else self._image(out)
        _check(lib().phi_grid(self._h, ctypes.c_void_p(y.data_ptr()),
                              ctypes.c_void_p(x.data_ptr()), _stream(stream)), "phi_grid")
        return x

    def _dde(self, a, b):
        a = torch.as_tensor(a)
        b = torch.as_tensor(b)
        if a.dim() != 2 or a.shape != b.shape or a.shape[0] != self.n_vis:
            raise ValueError(f"DDE kernels must both be ({self.n_vis}, taps)")
        return (a.to(self.device, self.complex_dtype).contiguous(),
                b.to(self.device, self.complex_dtype).contiguous())

    def degrid_dde(self, x, a, b, out=None, stream=None):
        """y = Phi_D x with the per-visibility separable DDE kernels a, b
        ((n_vis, taps) complex, taps odd; Sec. 5.2) convolved with the
        w-kernel.  The plan must be built without the conjugate fold."""
        x = self._image(x)
        a, b = self._dde(a, b)
        y = torch.empty(self.n_vis, dtype=self.complex_dtype, device=self.device) if out is None \
            else self._vis(out)
        _check(lib().phi_degrid_dde(self._h, ctypes.c_void_p(x.data_ptr()),
                                    ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()),
                                    a.shape[1], ctypes.c_void_p(y.data_ptr()), _stream(stream)),
               "phi_degrid_dde")
        return y

    def grid_dde(self, y, a, b, out=None, stream=None):
        """x = Re(Phi_D^H y), the adjoint of degrid_dde."""
        y = self._vis(y)
        a, b = self._dde(a, b)
        n = self.image_n
        x = torch.empty((n, n), dtype=self.real_dtype, device=self.device) if out is None \
            else self._image(out)
        _check(lib().phi_grid_dde(self._h, ctypes.c_void_p(y.data_ptr()),
                                  ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()),
                                  a.shape[1], ctypes.c_void_p(x.data_ptr()), _stream(stream)),
               "phi_grid_dde")
        return x

    def wkernel(self, rho, dw, stream=None):
        """[GC](rho, dw) for arrays of radii (grid pixels) and w offsets.
        Returns (complex tensor, number of points above tolerance)."""
        rho = torch.as_tensor(rho, dtype=torch.float64).to(self.device).contiguous().ravel()
        dw = torch.as_tensor(dw, dtype=torch.float64).to(self.device).contiguous().ravel()
        if rho.shape != dw.shape:
            raise ValueError("rho and dw must have the same size")
        k = torch.empty(rho.numel(), dtype=self.complex_dtype, device=self.device)
        bad = _i64(0)
        _check(lib().phi_wkernel(self._h, ctypes.c_void_p(rho.data_ptr()),
                                 ctypes.c_void_p(dw.data_ptr()), rho.numel(),
                                 ctypes.c_void_p(k.data_ptr()), ctypes.byref(bad),
                                 _stream(stream)), "phi_wkernel")
        return k, int(bad.value)

    # -- introspection --------------------------------------------------------
    def info(self) -> dict:
        s = PlanSummary()
        K = int(self.desc.n_stacks)
        wbar = (ctypes.c_double * K)()
        cnt = (ctypes.c_int64 * K)()
        jw = (ctypes.c_int32 * K)()
        _check(lib().phi_plan_info(self._h, ctypes.byref(s), wbar, cnt, jw), "phi_plan_info")
        out = {f: getattr(s, f) for f, _ in PlanSummary._fields_}
        out["wbar"] = list(wbar)
        out["counts"] = list(cnt)
        out["jw"] = list(jw)
        return out

    def stats(self, reset=False, stream=None):
        """(taps above tolerance, taps evaluated) since the last reset."""
        return self.stats_full(reset, stream)[:2]

    def stats_full(self, reset=False, stream=None):
        """(taps above tolerance, taps evaluated, tap-node evaluations)."""
        a, b, c = _i64(0), _i64(0), _i64(0)
        _check(lib().phi_plan_stats(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                    int(reset), _stream(stream)), "phi_plan_stats")
        return int(a.value), int(b.value), int(c.value)

    def set_timing(self, enable=True):
        _check(lib().phi_plan_set_timing(self._h, int(enable)), "phi_plan_set_timing")

    def timings(self, reset=False, stream=None):
        """{stage: (milliseconds, launches)} since the last reset (synchronises)."""
        ms = (ctypes.c_double * NUM_STAGES)()
        n = (ctypes.c_int64 * NUM_STAGES)()
        _check(lib().phi_plan_timings(self._h, ms, n, int(reset), _stream(stream)),
               "phi_plan_timings")
        return {STAGES[i]: (ms[i], int(n[i])) for i in range(NUM_STAGES)}


def wkernel_noalloc(params: WKernelParams, rho, dw, stream=None):
    """[GC](rho, dw) without a plan and without any device allocation inside
    the library (its scratch is a fixed array in the library itself), for
    callers that must not allocate device memory while running.  rho and dw
    must already be float64 CUDA tensors of equal size; returns (complex
    tensor, number of points above tolerance).  The output tensor is
    allocated here by PyTorch; callers that cannot allocate pass their own
    buffer to the C entry point directly."""
    if rho.dtype != torch.float64 or dw.dtype != torch.float64 or rho.shape != dw.shape:
        raise ValueError("rho and dw must be float64 tensors of the same shape")
    if not rho.is_cuda or not dw.is_cuda:
        raise ValueError("rho and dw must be on the GPU")
    rho = rho.contiguous().ravel()
    dw = dw.contiguous().ravel()
    cd = torch.complex128 if params.precision == PHI_F64 else torch.complex64
    k = torch.empty(rho.numel(), dtype=cd, device=rho.device)
    bad = _i64(0)
    _check(lib().phi_wkernel_noalloc(ctypes.byref(params), ctypes.c_void_p(rho.data_ptr()),
                                     ctypes.c_void_p(dw.data_ptr()), rho.numel(),
                                     ctypes.c_void_p(k.data_ptr()), ctypes.byref(bad),
                                     _stream(stream)), "phi_wkernel_noalloc")
    return k, int(bad.value)


__all__ = ["Plan", "PlanDesc", "PlanSummary", "PhiError", "WKernelParams", "default_desc", "lib",
           "lib_path", "wkernel_noalloc"]
