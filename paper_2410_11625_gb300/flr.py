"""ctypes binding of libflr.so (include/flr.h): argument marshalling only.

Every step of the FLR path runs in the library's CUDA kernels.  PyTorch is used for
device memory and streams: device entry points take CUDA float32 tensors and run on
the current torch stream.  Nothing here computes; a missing library raises.
"""
from __future__ import annotations

import ctypes
import os

from . import _build

FLR_OK = 0
STATUS = {0: "FLR_OK", -1: "FLR_ERR_ARG", -2: "FLR_ERR_ALIGN", -3: "FLR_ERR_CUDA",
          -4: "FLR_ERR_UNSUPPORTED", -5: "FLR_ERR_NOMEM", -6: "FLR_ERR_TIMEOUT"}

# every symbol include/flr.h declares
EXPORTS = ("flr_create", "flr_destroy", "flr_reserve", "flr_denoise", "flr_denoise_host",
           "flr_denoise_host_async", "flr_host_wait",
           "flr_get_stats", "flr_get_kernel_times", "flr_status_string", "flr_last_cuda_error",
           "flr_denoise_noalloc", "flr_backward", "flr_fast_create", "flr_fast_destroy",
           "flr_fast_denoise", "flr_fast_get_stats", "flr_fast_param_grad", "flr_denoise_batch", "flr_fast_reserve_batch",
           "flr_fast_denoise_batch", "flr_fast_batch_status", "flr_barrier_selftest",
           "flr_mbarrier_selftest", "flr_host_band_plan",
           "flnr_param_count", "flnr_create", "flnr_destroy", "flnr_set_weights", "flnr_get_weights",
           "flnr_get_state", "flnr_set_state",
           "flnr_guide_forward", "flnr_guide_backward", "flnr_zero_grads", "flnr_get_grads",
           "flnr_adam_step", "flnr_l1_loss", "flnr_smape_loss", "flnr_layer", "flnr_status", "flr_fp32_fma_peak")
BATCH_TIMEOUT = 1
FLAG_TIMING = 1
HOST_MAX_BANDS = 8  # FLR_HOST_MAX_BANDS


class FlrParams(ctypes.Structure):
    _fields_ = [("q", ctypes.c_int), ("radius", ctypes.c_int), ("coef_radius", ctypes.c_int),
                ("eps", ctypes.c_float), ("pivot_ratio", ctypes.c_float),
                ("flags", ctypes.c_uint)]


class FlrFastParams(ctypes.Structure):
    _fields_ = [("q", ctypes.c_int), ("factor", ctypes.c_int), ("scale", ctypes.c_int),
                ("sigma", ctypes.c_float), ("taps", ctypes.c_int), ("eps", ctypes.c_float),
                ("pivot_ratio", ctypes.c_float), ("flags", ctypes.c_uint), ("eps_mul", ctypes.c_float)]


FLR_FAST_APPENDIX = 1


class FlrFrame(ctypes.Structure):
    _fields_ = [("guide", ctypes.c_void_p), ("map_guide", ctypes.c_void_p), ("radiance", ctypes.c_void_p),
                ("out", ctypes.c_void_p), ("H", ctypes.c_int), ("W", ctypes.c_int)]


class FlrStats(ctypes.Structure):
    _fields_ = [("flagged", ctypes.c_ulonglong), ("resolved", ctypes.c_ulonglong),
                ("nonfinite", ctypes.c_ulonglong)]


class FlrKernelTimes(ctypes.Structure):
    _fields_ = [("fwd_ms", ctypes.c_double), ("fp64_ms", ctypes.c_double),
                ("apply_ms", ctypes.c_double), ("fwd_n", ctypes.c_ulonglong),
                ("fp64_n", ctypes.c_ulonglong), ("apply_n", ctypes.c_ulonglong)]


class FlrError(RuntimeError):
    def __init__(self, status, what):
        lib = _lib
        msg = STATUS.get(status, str(status))
        if status == -3 and lib is not None:
            msg += ": " + lib.flr_last_cuda_error().decode()
        super().__init__(f"{what} failed: {msg}")
        self.status = status


_lib = None


def library_path() -> str:
    return _build.LIBPATH


def load_library():
    """Load libflr.so (built by ``paper_2410_11625_gb300.build()``); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIBPATH
    if not os.path.exists(path):
        raise FileNotFoundError(f"{path} is missing: run paper_2410_11625_gb300.build() first")
    lib = ctypes.CDLL(path)
    vp, fp, ip = ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int
    lib.flr_create.argtypes = [ctypes.POINTER(FlrParams), ctypes.POINTER(ctypes.c_void_p)]
    lib.flr_destroy.argtypes = [vp]
    lib.flr_reserve.argtypes = [vp, ip, ip]
    lib.flr_denoise.argtypes = [vp, fp, fp, fp, fp, ip, ip, vp]
    lib.flr_denoise_host.argtypes = [vp, fp, fp, fp, fp, ip, ip, vp]
    lib.flr_denoise_host_async.argtypes = [vp, fp, fp, fp, fp, ip, ip, vp]
    lib.flr_host_wait.argtypes = [vp]
    lib.flr_host_band_plan.argtypes = [ip, ip, ip, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.flr_get_stats.argtypes = [vp, ctypes.POINTER(FlrStats)]
    lib.flr_get_kernel_times.argtypes = [vp, ctypes.POINTER(FlrKernelTimes), ip]
    lib.flr_backward.argtypes = [vp, fp, fp, fp, fp, fp, fp, fp, vp, ip, ip, vp]
    lib.flr_backward.restype = ctypes.c_int
    lib.flr_fast_create.argtypes = [ctypes.POINTER(FlrFastParams), ctypes.POINTER(ctypes.c_void_p)]
    lib.flr_fast_destroy.argtypes = [vp]
    lib.flr_fast_denoise.argtypes = [vp, fp, fp, fp, fp, ip, ip, vp]
    lib.flr_fast_get_stats.argtypes = [vp, ctypes.POINTER(FlrStats)]
    lib.flr_fast_param_grad.argtypes = [vp, fp, fp, fp, fp, vp, ip, ip, vp]
    lib.flr_fast_param_grad.restype = ctypes.c_int
    for name in ("flr_fast_create", "flr_fast_destroy", "flr_fast_denoise", "flr_fast_get_stats"):
        getattr(lib, name).restype = ctypes.c_int
    lib.flr_denoise_batch.argtypes = [vp, ip, ctypes.POINTER(FlrFrame), vp]
    lib.flr_fast_reserve_batch.argtypes = [vp, ip, ctypes.POINTER(FlrFrame)]
    lib.flr_fast_denoise_batch.argtypes = [vp, ip, ctypes.POINTER(FlrFrame), vp]
    lib.flr_fast_batch_status.argtypes = [vp]
    lib.flr_barrier_selftest.argtypes = [ip, ctypes.c_ulonglong, ctypes.POINTER(ctypes.c_int)]
    lib.flr_mbarrier_selftest.argtypes = [ip, ctypes.c_ulonglong, ctypes.POINTER(ctypes.c_int)]
    for name in ("flr_denoise_batch", "flr_fast_reserve_batch", "flr_fast_denoise_batch",
                 "flr_fast_batch_status", "flr_barrier_selftest", "flr_mbarrier_selftest"):
        getattr(lib, name).restype = ctypes.c_int
    lib.flr_fp32_fma_peak.argtypes = [ip, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    lib.flr_fp32_fma_peak.restype = ctypes.c_int
    lib.flr_denoise_noalloc.argtypes = [ctypes.POINTER(FlrParams), fp, fp, fp, fp, ip, ip, vp]
    lib.flr_denoise_noalloc.restype = ctypes.c_int
    lib.flr_status_string.argtypes = [ip]
    lib.flr_status_string.restype = ctypes.c_char_p
    lib.flr_last_cuda_error.argtypes = []
    lib.flr_last_cuda_error.restype = ctypes.c_char_p
    for name in ("flr_create", "flr_destroy", "flr_reserve", "flr_denoise", "flr_denoise_host",
                 "flr_denoise_host_async", "flr_host_wait", "flr_get_stats", "flr_get_kernel_times"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(status, what):
    if status != FLR_OK:
        raise FlrError(status, what)


def _dev_ptr(t, name, shape):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float32 or not t.is_contiguous():
        raise TypeError(f"{name} must be contiguous float32")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return ctypes.c_void_p(t.data_ptr())


def _host_ptr(a, name, shape):
    import numpy as np
    if not isinstance(a, np.ndarray) or a.dtype != np.float32 or not a.flags.c_contiguous:
        raise TypeError(f"{name} must be a C-contiguous float32 numpy array")
    if a.shape != tuple(shape):
        raise ValueError(f"{name} has shape {a.shape}, expected {tuple(shape)}")
    return ctypes.c_void_p(a.ctypes.data)


class FLR:
    """A libflr handle: FLR with fixed q, radius, coef_radius, eps and pivot_ratio."""

    def __init__(self, q=8, radius=8, coef_radius=None, eps=1e-3, pivot_ratio=1e-3,
                 timing=False):
        lib = load_library()
        self.q, self.radius = int(q), int(radius)
        self.coef_radius = self.radius if coef_radius is None else int(coef_radius)
        self.eps, self.pivot_ratio = float(eps), float(pivot_ratio)
        p = FlrParams(self.q, self.radius, self.coef_radius, self.eps, self.pivot_ratio,
                      FLAG_TIMING if timing else 0)
        h = ctypes.c_void_p()
        _check(lib.flr_create(ctypes.byref(p), ctypes.byref(h)), "flr_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load_library().flr_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reserve(self, H, W):
        _check(load_library().flr_reserve(self._h, int(H), int(W)), "flr_reserve")

    def denoise(self, guide, radiance, map_guide=None, out=None, stream=None):
        """Device FLR: guide [q,H,W], radiance [3,H,W] CUDA float32 -> out [3,H,W]."""
        import torch
        H, W = int(radiance.shape[-2]), int(radiance.shape[-1])
        g = _dev_ptr(guide, "guide", (self.q, H, W))
        r = _dev_ptr(radiance, "radiance", (3, H, W))
        m = None if map_guide is None else _dev_ptr(map_guide, "map_guide", (self.q, H, W))
        if out is None:
            out = torch.empty((3, H, W), dtype=torch.float32, device=radiance.device)
        o = _dev_ptr(out, "out", (3, H, W))
        if stream is None:
            stream = torch.cuda.current_stream(radiance.device)
        st = ctypes.c_void_p(stream.cuda_stream)
        _check(load_library().flr_denoise(self._h, g, m, r, o, H, W, st), "flr_denoise")
        return out

    def backward(self, guide, radiance, grad_out, map_guide=None, need_eps=False, stream=None,
                 grad_guide=None, grad_radiance=None, grad_map_guide=None):
        """Device FLR adjoint: gradients of <grad_out, I> for guide, radiance, map guide
        (when given) and eps.  Returns a dict of CUDA tensors (eps as a 1-element float64);
        grad_guide / grad_radiance / grad_map_guide may be given as preallocated outputs."""
        import torch
        H, W = int(radiance.shape[-2]), int(radiance.shape[-1])
        dev = radiance.device
        g = _dev_ptr(guide, "guide", (self.q, H, W))
        r = _dev_ptr(radiance, "radiance", (3, H, W))
        go = _dev_ptr(grad_out, "grad_out", (3, H, W))
        m = None if map_guide is None else _dev_ptr(map_guide, "map_guide", (self.q, H, W))
        gg = torch.empty((self.q, H, W), dtype=torch.float32, device=dev) if grad_guide is None else grad_guide
        gr = torch.empty((3, H, W), dtype=torch.float32, device=dev) if grad_radiance is None else grad_radiance
        _dev_ptr(gg, "grad_guide", (self.q, H, W))
        _dev_ptr(gr, "grad_radiance", (3, H, W))
        gm = None
        if map_guide is not None:
            gm = torch.empty((self.q, H, W), dtype=torch.float32, device=dev) if grad_map_guide is None else grad_map_guide
            _dev_ptr(gm, "grad_map_guide", (self.q, H, W))
        ge = torch.zeros(1, dtype=torch.float64, device=dev) if need_eps else None
        if stream is None:
            stream = torch.cuda.current_stream(dev)
        st = load_library().flr_backward(
            self._h, g, m, r, go, ctypes.c_void_p(gg.data_ptr()),
            None if gm is None else ctypes.c_void_p(gm.data_ptr()), ctypes.c_void_p(gr.data_ptr()),
            None if ge is None else ctypes.c_void_p(ge.data_ptr()), H, W, ctypes.c_void_p(stream.cuda_stream))
        _check(st, "flr_backward")
        res = {"guide": gg, "radiance": gr}
        if gm is not None:
            res["map_guide"] = gm
        if ge is not None:
            res["eps"] = ge
        return res

    def denoise_host(self, guide, radiance, map_guide=None, out=None, stream=None):
        """Host FLR: numpy float32 in and out; copies and waits inside the library."""
        import numpy as np
        H, W = radiance.shape[-2], radiance.shape[-1]
        g = _host_ptr(guide, "guide", (self.q, H, W))
        r = _host_ptr(radiance, "radiance", (3, H, W))
        m = None if map_guide is None else _host_ptr(map_guide, "map_guide", (self.q, H, W))
        if out is None:
            out = np.empty((3, H, W), np.float32)
        o = _host_ptr(out, "out", (3, H, W))
        st = ctypes.c_void_p(0 if stream is None else stream.cuda_stream)
        _check(load_library().flr_denoise_host(self._h, g, m, r, o, H, W, st), "flr_denoise_host")
        return out

    def denoise_host_async(self, guide, radiance, out, map_guide=None, stream=None):
        """Queue one frame of a host frame stream (numpy float32, page-locked for overlap);
        `out` and the inputs belong to the library until host_wait() returns."""
        H, W = radiance.shape[-2], radiance.shape[-1]
        g = _host_ptr(guide, "guide", (self.q, H, W))
        r = _host_ptr(radiance, "radiance", (3, H, W))
        m = None if map_guide is None else _host_ptr(map_guide, "map_guide", (self.q, H, W))
        o = _host_ptr(out, "out", (3, H, W))
        st = ctypes.c_void_p(0 if stream is None else stream.cuda_stream)
        _check(load_library().flr_denoise_host_async(self._h, g, m, r, o, H, W, st), "flr_denoise_host_async")
        return out

    def host_wait(self):
        """Wait until every frame queued by denoise_host_async is in host memory."""
        _check(load_library().flr_host_wait(self._h), "flr_host_wait")

    def denoise_batch(self, frames, stream=None):
        """Per-pixel FLR over frames in order: list of (guide, radiance, map_guide, out)."""
        import torch
        arr = (FlrFrame * len(frames))()
        for i, (g, y, z, o) in enumerate(frames):
            H, W = int(y.shape[-2]), int(y.shape[-1])
            arr[i] = FlrFrame(_dev_ptr(g, "guide", (self.q, H, W)).value,
                              None if z is None else _dev_ptr(z, "map_guide", (self.q, H, W)).value,
                              _dev_ptr(y, "radiance", (3, H, W)).value, _dev_ptr(o, "out", (3, H, W)).value, H, W)
        if stream is None:
            stream = torch.cuda.current_stream(frames[0][1].device)
        _check(load_library().flr_denoise_batch(self._h, len(frames), arr, ctypes.c_void_p(stream.cuda_stream)),
               "flr_denoise_batch")

    def kernel_times(self, reset=True):
        """Launch counts and summed CUDA-event kernel durations (ms) since the last reset."""
        t = FlrKernelTimes()
        _check(load_library().flr_get_kernel_times(self._h, ctypes.byref(t), int(reset)),
               "flr_get_kernel_times")
        return {"fwd_ms": t.fwd_ms, "fp64_ms": t.fp64_ms, "apply_ms": t.apply_ms,
                "fwd_n": int(t.fwd_n), "fp64_n": int(t.fp64_n), "apply_n": int(t.apply_n)}

    def stats(self):
        s = FlrStats()
        _check(load_library().flr_get_stats(self._h, ctypes.byref(s)), "flr_get_stats")
        return {"flagged": int(s.flagged), "resolved": int(s.resolved), "nonfinite": int(s.nonfinite)}


class FastFLR:
    """A fast-FLR handle (Sec. 3.2 block-downsampled moments; Sec. 3.2.1 with scale > 1)."""

    def __init__(self, q=8, factor=8, scale=1, sigma=1.25, taps=3, eps=1e-3, pivot_ratio=1e-3, appendix=None):
        """appendix = (eps_add, eps_mul): the Appendix's regularised normalised solve per block
        (flags FLR_FAST_APPENDIX) instead of the centred ridge with eps."""
        lib = load_library()
        self.q, self.factor, self.scale = int(q), int(factor), int(scale)
        if appendix is None:
            p = FlrFastParams(self.q, self.factor, self.scale, float(sigma), int(taps), float(eps),
                              float(pivot_ratio), 0, 0.0)
        else:
            p = FlrFastParams(self.q, self.factor, self.scale, float(sigma), int(taps), float(appendix[0]),
                              float(pivot_ratio), FLR_FAST_APPENDIX, float(appendix[1]))
        h = ctypes.c_void_p()
        _check(lib.flr_fast_create(ctypes.byref(p), ctypes.byref(h)), "flr_fast_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load_library().flr_fast_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def denoise(self, guide, radiance, map_guide=None, out=None, stream=None):
        """guide [q,Hi,Wi], radiance [3,Hi,Wi] (CUDA float32); map_guide [q,Hi*s,Wi*s]."""
        import torch
        Hi, Wi = int(radiance.shape[-2]), int(radiance.shape[-1])
        Ho, Wo = Hi * self.scale, Wi * self.scale
        g = _dev_ptr(guide, "guide", (self.q, Hi, Wi))
        r = _dev_ptr(radiance, "radiance", (3, Hi, Wi))
        m = None if map_guide is None else _dev_ptr(map_guide, "map_guide", (self.q, Ho, Wo))
        if out is None:
            out = torch.empty((3, Ho, Wo), dtype=torch.float32, device=radiance.device)
        o = _dev_ptr(out, "out", (3, Ho, Wo))
        if stream is None:
            stream = torch.cuda.current_stream(radiance.device)
        _check(load_library().flr_fast_denoise(self._h, g, m, r, o, Hi, Wi,
                                               ctypes.c_void_p(stream.cuda_stream)), "flr_fast_denoise")
        return out

    def param_grad(self, guide, radiance, grad_out, map_guide=None, stream=None):
        """dL/d(sigma, eps, eps_mul) for L = <grad_out, output> (flr_fast_param_grad): a CUDA
        float64 tensor of 3 values (eps_mul's is 0 without the Appendix solve)."""
        import torch
        Hi, Wi = int(radiance.shape[-2]), int(radiance.shape[-1])
        Ho, Wo = Hi * self.scale, Wi * self.scale
        g = _dev_ptr(guide, "guide", (self.q, Hi, Wi))
        r = _dev_ptr(radiance, "radiance", (3, Hi, Wi))
        m = None if map_guide is None else _dev_ptr(map_guide, "map_guide", (self.q, Ho, Wo))
        go = _dev_ptr(grad_out, "grad_out", (3, Ho, Wo))
        out = torch.zeros(3, dtype=torch.float64, device=radiance.device)
        if stream is None:
            stream = torch.cuda.current_stream(radiance.device)
        _check(load_library().flr_fast_param_grad(self._h, g, m, r, go, ctypes.c_void_p(out.data_ptr()), Hi, Wi,
                                                  ctypes.c_void_p(stream.cuda_stream)), "flr_fast_param_grad")
        return out

    def _frames(self, frames):
        arr = (FlrFrame * len(frames))()
        for i, (g, y, z, o) in enumerate(frames):
            Hi, Wi = int(y.shape[-2]), int(y.shape[-1])
            Ho, Wo = Hi * self.scale, Wi * self.scale
            arr[i] = FlrFrame(_dev_ptr(g, "guide", (self.q, Hi, Wi)).value,
                              None if z is None else _dev_ptr(z, "map_guide", (self.q, Ho, Wo)).value,
                              _dev_ptr(y, "radiance", (3, Hi, Wi)).value,
                              _dev_ptr(o, "out", (3, Ho, Wo)).value, Hi, Wi)
        return arr

    def reserve_batch(self, frames):
        """frames: list of (guide, radiance, map_guide or None, out) CUDA tensors."""
        arr = self._frames(frames)
        _check(load_library().flr_fast_reserve_batch(self._h, len(frames), arr), "flr_fast_reserve_batch")

    def denoise_batch(self, frames, stream=None):
        """One persistent launch over every frame: list of (guide, radiance, map_guide, out)."""
        import torch
        arr = self._frames(frames)
        if stream is None:
            stream = torch.cuda.current_stream(frames[0][1].device)
        _check(load_library().flr_fast_denoise_batch(self._h, len(frames), arr,
                                                     ctypes.c_void_p(stream.cuda_stream)), "flr_fast_denoise_batch")

    def batch_status(self):
        """FLR_OK (0) or FLR_ERR_TIMEOUT (-6) for the last batch (waits for it)."""
        return int(load_library().flr_fast_batch_status(self._h))

    def stats(self):
        s = FlrStats()
        _check(load_library().flr_fast_get_stats(self._h, ctypes.byref(s)), "flr_fast_get_stats")
        return {"flagged": int(s.flagged), "resolved": int(s.resolved)}


def fp32_fma_peak(iters=20000):
    """Measured FP32 FMA rate of the current device: (TFLOP/s, ms of the timed run)."""
    tf, ms = ctypes.c_double(), ctypes.c_double()
    _check(load_library().flr_fp32_fma_peak(int(iters), ctypes.byref(tf), ctypes.byref(ms)), "flr_fp32_fma_peak")
    return tf.value, ms.value


def host_band_plan(H, radius, coef_radius):
    """The row bands flr_denoise_host uses for H rows: lists c, in_end, out_lo of K + 1
    entries (host arithmetic only; see flr_host_band_plan)."""
    import numpy as np
    c, e, o = (np.zeros(HOST_MAX_BANDS + 1, np.int32) for _ in range(3))
    K = load_library().flr_host_band_plan(int(H), int(radius), int(coef_radius), c.ctypes.data, e.ctypes.data,
                                          o.ctypes.data)
    _check(min(K, 0), "flr_host_band_plan")
    return c[:K + 1].tolist(), e[:K + 1].tolist(), o[:K + 1].tolist()


def mbarrier_selftest(ctas=4, timeout_ns=20_000_000):
    """Status word of flr_mbarrier_selftest (1 = the never-completing wait ran out and the
    completing one did not)."""
    st = ctypes.c_int(0)
    _check(load_library().flr_mbarrier_selftest(int(ctas), ctypes.c_ulonglong(timeout_ns), ctypes.byref(st)),
           "flr_mbarrier_selftest")
    return st.value


def barrier_selftest(ctas=4, timeout_ns=50_000_000):
    """Run a grid barrier that can never complete; returns the device status word, which
    must be BATCH_TIMEOUT (the bounded wait ran out and the kernel returned)."""
    st = ctypes.c_int(0)
    _check(load_library().flr_barrier_selftest(int(ctas), ctypes.c_ulonglong(timeout_ns), ctypes.byref(st)),
           "flr_barrier_selftest")
    return int(st.value)


def denoise(guide, radiance, radius=8, eps=1e-3, coef_radius=None, map_guide=None,
            pivot_ratio=1e-3):
    """One-shot FLR on CUDA tensors (creates and frees a handle)."""
    f = FLR(int(guide.shape[0]), radius, coef_radius, eps, pivot_ratio)
    try:
        return f.denoise(guide, radiance, map_guide=map_guide)
    finally:
        import torch
        torch.cuda.current_stream(radiance.device).synchronize()
        f.close()


def _autograd_function():
    import torch

    class FLRFunction(torch.autograd.Function):
        """torch.autograd.Function around flr_denoise / flr_backward (CUDA tensors).

        apply(handle, guide, radiance, map_guide=None) -> I; the backward pass recomputes
        the window moments instead of keeping them from the forward.
        """

        @staticmethod
        def forward(ctx, handle, guide, radiance, map_guide=None):
            guide = guide.contiguous()
            radiance = radiance.contiguous()
            map_guide = None if map_guide is None else map_guide.contiguous()
            ctx.handle = handle
            ctx.has_map = map_guide is not None
            if ctx.has_map:
                ctx.save_for_backward(guide, radiance, map_guide)
            else:
                ctx.save_for_backward(guide, radiance)
            return handle.denoise(guide, radiance, map_guide=map_guide)

        @staticmethod
        def backward(ctx, grad_out):
            saved = ctx.saved_tensors
            guide, radiance = saved[0], saved[1]
            map_guide = saved[2] if ctx.has_map else None
            res = ctx.handle.backward(guide, radiance, grad_out.contiguous(), map_guide=map_guide)
            return None, res["guide"], res["radiance"], res.get("map_guide")

    return FLRFunction


_FLRFunction = None


def flr_autograd(handle, guide, radiance, map_guide=None):
    """Differentiable FLR: I = FLR(guide, radiance[, map_guide]) with CUDA-kernel backward."""
    global _FLRFunction
    if _FLRFunction is None:
        _FLRFunction = _autograd_function()
    return _FLRFunction.apply(handle, guide, radiance, map_guide)
