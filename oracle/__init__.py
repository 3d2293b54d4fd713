"""FP64 CPU oracle of Fast Local Regression (arXiv 2410.11625).

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package.  The GPU library never imports it, and it
never imports the GPU library.

The arithmetic lives in ``flr_oracle.c`` (plain C, double precision; every function
cites the passage of the paper it follows).  This module only marshals numpy arrays
into it through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "_lib")
_LIBPATH = os.path.join(_LIBDIR, "liboracle.so")
_SOURCES = ["flr_oracle.c"]

_lib = None


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` with gcc (OpenMP, no fast-math) and return its path."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    if not force and os.path.exists(_LIBPATH):
        newest = max(os.path.getmtime(s) for s in srcs)
        if os.path.getmtime(_LIBPATH) >= newest:
            return _LIBPATH
    os.makedirs(_LIBDIR, exist_ok=True)
    tmp = _LIBPATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
           "-ffp-contract=off", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIBPATH)
    return _LIBPATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIBPATH)
        dp = ctypes.POINTER(ctypes.c_double)
        fp = ctypes.POINTER(ctypes.c_float)
        lib.flr_oracle_forward.argtypes = [
            ctypes.c_int, ctypes.c_int, ctypes.c_int, fp, fp, fp,
            ctypes.c_int, ctypes.c_int, ctypes.c_double, dp, dp]
        lib.flr_oracle_forward.restype = ctypes.c_int
        lib.flr_oracle_backward.argtypes = [
            ctypes.c_int, ctypes.c_int, ctypes.c_int, fp, fp, fp, ctypes.c_int, ctypes.c_int,
            ctypes.c_double, dp, dp, dp, dp, dp]
        lib.flr_oracle_backward.restype = ctypes.c_int
        lib.flr_oracle_fast.argtypes = [
            ctypes.c_int, ctypes.c_int, ctypes.c_int, fp, fp, fp, ctypes.c_int, ctypes.c_int,
            ctypes.c_double, ctypes.c_int, ctypes.c_double, dp, dp]
        lib.flr_oracle_fast.restype = ctypes.c_int
        lib.flr_oracle_fast_reg.argtypes = [
            ctypes.c_int, ctypes.c_int, ctypes.c_int, fp, fp, fp, ctypes.c_int, ctypes.c_int,
            ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_double, dp, dp]
        lib.flr_oracle_fast_reg.restype = ctypes.c_int
        lib.flr_oracle_threads.argtypes = []
        lib.flr_oracle_threads.restype = ctypes.c_int
        lib.flr_oracle_set_threads.argtypes = [ctypes.c_int]
        lib.flr_oracle_set_threads.restype = None
        _lib = lib
    return _lib


def _fptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def _dptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _as_f32(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float32)


class OracleError(RuntimeError):
    pass


def threads() -> int:
    """Threads the oracle's parallel loops use."""
    return int(_load().flr_oracle_threads())


def set_threads(n: int) -> None:
    """Threads for the oracle's parallel loops from now on (for timing; results do not change)."""
    _load().flr_oracle_set_threads(int(n))


def flr_forward(guide, radiance, radius, eps, coef_radius=0, map_guide=None,
                return_coef=False):
    """FLR forward pass in FP64 (Sec. 3.1-3.2 and the Appendix of the paper).

    guide: [Q, H, W]; radiance: [3, H, W]; map_guide: [Q, H, W] or None (= guide).
    Inputs are rounded to float32 first (the precision the GPU path reads).
    Returns out [3, H, W] float64, and with ``return_coef`` also the per-pixel model
    A_k before averaging as [(Q+1), 3, H, W] (row 0 is the bias).
    """
    rad = _as_f32(radiance)
    if rad.ndim != 3 or rad.shape[0] != 3:
        raise ValueError("radiance must be [3, H, W]")
    _, H, W = rad.shape
    g = _as_f32(guide)
    if g is None:
        g = np.zeros((0, H, W), np.float32)
    q = g.shape[0]
    if g.shape[1:] != (H, W):
        raise ValueError("guide must be [Q, H, W] with the radiance's H, W")
    mg = _as_f32(map_guide)
    if mg is not None and mg.shape != g.shape:
        raise ValueError("map_guide must match guide")
    out = np.empty((3, H, W), np.float64)
    coef = np.empty((q + 1, 3, H, W), np.float64) if return_coef else None
    st = _load().flr_oracle_forward(q, H, W, _fptr(g) if q else None, _fptr(mg), _fptr(rad),
                                    int(radius), int(coef_radius), float(eps),
                                    _dptr(out), _dptr(coef))
    if st != 0:
        raise OracleError(f"flr_oracle_forward failed with status {st}")
    return (out, coef) if return_coef else out


def flr_backward(guide, radiance, grad_out, radius, eps, coef_radius=0, map_guide=None):
    """FP64 gradient of <grad_out, FLR(guide, radiance)> (reverse-mode through Sec. 3.1-3.2).

    Returns a dict with ``guide`` [Q,H,W], ``radiance`` [3,H,W], ``eps`` (float) and, when a
    separate ``map_guide`` is given, ``map_guide`` [Q,H,W].  Without a map guide the guide
    gradient includes the path through the applied guide.
    """
    rad = _as_f32(radiance)
    g = _as_f32(guide)
    q, H, W = g.shape
    mg = _as_f32(map_guide)
    go = np.ascontiguousarray(grad_out, dtype=np.float64)
    if go.shape != (3, H, W):
        raise ValueError("grad_out must be [3, H, W]")
    gg = np.empty((q, H, W), np.float64)
    gm = np.empty((q, H, W), np.float64) if mg is not None else None
    gr = np.empty((3, H, W), np.float64)
    ge = np.zeros(1, np.float64)
    st = _load().flr_oracle_backward(q, H, W, _fptr(g), _fptr(mg), _fptr(rad), int(radius),
                                     int(coef_radius), float(eps), _dptr(go), _dptr(gg),
                                     _dptr(gm), _dptr(gr), _dptr(ge))
    if st != 0:
        raise OracleError(f"flr_oracle_backward failed with status {st}")
    res = {"guide": gg, "radiance": gr, "eps": float(ge[0])}
    if gm is not None:
        res["map_guide"] = gm
    return res


def flr_fast(guide, radiance, factor=8, sigma_blocks=1.25, taps=3, eps=1e-3, map_guide=None,
             scale=1, return_coef=False, appendix=None):
    """Fast FLR in FP64 (Sec. 3.2, and Sec. 3.2.1 when ``scale`` > 1).

    guide [Q,Hi,Wi] and radiance [3,Hi,Wi] at the input resolution; map_guide [Q,Hi*scale,
    Wi*scale] (None: the guide, scale 1).  Moments are summed over factor x factor blocks,
    blurred by a Gaussian of ``sigma_blocks`` block units truncated at ``taps`` blocks,
    solved per block and bilinearly interpolated.  Returns out [3,Ho,Wo] (float64) and
    with ``return_coef`` the block models [(Q+1),3,Hb,Wb].

    ``appendix`` = (eps_add, eps_mul) solves each block with the Appendix's regularised
    normalised system (additive term eps_add used twice as printed, multiplicative term
    eps_mul in [0, 1]) instead of the centred ridge with ``eps``.
    """
    g = _as_f32(guide)
    rad = _as_f32(radiance)
    q, Hi, Wi = g.shape
    mg = _as_f32(map_guide)
    Ho, Wo = Hi * scale, Wi * scale
    if mg is not None and mg.shape != (q, Ho, Wo):
        raise ValueError("map_guide must be [Q, Hi*scale, Wi*scale]")
    Hb, Wb = -(-Hi // factor), -(-Wi // factor)
    out = np.empty((3, Ho, Wo), np.float64)
    coef = np.empty((q + 1, 3, Hb, Wb), np.float64) if return_coef else None
    if appendix is None:
        st = _load().flr_oracle_fast(q, Hi, Wi, _fptr(g), _fptr(rad), _fptr(mg), int(factor), int(scale),
                                     float(sigma_blocks), int(taps), float(eps), _dptr(out), _dptr(coef))
    else:
        st = _load().flr_oracle_fast_reg(q, Hi, Wi, _fptr(g), _fptr(rad), _fptr(mg), int(factor), int(scale),
                                         float(sigma_blocks), int(taps), float(appendix[0]), 1, float(appendix[1]),
                                         _dptr(out), _dptr(coef))
    if st != 0:
        raise OracleError(f"flr_oracle_fast failed with status {st}")
    return (out, coef) if return_coef else out


def flr_fast_param_grads(guide, radiance, grad_out, factor=8, sigma_blocks=1.25, taps=3, eps=1e-3, map_guide=None,
                         scale=1, appendix=None, rel_step=1e-3):
    """Derivatives of L = sum(grad_out * fast_FLR(...)) with respect to the Gaussian's
    standard deviation (``sigma_blocks``) and the regularisation terms: Sec. 3.2 learns the
    blur radius and the regularisers by backpropagation.  Keys: "sigma", "eps" (the ridge
    term, or the Appendix's additive term when ``appendix`` = (eps_add, eps_mul) is given)
    and, with ``appendix``, "eps_mul" (its multiplicative term).

    The derivative is taken from its definition on the FP64 forward pass above: central
    differences with step h = rel_step * theta and h / 2, combined by Richardson
    extrapolation (4 D(h/2) - D(h)) / 3, which cancels the h^2 error term (the remaining
    O(h^4) term and the rounding of the FP64 forward are far below 1e-8 relative for the
    parameter ranges used).  Only positive parameters get a derivative (a zero term, e.g.
    eps_mul = 0, sits at the edge of its domain and is left out of the result)."""
    g_out = np.asarray(grad_out, np.float64)
    base = dict(factor=factor, sigma_blocks=sigma_blocks, taps=taps, eps=eps, map_guide=map_guide, scale=scale)
    params = {"sigma": float(sigma_blocks)}
    if appendix is None:
        params["eps"] = float(eps)
    else:
        params["eps"], params["eps_mul"] = float(appendix[0]), float(appendix[1])

    def loss(name, value):
        kw = dict(base)
        app = None if appendix is None else [float(appendix[0]), float(appendix[1])]
        if name == "sigma":
            kw["sigma_blocks"] = value
        elif name == "eps" and app is None:
            kw["eps"] = value
        elif name == "eps":
            app[0] = value
        else:
            app[1] = value
        return float(np.sum(g_out * flr_fast(guide, radiance, appendix=app, **kw)))

    out = {}
    for name, theta in params.items():
        if not theta > 0.0:
            continue
        h = rel_step * theta

        def diff(step):
            return (loss(name, theta + step) - loss(name, theta - step)) / (2.0 * step)
        out[name] = (4.0 * diff(h / 2.0) - diff(h)) / 3.0
    return out
