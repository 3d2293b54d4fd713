"""Seeded synthetic inputs for FLR: procedural Lambertian rooms and random frames.

This module is an input generator only and holds none of FLR's arithmetic.  Both the
FP64 oracle (in the tests) and the GPU library (in the tests and the benchmark) consume
what it makes, which is why it lives apart from both.

``render(seed, H, W)`` gives the frame of the paper's workload shape (Sec. 4.1): eight
noise-free guides (albedo RGB, world normal xyz, normalised depth, ambient occlusion)
and the albedo-demodulated one-sample-per-pixel indirect radiance, traced by
``pathtracer.c``.  ``random_frame`` gives i.i.d. uniform frames and the adversarial
variants the parity tests use.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "_lib")
_LIBPATH = os.path.join(_LIBDIR, "libsynth.so")
_SOURCES = ["pathtracer.c", "scene.h"]
_GPU_LIBPATH = os.path.join(_LIBDIR, "libsynth_gpu.so")
_GPU_SOURCES = ["pathtracer_gpu.cu", "scene.h"]

GUIDE_CHANNELS = ("albedo_r", "albedo_g", "albedo_b", "normal_x", "normal_y", "normal_z",
                  "depth", "ao")

_lib = None


def build(force: bool = False) -> str:
    """Compile ``libsynth.so`` with gcc (OpenMP) and return its path."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    if not force and os.path.exists(_LIBPATH):
        if os.path.getmtime(_LIBPATH) >= max(os.path.getmtime(s) for s in srcs):
            return _LIBPATH
    os.makedirs(_LIBDIR, exist_ok=True)
    tmp = _LIBPATH + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-o", tmp]
                   + [s for s in srcs if s.endswith(".c")] + ["-lm"], check=True)
    os.replace(tmp, _LIBPATH)
    return _LIBPATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIBPATH)
        fp = ctypes.POINTER(ctypes.c_float)
        lib.synth_render.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_int, fp, fp, fp,
                                     ctypes.c_int]
        lib.synth_render.restype = ctypes.c_int
        lib.synth_render_noise.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                           ctypes.c_int, fp]
        lib.synth_render_noise.restype = ctypes.c_int
        lib.synth_build_scene.argtypes = [ctypes.c_uint64, ctypes.c_void_p]
        lib.synth_build_scene.restype = ctypes.c_int
        _lib = lib
    return _lib


_gpu_lib = None


def build_gpu(force: bool = False) -> str:
    """Compile ``libsynth_gpu.so`` (the reference renderer on the GPU) with nvcc for sm_103a,
    without fused multiply-adds so that its ray arithmetic rounds as the host's does."""
    srcs = [os.path.join(_HERE, s) for s in _GPU_SOURCES]
    if not force and os.path.exists(_GPU_LIBPATH):
        if os.path.getmtime(_GPU_LIBPATH) >= max(os.path.getmtime(s) for s in srcs):
            return _GPU_LIBPATH
    os.makedirs(_LIBDIR, exist_ok=True)
    tmp = _GPU_LIBPATH + f".tmp{os.getpid()}"
    nvcc = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-fmad=false", "-std=c++17",
                    "-Xcompiler", "-fPIC", "-shared", "-o", tmp, srcs[0]], check=True)
    os.replace(tmp, _GPU_LIBPATH)
    return _GPU_LIBPATH


def scene_record(seed: int) -> bytes:
    """The room of ``seed`` as the host builds it (a scene_t record)."""
    lib = _load()
    n = lib.synth_build_scene(ctypes.c_uint64(seed), None)
    buf = ctypes.create_string_buffer(n)
    lib.synth_build_scene(ctypes.c_uint64(seed), buf)
    return buf.raw


def render_reference_gpu(seed: int, H: int, W: int, spp: int, device="cuda"):
    """The ``spp``-sample reference [3, H, W] of ``render(seed, H, W, ref_spp=spp)`` traced on
    the GPU (same room, estimator and random numbers; a CUDA float32 tensor)."""
    import torch
    global _gpu_lib
    if _gpu_lib is None:
        build_gpu()
        lib = ctypes.CDLL(_GPU_LIBPATH)
        lib.synth_reference_gpu.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
        lib.synth_reference_gpu.restype = ctypes.c_int
        _gpu_lib = lib
    rec = scene_record(seed)
    out = torch.empty((3, H, W), dtype=torch.float32, device=device)
    st = _gpu_lib.synth_reference_gpu(rec, len(rec), ctypes.c_uint64(seed), int(H), int(W), int(spp),
                                      ctypes.c_void_p(out.data_ptr()),
                                      ctypes.c_void_p(torch.cuda.current_stream(out.device).cuda_stream))
    if st != 0:
        raise RuntimeError(f"synth_reference_gpu failed with status {st}")
    return out


def render(seed: int, H: int, W: int, ref_spp: int = 0):
    """Render the procedural room of ``seed`` at H x W.

    Returns ``(guide [8,H,W], radiance [3,H,W])`` as float32, plus the ``ref_spp``-sample
    reference [3,H,W] as a third element when ``ref_spp > 0``.
    """
    guide = np.empty((8, H, W), np.float32)
    rad = np.empty((3, H, W), np.float32)
    ref = np.empty((3, H, W), np.float32) if ref_spp > 0 else None
    fp = ctypes.POINTER(ctypes.c_float)
    st = _load().synth_render(ctypes.c_uint64(seed), H, W, guide.ctypes.data_as(fp),
                              rad.ctypes.data_as(fp),
                              None if ref is None else ref.ctypes.data_as(fp), int(ref_spp))
    if st != 0:
        raise ValueError("synth_render: bad arguments")
    return (guide, rad, ref) if ref is not None else (guide, rad)


def render_noise(seed: int, H: int, W: int, count: int, first: int = 0):
    """``count`` further independent 1 spp radiance renders [count,3,H,W] of the scene of
    ``seed`` (same guides and reference as ``render``), realisations first..first+count-1."""
    rad = np.empty((count, 3, H, W), np.float32)
    st = _load().synth_render_noise(ctypes.c_uint64(seed), H, W, ctypes.c_uint64(first), int(count),
                                    rad.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
    if st != 0:
        raise ValueError("synth_render_noise: bad arguments")
    return rad


def random_frame(seed: int, H: int, W: int, q: int = 8, kind: str = "uniform"):
    """Seeded random (guide [q,H,W], radiance [3,H,W]) float32 frames.

    kinds:
      uniform       i.i.d. U[0, 1] guides and radiance
      signed        guides U[-1, 1], radiance U[0, 1]
      const_guide   guide channel 1 constant over the frame (rank-deficient windows)
      dup_guide     guide channel 2 duplicates channel 0 (collinear guides)
      depth_offset  uniform guides with +100 added to the last guide channel
      heavy_tail    uniform guides; Pareto(alpha = 1.5) radiance: fireflies up to ~10^3
                    times the median at 10^5 pixels
    """
    rng = np.random.default_rng(seed)
    lo = -1.0 if kind == "signed" else 0.0
    g = rng.uniform(lo, 1.0, size=(q, H, W)).astype(np.float32)
    y = rng.uniform(0.0, 1.0, size=(3, H, W)).astype(np.float32)
    if kind == "const_guide" and q > 1:
        g[1] = np.float32(0.37)
    elif kind == "dup_guide" and q > 2:
        g[2] = g[0]
    elif kind == "depth_offset":
        g[q - 1] += np.float32(100.0)
    elif kind == "heavy_tail":
        u = rng.uniform(0.0, 1.0, size=(3, H, W))
        y = (0.2 * (1.0 - u) ** (-1.0 / 1.5)).astype(np.float32)
    elif kind not in ("uniform", "signed", "const_guide", "dup_guide"):
        raise ValueError(f"unknown kind {kind!r}")
    return g, y
