"""flr_denoise_noalloc, the entry point for callers that cannot allocate device memory.

Such a caller (a custom allocator or memory-pool callback, a host that forbids late
allocations, a plugin that only receives buffers) cannot create a handle, because a
handle allocates its workspace.  flr_denoise_noalloc keeps that workspace in a fixed
__device__ array instead.  These tests call it through the C ABI twice in a row on
different frames and check each result against the handle-based flr_denoise and against
the FP64 oracle, over the paths the call can take: the fused kernel with coefficient
averaging (r = rc = 5) and without (r = 8, rc = 0), every pixel re-solved in FP64
(pivot_ratio = 1), a separate map guide, and the unfused kernels (q = 4, r = 3).  The file
sits by itself and is collected last.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from helpers import TOL, rel_err, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def flr():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2410_11625_gb300 import flr as mod
    return mod


def noalloc(flr, params, G, Y, out, Z=None):
    import torch
    lib = flr.load_library()
    H, W = int(Y.shape[1]), int(Y.shape[2])
    return lib.flr_denoise_noalloc(ctypes.byref(params), ctypes.c_void_p(G.data_ptr()),
                                   None if Z is None else ctypes.c_void_p(Z.data_ptr()),
                                   ctypes.c_void_p(Y.data_ptr()), ctypes.c_void_p(out.data_ptr()), H, W,
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("q,r,rc,pivot,map_guide", [
    (8, 5, 5, 1e-3, False), (8, 8, 0, 1e-3, False), (8, 5, 5, 1.0, False), (8, 8, 0, 1.0, False),
    (8, 5, 5, 1e-3, True), (4, 3, 2, 1e-3, False),
])
def test_noalloc_matches_handle_path_and_oracle_twice(flr, q, r, rc, pivot, map_guide):
    import torch
    params = flr.FlrParams(q, r, rc, 1e-3, pivot, 0)
    ref_handle = flr.FLR(q=q, radius=r, coef_radius=rc, eps=1e-3, pivot_ratio=pivot)
    for seed, (H, W) in ((0, (256, 256)), (11, (200, 300))):
        if q == 8:
            g, y = synth.render(seed, H, W)
        else:
            g, y = synth.random_frame(seed, H, W, q)
        z = (g + synth.random_frame(seed + 7, H, W, q)[0] * 0.05).astype(np.float32) if map_guide else None
        G, Y = to_dev(g), to_dev(y)
        Z = None if z is None else to_dev(z)
        out = torch.empty((3, H, W), device="cuda")
        st = noalloc(flr, params, G, Y, out, Z)
        assert st == 0, flr.STATUS.get(st, st)
        ref = ref_handle.denoise(G, Y, map_guide=Z)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert rel_err(got, ref.cpu().numpy().astype(np.float64)) <= TOL
        oref = oracle.flr_forward(g, y, r, 1e-3, coef_radius=rc, map_guide=z)
        if pivot >= 1.0 and rc == 0:  # every result from the FP64 re-solve
            assert rel_err(got, oref) <= 2e-6
        elif z is not None:  # rendered guides with a perturbed map guide: absolute bar
            assert np.max(np.abs(got - oref)) <= 1e-4 * np.sqrt(np.mean(oref ** 2))
        else:
            assert rel_err(got, oref) <= TOL
    ref_handle.close()


def test_noalloc_rejects_frames_beyond_its_array(flr):
    import torch
    params = flr.FlrParams(8, 5, 5, 1e-3, 1e-3, 0)
    big = torch.zeros((8, 257, 256), device="cuda")
    out = torch.zeros((3, 257, 256), device="cuda")
    st = noalloc(flr, params, big, big[:3], out)
    assert st == -4
