"""The fused forward path (flr_fused.cu) through the C ABI, against the FP64 oracle.

flr_denoise takes the fused kernel for q = 8 with (r, rc) = (8, 8), (8, 0) or (5, 5) and
16-byte rows; these tests cover what is particular to it:
  - flagged pixels: with pivot_ratio = 1 every pixel is flagged, left out of the fused
    average and given its FP64 model by the correction kernel, deterministically;
  - a separate map guide read by TMA for the apply;
  - strip and segment edges, windows larger than the image, ragged strips;
  - the 1080p launch geometry of the backward pass (which recomputes the models with the
    unfused kernels) on sampled blocks;
  - the shared-memory setting of the generic forward kernel, which handles of different
    radii share, is only ever raised.
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


def run(flr, g, y, r, rc, eps=1e-3, pivot_ratio=1e-3, map_guide=None):
    import torch
    f = flr.FLR(q=g.shape[0], radius=r, coef_radius=rc, eps=eps, pivot_ratio=pivot_ratio)
    out = f.denoise(to_dev(g), to_dev(y), map_guide=None if map_guide is None else to_dev(map_guide))
    torch.cuda.synchronize()
    res = out.cpu().numpy()
    st = f.stats()
    f.close()
    return res, st


@pytest.mark.parametrize("r,rc", [(8, 8), (5, 5), (8, 0)])
def test_every_pixel_flagged_gets_its_fp64_model(flr, r, rc):
    """pivot_ratio = 1 flags every solve: the fused kernel averages nothing and the FP64
    correction adds every model's share (rc > 0) or writes every result (rc = 0)."""
    g, y = synth.render(6, 64, 200)
    eps = 1e-3
    ref = oracle.flr_forward(g, y, r, eps, coef_radius=rc)
    got, st = run(flr, g, y, r, rc, eps=eps, pivot_ratio=1.0)
    assert st["flagged"] == 64 * 200 and st["resolved"] == st["flagged"]
    assert np.all(np.isfinite(got))
    assert rel_err(got, ref) <= (2e-6 if rc == 0 else TOL)


def test_flagged_result_is_deterministic(flr):
    """The flagged pixels are listed in (row, column) order per CTA and corrected one after
    the other, so two runs agree bit for bit."""
    g, y = synth.render(7, 64, 160)
    a, _ = run(flr, g, y, 8, 8, eps=1e-5, pivot_ratio=0.3)
    b, st = run(flr, g, y, 8, 8, eps=1e-5, pivot_ratio=0.3)
    assert st["flagged"] > 0
    assert np.array_equal(a, b)


@pytest.mark.parametrize("r,rc", [(8, 8), (8, 0), (5, 5)])
def test_separate_map_guide(flr, r, rc):
    """Random full-rank model and map guides: the apply reads the map guide's rows, staged
    by TMA (rc > 0) or from global memory (rc = 0)."""
    g, y = synth.random_frame(81, 96, 176, 8)
    z, _ = synth.random_frame(82, 96, 176, 8)
    ref = oracle.flr_forward(g, y, r, 1e-3, coef_radius=rc, map_guide=z)
    got, _ = run(flr, g, y, r, rc, map_guide=z)
    assert rel_err(got, ref) <= TOL


@pytest.mark.parametrize("H,W,r,rc", [
    (3, 40, 8, 8), (40, 4, 8, 8), (7, 164, 5, 5), (333, 84, 8, 8), (61, 332, 8, 0), (250, 404, 5, 5),
])
def test_edges_and_ragged_strips(flr, H, W, r, rc):
    """Windows larger than the image, a single strip narrower than one window, ragged last
    strips and segments (uniform guides, so every window is well conditioned)."""
    g, y = synth.random_frame(H * 7 + W, H, W, 8)
    ref = oracle.flr_forward(g, y, r, 1e-3, coef_radius=rc)
    got, st = run(flr, g, y, r, rc)
    assert np.all(np.isfinite(got))
    assert rel_err(got, ref) <= TOL


def test_generic_kernel_shared_memory_is_only_raised(flr):
    """Handles of one guide count and different radii share the generic forward kernel; a
    later handle with a smaller radius must not take shared memory from an earlier, larger
    one (q = 4 runs the unfused kernels)."""
    import torch
    g, y = synth.random_frame(5, 80, 120, 4)
    big = flr.FLR(q=4, radius=12, coef_radius=3, eps=1e-3)
    small = flr.FLR(q=4, radius=2, coef_radius=1, eps=1e-3)
    out_small = small.denoise(to_dev(g), to_dev(y))
    out_big = big.denoise(to_dev(g), to_dev(y))
    torch.cuda.synchronize()
    assert rel_err(out_big.cpu().numpy(), oracle.flr_forward(g, y, 12, 1e-3, coef_radius=3)) <= TOL
    assert rel_err(out_small.cpu().numpy(), oracle.flr_forward(g, y, 2, 1e-3, coef_radius=1)) <= TOL
    # the entry point without a handle, at the larger radius, after the smaller handle
    lib = flr.load_library()
    p = flr.FlrParams(4, 12, 3, 1e-3, 1e-3, 0)
    out = torch.empty((3, 80, 120), device="cuda")
    G, Y = to_dev(g), to_dev(y)
    st = lib.flr_denoise_noalloc(ctypes.byref(p), ctypes.c_void_p(G.data_ptr()), None, ctypes.c_void_p(Y.data_ptr()),
                                 ctypes.c_void_p(out.data_ptr()), 80, 120,
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert st == 0
    assert rel_err(out.cpu().numpy(), oracle.flr_forward(g, y, 12, 1e-3, coef_radius=3)) <= TOL
    big.close()
    small.close()
