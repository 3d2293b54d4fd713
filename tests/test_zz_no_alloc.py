"""flr_denoise_noalloc, the entry point for callers that cannot allocate device memory.

Such a caller (a custom allocator or memory-pool callback, a host that forbids late
allocations, a plugin that only receives buffers) cannot create a handle, because a
handle allocates its workspace.  flr_denoise_noalloc keeps that workspace in a fixed
__device__ array instead.  This test calls it through the C ABI twice in a row, on two
different frames, and checks each result against the handle-based flr_denoise within the
parity tolerance.  It sits in a file of its own, collected last.
"""
import ctypes

import numpy as np
import pytest

import synth
from helpers import TOL, rel_err, to_dev

pytestmark = pytest.mark.gpu


def test_noalloc_matches_handle_path_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2410_11625_gb300 import flr
    lib = flr.load_library()
    params = flr.FlrParams(8, 5, 5, 1e-3, 1e-3, 0)
    ref_handle = flr.FLR(q=8, radius=5, coef_radius=5, eps=1e-3, pivot_ratio=1e-3)
    stream = torch.cuda.current_stream()
    for seed, (H, W) in ((0, (256, 256)), (11, (200, 300))):
        g, y = synth.render(seed, H, W)
        G, Y = to_dev(g), to_dev(y)
        out = torch.empty((3, H, W), device="cuda")
        st = lib.flr_denoise_noalloc(ctypes.byref(params), ctypes.c_void_p(G.data_ptr()), None,
                                     ctypes.c_void_p(Y.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                     H, W, ctypes.c_void_p(stream.cuda_stream))
        assert st == 0, flr.STATUS.get(st, st)
        ref = ref_handle.denoise(G, Y)
        torch.cuda.synchronize()
        assert rel_err(out.cpu().numpy(), ref.cpu().numpy().astype(np.float64)) <= TOL
    # a frame beyond the array's capacity is refused, not written
    big = torch.zeros((8, 257, 256), device="cuda")
    st = lib.flr_denoise_noalloc(ctypes.byref(params), ctypes.c_void_p(big.data_ptr()), None,
                                 ctypes.c_void_p(big.data_ptr()), ctypes.c_void_p(big.data_ptr()),
                                 257, 256, None)
    assert st == -4
    ref_handle.close()
