"""Batched serving pattern (Sec. 3.2.1 joint denoising and upsampling, several frames of
mixed sizes): one persistent cooperative launch, CUDA-graph capture, bounded device waits.
"""
import time

import numpy as np
import pytest

import oracle
import synth
from helpers import TOL, to_dev

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


SIZES = [(90, 160), (54, 96), (120, 200), (45, 80)]  # input sizes; output is 2x


def make_frames(scale):
    import torch
    frames, host = [], []
    for k, (H, W) in enumerate(SIZES):
        g_lo, y_lo = synth.render(10 + k, H, W)
        g_hi, _ = synth.render(10 + k, H * scale, W * scale)
        out = torch.empty((3, H * scale, W * scale), device="cuda")
        frames.append((to_dev(g_lo), to_dev(y_lo), to_dev(g_hi), out))
        host.append((g_lo, y_lo, g_hi))
    return frames, host


def test_batch_equals_per_frame_and_oracle(flr):
    import torch
    frames, host = make_frames(2)
    f = flr.FastFLR(q=8, factor=4, scale=2)
    f.denoise_batch(frames)
    assert f.batch_status() == 0
    batch = [o.clone() for (_, _, _, o) in frames]
    for (g, y, z, o), b in zip(frames, batch):
        single = f.denoise(g, y, map_guide=z)
        torch.cuda.synchronize()
        assert torch.equal(single, b)
    for (g_lo, y_lo, g_hi), b in zip(host, batch):
        ref = oracle.flr_fast(g_lo, y_lo, factor=4, map_guide=g_hi, scale=2)
        err = float(np.max(np.abs(b.cpu().numpy() - ref)) / np.sqrt(np.mean(ref ** 2)))
        assert err <= TOL
    f.close()


def test_batch_captured_in_cuda_graph(flr):
    import torch
    frames, _ = make_frames(2)
    f = flr.FastFLR(q=8, factor=4, scale=2)
    f.reserve_batch(frames)
    f.denoise_batch(frames)  # eager reference
    torch.cuda.synchronize()
    eager = [o.clone() for (_, _, _, o) in frames]
    for (_, _, _, o) in frames:
        o.zero_()
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            f.denoise_batch(frames, stream=s)
    for _ in range(3):
        graph.replay()
    torch.cuda.synchronize()
    assert f.batch_status() == 0
    for (_, _, _, o), e in zip(frames, eager):
        assert torch.equal(o, e)
    f.close()


def test_bounded_wait_reports_timeout(flr):
    t0 = time.time()
    status = flr.barrier_selftest(ctas=4, timeout_ns=50_000_000)
    assert status == flr.BATCH_TIMEOUT
    assert time.time() - t0 < 10.0


def test_bounded_mbarrier_wait_reports_timeout(flr):
    """The mbarrier wait of the TMA / tensor-core kernels gives up after its limit: a phase
    that never completes sets bit 0 only (the completing one is not reported), in bounded
    time, and the context stays usable afterwards."""
    import torch
    t0 = time.time()
    assert flr.mbarrier_selftest(ctas=8, timeout_ns=20_000_000) == 1
    assert time.time() - t0 < 10.0
    x = torch.ones(16, device="cuda")
    assert float((x * 2).sum().item()) == 32.0


def test_per_pixel_batch_equals_per_frame(flr):
    import torch
    f = flr.FLR(q=8, radius=5, coef_radius=5)
    frames = []
    for k, (H, W) in enumerate(SIZES):
        g, y = synth.render(20 + k, H, W)
        frames.append((to_dev(g), to_dev(y), None, torch.empty((3, H, W), device="cuda")))
    f.denoise_batch(frames)
    torch.cuda.synchronize()
    for (g, y, _, o) in frames:
        assert torch.equal(f.denoise(g, y), o)
    f.close()


def test_batch_with_guide_network(flr):
    """The serving step with the FLNR guide network (serving.GuidedBatch): per frame size,
    the network's forward pass over the half-resolution inputs gives the model guides, then
    one persistent fast-FLR launch does joint denoising and 2x upsampling of every frame;
    the step is a captured CUDA graph, replayed twice.  The map guides are the same
    network's output on the full-resolution inputs (guides from one distribution, as the
    model and map guides of FLNR are).  The model guides equal a separate forward pass of
    the network, bit for bit, and each frame's result meets the FP64 oracle of fast FLR run
    on those guides (the map guide differs from the model guide: the absolute bar of the
    joint-upsampling tests)."""
    import torch

    from paper_2410_11625_gb300 import flnr, serving
    weights = flnr.init_weights(3)
    hi_net = flnr.FLNR(2 * 96 * 128, weights)
    groups = []
    for i, (h, w) in enumerate([(32, 48), (48, 64)]):
        xs, xs_hi = [], []
        for j in range(2):
            g_lo, y_lo = synth.render(40 + 2 * i + j, h, w)
            g_hi, y_hi = synth.render(40 + 2 * i + j, 2 * h, 2 * w)
            xs.append(np.concatenate([g_lo, y_lo]))
            xs_hi.append(np.concatenate([g_hi, y_hi]))
        z = hi_net.forward(torch.from_numpy(np.stack(xs_hi)).cuda()).clone()
        groups.append((torch.from_numpy(np.stack(xs)).cuda(), z, torch.empty((2, 3, 2 * h, 2 * w), device="cuda")))
    torch.cuda.synchronize()
    hi_net.close()
    b = serving.GuidedBatch(groups, weights, factor=4)
    b.run()
    b.run()
    assert b.status() == 0
    net = flnr.FLNR(2 * 48 * 64, weights)
    for (x, z, o), e in zip(groups, b.enh):
        assert torch.equal(net.forward(x), e)
        for n in range(x.shape[0]):
            ref = oracle.flr_fast(e[n].cpu().numpy(), x[n, 8:].cpu().numpy(), factor=4,
                                  map_guide=z[n].cpu().numpy(), scale=2)
            got = o[n].cpu().numpy()
            assert np.max(np.abs(got - ref)) <= TOL * np.sqrt(np.mean(ref ** 2))
    net.close()
    b.close()
