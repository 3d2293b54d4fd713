"""Batched serving step with the FLNR guide network: joint denoising and 2x upsampling of
frames of mixed sizes (Sec. 3.2.1) with model guides enhanced by the network (Sec. 3.3).

One step: for every group of same-size frames, the network's forward pass over the group's
half-resolution inputs (guides and noisy radiance, concatenated channel-wise) gives the
enhanced model guides; then ONE persistent cooperative fast-FLR launch fits every frame's
block models on its enhanced guides and half-resolution radiance and applies them to its
full-resolution map guides.  The whole step is captured once in a CUDA graph and replayed.
Launch arrangement only: every step runs in libflr.so's kernels.
"""
from __future__ import annotations

from . import flnr, flr


class GuidedBatch:
    """groups: list of (xin [N,11,h,w], map_guide [N,8,2h,2w], out [N,3,2h,2w]) CUDA float32
    tensors, one entry per frame size (xin = guides then radiance, as the network reads it).
    weights: the network's parameters (flnr.init_weights layout)."""

    def __init__(self, groups, weights, factor=4, sigma=1.25, taps=3, eps=1e-3, pivot_ratio=1e-3, graph=True):
        import torch
        self.groups = groups
        dev = groups[0][0].device
        self.max_px = max(int(x.shape[0] * x.shape[2] * x.shape[3]) for x, _, _ in groups)
        self.net = flnr.FLNR(self.max_px, weights)
        self.enh = [torch.empty((x.shape[0], 8, x.shape[2], x.shape[3]), dtype=torch.float32, device=dev)
                    for x, _, _ in groups]
        self.frames = []
        for (x, z, o), e in zip(groups, self.enh):
            for n in range(x.shape[0]):
                self.frames.append((e[n], x[n, 8:11], z[n], o[n]))
        self.flr = flr.FastFLR(q=8, factor=factor, scale=2, sigma=sigma, taps=taps, eps=eps,
                               pivot_ratio=pivot_ratio)
        self.flr.reserve_batch(self.frames)
        self.stream = torch.cuda.Stream(dev)
        self.graph = None
        if graph:
            with torch.cuda.stream(self.stream):
                self._step()  # eager once: kernel attributes set outside the capture
                self.stream.synchronize()
                self.graph = torch.cuda.CUDAGraph()
                with torch.cuda.graph(self.graph, stream=self.stream):
                    self._step()

    def _step(self):
        for (x, _, _), e in zip(self.groups, self.enh):
            self.net.forward(x, out=e)
        self.flr.denoise_batch(self.frames, stream=self.stream)

    def run(self):
        """One serving step on the batch's stream (the graph when captured)."""
        import torch
        with torch.cuda.stream(self.stream):
            if self.graph is not None:
                self.graph.replay()
            else:
                self._step()

    def status(self):
        """Waits for the step; FLR_OK (0), or FLR_ERR_TIMEOUT (-6) if a bounded wait of the
        fast-FLR batch ran out; raises flr.FlrError if one of the network's did."""
        s = self.flr.batch_status()
        self.net.status()
        return s

    def close(self):
        self.graph = None
        self.flr.close()
        self.net.close()
