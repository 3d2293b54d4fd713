"""FLNR training and evaluation (Sec. 3.3): the guide network is trained end to end
through FLR, on crops of the project's own rendered scenes.

One training step (batch B of c x c crops):
  X' = FLNR(X || Y)                      flnr_guide_forward
  I_b = FLR(X'_b, Y_b), per crop         flr_denoise (8 outputs: X' is both model and map
                                         guide; 16 outputs, Sec. 3.3's two sets: channels
                                         0-7 fit the models, 8-15 are the map guide)
  L = mean |I - I_ref|, dL/dI             flnr_l1_loss (config 4), or Sec. 3.3's SMAPE
                                         mean |I - I_ref| / (|I| + |I_ref| + 0.01)
                                         (flnr_smape_loss, loss="smape")
  dL/dX'_b = FLR adjoint, per crop       flr_backward
  parameter gradients                     flnr_guide_backward
  Adam on the FP32 master weights         flnr_adam_step (BF16 copies refreshed)
Every step runs in the library's kernels; this module samples crops on the host and
moves them to the device, and writes and reads training checkpoints (save_checkpoint,
load_checkpoint: weights, Adam moments, step count, learning rate, sampler state).  Data: `synth.render` scenes with 1 spp inputs and high-spp
references; held-out evaluation scenes use seeds >= 1,000,000.
"""
from __future__ import annotations

import json
import math
import struct
import zlib

import numpy as np

from . import flnr as _flnr
from . import flr as _flr

EVAL_SEED0 = 1_000_000


def render_scenes(seeds, H, W, ref_spp=1024, noise=1, gpu_ref=False):
    """Per seed: (x [11,H,W], ref [3,H,W], albedo [3,H,W], extra [noise-1,3,H,W]) float32,
    x = guides ++ 1 spp radiance; `extra` holds further independent 1 spp renders of the
    same scene (cheap next to the reference), which training draws from as well.  With
    gpu_ref the reference is traced by the input generator's GPU renderer (the same room,
    estimator and random numbers as the host's)."""
    import synth
    out = []
    for s in seeds:
        if gpu_ref:
            g, y = synth.render(int(s), H, W)
            ref = synth.render_reference_gpu(int(s), H, W, ref_spp).cpu().numpy()
        else:
            g, y, ref = synth.render(int(s), H, W, ref_spp=ref_spp)
        extra = synth.render_noise(int(s), H, W, noise - 1) if noise > 1 else np.empty((0, 3, H, W), np.float32)
        out.append((np.ascontiguousarray(np.concatenate([g, y])), ref, g[:3].copy(), extra))
    return out


def sample_batch(rng, scenes, batch, crop):
    """Random crops (random scene, noise realisation, position, horizontal / vertical flips):
    x [B,11,c,c], ref [B,3,c,c]."""
    xs = np.empty((batch, 11, crop, crop), np.float32)
    rs = np.empty((batch, 3, crop, crop), np.float32)
    for b in range(batch):
        x, ref, _, extra = scenes[rng.integers(len(scenes))]
        H, W = x.shape[1:]
        i, j = rng.integers(0, H - crop + 1), rng.integers(0, W - crop + 1)
        k = rng.integers(len(extra) + 1)
        cx = x[:, i:i + crop, j:j + crop]
        if k > 0:
            cx = np.concatenate([cx[:8], extra[k - 1][:, i:i + crop, j:j + crop]])
        cr = ref[:, i:i + crop, j:j + crop]
        if rng.random() < 0.5:
            cx, cr = cx[:, :, ::-1], cr[:, :, ::-1]
        if rng.random() < 0.5:
            cx, cr = cx[:, ::-1], cr[:, ::-1]
        xs[b], rs[b] = cx, cr
    return xs, rs


class Trainer:
    """Holds the network, the FLR handle and the device buffers of one batch shape."""

    def __init__(self, weights, batch=16, crop=128, radius=8, eps=1e-3, lr=1e-3, device="cuda", graph=True,
                 loss="l1"):
        import torch
        if loss not in ("l1", "smape"):
            raise ValueError("loss must be 'l1' or 'smape'")
        self.B, self.c, self.lr = batch, crop, lr
        self.loss_fn = _flnr.l1_loss if loss == "l1" else _flnr.smape_loss
        self.net = _flnr.FLNR(batch * crop * crop, weights)
        # one FLR handle and stream per crop: the crops' FLR passes and adjoints (small
        # grids each) run concurrently, and no two of them share a handle's workspace.
        # These handles only ever see crops, so their buffers never move once the step is
        # captured in a graph; `flr` is a separate handle for evaluation at other sizes.
        self.flrs = [_flr.FLR(q=8, radius=radius, eps=eps) for _ in range(batch)]
        for f in self.flrs:
            f.reserve(crop, crop)
        self.flr = _flr.FLR(q=8, radius=radius, eps=eps)
        self.streams = [torch.cuda.Stream() for _ in range(batch)]
        opt = dict(dtype=torch.float32, device=device)
        self.x_host = torch.empty((batch, 11, crop, crop), dtype=torch.float32).pin_memory()
        self.r_host = torch.empty((batch, 3, crop, crop), dtype=torch.float32).pin_memory()
        self.x = torch.empty((batch, 11, crop, crop), **opt)
        self.ref = torch.empty((batch, 3, crop, crop), **opt)
        self.outputs = self.net.outputs
        self.guides = torch.empty((batch, self.outputs, crop, crop), **opt)
        self.out = torch.empty((batch, 3, crop, crop), **opt)
        self.g_guides = torch.empty((batch, self.outputs, crop, crop), **opt)
        self.g_rad = torch.empty((batch, 3, crop, crop), **opt)
        self.steps = 0
        # After two eager warm-up steps the device part of a step (network forward, FLR per
        # crop, L1, FLR adjoint per crop, network backward: about 200 launches on B + 1
        # streams) is captured once in a CUDA graph and replayed.  The batch's H2D copy and Adam stay outside the
        # graph: the host buffer is refilled every step, and the step count and learning rate
        # enter Adam's arguments.
        self.use_graph = graph
        self.graph = None
        self.loss_static = None
        self.h2d_done = torch.cuda.Event()
        self.h2d_pending = False

    def _per_crop(self, fn):
        """Runs fn(b) for every crop on its own stream, forked from and joined back into
        the current stream."""
        import torch
        cur = torch.cuda.current_stream()
        for b in range(self.B):
            self.streams[b].wait_stream(cur)
            with torch.cuda.stream(self.streams[b]):
                fn(b)
        for b in range(self.B):
            cur.wait_stream(self.streams[b])

    def _device_step(self):
        """Forward, loss and gradients of the batch already on the device; returns the loss."""
        self.net.forward(self.x, out=self.guides)
        if self.outputs == 16:  # model guides 0-7, map guides 8-15
            self._per_crop(lambda b: self.flrs[b].denoise(self.guides[b, :8], self.x[b, 8:11],
                                                         map_guide=self.guides[b, 8:], out=self.out[b]))
        else:
            self._per_crop(lambda b: self.flrs[b].denoise(self.guides[b], self.x[b, 8:11], out=self.out[b]))
        loss, g_out = self.loss_fn(self.out, self.ref)
        if self.outputs == 16:
            self._per_crop(lambda b: self.flrs[b].backward(
                self.guides[b, :8], self.x[b, 8:11], g_out[b], map_guide=self.guides[b, 8:],
                grad_guide=self.g_guides[b, :8], grad_map_guide=self.g_guides[b, 8:], grad_radiance=self.g_rad[b]))
        else:
            self._per_crop(lambda b: self.flrs[b].backward(self.guides[b], self.x[b, 8:11], g_out[b],
                                                          grad_guide=self.g_guides[b], grad_radiance=self.g_rad[b]))
        self.net.zero_grads(self.x)
        self.net.backward(self.g_guides)
        return loss

    def step(self, xs, rs):
        """One optimisation step on host crops; returns the loss as a device tensor."""
        import torch
        if self.h2d_pending:
            self.h2d_done.synchronize()  # the previous step's copies have read the host buffers
        self.x_host.numpy()[...] = xs
        self.r_host.numpy()[...] = rs
        self.x.copy_(self.x_host, non_blocking=True)
        self.ref.copy_(self.r_host, non_blocking=True)
        self.h2d_done.record()
        self.h2d_pending = True
        if self.graph is None and self.use_graph and self.steps >= 2:
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, capture_error_mode="relaxed"):
                self.loss_static = self._device_step()
            self.graph = graph
        if self.graph is not None:
            self.graph.replay()
            loss = self.loss_static.clone()
        else:
            loss = self._device_step()
        self.steps += 1
        self.net.adam_step(self.steps, lr=self.lr, stream_of=self.x)
        return loss

    def train(self, scenes, steps, seed=0, lr_final=None, log_every=0, rng=None, t0=0, total=None):
        """`steps` Adam steps on random crops of `scenes`, with the learning rate on a cosine
        from self.lr down to lr_final over `total` steps (default: `steps`), starting at step
        t0 of that schedule.  Crops are drawn from `rng` (a numpy Generator; default: a new
        one seeded with `seed`).  A run resumed from a checkpoint passes the generator that
        load_checkpoint returns and t0 = the steps already taken, so that it draws and
        schedules exactly what the uninterrupted run would have."""
        rng = np.random.default_rng(seed) if rng is None else rng
        total = steps if total is None else total
        lr0, lr1 = self.lr, (self.lr if lr_final is None else lr_final)
        losses = []
        for t in range(steps):
            self.lr = lr1 + 0.5 * (lr0 - lr1) * (1 + math.cos(math.pi * (t0 + t) / max(total, 1)))
            loss = self.step(*sample_batch(rng, scenes, self.B, self.c))
            if log_every and (t % log_every == 0 or t == steps - 1):
                losses.append((t0 + t, float(loss.item())))
        self.lr = lr0
        return losses


# ---- checkpoints ---------------------------------------------------------------------
# A file holds everything a training run needs to continue where it stopped: the network's
# FP32 master weights and Adam moments (flnr_get_state), the Adam step count, the base
# learning rate and the state of the crop sampler's random generator.  Layout: the 8-byte
# magic, a little-endian u32 header length, the header (UTF-8 JSON), the state as
# little-endian float32, and a u32 CRC-32 of everything before it.
CKPT_MAGIC = b"FLNRCKP1"
CKPT_VERSION = 1


def pack_checkpoint(state, meta):
    """Bytes of a checkpoint: state (float32 array) and meta (JSON-serialisable dict)."""
    state = np.ascontiguousarray(state, dtype="<f4")
    head = dict(meta, version=CKPT_VERSION, floats=int(state.size))
    hj = json.dumps(head, sort_keys=True).encode("utf-8")
    body = CKPT_MAGIC + struct.pack("<I", len(hj)) + hj + state.tobytes()
    return body + struct.pack("<I", zlib.crc32(body) & 0xFFFFFFFF)


def unpack_checkpoint(blob):
    """(state float32 array, meta dict) from pack_checkpoint's bytes; raises ValueError on a
    wrong magic, version, length or CRC."""
    if len(blob) < len(CKPT_MAGIC) + 8 or blob[:len(CKPT_MAGIC)] != CKPT_MAGIC:
        raise ValueError("not an FLNR checkpoint")
    body, (crc,) = blob[:-4], struct.unpack("<I", blob[-4:])
    if zlib.crc32(body) & 0xFFFFFFFF != crc:
        raise ValueError("checkpoint CRC mismatch (file damaged)")
    (hl,) = struct.unpack("<I", body[len(CKPT_MAGIC):len(CKPT_MAGIC) + 4])
    p = len(CKPT_MAGIC) + 4
    meta = json.loads(body[p:p + hl].decode("utf-8"))
    if meta.get("version") != CKPT_VERSION:
        raise ValueError(f"checkpoint version {meta.get('version')} (expected {CKPT_VERSION})")
    data = body[p + hl:]
    if len(data) != 4 * meta["floats"]:
        raise ValueError("checkpoint length does not match its header")
    return np.frombuffer(data, dtype="<f4").astype(np.float32), meta


def save_checkpoint(path, trainer, rng=None):
    """Writes trainer's optimiser state, step count and base learning rate, and the state of
    rng (the crop sampler's numpy Generator), to path (replaced atomically)."""
    import os
    meta = {"outputs": trainer.outputs, "params": trainer.net.count, "steps": trainer.steps, "lr": trainer.lr,
            "rng": None if rng is None else rng.bit_generator.state}
    blob = pack_checkpoint(trainer.net.get_state(), meta)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "wb") as f:
        f.write(blob)
    os.replace(tmp, path)


def load_checkpoint(path, trainer):
    """Restores what save_checkpoint wrote into trainer (same network size); returns the
    crop sampler's generator in its saved state (None if none was saved)."""
    with open(path, "rb") as f:
        state, meta = unpack_checkpoint(f.read())
    if meta["outputs"] != trainer.outputs or meta["params"] != trainer.net.count:
        raise ValueError("checkpoint is for a network of another size")
    trainer.net.set_state(state)
    trainer.steps = int(meta["steps"])
    trainer.lr = float(meta["lr"])
    if meta.get("rng") is None:
        return None
    rng = np.random.Generator(getattr(np.random, meta["rng"]["bit_generator"])())
    rng.bit_generator.state = meta["rng"]
    return rng


def psnr(img, ref):
    """PSNR in dB of the albedo-modulated images clamped to [0, 1] (peak 1)."""
    a = np.clip(np.asarray(img, np.float64), 0.0, 1.0)
    b = np.clip(np.asarray(ref, np.float64), 0.0, 1.0)
    return float(10.0 * np.log10(1.0 / max(np.mean((a - b) ** 2), 1e-20)))


def evaluate(net, flr, scenes):
    """PSNR of plain FLR (rendered guides) and of FLNR (network guides) against each
    scene's reference, after albedo modulation.  Returns two lists."""
    import torch
    p_flr, p_flnr = [], []
    for x, ref, alb, _ in scenes:
        xd = torch.from_numpy(x[None]).cuda()
        y = xd[0, 8:11]
        plain = flr.denoise(xd[0, :8], y).cpu().numpy()
        guides = net.forward(xd)
        if guides.shape[1] == 16:  # model and map guide sets
            learned = flr.denoise(guides[0, :8], y, map_guide=guides[0, 8:]).cpu().numpy()
        else:
            learned = flr.denoise(guides[0], y).cpu().numpy()
        p_flr.append(psnr(plain * alb, ref * alb))
        p_flnr.append(psnr(learned * alb, ref * alb))
    return p_flr, p_flnr
