#!/usr/bin/env python3
"""Benchmark of the FLR hot path: ms per 1920x1080 frame on GB300.

Besides the headline, `rows` reports the other parts of the path: the FLR adjoint, the
paper's fast FLR, joint 2x upsampling, batched serving, and FLNR (training on rendered
crops, PSNR against high-spp references on held-out rooms, 1080p inference time).

One step = one full FLR pass over one frame whose inputs are already in HBM: the fused
kernel (windowed moments, per-pixel Cholesky solve, coefficient averaging and apply) and
the FP64 correction of flagged pixels.  Four rendered frames rotate, so every step reads inputs larger than L2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 it runs under torchrun, one independent replica per GPU (frames are
independent; no collective on the data path), and reports the whole job's ms per frame.
`--impl reference` times the FP64 CPU oracle on the host cores instead (a slow
reference program, on bounded row bands of the same workload).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

H, W, Q, R, RC, EPS, TAU = 1080, 1920, 8, 8, 8, 1e-3, 1e-3
N_FRAMES = 4
METRIC = "ms per 1080p frame (FLR)"
UNIT = "ms/frame"
WORKLOAD = ("FLR forward, 1920x1080, Q=8 rendered guides (albedo RGB, normal xyz, depth, AO), "
            "1spp albedo-demodulated indirect RGB, r=8, rc=8, eps=1e-3, pivot ratio 1e-3")
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
N_SM, FP32_LANES = 152, 128
FWD_SOURCES = ["paper_2410_11625_gb300/csrc/flr_fused.cu", "paper_2410_11625_gb300/csrc/flr_internal.cuh",
               "paper_2410_11625_gb300/csrc/flr_device.cuh", "paper_2410_11625_gb300/csrc/flr_tmem.cuh"]
FWD_PROFILE = os.path.join(ROOT, "profiles", "flr_fused_1080p_r8.txt")


def fwd_flops_per_pixel(q: int) -> int:
    """Algorithmic FP32 flops per pixel of the per-pixel model (FMA = 2): products, window
    sums, centring, Cholesky, three triangular solves and the bias."""
    products = q * (q + 1) // 2 + 3 * q                 # x x^T upper triangle and x y^T
    box_sums = 4 * (products + q + 3)                   # 2 passes x (add + subtract)
    centring = (q + 3) + 2 * (q * (q + 1) // 2 + 3 * q) + q
    chol = 2 * (q * (q - 1) // 2 + sum((q - 1 - j) * j for j in range(q))) + q * (q - 1) // 2 + 2 * q
    solves = 6 * q * q                                  # 3 RHS x (forward + backward)
    bias = 3 * 2 * q                                    # b = mu_y - a^T mu
    return products + box_sums + centring + chol + solves + bias


def path_flops_per_pixel(q: int, rc: int) -> int:
    """The whole FLR path per output pixel: the model, then (rc > 0) the box average of its
    3 (q + 1) coefficients (2 passes x add + subtract), and the apply (3 x (q + 1) FMA)."""
    average = 4 * 3 * (q + 1) if rc > 0 else 0
    return fwd_flops_per_pixel(q) + average + 2 * 3 * (q + 1)


def frame_bytes(q: int) -> int:
    """Algorithmic HBM bytes of one frame: read guides + radiance, write the result."""
    return 4 * H * W * (q + 3 + 3)


def load_peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def sha_of(paths):
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def profiled_traffic():
    """DRAM bytes per launch of the fused forward kernel from the committed ncu summary, if
    the kernel source has not changed since it was captured; else None."""
    try:
        text = open(FWD_PROFILE).read()
    except OSError:
        return None
    vals = {}
    for line in text.splitlines():
        if ":" in line:
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("source_sha256") != sha_of(FWD_SOURCES):
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50", "-i", str(self.dev)],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(n_gpus, backend="nccl"):
    """Rank, world size and local rank from the torchrun environment; for N > 1 one process
    group (NCCL on the GPUs; the CPU tests use gloo).  It carries only the barrier and the
    max-reduce of the timed region: the replicas share no data."""
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world != n_gpus:
        raise SystemExit(f"--gpus {n_gpus} but WORLD_SIZE={world}: launch N>1 with torchrun")
    if world > 1:
        import torch.distributed as dist
        if backend == "nccl":
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group(backend)
    return world, rank, local


def frame_seeds(rank):
    """Scene seeds of a rank's rotating frames: every replica renders its own frames."""
    return [1 + N_FRAMES * rank + i for i in range(N_FRAMES)]


def reduce_max(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def cpu_oracle_band(frame, rows):
    """Time the FP64 oracle on the band of `rows` rows around the frame's middle."""
    import oracle
    g, y = frame
    y0 = (H - rows) // 2
    t = time.perf_counter()
    oracle.flr_forward(g[:, y0:y0 + rows], y[:, y0:y0 + rows], R, EPS, coef_radius=RC)
    return time.perf_counter() - t


def cpu_baseline(frame):
    """The FP64 oracle on whole 1080p frames: all host cores (median of 5 runs after one
    warm-up) and one core (median of 3); about 25 s of CPU work on 16 Arm cores."""
    import oracle
    n_all = os.cpu_count() or 1
    oracle.set_threads(n_all)
    cpu_oracle_band(frame, H)
    t_all = statistics.median(cpu_oracle_band(frame, H) for _ in range(5))
    oracle.set_threads(1)
    t_one = statistics.median(cpu_oracle_band(frame, H) for _ in range(3))
    oracle.set_threads(n_all)
    return {"value": round(t_all * 1e3, 2), "unit": UNIT, "cores": n_all, "kind": "oracle",
            "sample": f"FP64 oracle on whole {W}x{H} frames (r=8, rc=8): median of 5 runs on {n_all} threads",
            "single_thread": {"value": round(t_one * 1e3, 2), "unit": UNIT, "cores": 1,
                              "sample": "the same frame, median of 3 runs on one thread"}}


def sampled_parity(got, frame, blocks=12, B=32, seed=0):
    """max relative error, |got - ref| / max(|ref|, 1% of RMS(ref)), of the timed frame's
    result against the oracle on sampled B x B blocks (corners, edges, random interior), each
    computed by the oracle on the block plus its radius-(r + rc) halo, which holds every input
    its outputs depend on."""
    import numpy as np

    import oracle
    g, y = frame
    rng = np.random.default_rng(seed)
    halo = R + RC
    where = [(0, 0), (0, W - B), (H - B, 0), (H - B, W - B)]
    where += [(int(rng.integers(0, H - B)), int(rng.integers(0, W - B))) for _ in range(blocks - 4)]
    worst = 0.0
    for by, bx in where:
        y0, y1 = max(0, by - halo), min(H, by + B + halo)
        x0, x1 = max(0, bx - halo), min(W, bx + B + halo)
        ref = oracle.flr_forward(g[:, y0:y1, x0:x1], y[:, y0:y1, x0:x1], R, EPS, coef_radius=RC)
        ref = ref[:, by - y0:by - y0 + B, bx - x0:bx - x0 + B]
        part = np.asarray(got[:, by:by + B, bx:bx + B], np.float64)
        rms = np.sqrt(np.mean(ref ** 2))
        worst = max(worst, float(np.max(np.abs(part - ref) / np.maximum(np.abs(ref), 0.01 * rms))))
    return worst, len(where)


def serving_batch(flr, torch, np, dev, stream, n_iter=100):
    """8 frames of mixed sizes (720p / 1080p / 1440p output, 2x joint upsampling from half
    resolution) in one persistent launch, captured in a CUDA graph and replayed."""
    import synth
    sizes = [(720, 1280), (1080, 1920), (1440, 2560)]
    scenes = {hw: synth.render(100 + i, *hw) for i, hw in enumerate(sizes)}
    frames = []
    for k in range(8):
        Ho, Wo = sizes[k % 3]
        g, y = scenes[(Ho, Wo)]
        frames.append((torch.from_numpy(np.ascontiguousarray(g[:, ::2, ::2])).to(dev),
                       torch.from_numpy(np.ascontiguousarray(y[:, ::2, ::2])).to(dev),
                       torch.from_numpy(g).to(dev), torch.empty((3, Ho, Wo), device=dev)))
    f = flr.FastFLR(q=Q, factor=4, scale=2, sigma=1.25, taps=3, eps=EPS, pivot_ratio=TAU)
    f.reserve_batch(frames)
    s = torch.cuda.Stream(dev)
    with torch.cuda.stream(s):
        f.denoise_batch(frames, stream=s)
        s.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=s):
            f.denoise_batch(frames, stream=s)
        for _ in range(5):
            graph.replay()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_iter)]
        for e0, e1 in evs:
            e0.record(s)
            graph.replay()
            e1.record(s)
        s.synchronize()
    lat = sorted(e0.elapsed_time(e1) for e0, e1 in evs)
    status = f.batch_status()
    f.close()
    px = sum(h * w for (h, w) in [sizes[k % 3] for k in range(8)])
    mean = sum(lat) / len(lat)
    return {"frames": 8, "outputs": "3x 1280x720, 3x 1920x1080, 2x 2560x1440", "inputs": "half resolution",
            "launches_per_batch": 1, "graph": True, "batch_latency_ms_p50": round(lat[len(lat) // 2], 4),
            "batch_latency_ms_p99": round(lat[min(len(lat) - 1, int(0.99 * len(lat)))], 4),
            "frames_per_s": round(8 / (mean * 1e-3), 1), "output_mpix_per_s": round(px / (mean * 1e-3) / 1e6, 1),
            "status": "ok" if status == 0 else "timeout",
            "what": "flr_fast_denoise_batch: one persistent cooperative kernel, 4 stages x 8 frames"}


def serving_batch_flnr(torch, np, dev, weights, n_iter=100):
    """The same 8 frames with the FLNR guide network in the step (config of the batched serving
    pattern: FP32 FLR plus the BF16 guide CNN): per frame size, the network's forward over the
    half-resolution inputs gives the model guides, then one persistent fast-FLR launch; the
    step is one captured CUDA graph."""
    import synth
    from paper_2410_11625_gb300 import serving
    sizes = [(720, 1280), (1080, 1920), (1440, 2560)]
    groups = []
    for i, (Ho, Wo) in enumerate(sizes):
        g, y = synth.render(100 + i, Ho, Wo)
        n = 3 if i < 2 else 2
        lo = np.concatenate([g[:, ::2, ::2], y[:, ::2, ::2]])
        x = torch.from_numpy(np.ascontiguousarray(np.repeat(lo[None], n, axis=0))).to(dev)
        z = torch.from_numpy(np.ascontiguousarray(np.repeat(g[None], n, axis=0))).to(dev)
        groups.append((x, z, torch.empty((n, 3, Ho, Wo), device=dev)))
    b = serving.GuidedBatch(groups, weights, factor=4)
    for _ in range(5):
        b.run()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_iter)]
    for e0, e1 in evs:
        e0.record(b.stream)
        b.run()
        e1.record(b.stream)
    b.stream.synchronize()
    lat = sorted(e0.elapsed_time(e1) for e0, e1 in evs)
    status = b.status()
    b.close()
    px = 3 * 1280 * 720 + 3 * 1920 * 1080 + 2 * 2560 * 1440
    mean = sum(lat) / len(lat)
    return {"frames": 8, "outputs": "3x 1280x720, 3x 1920x1080, 2x 2560x1440", "inputs": "half resolution",
            "launches_per_batch": "3 network forward passes (one per frame size, 8 kernels each) + 1 persistent FLR",
            "graph": True, "batch_latency_ms_p50": round(lat[len(lat) // 2], 4),
            "batch_latency_ms_p99": round(lat[min(len(lat) - 1, int(0.99 * len(lat)))], 4),
            "frames_per_s": round(8 / (mean * 1e-3), 1), "output_mpix_per_s": round(px / (mean * 1e-3) / 1e6, 1),
            "status": "ok" if status == 0 else "timeout",
            "what": "serving.GuidedBatch: FLNR (BF16 tcgen05) model guides at half resolution + "
                    "flr_fast_denoise_batch, one CUDA graph"}


ROW_NAMES = ("backward", "fast", "joint", "serving", "flnr")

# FLNR network (Sec. 3.3): multiply-accumulates per full-resolution pixel, layer by layer
# (Cin x Cout x k^2 per output pixel, divided by 4 at half and 16 at quarter resolution; the
# stride-2 encoder convolutions e1b and e2b produce half- and quarter-resolution outputs)
FLNR_MACS_PER_PIXEL = (11 * 16 * 9 + 16 * 16 + 16 * 32 * 9 + (32 * 32 * 9) / 4 + (32 * 64 * 9) / 4
                       + (64 * 64 * 9) / 16 + (96 * 32 * 9 + 32 * 32 * 9) / 4 + 48 * 16 * 9 + 16 * 16 * 9
                       + 16 * 16 * 9 + 16 * 8)


def flnr_rows(frames, dev_frames, torch, np, dev, timed, train_steps, full_hd_rooms=0):
    """FLNR rows: training on rendered crops, PSNR against 1024 spp references on held-out
    rooms, 1080p inference time (network + FLR on its guides), training-step time."""
    from paper_2410_11625_gb300 import flnr, flnr_train, flr
    rows = {}
    if train_steps <= 0:  # timing only, with the initial weights
        return flnr_inference_row(flnr.init_weights(0), dev_frames, torch, dev, timed, rows)
    t0 = time.perf_counter()
    n_train = 192  # the two-set head needs the data: 64 rooms -0.37 dB against FLR, 192 rooms +0.85 dB
    scenes = flnr_train.render_scenes(range(1, n_train + 1), 192, 192, ref_spp=1024, noise=8, gpu_ref=True)
    n_eval = 16
    held_out = flnr_train.render_scenes(range(flnr_train.EVAL_SEED0, flnr_train.EVAL_SEED0 + n_eval), 256, 256,
                                        ref_spp=1024, gpu_ref=True)
    t_render = time.perf_counter() - t0
    tr = flnr_train.Trainer(flnr.init_weights(0), batch=16, crop=128, lr=2e-3)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tr.train(scenes, train_steps, seed=0, lr_final=1e-4)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    p_flr, p_net = flnr_train.evaluate(tr.net, tr.flr, held_out)
    rows["flnr_psnr"] = {
        "psnr_flr_db": round(float(np.mean(p_flr)), 3), "psnr_flnr_db": round(float(np.mean(p_net)), 3),
        "gain_db": round(float(np.mean(p_net) - np.mean(p_flr)), 3),
        "per_scene_gain_db": [round(a - b, 2) for a, b in zip(p_net, p_flr)],
        "psnr_flr_per_scene_db": [round(float(a), 2) for a in p_flr],
        "rooms_improved": int(sum(a > b for a, b in zip(p_net, p_flr))),
        "what": (f"{n_eval} held-out rooms (seeds {flnr_train.EVAL_SEED0}..{flnr_train.EVAL_SEED0 + n_eval - 1}, "
                 f"256x256) vs 1024 spp references, albedo-modulated, "
                 f"clamped to [0,1]; network trained here for {train_steps} steps (batch 16 x 128^2 crops of {n_train} "
                 f"rooms, 8 noise realisations each, L1, Adam lr 2e-3 cosine to 1e-4) in {t_train:.1f} s; "
                 f"rendering {t_render:.1f} s (guides and 1 spp on the host, references on the GPU)"),
    }
    # the two guide sets of Sec. 3.3 (16 outputs: model guides, map guides), same recipe
    tr2 = flnr_train.Trainer(flnr.init_weights(0, 16), batch=16, crop=128, lr=2e-3)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tr2.train(scenes, train_steps, seed=0, lr_final=1e-4)
    torch.cuda.synchronize()
    t_train2 = time.perf_counter() - t0
    _, p_2q = flnr_train.evaluate(tr2.net, tr2.flr, held_out)
    rows["flnr_2q_psnr"] = {
        "psnr_flnr_2q_db": round(float(np.mean(p_2q)), 3), "gain_db": round(float(np.mean(p_2q) - np.mean(p_flr)), 3),
        "per_scene_gain_db": [round(a - b, 2) for a, b in zip(p_2q, p_flr)],
        "rooms_improved": int(sum(a > b for a, b in zip(p_2q, p_flr))),
        "what": f"as flnr_psnr with a 16-output head: channels 0-7 fit the models, 8-15 are FLR's map guide; "
                f"trained {train_steps} steps in {t_train2:.1f} s"}
    xs, rs = flnr_train.sample_batch(np.random.default_rng(1), scenes, 16, 128)
    t_step2 = timed(lambda i: tr2.step(xs, rs), 50)
    tr2.net.close()
    # Sec. 3.3's SMAPE loss instead of config 4's L1, same recipe otherwise
    tr3 = flnr_train.Trainer(flnr.init_weights(0), batch=16, crop=128, lr=2e-3, loss="smape")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tr3.train(scenes, train_steps, seed=0, lr_final=1e-4)
    torch.cuda.synchronize()
    t_train3 = time.perf_counter() - t0
    _, p_sm = flnr_train.evaluate(tr3.net, tr3.flr, held_out)
    tr3.net.close()
    rows["flnr_smape_psnr"] = {
        "psnr_flnr_smape_db": round(float(np.mean(p_sm)), 3), "gain_db": round(float(np.mean(p_sm) - np.mean(p_flr)), 3),
        "per_scene_gain_db": [round(a - b, 2) for a, b in zip(p_sm, p_flr)],
        "rooms_improved": int(sum(a > b for a, b in zip(p_sm, p_flr))),
        "what": f"as flnr_psnr trained on SMAPE |I - R| / (|I| + |R| + 0.01) (Sec. 3.3) instead of L1; "
                f"trained {train_steps} steps in {t_train3:.1f} s"}
    t_step = timed(lambda i: tr.step(xs, rs), 50)
    rows["flnr_train_step"] = {"ms_per_step": round(t_step, 4), "ms_per_step_2q": round(t_step2, 4),
                               "what": "batch 16 x 128x128: FLNR fwd, 16 x FLR, L1, 16 x FLR adjoint, FLNR bwd, Adam; "
                                       "includes the pinned H2D copy of the batch"}
    weights = tr.net.get_weights()
    tr.net.close()
    if full_hd_rooms > 0:
        # the same network (fully convolutional) on 1920x1080 held-out rooms
        t0 = time.perf_counter()
        seeds = range(flnr_train.EVAL_SEED0 + 100, flnr_train.EVAL_SEED0 + 100 + full_hd_rooms)
        big = flnr_train.render_scenes(seeds, H, W, ref_spp=1024, gpu_ref=True)
        t_big = time.perf_counter() - t0
        net_big = flnr.FLNR(H * W, weights)
        f_big = flr.FLR(q=8, radius=8, eps=1e-3)
        pf, pn = flnr_train.evaluate(net_big, f_big, big)
        net_big.close()
        f_big.close()
        rows["flnr_psnr_1080p"] = {
            "psnr_flr_db": round(float(np.mean(pf)), 3), "psnr_flnr_db": round(float(np.mean(pn)), 3),
            "gain_db": round(float(np.mean(pn) - np.mean(pf)), 3),
            "per_scene_gain_db": [round(a - b, 2) for a, b in zip(pn, pf)],
            "what": (f"{full_hd_rooms} held-out rooms (seeds {seeds[0]}..{seeds[-1]}) at {W}x{H} vs 1024 spp "
                     f"references (GPU path tracer; guides and 1 spp on the host: {t_big:.0f} s), FLR r=8 with "
                     f"rendered vs network guides; network as flnr_psnr")}
    return flnr_inference_row(weights, dev_frames, torch, dev, timed, rows)


def flnr_inference_row(weights, dev_frames, torch, dev, timed, rows):
    """1080p inference: the network, FLR on its guides, and both in sequence."""
    from paper_2410_11625_gb300 import flnr, flr
    net = flnr.FLNR(H * W, weights)
    f = flr.FLR(q=Q, radius=R, coef_radius=RC, eps=EPS, pivot_ratio=TAU)
    f.reserve(H, W)
    xin = [torch.cat([g, y]).unsqueeze(0).contiguous() for g, y in dev_frames]
    guides = torch.empty((1, 8, H, W), dtype=torch.float32, device=dev)
    out = torch.empty((3, H, W), dtype=torch.float32, device=dev)
    t_net = timed(lambda i: net.forward(xin[i % len(xin)], out=guides), 50)
    net.forward(xin[0], out=guides)
    t_flr = timed(lambda i: f.denoise(guides[0], dev_frames[0][1], out=out), 50)

    def both(i):
        net.forward(xin[i % len(xin)], out=guides)
        f.denoise(guides[0], dev_frames[i % len(xin)][1], out=out)
    t_both = timed(both, 50)
    tflops = 2 * FLNR_MACS_PER_PIXEL * H * W / (t_net * 1e-3) / 1e12
    peak = float(load_peaks()[0]["bf16_tflops"])
    rows["flnr_1080p"] = {"ms_per_frame": round(t_both, 4), "net_ms": round(t_net, 4), "flr_on_net_guides_ms": round(t_flr, 4),
                          "net_tflops": round(tflops, 2), "net_tensor_frac": round(tflops / peak, 4),
                          "net_macs_per_pixel": FLNR_MACS_PER_PIXEL,
                          "what": "FLNR guide network (BF16 tcgen05 implicit-GEMM convs with TMA-staged tiles, FP32 "
                                  "accumulation in TMEM) + FP32 FLR r=8 on its guides, 1920x1080; tensor fraction of "
                                  "measured dense bf16 peak"}
    f.close()
    net.close()
    # the network's backward pass alone at the training batch shape (16 x 128^2 crops): its
    # activation gradients, input- and weight-gradient convolutions and their reductions
    tb = flnr.FLNR(16 * 128 * 128, weights)
    gen = torch.Generator(device=dev)
    gen.manual_seed(0)
    xb = torch.rand((16, 11, 128, 128), device=dev, generator=gen)
    gb = torch.randn((16, tb.outputs, 128, 128), device=dev, generator=gen) * 1e-3
    tb.forward(xb)

    def bwd(i):
        tb.zero_grads(xb)
        tb.backward(gb)
    rows["flnr_backward_16x128"] = {"ms": round(timed(bwd, 20), 4),
                                    "what": "FLNR backward pass (tcgen05 input- and weight-gradient convolutions, "
                                            "fixed-order reductions) on a 16 x 128x128 batch, without FLR"}
    tb.close()
    return rows


def run_ours(args):
    import numpy as np
    import torch

    import synth
    from paper_2410_11625_gb300 import build, flr

    world, rank, local = dist_setup(args.gpus)
    build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    frames = [synth.render(seed, H, W) for seed in frame_seeds(rank)]
    dev_frames = [(torch.from_numpy(g).to(dev), torch.from_numpy(y).to(dev)) for g, y in frames]
    host_frames = [(torch.from_numpy(g).pin_memory(), torch.from_numpy(y).pin_memory()) for g, y in frames]
    out = torch.empty((3, H, W), dtype=torch.float32, device=dev)
    host_out = torch.empty((3, H, W), dtype=torch.float32).pin_memory()

    f = flr.FLR(q=Q, radius=R, coef_radius=RC, eps=EPS, pivot_ratio=TAU, timing=True)
    f.reserve(H, W)
    stream = torch.cuda.current_stream(dev)
    for i in range(args.warmup):
        f.denoise(*dev_frames[i % N_FRAMES], out=out)
    torch.cuda.synchronize()
    f.kernel_times(reset=True)

    clocks = Clocks(local)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for i in range(args.steps):
        f.denoise(*dev_frames[i % N_FRAMES], out=out)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    t_ms = reduce_max(ev0.elapsed_time(ev1), world)
    kt = f.kernel_times(reset=True)
    flagged = f.stats()["flagged"]

    # end to end through the host-buffer entry points: every frame's inputs copied in from
    # page-locked host memory, FLR, its result copied back.  (1) the frame stream
    # (flr_denoise_host_async per frame, one flr_host_wait): copies overlap across frames;
    # (2) one synchronous flr_denoise_host call per frame: copies overlap within a frame only.
    n_e2e = max(3, min(args.steps, 100))
    host_outs = [torch.empty((3, H, W), dtype=torch.float32).pin_memory() for _ in range(N_FRAMES)]
    for i in range(2):
        g, y = host_frames[i % N_FRAMES]
        f.denoise_host_async(g.numpy(), y.numpy(), host_outs[i % N_FRAMES].numpy(), stream=stream)
    f.host_wait()
    barrier(world)
    t0 = time.perf_counter()
    for i in range(n_e2e):
        g, y = host_frames[i % N_FRAMES]
        f.denoise_host_async(g.numpy(), y.numpy(), host_outs[i % N_FRAMES].numpy(), stream=stream)
    f.host_wait()
    e2e_s = reduce_max(time.perf_counter() - t0, world)
    last = (n_e2e - 1) % N_FRAMES
    f.denoise(*dev_frames[last], out=out)
    e2e_exact = bool(torch.equal(out.cpu(), host_outs[last]))
    for i in range(2):
        g, y = host_frames[i % N_FRAMES]
        f.denoise_host(g.numpy(), y.numpy(), out=host_out.numpy(), stream=stream)
    barrier(world)
    t0 = time.perf_counter()
    for i in range(n_e2e):
        g, y = host_frames[i % N_FRAMES]
        f.denoise_host(g.numpy(), y.numpy(), out=host_out.numpy(), stream=stream)
    e2e_sync_s = reduce_max(time.perf_counter() - t0, world)
    f.close()

    # the other rows of the path, on the same frames (CUDA events on the launching stream)
    def timed(fn, n, warm=5):
        for i in range(warm):
            fn(i)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(n):
            fn(i)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n

    rows = {}
    want = set(ROW_NAMES) if args.rows == "all" else set(args.rows.split(",")) - {"none"}
    if "backward" in want:
        fb = flr.FLR(q=Q, radius=R, coef_radius=RC, eps=EPS, pivot_ratio=TAU)
        gout = torch.randn((3, H, W), dtype=torch.float32, device=dev)
        rows["backward_1080p"] = {"ms_per_frame": round(timed(lambda i: fb.backward(*dev_frames[i % N_FRAMES], gout), 20), 4),
                                  "what": "flr_backward: guide, radiance gradients, r=rc=8"}
        fb.close()
    if "fast" in want:
        ff = flr.FastFLR(q=Q, factor=8, scale=1, sigma=1.25, taps=3, eps=EPS, pivot_ratio=TAU)
        t_fast = timed(lambda i: ff.denoise(*dev_frames[i % N_FRAMES], out=out), 200)
        ff.close()
        rows["fast_flr_1080p"] = {"ms_per_frame": round(t_fast, 5),
                                  "hbm_frac": round(frame_bytes(Q) / (t_fast * 1e-3) / 1e9 / float(load_peaks()[0]["hbm_gbs"]), 4),
                                  "what": "Sec. 3.2 fast FLR: 8x8 block moments, Gaussian sigma 1.25 blocks, 3 taps"}
    if "joint" in want:
        lo = [(torch.from_numpy(np.ascontiguousarray(g[:, ::2, ::2])).to(dev),
               torch.from_numpy(np.ascontiguousarray(y[:, ::2, ::2])).to(dev)) for g, y in frames[:2]]
        fj = flr.FastFLR(q=Q, factor=4, scale=2, sigma=1.25, taps=3, eps=EPS, pivot_ratio=TAU)
        t_joint = timed(lambda i: fj.denoise(*lo[i % 2], map_guide=dev_frames[i % 2][0], out=out), 200)
        fj.close()
        rows["joint_upsample_2x_1080p"] = {"ms_per_frame": round(t_joint, 5),
                                           "what": "Sec. 3.2.1: 960x540 radiance and model guides, 1920x1080 map guide and output"}
    if "serving" in want:
        rows["batch_serving"] = serving_batch(flr, torch, np, dev, stream)
        from paper_2410_11625_gb300 import flnr as _flnr
        rows["batch_serving_flnr"] = serving_batch_flnr(torch, np, dev, _flnr.init_weights(0))
    if rank == 0 and "flnr" in want:
        rows.update(flnr_rows(frames, dev_frames, torch, np, dev, timed, args.flnr_steps, full_hd_rooms=8))

    # parity of the timed configuration: the last timed frame against the oracle on blocks
    f2 = flr.FLR(q=Q, radius=R, coef_radius=RC, eps=EPS, pivot_ratio=TAU)
    res = f2.denoise(*dev_frames[0], out=out).cpu().numpy()
    f2.close()
    # measured FP32 FMA rate, the denominator of the ALU roofline
    fma_tflops, fma_ms = flr.fp32_fma_peak(20000)

    if rank != 0:
        return
    peaks, peak_src = load_peaks()
    max_rel, n_blocks = sampled_parity(res, frames[0])
    value = t_ms / (args.steps * world)
    fwd_avg_ms = kt["fwd_ms"] / max(1, kt["fwd_n"])
    flops = path_flops_per_pixel(Q, RC) * H * W
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    nominal = N_SM * FP32_LANES * 2 * sm_max * 1e6 / 1e12
    achieved = flops / (fwd_avg_ms * 1e-3) / 1e12
    hbm_peak = float(peaks["hbm_gbs"])
    frame_gbs = frame_bytes(Q) / (value * 1e-3) / 1e9
    traffic = profiled_traffic()
    cpu = cpu_baseline(frames[0])

    line = {
        "metric": METRIC, "value": round(value, 5), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t_ms / args.steps, 5),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic: seeded procedural Lambertian rooms rendered by the project's path tracer",
        "config": {"workload": WORKLOAD, "H": H, "W": W, "q": Q, "radius": R, "coef_radius": RC,
                   "eps": EPS, "pivot_ratio": TAU, "frames_rotated": N_FRAMES,
                   "l2": f"inputs larger than L2: {N_FRAMES} frames x {4 * H * W * (Q + 3) / 1e6:.1f} MB rotate",
                   "parallelism": f"{world} independent replica(s), no collective on the data path"},
        "e2e": {"value": round(e2e_s * 1e3 / (n_e2e * world), 5), "unit": UNIT,
                "h2d_bytes_per_step": 4 * H * W * (Q + 3), "d2h_bytes_per_step": 4 * H * W * 3,
                "steps": n_e2e, "result_equals_device_path": e2e_exact,
                "api": ("flr_denoise_host_async per frame + one flr_host_wait (page-locked host buffers; "
                        "frame i+1 copied in while frame i runs, frame i copied out while frame i+1 runs)"),
                "sync_per_frame": {"value": round(e2e_sync_s * 1e3 / (n_e2e * world), 5), "unit": UNIT,
                                   "api": "flr_denoise_host, one synchronous call per frame (row bands)"}},
        "roofline": {"bound": "alu", "kernel": "flr_fused_kernel<8,8,8>", "achieved": round(achieved, 3),
                     "peak": round(fma_tflops, 2), "unit": "TFLOP/s", "frac": round(achieved / fma_tflops, 4),
                     "traffic": traffic,
                     "peak_source": (f"measured: flr_fp32_fma_peak, independent FP32 FMA chains on every SM "
                                     f"({fma_ms:.2f} ms run); nominal 152 SMs x 128 lanes x 2 x {sm_max:.0f} MHz "
                                     f"= {nominal:.1f}"),
                     "flops_per_pixel": path_flops_per_pixel(Q, RC), "avg_launch_ms": round(fwd_avg_ms, 5)},
        "hbm": {"algorithmic_bytes_per_frame": frame_bytes(Q), "achieved_gbs": round(frame_gbs, 1),
                "peak_gbs": hbm_peak, "frac": round(frame_gbs / hbm_peak, 4),
                "peak_source": f"{peak_src} copy bandwidth"},
        "parity": {"max_rel_err": float(f"{max_rel:.3e}"), "bar": 1e-4, "blocks": n_blocks,
                   "what": "the timed configuration's result on frame seed 1 vs the FP64 oracle, 32x32 blocks "
                           "(corners + random) with their radius-16 halo; error relative to the value, floored at 1% of the RMS"},
        "cpu_baseline": cpu,
        "gpu_launches": int(kt["fwd_n"] + kt["fp64_n"] + kt["apply_n"]),
        "flagged_pixels_last_frame": flagged,
    }
    line["kernels"] = {
        "flr_fused": {"launches": kt["fwd_n"], "avg_ms": round(kt["fwd_ms"] / max(1, kt["fwd_n"]), 5)},
        "flr_fused_fix": {"launches": kt["fp64_n"], "avg_ms": round(kt["fp64_ms"] / max(1, kt["fp64_n"]), 5)},
    }
    line["rows"] = rows
    if clk is not None:
        line["clocks"] = clk
    print(json.dumps(line), flush=True)


def run_reference(args):
    """The FP64 CPU oracle as the reference program, on bounded row bands."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    import synth
    frame = synth.render(1, H, W)
    oracle.build()
    # size the band so the whole run stays within about two minutes
    t_probe = cpu_oracle_band(frame, 8) / 8
    budget = 100.0 / max(1, args.steps + args.warmup)
    rows = int(max(1, min(H // 4, budget / max(t_probe, 1e-6))))
    for _ in range(args.warmup):
        cpu_oracle_band(frame, rows)
    times = [cpu_oracle_band(frame, rows) for _ in range(args.steps)]
    ms_frame = sum(times) / len(times) * 1e3 * (H / rows)
    sample = f"FP64 oracle on a {W}x{rows} row band per step (r=8, rc=8), scaled x{H / rows:g} to a frame"
    line = {
        "metric": METRIC, "value": round(ms_frame, 3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * sum(times) / len(times), 3),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic: seeded procedural Lambertian rooms rendered by the project's path tracer",
        "config": {"workload": WORKLOAD, "H": H, "W": W, "q": Q, "radius": R, "coef_radius": RC,
                   "eps": EPS},
        "impl": "reference",
        "cpu_baseline": {"value": round(ms_frame, 3), "unit": UNIT, "cores": oracle.threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": round(ms_frame, 3), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--rows", default="all",
                    help="comma list of extra rows to run: " + ",".join(ROW_NAMES) + " (or all, none)")
    ap.add_argument("--flnr-steps", type=int, default=6000,
                    help="FLNR training steps before its PSNR and 1080p rows (0: 1080p timing only)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
