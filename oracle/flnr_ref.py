"""FP64 CPU oracle of the FLNR guide network (Sec. 3.3), in plain PyTorch CPU float64 ops.

TEST INFRASTRUCTURE: only tests, the smoke check and the benchmark's CPU leg use it.

The network maps the 11 input channels (Q = 8 guides and the noisy RGB radiance,
concatenated channel-wise, Sec. 3.3) to 8 enhanced guide channels through a 3-level U-Net
(Sec. 3.3's blocks; widths 16 / 32 / 64, ReLU as the activation):
  input              guides X unchanged, radiance Y as log(1 + max(Y, 0))
  input projection   conv3x3 11->16, ReLU;  conv1x1 16->16, ReLU                    -> f0 (H)
  encoder level 1    conv3x3 16->32, ReLU;  conv3x3 32->32 stride 2, ReLU           -> f1 (H/2)
  encoder level 2    conv3x3 32->64, ReLU;  conv3x3 64->64 stride 2, ReLU           -> f2 (H/4)
  decoder level 1    nearest 2x up(f2) ++ f1;  conv3x3 96->32, ReLU;  conv3x3 32->32, ReLU -> d1
  decoder level 0    nearest 2x up(d1) ++ f0;  conv3x3 48->16, ReLU;  conv3x3 16->16, ReLU -> d0
  output             conv3x3 16->16, ReLU;  conv1x1 16->Q';  sigmoid               -> X'
Q' = 8 (one set of enhanced guides, used both to fit and to apply the regression), or the
paper's two sets (Sec. 3.3): Q' = 2Q = 16 outputs, channels 0-7 the model guides X'_model
and channels 8-15 the map guides X'_map.
Sec. 3.3: each encoder block is two 3x3 convolutions, the second striding by 2 to
downsample (no separate pooling).  Every 3x3 convolution has zero padding 1; a stride-2 one
gives output (i, j) from inputs (2i + u - 1, 2j + v - 1).  H and W must be multiples of 4.
Weights are [Cout][Cin][kh][kw] with a bias per output channel.

`bf16_storage=True` takes the network's rounding decisions in the precision a BF16
implementation stores (every product and sum still in float64): the input, the weights and
each ReLU output are rounded to bfloat16 (round to nearest even) on the forward pass; on
the reverse pass the gradient with respect to each pre-activation and each concatenation is
rounded to bfloat16.  The ReLU masks are then
the same on both sides, which the comparison of gradients needs: a mask decided
differently at one pixel changes that pixel's whole contribution to a weight gradient.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.nn.functional as F

# (name, kind, cin, cout, kernel) in execution order; kind: conv with ReLU ("cr"),
# conv without activation ("c")
LAYERS = [
    ("in0", "cr", 11, 16, 3), ("in1", "cr", 16, 16, 1),
    ("e1a", "cr", 16, 32, 3), ("e1b", "cr", 32, 32, 3),
    ("e2a", "cr", 32, 64, 3), ("e2b", "cr", 64, 64, 3),
    ("d1a", "cr", 96, 32, 3), ("d1b", "cr", 32, 32, 3),
    ("d0a", "cr", 48, 16, 3), ("d0b", "cr", 16, 16, 3),
    ("o0", "cr", 16, 16, 3), ("o1", "c", 16, 8, 1),
]


def init_weights(seed=0, outputs=8):
    """He-uniform weights and zero biases, float32 (the dtype the GPU master copy keeps);
    the output projection o1 at a tenth of its He bound, with `outputs` (8, or 16 for the
    model and map sets of Sec. 3.3) output channels; with 16, the map rows of o1 start as a
    copy of the model rows, so the network starts as the 8-output one."""
    rng = np.random.default_rng(seed)
    params = {}
    for name, _, cin, cout, k in LAYERS:
        if name == "o1":
            cout = outputs
        bound = np.sqrt(6.0 / (cin * k * k)) * (0.1 if name == "o1" else 1.0)
        params[name + ".w"] = rng.uniform(-bound, bound, size=(cout, cin, k, k)).astype(np.float32)
        params[name + ".b"] = np.zeros(cout, np.float32)
    if outputs == 16:  # the map set starts as a copy of the model set
        params["o1.w"][8:] = params["o1.w"][:8]
    return params


def round_bf16(t):
    """Round float64 values to bfloat16 (nearest even) through float32, returned as float64."""
    return t.to(torch.float32).to(torch.bfloat16).to(torch.float64)


class _RoundValue(torch.autograd.Function):
    """Forward: round to bfloat16.  Backward: the gradient passes unchanged."""

    @staticmethod
    def forward(ctx, t):
        return round_bf16(t)

    @staticmethod
    def backward(ctx, g):
        return g


class _RoundGrad(torch.autograd.Function):
    """Forward: identity.  Backward: the incoming gradient is rounded to bfloat16."""

    @staticmethod
    def forward(ctx, t):
        return t.clone()

    @staticmethod
    def backward(ctx, g):
        return round_bf16(g)


def forward(x, params, bf16_storage=False):
    """x: [N, 11, H, W] float64 tensor; params: dict of float64 tensors. Returns [N, 8, H, W]."""
    R = _RoundValue.apply if bf16_storage else (lambda t: t)
    G = _RoundGrad.apply if bf16_storage else (lambda t: t)

    def conv(t, name, relu, stride=1):
        w, b = R(params[name + ".w"]), params[name + ".b"]
        z = G(F.conv2d(t, w, b, stride=stride, padding=w.shape[-1] // 2))
        return R(F.relu(z)) if relu else z

    def upcat(lo, skip):
        return G(torch.cat([F.interpolate(lo, scale_factor=2, mode="nearest"), skip], dim=1))

    x = torch.cat([x[:, :8], torch.log1p(torch.clamp(x[:, 8:], min=0.0))], dim=1)
    f0 = conv(conv(R(x), "in0", True), "in1", True)
    f1 = conv(conv(f0, "e1a", True), "e1b", True, stride=2)
    f2 = conv(conv(f1, "e2a", True), "e2b", True, stride=2)
    d1 = conv(conv(upcat(f2, f1), "d1a", True), "d1b", True)
    d0 = conv(conv(upcat(d1, f0), "d0a", True), "d0b", True)
    return torch.sigmoid(conv(conv(d0, "o0", True), "o1", False))


def forward_backward(x, params, grad_out, bf16_storage=False):
    """FP64 forward and reverse-mode gradients (torch autograd on CPU).

    x [N,11,H,W], params (numpy float32/float64 dict), grad_out [N,8,H,W] (dL/dX').
    Returns (out, grads) with grads[name] for every parameter and grads["input"].
    """
    xt = torch.tensor(np.asarray(x, np.float64), requires_grad=True)
    pt = {k: torch.tensor(np.asarray(v, np.float64), requires_grad=True) for k, v in params.items()}
    out = forward(xt, pt, bf16_storage)
    out.backward(torch.tensor(np.asarray(grad_out, np.float64)))
    grads = {k: v.grad.numpy() for k, v in pt.items()}
    grads["input"] = xt.grad.numpy()
    return out.detach().numpy(), grads


def conv2d_direct(x, w, b, stride=1):
    """Reference 2-D convolution by explicit summation (zero padding k//2):
    y[n, o, i, j] = b[o] + sum_{c, u, v} w[o, c, u, v] x[n, c, s i + u - k//2, s j + v - k//2]
    for output (i, j), i < ceil(H / s), j < ceil(W / s)."""
    N, C, H, W = x.shape
    O, _, k, _ = w.shape
    p = k // 2
    Ho, Wo = (H + stride - 1) // stride, (W + stride - 1) // stride
    xp = np.zeros((N, C, H + 2 * p + stride, W + 2 * p + stride))
    xp[:, :, p:p + H, p:p + W] = x
    y = np.zeros((N, O, Ho, Wo)) + b[None, :, None, None]
    for u in range(k):
        for v in range(k):
            tap = xp[:, :, u:u + stride * Ho:stride, v:v + stride * Wo:stride]
            y += np.einsum("oc,nchw->nohw", w[:, :, u, v], tap)
    return y
