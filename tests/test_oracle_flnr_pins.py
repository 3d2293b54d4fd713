"""Pins of the FLNR network oracle (oracle/flnr_ref.py, PyTorch CPU float64).

* torch's conv2d as used (cross-correlation, zero padding k//2) equals an explicit
  summation over taps, for 3x3 and 1x1 kernels, at stride 1 and at the encoder's stride 2
  (Sec. 3.3), which is also the stride-1 result at even rows and columns and, on a tiny
  input, a pure-Python loop over every output, channel and tap;
* the autograd gradients equal Richardson central differences of the forward pass, for
  weights, biases of several layers and the input (steps of 1e-6 keep every ReLU on one
  side of its kink);
* shapes and the sigmoid's open range.
"""
import numpy as np
import pytest
import torch

from oracle import flnr_ref


@pytest.mark.parametrize("k", [3, 1])
def test_conv_matches_explicit_sum(k):
    rng = np.random.default_rng(k)
    x = rng.normal(size=(2, 5, 9, 7))
    w = rng.normal(size=(4, 5, k, k))
    b = rng.normal(size=4)
    ref = flnr_ref.conv2d_direct(x, w, b)
    got = torch.nn.functional.conv2d(torch.tensor(x), torch.tensor(w), torch.tensor(b), padding=k // 2).numpy()
    assert np.max(np.abs(got - ref)) < 1e-12


@pytest.mark.parametrize("H,W", [(8, 12), (9, 7)])
def test_stride_two_conv_matches_explicit_sum_and_subsampling(H, W):
    rng = np.random.default_rng(H * W)
    x = rng.normal(size=(2, 5, H, W))
    w = rng.normal(size=(4, 5, 3, 3))
    b = rng.normal(size=4)
    ref = flnr_ref.conv2d_direct(x, w, b, stride=2)
    assert ref.shape == (2, 4, (H + 1) // 2, (W + 1) // 2)
    got = torch.nn.functional.conv2d(torch.tensor(x), torch.tensor(w), torch.tensor(b), stride=2, padding=1).numpy()
    assert np.max(np.abs(got - ref)) < 1e-12
    full = flnr_ref.conv2d_direct(x, w, b)
    assert np.max(np.abs(full[:, :, ::2, ::2] - ref)) < 1e-12


def test_stride_two_conv_brute_force():
    """Output (i, j) of a stride-2 3x3 convolution with zero padding 1 reads inputs
    (2i - 1 .. 2i + 1, 2j - 1 .. 2j + 1); written out element by element."""
    rng = np.random.default_rng(4)
    x = rng.normal(size=(1, 2, 5, 6))
    w = rng.normal(size=(3, 2, 3, 3))
    b = rng.normal(size=3)
    ref = flnr_ref.conv2d_direct(x, w, b, stride=2)
    for o in range(3):
        for i in range(3):
            for j in range(3):
                acc = b[o]
                for c in range(2):
                    for u in range(3):
                        for v in range(3):
                            yy, xx = 2 * i + u - 1, 2 * j + v - 1
                            if 0 <= yy < 5 and 0 <= xx < 6:
                                acc += w[o, c, u, v] * x[0, c, yy, xx]
                assert abs(acc - ref[0, o, i, j]) < 1e-12


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    params = {k: v.astype(np.float64) for k, v in flnr_ref.init_weights(3).items()}
    for k in params:
        if k.endswith(".b"):
            params[k] = rng.normal(scale=0.1, size=params[k].shape)
    x = rng.uniform(size=(1, 11, 16, 20))
    G = rng.normal(size=(1, 8, 16, 20))
    out, grads = flnr_ref.forward_backward(x, params, G)
    assert out.shape == (1, 8, 16, 20) and np.all((out > 0) & (out < 1))

    def loss(p, xx):
        pt = {kk: torch.tensor(v) for kk, v in p.items()}
        return float((flnr_ref.forward(torch.tensor(xx), pt).numpy() * G).sum())

    def rich(f, h):
        return (4 * (f(h / 2) - f(-h / 2)) / h - (f(h) - f(-h)) / (2 * h)) / 3

    for name, idx in [("in0.w", (3, 7, 1, 2)), ("e2b.w", (10, 20, 0, 1)), ("d1a.w", (5, 70, 2, 2)),
                      ("o1.w", (6, 9, 0, 0)), ("o0.b", (4,)), ("e1a.b", (17,)), ("e1b.w", (2, 9, 2, 0)),
                      ("e2a.w", (40, 3, 1, 1)), ("e1b.b", (30,))]:
        def f(t, name=name, idx=idx):
            p = dict(params)
            p[name] = params[name].copy()
            p[name][idx] += t
            return loss(p, x)
        fd = rich(f, 1e-6)
        assert abs(fd - grads[name][idx]) <= 1e-6 * max(1.0, abs(fd)), name
    for idx in [(0, 2, 5, 5), (0, 10, 15, 19)]:
        def fx(t, idx=idx):
            xx = x.copy()
            xx[idx] += t
            return loss(params, xx)
        fd = rich(fx, 1e-6)
        assert abs(fd - grads["input"][idx]) <= 1e-6 * max(1.0, abs(fd))


def test_two_output_sets_share_the_network():
    """Sec. 3.3's 2Q outputs: the 16-channel head's first 8 channels equal the 8-channel
    network whose o1 holds the first 8 rows of the 16-channel o1, and the other 8 follow the
    same features with the remaining rows (the layers before o1 are shared)."""
    rng = np.random.default_rng(12)
    p16 = {k: v.astype(np.float64) for k, v in flnr_ref.init_weights(4, outputs=16).items()}
    assert p16["o1.w"].shape == (16, 16, 1, 1) and p16["o1.b"].shape == (16,)
    assert np.array_equal(p16["o1.w"][8:], p16["o1.w"][:8])  # the map set starts as the model set
    p16["o1.w"][8:] = rng.normal(scale=0.2, size=(8, 16, 1, 1))  # distinct halves for the check
    p16["o1.b"] = rng.normal(scale=0.1, size=16)
    x = rng.uniform(size=(1, 11, 8, 12))
    out16 = flnr_ref.forward(torch.tensor(x), {k: torch.tensor(v) for k, v in p16.items()}).numpy()
    assert out16.shape == (1, 16, 8, 12)
    for half in (slice(0, 8), slice(8, 16)):
        p8 = dict(p16)
        p8["o1.w"], p8["o1.b"] = p16["o1.w"][half], p16["o1.b"][half]
        out8 = flnr_ref.forward(torch.tensor(x), {k: torch.tensor(v) for k, v in p8.items()}).numpy()
        assert np.max(np.abs(out8 - out16[:, half])) < 1e-14


def bf16_bits(a):
    """Round-to-nearest-even of float32 values to bfloat16, by integer arithmetic on the
    IEEE-754 bit patterns (finite inputs): keep the top 16 bits, adding 0x7FFF plus the
    lowest kept bit before truncating."""
    u = np.asarray(a, np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def test_bf16_rounding_is_nearest_even():
    rng = np.random.default_rng(5)
    v = np.concatenate([rng.normal(size=4000) * 10.0 ** rng.integers(-6, 6, 4000),
                        # exact ties between two bfloat16 neighbours, both parities
                        np.array([1 + 2 ** -8, 1 + 3 * 2 ** -8, -(1 + 2 ** -8), 2 ** -8 + 2 ** -16, 0.0])])
    got = flnr_ref.round_bf16(torch.tensor(v)).numpy()
    assert np.array_equal(got, bf16_bits(v.astype(np.float32)))
    assert got[-5] == 1.0 and got[-4] == 1 + 4 * 2 ** -8 and got[-3] == -1.0


def test_bf16_storage_forward_matches_explicit_rounding():
    """The emulated forward equals a numpy restatement: log(1 + max(Y, 0)) radiance input,
    explicit-sum convolutions in float64 with bit-level bfloat16 rounding of the input,
    weights and ReLU outputs (Sec. 3.3's network, stride-2 encoder convolutions)."""
    rng = np.random.default_rng(7)
    params = flnr_ref.init_weights(4)
    for k in params:
        if k.endswith(".b"):
            params[k] = rng.normal(scale=0.05, size=params[k].shape).astype(np.float32)
    x = rng.uniform(size=(1, 11, 8, 12))
    x[:, 8:] = rng.normal(size=(1, 3, 8, 12)) * 3.0  # negative and firefly-like radiance
    pt = {k: torch.tensor(v.astype(np.float64)) for k, v in params.items()}
    got = flnr_ref.forward(torch.tensor(x), pt, bf16_storage=True).numpy()

    def conv(t, n, relu=True, stride=1):
        z = flnr_ref.conv2d_direct(t, bf16_bits(params[n + ".w"]), params[n + ".b"].astype(np.float64),
                                   stride=stride)
        return bf16_bits(np.maximum(z, 0.0)) if relu else z

    def up(t):
        return t.repeat(2, axis=2).repeat(2, axis=3)

    xin = np.concatenate([x[:, :8], np.log1p(np.maximum(x[:, 8:], 0.0))], axis=1)
    f0 = conv(conv(bf16_bits(xin), "in0"), "in1")
    f1 = conv(conv(f0, "e1a"), "e1b", stride=2)
    f2 = conv(conv(f1, "e2a"), "e2b", stride=2)
    d1 = conv(conv(np.concatenate([up(f2), f1], 1), "d1a"), "d1b")
    d0 = conv(conv(np.concatenate([up(d1), f0], 1), "d0a"), "d0b")
    ref = 1.0 / (1.0 + np.exp(-conv(conv(d0, "o0"), "o1", relu=False)))
    assert np.max(np.abs(got - ref)) < 1e-12


def test_bf16_storage_gradients_of_the_head():
    """Under BF16 storage the output bias gradient is the pixel sum of the bfloat16-rounded
    sigmoid gradient g s (1 - s), and the emulated gradients stay close to the float64 ones
    (a few bfloat16 rounding units of the gradient's scale)."""
    rng = np.random.default_rng(8)
    params = flnr_ref.init_weights(6)
    x = rng.uniform(size=(1, 11, 12, 16))
    G = rng.normal(size=(1, 8, 12, 16))
    out, g16 = flnr_ref.forward_backward(x, params, G, bf16_storage=True)
    ref_b = bf16_bits((G * out * (1.0 - out)).astype(np.float32)).sum(axis=(0, 2, 3))
    assert np.max(np.abs(g16["o1.b"] - ref_b)) < 1e-9
    out64, g64 = flnr_ref.forward_backward(x, params, G)
    assert np.max(np.abs(out - out64)) < 3e-2
    for name in ("o1.w", "o0.w", "d0b.w"):
        a, b = g16[name], g64[name]
        assert np.sum(a * b) / np.linalg.norm(a) / np.linalg.norm(b) > 0.95, name
