"""Pins of the FLNR network oracle (oracle/flnr_ref.py, PyTorch CPU float64).

* torch's conv2d as used (cross-correlation, zero padding k//2) equals an explicit
  summation over taps, for 3x3 and 1x1 kernels;
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
                      ("o1.w", (6, 9, 0, 0)), ("o0.b", (4,)), ("e1a.b", (17,))]:
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
