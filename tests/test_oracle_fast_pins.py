"""Pins of the FP64 fast-FLR oracle (Sec. 3.2 and 3.2.1) to things other than itself.

* Per-block weighted least squares (the WLS equation of Sec. 3.2) solved by numpy's SVD
  lstsq on the explicit sqrt(w)-scaled window rows plus sqrt(n eps) ridge rows, where a
  pixel's weight is the product of the 1-D Gaussian weights of its block's offsets.
* Exact affine recovery (also through 2x and 4x joint upsampling with a full-resolution
  map guide), constant radiance, and the eps -> infinity limit: block models reduce to
  Gaussian-weighted block means of Y, bilinearly interpolated (computed here with numpy).
"""
import numpy as np
import pytest

import oracle
import synth


def gauss(sigma, taps):
    d = np.arange(-taps, taps + 1)
    return np.exp(-d ** 2 / (2.0 * sigma ** 2))


def brute_block_models(g, y, F, sigma, taps, eps):
    q, H, W = g.shape
    Hb, Wb = -(-H // F), -(-W // F)
    w1 = gauss(sigma, taps)
    A = np.zeros((q + 1, 3, Hb, Wb))
    ys, xs = np.mgrid[0:H, 0:W]
    for by in range(Hb):
        for bx in range(Wb):
            dy = ys // F - by
            dx = xs // F - bx
            m = (np.abs(dy) <= taps) & (np.abs(dx) <= taps)
            wt = w1[dy[m] + taps] * w1[dx[m] + taps]
            X = np.concatenate([np.ones((wt.size, 1)), g[:, m].T.astype(np.float64)], axis=1)
            Y = y[:, m].T.astype(np.float64)
            sw = np.sqrt(wt)[:, None]
            n = wt.sum()
            reg = np.concatenate([np.zeros((q, 1)), np.sqrt(n * eps) * np.eye(q)], axis=1)
            Xa = np.concatenate([X * sw, reg])
            Ya = np.concatenate([Y * sw, np.zeros((q, 3))])
            A[:, :, by, bx] = np.linalg.lstsq(Xa, Ya, rcond=None)[0]
    return A


@pytest.mark.parametrize("H,W,F,sigma,taps", [(24, 40, 8, 1.25, 3), (21, 30, 4, 0.8, 2), (9, 13, 8, 2.0, 1)])
def test_block_models_match_weighted_least_squares(H, W, F, sigma, taps):
    g, y = synth.random_frame(H * W, H, W, 4)
    _, coef = oracle.flr_fast(g, y, factor=F, sigma_blocks=sigma, taps=taps, eps=1e-3, return_coef=True)
    ref = brute_block_models(g, y, F, sigma, taps, 1e-3)
    assert np.max(np.abs(coef - ref)) <= 1e-9 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("scale", [1, 2, 4])
def test_affine_radiance_is_recovered_exactly(scale):
    rng = np.random.default_rng(1)
    H, W, q = 32, 48, 5
    g, _ = synth.random_frame(2, H, W, q)
    g = (np.round(g * 256) / 256).astype(np.float32)
    Am = np.round(rng.normal(size=(q, 3)) * 16) / 16
    c = np.round(rng.normal(size=3) * 16) / 16
    y = (np.einsum("qhw,qc->chw", g.astype(np.float64), Am) + c[:, None, None]).astype(np.float32)
    z = None
    if scale > 1:
        z, _ = synth.random_frame(3, H * scale, W * scale, q)
    out = oracle.flr_fast(g, y, factor=8 // min(scale, 4) if scale > 1 else 8, sigma_blocks=1.25,
                          taps=3, eps=0.0, map_guide=z, scale=scale)
    zz = g if z is None else z
    ref = np.einsum("qhw,qc->chw", zz.astype(np.float64), Am) + c[:, None, None]
    assert np.max(np.abs(out - ref)) <= 1e-9


def test_constant_radiance_is_invariant():
    g, _ = synth.random_frame(4, 40, 56, 8)
    y = np.full((3, 40, 56), 0.75, np.float32)
    out = oracle.flr_fast(g, y, eps=1e-3)
    assert np.max(np.abs(out - 0.75)) <= 1e-12


def bilinear(blocks, Ho, Wo, F, s):
    Hb, Wb = blocks.shape
    u = np.clip((np.arange(Ho) + 0.5) / (F * s) - 0.5, 0, Hb - 1)
    v = np.clip((np.arange(Wo) + 0.5) / (F * s) - 0.5, 0, Wb - 1)
    i0 = np.minimum(np.floor(u).astype(int), max(Hb - 2, 0))
    j0 = np.minimum(np.floor(v).astype(int), max(Wb - 2, 0))
    i1 = np.minimum(i0 + 1, Hb - 1)
    j1 = np.minimum(j0 + 1, Wb - 1)
    fy = (u - i0)[:, None]
    fx = (v - j0)[None, :]
    return ((1 - fy) * ((1 - fx) * blocks[np.ix_(i0, j0)] + fx * blocks[np.ix_(i0, j1)]) +
            fy * ((1 - fx) * blocks[np.ix_(i1, j0)] + fx * blocks[np.ix_(i1, j1)]))


def test_huge_eps_is_blurred_block_mean_bilinearly_interpolated():
    H, W, F, sigma, taps = 45, 70, 8, 1.25, 3
    g, y = synth.random_frame(5, H, W, 3)
    out = oracle.flr_fast(g, y, factor=F, sigma_blocks=sigma, taps=taps, eps=1e12)
    Hb, Wb = -(-H // F), -(-W // F)
    w1 = gauss(sigma, taps)
    for c in range(3):
        pad = np.zeros((Hb * F, Wb * F))
        pad[:H, :W] = y[c]
        cnt = np.zeros_like(pad)
        cnt[:H, :W] = 1.0
        sums = pad.reshape(Hb, F, Wb, F).sum(axis=(1, 3))
        ns = cnt.reshape(Hb, F, Wb, F).sum(axis=(1, 3))

        def blur(a):
            t = np.zeros_like(a)
            for d in range(-taps, taps + 1):
                sh = np.zeros_like(a)
                if d >= 0:
                    sh[:, :Wb - d] = a[:, d:]
                else:
                    sh[:, -d:] = a[:, :Wb + d]
                t += w1[d + taps] * sh
            u = np.zeros_like(a)
            for d in range(-taps, taps + 1):
                sh = np.zeros_like(a)
                if d >= 0:
                    sh[:Hb - d] = t[d:]
                else:
                    sh[-d:] = t[:Hb + d]
                u += w1[d + taps] * sh
            return u
        means = blur(sums) / blur(ns)
        ref = bilinear(means, H, W, F, 1)
        assert np.max(np.abs(out[c] - ref)) <= 1e-9
