"""Pins of the FP64 fast-FLR oracle (Sec. 3.2 and 3.2.1) to things other than itself.

* Per-block weighted least squares (the WLS equation of Sec. 3.2) solved by numpy's SVD
  lstsq on the explicit sqrt(w)-scaled window rows plus sqrt(n eps) ridge rows, where a
  pixel's weight is the product of the 1-D Gaussian weights of its block's offsets.
* The Appendix's regularised normalised solve (additive and multiplicative terms) against
  the same weighted least squares with the penalty its normalisation amounts to, solved
  by lstsq on augmented rows; with both terms zero it is the plain weighted solve.
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


def brute_block_models_appendix(g, y, F, sigma, taps, e_add, e_mul):
    """The Appendix's regularised normalised solve, derived independently of its printed
    steps: with D_s = diag(sigma^), C^ + e_add I = D_s^-1 (W^ + e_add D_s^2) D_s^-1, so the
    un-normalised model is a = (W^ + e_add diag(W^))^-1 D with
    W^ = W + e_mul (mu mu^T + diag(mu^2)) + e_add I -- the weighted least squares with the
    penalty n a^T R a, R = e_mul (mu mu^T + diag(mu^2)) + e_add I + e_add diag(W^), on the
    guide coefficients only.  Solved here by lstsq on the sqrt(w)-scaled rows plus
    sqrt(n) L^T rows (R = L L^T), with mu and W the weighted window statistics."""
    q, H, W = g.shape
    Hb, Wb = -(-H // F), -(-W // F)
    w1 = gauss(sigma, taps)
    A = np.zeros((q + 1, 3, Hb, Wb))
    ys, xs = np.mgrid[0:H, 0:W]
    for by in range(Hb):
        for bx in range(Wb):
            dy, dx = ys // F - by, xs // F - bx
            m = (np.abs(dy) <= taps) & (np.abs(dx) <= taps)
            wt = w1[dy[m] + taps] * w1[dx[m] + taps]
            Xg = g[:, m].T.astype(np.float64)
            n = wt.sum()
            mu = (wt[:, None] * Xg).sum(0) / n
            Wc = ((wt[:, None] * (Xg - mu)).T @ (Xg - mu)) / n
            Wh = Wc + e_mul * (np.outer(mu, mu) + np.diag(mu ** 2)) + e_add * np.eye(q)
            R = e_mul * (np.outer(mu, mu) + np.diag(mu ** 2)) + e_add * np.eye(q) + e_add * np.diag(np.diag(Wh))
            L = np.linalg.cholesky(R)
            X = np.concatenate([np.ones((wt.size, 1)), Xg], axis=1)
            sw = np.sqrt(wt)[:, None]
            reg = np.concatenate([np.zeros((q, 1)), np.sqrt(n) * L.T], axis=1)
            Xa = np.concatenate([X * sw, reg])
            Ya = np.concatenate([y[:, m].T.astype(np.float64) * sw, np.zeros((q, 3))])
            A[:, :, by, bx] = np.linalg.lstsq(Xa, Ya, rcond=None)[0]
    return A


@pytest.mark.parametrize("e_add,e_mul", [(1e-3, 0.0), (1e-4, 1e-4), (3e-3, 0.2), (0.0, 0.05)])
@pytest.mark.parametrize("H,W,F,sigma,taps", [(24, 40, 8, 1.25, 3), (21, 30, 4, 0.8, 2)])
def test_appendix_solve_matches_augmented_least_squares(H, W, F, sigma, taps, e_add, e_mul):
    """Appendix: W^ = S/n + e_mul diag(mu^T mu) + e_add I - (1 - e_mul) mu^T mu, normalised
    by sigma^ = sqrt(diag W^), solved with (C^ + e_add I), un-normalised."""
    g, y = synth.random_frame(H * W + 5, H, W, 4)
    g = g + 0.7  # guides with nonzero means, so the multiplicative term acts
    _, coef = oracle.flr_fast(g, y, factor=F, sigma_blocks=sigma, taps=taps, return_coef=True,
                              appendix=(e_add, e_mul))
    ref = brute_block_models_appendix(g, y, F, sigma, taps, e_add, e_mul)
    assert np.max(np.abs(coef - ref)) <= 1e-8 * max(1.0, np.max(np.abs(ref)))


def test_appendix_without_regularisers_is_plain_weighted_least_squares():
    """With both terms zero the normalisation cancels: the unregularised WLS models (the
    ridge pin at eps = 0) come back, so the printed steps add no bias of their own."""
    g, y = synth.random_frame(77, 24, 32, 4)
    _, coef = oracle.flr_fast(g, y, factor=8, sigma_blocks=1.25, taps=3, return_coef=True, appendix=(0.0, 0.0))
    ref = brute_block_models(g, y, 8, 1.25, 3, 0.0)
    assert np.max(np.abs(coef - ref)) <= 1e-8 * max(1.0, np.max(np.abs(ref)))


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


def brute_fast_forward(g, y, F, sigma, taps, eps):
    """Fast FLR written with numpy: brute weighted least squares per block (above) and the
    bilinear interpolation of the block models at every pixel (block centres at
    ((i + 1/2) F - 1/2), clamped at the outermost centres), applied to (1, guides)."""
    A = brute_block_models(g, y, F, sigma, taps, eps)
    q, H, W = g.shape
    Hb, Wb = A.shape[2:]

    def axis(n, nb):
        u = np.clip((np.arange(n) + 0.5) / F - 0.5, 0, nb - 1)
        i0 = np.minimum(np.floor(u).astype(int), max(nb - 2, 0))
        i1 = np.minimum(i0 + 1, nb - 1)
        return i0, i1, u - i0
    r0, r1, fy = axis(H, Hb)
    c0, c1, fx = axis(W, Wb)
    Ai = (A[:, :, r0][:, :, :, c0] * (1 - fy)[:, None] * (1 - fx)[None, :] +
          A[:, :, r0][:, :, :, c1] * (1 - fy)[:, None] * fx[None, :] +
          A[:, :, r1][:, :, :, c0] * fy[:, None] * (1 - fx)[None, :] +
          A[:, :, r1][:, :, :, c1] * fy[:, None] * fx[None, :])
    z = np.concatenate([np.ones((1, H, W)), g.astype(np.float64)])
    return np.einsum("ichw,ihw->chw", Ai, z)


def test_sigma_derivative_matches_the_numpy_forward():
    """Sec. 3.2's learned blur radius: d/dsigma of <G, fast FLR> from the oracle equals the
    same Richardson difference of the independent numpy forward."""
    g, y = synth.random_frame(91, 24, 40, 4)
    G = np.random.default_rng(2).normal(size=(3, 24, 40))
    sig, eps = 1.1, 1e-3
    got = oracle.flr_fast_param_grads(g, y, G, factor=8, sigma_blocks=sig, taps=3, eps=eps)
    assert np.max(np.abs(oracle.flr_fast(g, y, factor=8, sigma_blocks=sig, taps=3, eps=eps)
                         - brute_fast_forward(g, y, 8, sig, 3, eps))) < 1e-9

    def f(s):
        return np.sum(G * brute_fast_forward(g, y, 8, s, 3, eps))
    h = 1e-3 * sig
    d = lambda st: (f(sig + st) - f(sig - st)) / (2 * st)
    ref = (4 * d(h / 2) - d(h)) / 3
    assert abs(got["sigma"] - ref) <= 1e-7 * max(1.0, abs(ref))


@pytest.mark.parametrize("appendix", [None, (1e-3, 0.0), (2e-3, 0.3)])
def test_regulariser_derivatives_closed_form_on_one_block(appendix):
    """A frame of one block has one model, applied at every pixel: out = b + a^T z with
    a = M^-1 D.  Differentiating M a = D gives da = -M^-1 (dM) a and db = -mu^T da, with
    dM / d eps = I for the ridge; for the Appendix's M = W^ + e_add diag(W^),
    W^ = W + e_mul (mu mu^T + diag mu^2) + e_add I:
    dM / d e_add = I + diag(W^) + e_add I and
    dM / d e_mul = (mu mu^T + diag mu^2) + 2 e_add diag(mu^2)."""
    F, q = 8, 4
    g, y = synth.random_frame(17, F, F, q)
    g = (g + 0.6).astype(np.float32)
    G = np.random.default_rng(5).normal(size=(3, F, F))
    X = g.reshape(q, -1).T.astype(np.float64)
    Y = y.reshape(3, -1).T.astype(np.float64)
    n = X.shape[0]
    mu, muy = X.mean(0), Y.mean(0)
    Wc = (X - mu).T @ (X - mu) / n
    D = (X - mu).T @ (Y - muy) / n
    if appendix is None:
        e_add, e_mul = 1e-3, None
        M = Wc + e_add * np.eye(q)
        dMs = {"eps": np.eye(q)}
    else:
        e_add, e_mul = appendix
        P = np.outer(mu, mu) + np.diag(mu ** 2)
        Wh = Wc + e_mul * P + e_add * np.eye(q)
        M = Wh + e_add * np.diag(np.diag(Wh))
        dMs = {"eps": np.eye(q) + np.diag(np.diag(Wh)) + e_add * np.eye(q)}
        if e_mul > 0:
            dMs["eps_mul"] = P + 2 * e_add * np.diag(mu ** 2)
    a = np.linalg.solve(M, D)
    got = oracle.flr_fast_param_grads(g, y, G, factor=F, sigma_blocks=1.25, taps=3, eps=e_add, appendix=appendix)
    assert set(got) == {"sigma"} | set(dMs)
    for name, dM in dMs.items():
        da = -np.linalg.solve(M, dM @ a)
        db = -mu @ da
        dout = db[:, None] + da.T @ X.T  # [3][pixels]
        ref = float(np.sum(G.reshape(3, -1) * dout))
        assert abs(got[name] - ref) <= 1e-7 * max(1.0, abs(ref)), (name, got[name], ref)
