"""Pins of the FP64 oracle to things other than itself (CPU only).

Each test checks the oracle against something the paper or the mathematics fixes:
brute-force least squares on the explicit window matrices (Eqs. matX, matY, argmin),
exact rational arithmetic, closed-form invariants of the local affine model, and limits
that reduce FLR to a plain box filter.  A dropped term, a wrong sign or index, a
transposed operand or a mis-clipped window in the oracle fails at least one of them.
"""
from fractions import Fraction

import numpy as np
import pytest
from scipy.signal import convolve2d

import oracle
import synth


def brute_force(guide, rad, r, rc, eps, map_guide=None):
    """Per-pixel regularised least squares on explicit window matrices.

    For every pixel k: X_k = [1 | guides] over the clipped window, Y_k the radiance rows
    (Eqs. matX, matY).  The ridge term n_k * eps * ||a||^2 (bias unpenalised) is appended
    as sqrt(n_k * eps) * [0 | I] rows with zero targets and the augmented system is
    solved by numpy's SVD least squares, a different algorithm from the oracle's
    normal equations and Cholesky.  Then the coefficients are averaged over the clipped
    radius-rc window and applied to the centre pixel (Sec. 3.1).
    """
    g = guide.astype(np.float64)
    y = rad.astype(np.float64)
    z = g if map_guide is None else map_guide.astype(np.float64)
    q, H, W = g.shape
    A = np.zeros((H, W, q + 1, 3))
    for ky in range(H):
        for kx in range(W):
            ys = slice(max(0, ky - r), min(H, ky + r + 1))
            xs = slice(max(0, kx - r), min(W, kx + r + 1))
            X = g[:, ys, xs].reshape(q, -1).T
            n = X.shape[0]
            X = np.concatenate([np.ones((n, 1)), X], axis=1)
            Y = y[:, ys, xs].reshape(3, -1).T
            if eps > 0 and q > 0:
                reg = np.concatenate([np.zeros((q, 1)), np.sqrt(n * eps) * np.eye(q)], axis=1)
                X = np.concatenate([X, reg], axis=0)
                Y = np.concatenate([Y, np.zeros((q, 3))], axis=0)
            A[ky, kx] = np.linalg.lstsq(X, Y, rcond=None)[0]
    out = np.zeros((3, H, W))
    for iy in range(H):
        for ix in range(W):
            ys = slice(max(0, iy - rc), min(H, iy + rc + 1))
            xs = slice(max(0, ix - rc), min(W, ix + rc + 1))
            Abar = A[ys, xs].reshape(-1, q + 1, 3).mean(axis=0)
            xvec = np.concatenate([[1.0], z[:, iy, ix]])
            out[:, iy, ix] = xvec @ Abar
    return out, A.transpose(2, 3, 0, 1)


def rel_err(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


@pytest.mark.parametrize("H,W,q,r,rc,eps,seed", [
    (9, 7, 3, 2, 0, 1e-3, 0),
    (9, 7, 3, 2, 2, 1e-3, 1),
    (16, 16, 8, 5, 5, 1e-3, 2),
    (5, 40, 8, 8, 8, 1e-3, 3),    # window larger than the image in y
    (12, 6, 4, 3, 1, 1e-2, 4),
    (7, 9, 1, 1, 3, 1e-4, 5),
    (11, 10, 8, 2, 2, 0.0, 6),     # unregularised, full-rank i.i.d. guides
])
def test_oracle_matches_brute_force_least_squares(H, W, q, r, rc, eps, seed):
    g, y = synth.random_frame(seed, H, W, q)
    out, coef = oracle.flr_forward(g, y, r, eps, coef_radius=rc, return_coef=True)
    ref_out, ref_coef = brute_force(g, y, r, rc, eps)
    assert rel_err(coef, ref_coef) < 1e-9
    assert rel_err(out, ref_out) < 1e-10


def test_oracle_map_guide_matches_brute_force():
    g, y = synth.random_frame(11, 10, 12, 4)
    z, _ = synth.random_frame(12, 10, 12, 4)
    out = oracle.flr_forward(g, y, 2, 1e-3, coef_radius=1, map_guide=z)
    ref_out, _ = brute_force(g, y, 2, 1, 1e-3, map_guide=z)
    assert rel_err(out, ref_out) < 1e-10


def _solve_exact(M, rhs):
    """Gauss-Jordan elimination over the rationals (no rounding anywhere)."""
    n = len(M)
    aug = [list(M[i]) + list(rhs[i]) for i in range(n)]
    for c in range(n):
        p = next(i for i in range(c, n) if aug[i][c] != 0)
        aug[c], aug[p] = aug[p], aug[c]
        piv = aug[c][c]
        aug[c] = [v / piv for v in aug[c]]
        for i in range(n):
            if i != c and aug[i][c] != 0:
                f = aug[i][c]
                aug[i] = [a - f * b for a, b in zip(aug[i], aug[c])]
    return [row[n:] for row in aug]


def test_oracle_matches_exact_rational_normal_equations():
    """Eq. closed_form with the ridge on the guide rows, in exact rational arithmetic."""
    H, W, q, r, rc = 4, 5, 2, 1, 1
    eps = Fraction(1, 100)
    g, y = synth.random_frame(21, H, W, q)
    gq = [[[Fraction(float(g[c, i, j])) for j in range(W)] for i in range(H)] for c in range(q)]
    yq = [[[Fraction(float(y[c, i, j])) for j in range(W)] for i in range(H)] for c in range(3)]
    A = {}
    for ky in range(H):
        for kx in range(W):
            rows = [(i, j) for i in range(max(0, ky - r), min(H, ky + r + 1))
                    for j in range(max(0, kx - r), min(W, kx + r + 1))]
            n = len(rows)
            xs = [[Fraction(1)] + [gq[c][i][j] for c in range(q)] for i, j in rows]
            ys = [[yq[c][i][j] for c in range(3)] for i, j in rows]
            XtX = [[sum(x[a] * x[b] for x in xs) for b in range(q + 1)] for a in range(q + 1)]
            XtY = [[sum(x[a] * t[c] for x, t in zip(xs, ys)) for c in range(3)]
                   for a in range(q + 1)]
            for a in range(1, q + 1):
                XtX[a][a] += n * eps
            A[ky, kx] = _solve_exact(XtX, XtY)
    out = oracle.flr_forward(g, y, r, float(eps), coef_radius=rc)
    for iy in range(H):
        for ix in range(W):
            ks = [(i, j) for i in range(max(0, iy - rc), min(H, iy + rc + 1))
                  for j in range(max(0, ix - rc), min(W, ix + rc + 1))]
            for c in range(3):
                v = Fraction(0)
                for k in ks:
                    Ak = A[k]
                    v += Ak[0][c] + sum(Ak[a + 1][c] * gq[a][iy][ix] for a in range(q))
                v /= len(ks)
                assert abs(float(v) - out[c, iy, ix]) <= 1e-12 * max(1.0, abs(float(v)))


@pytest.mark.parametrize("rc", [0, 3])
def test_affine_radiance_is_recovered_exactly(rc):
    """If Y = X A + c exactly, every window's least-squares fit is exact (eps = 0)."""
    # guides on a 2^-8 grid and coefficients on a 2^-4 grid keep Y exact in float32
    rng = np.random.default_rng(5)
    g, _ = synth.random_frame(31, 24, 20, 5)
    g = (np.round(g * 256) / 256).astype(np.float32)
    Amat = np.round(rng.normal(size=(5, 3)) * 16) / 16
    c = np.round(rng.normal(size=3) * 16) / 16
    y64 = np.einsum("qhw,qc->chw", g.astype(np.float64), Amat) + c[:, None, None]
    y = y64.astype(np.float32)
    assert np.array_equal(y.astype(np.float64), y64)
    out = oracle.flr_forward(g, y, 3, 0.0, coef_radius=rc)
    assert np.max(np.abs(out - y64)) < 1e-9


@pytest.mark.parametrize("rc", [0, 4])
def test_constant_radiance_is_invariant(rc):
    g, _ = synth.random_frame(32, 20, 26, 8)
    y = np.full((3, 20, 26), 0.625, np.float32)
    y[1] = 1.5
    out = oracle.flr_forward(g, y, 4, 1e-3, coef_radius=rc)
    assert np.max(np.abs(out - y.astype(np.float64))) < 1e-12


@pytest.mark.parametrize("rc", [0, 2])
def test_guide_shift_invariance(rc):
    """The bias column absorbs a constant added to a guide (centred form)."""
    g, y = synth.random_frame(33, 18, 22, 6)
    g = (np.round(g * 1024) / 1024).astype(np.float32)  # g + shift stays exact in float32
    shift = np.array([0.5, -2.0, 10.0, 0.0, 3.25, -0.75], np.float32)[:, None, None]
    out0 = oracle.flr_forward(g, y, 3, 1e-3, coef_radius=rc)
    out1 = oracle.flr_forward(g + shift, y, 3, 1e-3, coef_radius=rc)
    assert np.max(np.abs(out0 - out1)) < 1e-9


def test_linear_in_radiance():
    """out(alpha Y + beta) = alpha out(Y) + beta; inputs on a 2^-10 grid stay exact in float32."""
    g, y = synth.random_frame(34, 16, 16, 8)
    y = np.round(y * 1024) / 1024
    alpha, beta = 2.0, -0.75
    out0 = oracle.flr_forward(g, y, 3, 1e-3, coef_radius=3)
    out1 = oracle.flr_forward(g, (alpha * y + beta).astype(np.float32), 3, 1e-3, coef_radius=3)
    assert np.max(np.abs(out1 - (alpha * out0 + beta))) < 1e-11


def test_guide_permutation_invariance():
    g, y = synth.random_frame(35, 15, 17, 8)
    perm = [3, 0, 7, 1, 6, 2, 5, 4]
    out0 = oracle.flr_forward(g, y, 4, 1e-3, coef_radius=2)
    out1 = oracle.flr_forward(g[perm], y, 4, 1e-3, coef_radius=2)
    assert np.max(np.abs(out0 - out1)) < 1e-11


def test_transpose_and_flip_commute():
    g, y = synth.random_frame(36, 14, 19, 4)
    out = oracle.flr_forward(g, y, 3, 1e-3, coef_radius=2)
    out_t = oracle.flr_forward(g.transpose(0, 2, 1), y.transpose(0, 2, 1), 3, 1e-3, coef_radius=2)
    assert np.max(np.abs(out_t.transpose(0, 2, 1) - out)) < 1e-11
    out_f = oracle.flr_forward(g[:, ::-1, :], y[:, ::-1, :], 3, 1e-3, coef_radius=2)
    assert np.max(np.abs(out_f[:, ::-1, :] - out)) < 1e-11
    out_f = oracle.flr_forward(g[:, :, ::-1], y[:, :, ::-1], 3, 1e-3, coef_radius=2)
    assert np.max(np.abs(out_f[:, :, ::-1] - out)) < 1e-11


def clipped_box_mean(img, rad):
    k = np.ones((2 * rad + 1, 2 * rad + 1))
    num = convolve2d(img, k, mode="same", boundary="fill")
    den = convolve2d(np.ones_like(img), k, mode="same", boundary="fill")
    return num / den


def test_huge_eps_reduces_to_box_filter():
    """eps -> infinity forces a -> 0, so each model is the window mean of Y."""
    g, y = synth.random_frame(37, 21, 23, 8)
    r, rc = 4, 3
    out = oracle.flr_forward(g, y, r, 1e12, coef_radius=rc)
    ref = np.stack([clipped_box_mean(clipped_box_mean(y[c].astype(np.float64), r), rc)
                    for c in range(3)])
    assert np.max(np.abs(out - ref)) < 1e-9


def test_zero_guides_is_box_filter():
    _, y = synth.random_frame(38, 13, 29, 1)
    out = oracle.flr_forward(None, y, 5, 1e-3, coef_radius=2)
    ref = np.stack([clipped_box_mean(clipped_box_mean(y[c].astype(np.float64), 5), 2)
                    for c in range(3)])
    assert np.max(np.abs(out - ref)) < 1e-12


def test_zero_radius_is_identity():
    g, y = synth.random_frame(39, 9, 11, 8)
    out = oracle.flr_forward(g, y, 0, 1e-3, coef_radius=0)
    assert np.max(np.abs(out - y.astype(np.float64))) < 1e-12


def test_unregularised_rank_deficient_window_is_reported():
    g, y = synth.random_frame(40, 8, 8, 3, kind="const_guide")
    with pytest.raises(oracle.OracleError):
        oracle.flr_forward(g, y, 2, 0.0)


def test_rendered_frame_denoises():
    """On a rendered room, FLR output is closer to a many-sample reference than the input."""
    g, y, ref = synth.render(7, 48, 64, ref_spp=256)
    out = oracle.flr_forward(g, y, 6, 1e-3, coef_radius=6)
    mse_in = np.mean((y.astype(np.float64) - ref) ** 2)
    mse_out = np.mean((out - ref) ** 2)
    assert mse_out < 0.25 * mse_in
