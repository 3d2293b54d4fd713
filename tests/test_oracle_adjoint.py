"""Pins of the oracle's FP64 backward pass to things other than itself (CPU only).

* Richardson-extrapolated central finite differences of L = <G, I> with respect to single
  guide, map-guide and radiance values and to eps.  Inputs sit on a 2^-12 grid and the
  steps are powers of two, so every perturbed input is exact in float32.
* Euler's identity: I is linear and homogeneous in Y (a = M^-1 D and b are linear in Y),
  so <G, I(Y)> = <dL/dY, Y> exactly.
* Shift invariance: adding t to a guide channel (model and map guide together) leaves I
  unchanged, so the guide gradient of every channel sums to zero over the image.
"""
import numpy as np
import pytest

import oracle
import synth


def grid_frame(seed, H, W, q, kind="uniform"):
    g, y = synth.random_frame(seed, H, W, q, kind=kind)
    g = (np.round(g * 4096) / 4096).astype(np.float32)
    y = (np.round(y * 4096) / 4096).astype(np.float32)
    return g, y


def loss(g, y, G, r, rc, eps, z=None):
    return float(np.sum(G * oracle.flr_forward(g, y, r, eps, coef_radius=rc, map_guide=z)))


def richardson(f, h):
    d1 = (f(h) - f(-h)) / (2 * h)
    d2 = (f(h / 2) - f(-h / 2)) / h
    return (4 * d2 - d1) / 3


@pytest.mark.parametrize("rc", [0, 2])
def test_backward_matches_finite_differences(rc):
    H, W, q, r, eps = 10, 12, 3, 2, 1e-2
    g, y = grid_frame(3, H, W, q)
    G = np.random.default_rng(4).normal(size=(3, H, W))
    bw = oracle.flr_backward(g, y, G, r, eps, coef_radius=rc)
    rng = np.random.default_rng(5)
    h = 2.0 ** -7
    for _ in range(6):
        c, i, j = int(rng.integers(q)), int(rng.integers(H)), int(rng.integers(W))

        def fg(t):
            g2 = g.copy()
            g2[c, i, j] += np.float32(t)
            return loss(g2, y, G, r, rc, eps)
        fd = richardson(fg, h)
        assert abs(fd - bw["guide"][c, i, j]) <= 1e-7 * max(1.0, abs(fd))

        c3 = int(rng.integers(3))

        def fy(t):
            y2 = y.copy()
            y2[c3, i, j] += np.float32(t)
            return loss(g, y2, G, r, rc, eps)
        fd = richardson(fy, h)
        assert abs(fd - bw["radiance"][c3, i, j]) <= 1e-7 * max(1.0, abs(fd))

    fe = richardson(lambda t: loss(g, y, G, r, rc, eps + t), 2.0 ** -12)
    assert abs(fe - bw["eps"]) <= 1e-6 * max(1.0, abs(fe))


def test_map_guide_gradient_matches_finite_differences():
    H, W, q, r, rc, eps = 9, 11, 2, 2, 1, 1e-2
    g, y = grid_frame(6, H, W, q)
    z, _ = grid_frame(7, H, W, q)
    G = np.random.default_rng(8).normal(size=(3, H, W))
    bw = oracle.flr_backward(g, y, G, r, eps, coef_radius=rc, map_guide=z)
    rng = np.random.default_rng(9)
    for _ in range(5):
        c, i, j = int(rng.integers(q)), int(rng.integers(H)), int(rng.integers(W))

        def fz(t):
            z2 = z.copy()
            z2[c, i, j] += np.float32(t)
            return loss(g, y, G, r, rc, eps, z=z2)

        def fg(t):
            g2 = g.copy()
            g2[c, i, j] += np.float32(t)
            return loss(g2, y, G, r, rc, eps, z=z)
        assert abs(richardson(fz, 2.0 ** -7) - bw["map_guide"][c, i, j]) <= 1e-7
        fd = richardson(fg, 2.0 ** -7)
        assert abs(fd - bw["guide"][c, i, j]) <= 1e-7 * max(1.0, abs(fd))


@pytest.mark.parametrize("rc", [0, 3])
def test_euler_identity_in_radiance(rc):
    H, W, q, r = 20, 23, 8, 4
    g, y = synth.random_frame(11, H, W, q)
    G = np.random.default_rng(12).normal(size=(3, H, W))
    out = oracle.flr_forward(g, y, r, 1e-3, coef_radius=rc)
    bw = oracle.flr_backward(g, y, G, r, 1e-3, coef_radius=rc)
    lhs = float(np.sum(G * out))
    rhs = float(np.sum(bw["radiance"] * y.astype(np.float64)))
    assert abs(lhs - rhs) <= 1e-10 * max(1.0, abs(lhs))


@pytest.mark.parametrize("rc", [0, 3])
def test_guide_gradient_sums_to_zero_per_channel(rc):
    H, W, q, r = 18, 21, 5, 3
    g, y = synth.random_frame(13, H, W, q)
    G = np.random.default_rng(14).normal(size=(3, H, W))
    bw = oracle.flr_backward(g, y, G, r, 1e-3, coef_radius=rc)
    scale = np.max(np.abs(bw["guide"]))
    assert np.max(np.abs(bw["guide"].sum(axis=(1, 2)))) <= 1e-9 * scale * H * W


def test_gradient_is_local_to_the_block_and_its_halo():
    """With grad_out nonzero only in a block, the gradient lives in the block plus its
    radius-(r + rc) halo and depends only on the inputs there (each output reads the models
    of its rc-window, each model the inputs of its r-window, clipped alike at the frame
    edge).  So the adjoint of the frame equals the sum of the adjoints of disjoint crops,
    exactly: the premise of the GPU test that checks a 1080p frame block by block."""
    H, W, r, rc, B = 120, 160, 4, 3, 12
    R = r + rc
    g, y = synth.render(2, H, W)
    blocks = [(0, 0), (H - B, W - B), (50, 70)]
    G = np.zeros((3, H, W), np.float32)
    rng = np.random.default_rng(0)
    for by, bx in blocks:
        G[:, by:by + B, bx:bx + B] = rng.normal(size=(3, B, B))
    full = oracle.flr_backward(g, y, G, r, 1e-3, coef_radius=rc)
    acc = {k: np.zeros_like(full[k]) for k in ("guide", "radiance")}
    e = 0.0
    for by, bx in blocks:
        y0, y1, x0, x1 = max(0, by - R), min(H, by + B + R), max(0, bx - R), min(W, bx + B + R)
        part = oracle.flr_backward(g[:, y0:y1, x0:x1], y[:, y0:y1, x0:x1], G[:, y0:y1, x0:x1], r, 1e-3,
                                   coef_radius=rc)
        for k in acc:
            acc[k][:, y0:y1, x0:x1] += part[k]
        e += part["eps"]
    for k in acc:
        assert np.max(np.abs(acc[k] - full[k])) <= 1e-12 * np.sqrt(np.mean(full[k] ** 2)), k
    assert abs(e - full["eps"]) <= 1e-12 * abs(full["eps"])
