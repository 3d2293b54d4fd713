"""The seeded input generator: determinism, guide ranges, and that the 1 spp renders are
unbiased samples of the radiance the reference estimates (the mean of many independent
noise realisations approaches the reference, at the Monte Carlo rate)."""
import numpy as np

import synth


def test_render_is_deterministic_and_guides_are_in_range():
    g, y, r = synth.render(7, 24, 40, ref_spp=16)
    g2, y2 = synth.render(7, 24, 40)
    assert np.array_equal(g, g2) and np.array_equal(y, y2)
    assert np.all((g[:3] >= 0.1) & (g[:3] <= 0.9))  # albedo
    assert np.allclose(np.sum(g[3:6].astype(np.float64) ** 2, axis=0), 1.0, atol=1e-5)  # unit normals
    assert np.all((g[6] > 0) & (g[6] <= 1)) and np.all((g[7] >= 0) & (g[7] <= 1))  # depth, AO
    assert np.all(y >= 0) and np.all(r >= 0)


def test_noise_realisations_average_to_the_reference():
    H, W = 32, 48
    g, y, ref = synth.render(3, H, W, ref_spp=2048)
    n = synth.render_noise(3, H, W, 512)
    assert not np.array_equal(n[0], y) and not np.array_equal(n[0], n[1])
    assert np.array_equal(n[5:9], synth.render_noise(3, H, W, 4, first=5))
    # mean absolute deviation from the reference shrinks like 1/sqrt(samples)
    d1 = np.abs(n[0] - ref).mean()
    d512 = np.abs(n.mean(axis=0) - ref).mean()
    assert d512 < d1 / 8
    assert abs(n.mean() - ref.mean()) < 0.05 * ref.mean()
