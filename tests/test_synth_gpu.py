"""The input generator's GPU reference renderer (synth.render_reference_gpu) against the
host renderer: the same room, estimator and counter-based random numbers, so the
references agree pixel by pixel up to rounding, except where a device cosf / sinf that
differs from the host's by an ulp turns a grazing ray into a different hit."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


@pytest.mark.parametrize("seed,H,W,spp", [(3, 48, 64, 16), (1000008, 37, 53, 64)])
def test_gpu_reference_matches_host_renderer(torch, seed, H, W, spp):
    _, _, ref = synth.render(seed, H, W, ref_spp=spp)
    got = synth.render_reference_gpu(seed, H, W, spp).cpu().numpy()
    assert got.shape == ref.shape and np.all(np.isfinite(got))
    d = np.abs(got - ref)
    scale = float(np.sqrt(np.mean(ref ** 2)))
    close = d <= 1e-5 * scale + 1e-6 * np.abs(ref)
    assert np.mean(close) >= 0.98, np.mean(close)
    # the rest differ by a few samples' worth of radiance at most
    assert abs(float(got.mean() - ref.mean())) <= 1e-3 * scale
