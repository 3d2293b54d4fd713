"""Host-side parts of FLNR on the CPU: the layer table agrees with the oracle's network
and the library's parameter count, the flat parameter layout round-trips, the seeded
initialisation matches the oracle's, training crops are windows of the rendered scenes,
PSNR and the bench's multiply-accumulate count follow their definitions, and the training
checkpoint format round-trips and detects damage."""
import numpy as np
import pytest

import bench
from oracle import flnr_ref
from paper_2410_11625_gb300 import flnr, flnr_train


def test_layer_table_matches_the_oracle_network():
    assert [(n, ci, co, k) for n, ci, co, k in flnr.LAYERS] == \
        [(n, ci, co, k) for n, _, ci, co, k in flnr_ref.LAYERS]


@pytest.mark.parametrize("outputs", [8, 16])
def test_parameter_count_and_flat_layout(tmp_path, outputs):
    import __graft_entry__
    __graft_entry__.build()
    n = sum(co * ci * k * k + co for _, ci, co, k in flnr.layers(outputs))
    assert flnr._lib().flnr_param_count(outputs) == n
    assert flnr._lib().flnr_param_count(12) == 0  # 8 or 16 outputs only
    p = flnr.init_weights(3, outputs)
    flat = flnr.flatten(p)
    assert flat.dtype == np.float32 and flat.size == n
    q = flnr.unflatten(flat, outputs)
    assert set(q) == set(p) and all(np.array_equal(q[k], p[k]) for k in p)
    # the first layer's weights lead, its biases follow, then the next layer
    ci, co, k = flnr.LAYERS[0][1:]
    assert np.array_equal(flat[:co * ci * k * k], p["in0.w"].ravel())
    assert np.array_equal(flat[co * ci * k * k:co * ci * k * k + co], p["in0.b"])


@pytest.mark.parametrize("outputs", [8, 16])
def test_initialisation_matches_the_oracle(outputs):
    a, b = flnr.init_weights(7, outputs), flnr_ref.init_weights(7, outputs)
    assert set(a) == set(b) and all(np.array_equal(a[k], b[k]) for k in a)
    assert a["o1.w"].shape == (outputs, 16, 1, 1)
    bound = np.sqrt(6.0 / (16 * 1 * 1)) * 0.1  # o1 at a tenth of its He bound
    assert np.max(np.abs(a["o1.w"])) <= bound and np.all(a["o1.b"] == 0)


def test_training_crops_are_windows_of_the_scenes():
    rng = np.random.default_rng(0)
    H, W, crop = 20, 24, 8
    scenes = []
    for s in range(3):
        x = rng.normal(size=(11, H, W)).astype(np.float32)
        extra = rng.normal(size=(2, 3, H, W)).astype(np.float32)
        scenes.append((x, rng.normal(size=(3, H, W)).astype(np.float32), x[:3].copy(), extra))
    xs, rs = flnr_train.sample_batch(np.random.default_rng(5), scenes, 16, crop)
    xs2, rs2 = flnr_train.sample_batch(np.random.default_rng(5), scenes, 16, crop)
    assert np.array_equal(xs, xs2) and np.array_equal(rs, rs2)  # seeded
    for b in range(16):
        found = False
        for x, ref, _, extra in scenes:
            for rad in [x[8:]] + list(extra):
                full = np.concatenate([x[:8], rad])
                for fy in (False, True):
                    for fx in (False, True):
                        f = full[:, ::-1] if fy else full
                        f = f[:, :, ::-1] if fx else f
                        r = ref[:, ::-1] if fy else ref
                        r = r[:, :, ::-1] if fx else r
                        for i in range(H - crop + 1):
                            for j in range(W - crop + 1):
                                if np.array_equal(f[:, i:i + crop, j:j + crop], xs[b]):
                                    assert np.array_equal(r[:, i:i + crop, j:j + crop], rs[b])
                                    found = True
        assert found, b


def test_psnr_definition():
    a = np.full((3, 4, 4), 0.5)
    assert flnr_train.psnr(a + 0.1, a) == pytest.approx(20.0)
    assert flnr_train.psnr(a, a) == pytest.approx(200.0)  # mean square error floored at 1e-20
    assert flnr_train.psnr(np.full((3, 2, 2), 2.0), np.ones((3, 2, 2))) == pytest.approx(200.0)  # clamped to [0, 1]


def test_bench_multiply_accumulates_per_pixel():
    # output resolution of each layer (Sec. 3.3: the second convolution of an encoder block
    # strides by 2): full for in*, e1a, d0*, o*; half for e1b, e2a, d1*; quarter for e2b
    scale = {"in0": 1, "in1": 1, "e1a": 1, "e1b": 4, "e2a": 4, "e2b": 16, "d1a": 4, "d1b": 4,
             "d0a": 1, "d0b": 1, "o0": 1, "o1": 1}
    macs = sum(ci * co * k * k / scale[n] for n, ci, co, k in flnr.LAYERS)
    assert bench.FLNR_MACS_PER_PIXEL == pytest.approx(macs) == pytest.approx(36528.0)


def test_checkpoint_file_round_trip_and_damage_detection():
    """The checkpoint format (magic, JSON header, float32 state, CRC-32) round-trips the state,
    the metadata and a numpy generator's state exactly, and rejects damaged files."""
    from paper_2410_11625_gb300 import flnr_train as ft
    state = np.random.default_rng(0).standard_normal(3 * 1000).astype(np.float32)
    rng = np.random.default_rng(5)
    rng.integers(10, size=7)
    blob = ft.pack_checkpoint(state, {"steps": 3, "lr": 2e-3, "rng": rng.bit_generator.state})
    got, meta = ft.unpack_checkpoint(blob)
    assert np.array_equal(got, state) and meta["steps"] == 3 and meta["lr"] == 2e-3
    again = np.random.Generator(getattr(np.random, meta["rng"]["bit_generator"])())
    again.bit_generator.state = meta["rng"]
    assert np.array_equal(again.integers(1 << 30, size=8), rng.integers(1 << 30, size=8))
    damaged = bytearray(blob)
    damaged[len(blob) // 2] ^= 0x10
    with pytest.raises(ValueError, match="CRC"):
        ft.unpack_checkpoint(bytes(damaged))
    with pytest.raises(ValueError, match="not an FLNR checkpoint"):
        ft.unpack_checkpoint(b"XXXXXXXX" + blob[8:])
    with pytest.raises(ValueError):
        ft.unpack_checkpoint(blob[:-9] + blob[-4:])  # truncated payload, CRC no longer matches
