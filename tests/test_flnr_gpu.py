"""FLNR on the GPU (Sec. 3.3) against the FP64 network oracle (oracle/flnr_ref.py).

Per layer (flnr_layer, the kernels the network launches, on the same bfloat16 inputs as
the oracle): forward, masked and unmasked input gradient and weight gradient, element by
element within a bound derived from the arithmetic.  Layers 3 and 5 (the second
convolution of each encoder block) stride by 2 (Sec. 3.3) and are compared with float64
library convolutions of stride 2.  A kernel computes a sum of n
products of bfloat16 values in FP32 and, for stored results, rounds the sum to bfloat16
(round to nearest even).  The products are exact in FP32; the accumulation error is at
most n * 2^-23 * S, with S the sum of the absolute values of the terms (twice the
textbook n * u bound, since the tensor-core accumulation order and rounding are not
specified); the final rounding to bfloat16 (8 significant bits, unit roundoff 2^-8)
adds at most 2^-8 of the value.  So
    |gpu - ref| <= 2^-8 |ref| + (1 + 2^-8) n 2^-23 S.
The whole network, whose bfloat16 roundings cascade, is compared with the oracle's
BF16-storage mode (same rounding points, so the same ReLU decisions except where an FP32
sum lands next to a bfloat16 rounding boundary), and end to end through FLR by a
directional finite difference.  Adam and the L1 loss are checked against their formulas.
"""
import numpy as np
import pytest
import torch
import torch.nn.functional as F

from helpers import to_dev
from oracle import flnr_ref
from paper_2410_11625_gb300 import flnr
from paper_2410_11625_gb300 import flr as flrmod

pytestmark = pytest.mark.gpu


def pad16(c):
    return 16 * ((c + 15) // 16)


def params_with_bias(seed, outputs=8):
    rng = np.random.default_rng(seed + 100)
    p = flnr_ref.init_weights(seed, outputs)
    for k in p:
        if k.endswith(".b"):
            p[k] = rng.normal(scale=0.1, size=p[k].shape).astype(np.float32)
    return p


def bf16_tensor(a):
    """(CUDA bfloat16 tensor, its exact values as float64 numpy)."""
    t = torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda().to(torch.bfloat16)
    return t, t.float().cpu().numpy().astype(np.float64)


def nchw(a):
    return torch.from_numpy(np.ascontiguousarray(a.transpose(0, 3, 1, 2)))


def check_bound(got, ref, S, n, what):
    bound = 2.0 ** -8 * np.abs(ref) + (1 + 2.0 ** -8) * n * 2.0 ** -23 * S
    excess = np.abs(got - ref) - bound
    assert np.all(excess <= 0), f"{what}: {np.sum(excess > 0)} elements over the bound, worst {excess.max():.3e}"


SIZES = [(2, 20, 36), (1, 4, 4), (1, 68, 40)]
STRIDE = {3: 2, 5: 2}  # layer -> stride (1 for the others)


@pytest.fixture(scope="module")
def net():
    # the gradient ops of a stride-2 layer spread dz onto its input grid in the network's
    # scratch: room for 2 x 152 x 256 pixels x 64 channels
    return flnr.FLNR(2 * 2 * 152 * 256, params_with_bias(11))


@pytest.mark.parametrize("l", range(12))
@pytest.mark.parametrize("N,H,W", SIZES)
def test_layer_forward(net, l, N, H, W):
    name, cin, cout, k = flnr.LAYERS[l]
    rng = np.random.default_rng(1000 * l + H)
    net.set_weights(params_with_bias(11))
    p = params_with_bias(11)
    w = flnr_ref.round_bf16(torch.tensor(p[name + ".w"].astype(np.float64))).numpy()
    b = p[name + ".b"].astype(np.float64)
    # ReLU-like non-negative inputs in every channel, padding channels included (their
    # weights must be zero)
    x, xv = bf16_tensor(np.abs(rng.normal(size=(N, H, W, pad16(cin)))))
    s = STRIDE.get(l, 1)
    z = F.conv2d(nchw(xv[..., :cin]), torch.tensor(w), torch.tensor(b), stride=s, padding=k // 2).numpy()
    S = F.conv2d(nchw(np.abs(xv[..., :cin])), torch.tensor(np.abs(w)), torch.tensor(np.abs(b)), stride=s,
                 padding=k // 2).numpy()
    n = cin * k * k + 1
    if l == 11:
        out = torch.empty((N, 8, H, W), dtype=torch.float32, device="cuda")
        net.layer(l, net.OP_FORWARD, x, out=out)
        got = out.cpu().numpy().astype(np.float64)
        ref = 1.0 / (1.0 + np.exp(-z))
        assert np.max(np.abs(got - ref) - (0.25 * n * 2.0 ** -23 * S + 3e-7)) <= 0
        return
    out = torch.empty((N, H // s, W // s, pad16(cout)), dtype=torch.bfloat16, device="cuda")
    net.layer(l, net.OP_FORWARD, x, out=out)
    got = out.float().cpu().numpy().astype(np.float64)
    assert np.all(got[..., cout:] == 0)
    got = got[..., :cout].transpose(0, 3, 1, 2)
    check_bound(got, np.maximum(z, 0.0), S, n, f"{name} forward")
    exact = flnr_ref.round_bf16(torch.tensor(np.maximum(z, 0.0))).numpy()
    assert np.mean(got != exact) <= 0.01


@pytest.mark.parametrize("l,ca", [(6, 64), (8, 32)])
@pytest.mark.parametrize("N,H,W", SIZES + [(1, 544, 400)])
def test_decoder_layer_forms_the_concatenation_on_load(net, l, ca, N, H, W):
    """Layers 6 and 8 read up2(lo) ++ skip directly (the network's fused form: the four
    parity classes of each output block read the low-resolution map and the skip's parity
    planes).  544 x 400 gives every CTA several blocks."""
    name, cin, cout, k = flnr.LAYERS[l]
    rng = np.random.default_rng(4000 * l + H)
    p = params_with_bias(11)
    net.set_weights(p)
    w = flnr_ref.round_bf16(torch.tensor(p[name + ".w"].astype(np.float64))).numpy()
    b = p[name + ".b"].astype(np.float64)
    lo, lov = bf16_tensor(np.abs(rng.normal(size=(N, H // 2, W // 2, ca))))
    sk, skv = bf16_tensor(np.abs(rng.normal(size=(N, H, W, cin - ca))))
    xv = np.concatenate([lov.repeat(2, axis=1).repeat(2, axis=2), skv], axis=3)
    out = torch.empty((N, H, W, pad16(cout)), dtype=torch.bfloat16, device="cuda")
    net.layer(l, net.OP_FORWARD, lo, b=sk, out=out, size=(N, H, W))
    got = out.float().cpu().numpy().astype(np.float64)[..., :cout].transpose(0, 3, 1, 2)
    z = F.conv2d(nchw(xv), torch.tensor(w), torch.tensor(b), padding=1).numpy()
    S = F.conv2d(nchw(np.abs(xv)), torch.tensor(np.abs(w)), torch.tensor(np.abs(b)), padding=1).numpy()
    check_bound(got, np.maximum(z, 0.0), S, cin * 9 + 1, f"{name} fused concatenation")


@pytest.mark.parametrize("l", [3, 5])
@pytest.mark.parametrize("N,H,W", [(2, 544, 800), (1, 6, 1030)])
def test_stride_two_layer_many_tiles(net, l, N, H, W):
    """The stride-2 encoder convolutions on inputs that give every CTA several 16 x 8 output
    tiles (the staging ring and both accumulators wrap), a ragged last tile row and column
    (544 x 800 -> 272 x 400; 6 x 1030 -> 3 x 515), and signed inputs."""
    name, cin, cout, k = flnr.LAYERS[l]
    rng = np.random.default_rng(5000 * l + H)
    p = params_with_bias(11)
    net.set_weights(p)
    w = flnr_ref.round_bf16(torch.tensor(p[name + ".w"].astype(np.float64))).numpy()
    b = p[name + ".b"].astype(np.float64)
    x, xv = bf16_tensor(rng.normal(size=(N, H, W, pad16(cin))))
    out = torch.empty((N, H // 2, W // 2, pad16(cout)), dtype=torch.bfloat16, device="cuda")
    net.layer(l, net.OP_FORWARD, x, out=out)
    net.status()
    z = F.conv2d(nchw(xv[..., :cin]), torch.tensor(w), torch.tensor(b), stride=2, padding=1).numpy()
    S = F.conv2d(nchw(np.abs(xv[..., :cin])), torch.tensor(np.abs(w)), torch.tensor(np.abs(b)), stride=2,
                 padding=1).numpy()
    got = out.float().cpu().numpy().astype(np.float64)[..., :cout].transpose(0, 3, 1, 2)
    check_bound(got, np.maximum(z, 0.0), S, cin * 9 + 1, f"{name} stride-2 forward")


@pytest.mark.parametrize("l", range(12))
@pytest.mark.parametrize("masked", [False, True])
@pytest.mark.parametrize("N,H,W", SIZES[:2])
def test_layer_input_gradient(net, l, masked, N, H, W):
    name, cin, cout, k = flnr.LAYERS[l]
    rng = np.random.default_rng(2000 * l + 7 * H + masked)
    p = params_with_bias(11)
    net.set_weights(p)
    w = flnr_ref.round_bf16(torch.tensor(p[name + ".w"].astype(np.float64))).numpy()
    s = STRIDE.get(l, 1)
    dz, dzv = bf16_tensor(rng.normal(size=(N, H // s, W // s, pad16(cout))))
    mask = mv = None
    if masked:
        mask, mv = bf16_tensor(np.maximum(rng.normal(size=(N, H, W, pad16(cin))), 0.0))
    out = torch.empty((N, H, W, pad16(cin)), dtype=torch.bfloat16, device="cuda")
    net.layer(l, net.OP_DGRAD, dz, mask=mask, out=out, size=(N, H, W))
    got = out.float().cpu().numpy().astype(np.float64)
    assert np.all(got[..., cin:] == 0)
    got = got[..., :cin].transpose(0, 3, 1, 2)
    # the adjoint of a stride-s convolution with zero padding k // 2 onto the H x W input
    ref = F.conv_transpose2d(nchw(dzv[..., :cout]), torch.tensor(w), stride=s, padding=k // 2,
                             output_padding=s - 1).numpy()
    S = F.conv_transpose2d(nchw(np.abs(dzv[..., :cout])), torch.tensor(np.abs(w)), stride=s, padding=k // 2,
                           output_padding=s - 1).numpy()
    assert ref.shape[2:] == (H, W)
    if masked:
        keep = (mv[..., :cin] > 0).transpose(0, 3, 1, 2)
        assert np.all(got[~keep] == 0)
        ref, S = ref * keep, S * keep
    check_bound(got, ref, S, cout * k * k, f"{name} dgrad")


@pytest.mark.parametrize("l", range(12))
@pytest.mark.parametrize("N,H,W", [(2, 20, 36), (2, 152, 256)])
def test_layer_weight_gradient(net, l, N, H, W):
    name, cin, cout, k = flnr.LAYERS[l]
    rng = np.random.default_rng(3000 * l + H)
    net.set_weights(params_with_bias(11))
    s = STRIDE.get(l, 1)
    x, xv = bf16_tensor(np.abs(rng.normal(size=(N, H, W, pad16(cin)))))
    dz, dzv = bf16_tensor(rng.normal(size=(N, H // s, W // s, pad16(cout))))
    net.zero_grads(x)
    net.layer(l, net.OP_WGRAD, x, b=dz)
    torch.cuda.synchronize()
    g = flnr.unflatten(net.grads())
    xt = nchw(xv[..., :cin])
    wt = torch.zeros((cout, cin, k, k), dtype=torch.float64, requires_grad=True)
    F.conv2d(xt, wt, stride=s, padding=k // 2).backward(nchw(dzv[..., :cout]))
    wa = torch.zeros((cout, cin, k, k), dtype=torch.float64, requires_grad=True)
    F.conv2d(xt.abs(), wa, stride=s, padding=k // 2).backward(nchw(np.abs(dzv[..., :cout])))
    n = N * H * W  # the kernels sum over the input grid (zeros where a stride-2 dz is absent)
    bound = n * 2.0 ** -23 * wa.grad.numpy()
    assert np.all(np.abs(g[name + ".w"] - wt.grad.numpy()) <= bound), name
    db = dzv[..., :cout].sum(axis=(0, 1, 2))
    assert np.all(np.abs(g[name + ".b"] - db) <= n * 2.0 ** -23 * np.abs(dzv[..., :cout]).sum(axis=(0, 1, 2)))
    # the typical error is far below the worst-case bound
    rel = np.linalg.norm(g[name + ".w"] - wt.grad.numpy()) / np.linalg.norm(wt.grad.numpy())
    assert rel <= 1e-5, (name, rel)
    # other layers untouched
    for other, *_ in flnr.LAYERS:
        if other != name:
            assert not np.any(g[other + ".w"]) and not np.any(g[other + ".b"])


def network_case(N, H, W, seed):
    rng = np.random.default_rng(seed)
    x = rng.uniform(size=(N, 11, H, W)).astype(np.float32)
    x[:, 8:] = (0.2 * (1.0 - rng.uniform(size=(N, 3, H, W))) ** (-1.0 / 1.5)).astype(np.float32)  # heavy tail
    G = rng.normal(size=(N, 8, H, W)).astype(np.float32)
    return x, G


@pytest.mark.parametrize("N,H,W,outputs", [(2, 32, 48, 8), (1, 44, 52, 8), (1, 4, 4, 8), (2, 32, 48, 16)])
def test_network_matches_bf16_storage_oracle(N, H, W, outputs):
    """outputs = 16: the model and map guide sets of Sec. 3.3 from one 16-channel head."""
    p = params_with_bias(3, outputs)
    x, G = network_case(N, H, W, H)
    if outputs == 16:
        G = np.concatenate([G, -0.5 * G[:, ::-1]], axis=1)
    x[:, 8:, ::7, ::5] = -0.3  # negative radiance: the input transform's zero-gradient branch
    ref, g_ref = flnr_ref.forward_backward(x, p, G, bf16_storage=True)
    ref64, _ = flnr_ref.forward_backward(x, p, G)
    net = flnr.FLNR(N * H * W, p)
    out = net.forward(to_dev(x))
    net.zero_grads(out)
    g_in = torch.full((N, 11, H, W), float("nan"), device="cuda")
    net.backward(to_dev(G), grad_in=g_in)
    torch.cuda.synchronize()
    # dL/d(input): guides directly, radiance through log(1 + max(Y, 0)); zero where Y < 0
    gi, gi_ref = g_in.cpu().numpy().astype(np.float64), g_ref["input"]
    assert np.all(np.isfinite(gi)) and np.all(gi[:, 8:][x[:, 8:] < 0] == 0)
    for sl in (slice(0, 8), slice(8, 11)):
        a, b = gi[:, sl], gi_ref[:, sl]
        cos = np.sum(a * b) / max(np.linalg.norm(a) * np.linalg.norm(b), 1e-30)
        rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
        assert cos >= 0.998 and rel <= 6e-2, ("input", sl, cos, rel)
    got = out.cpu().numpy()
    err = np.abs(got - ref)
    # outputs in (0, 1): a bfloat16 unit at 1 is 2^-8; rounding flips near boundaries cascade
    # into a few such units at most, and rarely
    assert err.max() <= 8e-3 and np.sqrt(np.mean(err ** 2)) <= 1e-3, (err.max(), np.sqrt(np.mean(err ** 2)))
    assert np.sqrt(np.mean((got - ref64) ** 2)) <= 4e-3
    assert got.shape == (N, outputs, H, W)
    g = flnr.unflatten(net.grads(), outputs)
    for name, *_ in flnr.LAYERS:
        for s in (".w", ".b"):
            a, b = g[name + s].astype(np.float64), g_ref[name + s]
            # a ReLU decided differently at m of the P pixels moves a pixel-summed gradient by
            # about sqrt(m / P) of its size: rare flips stay within a few percent
            cos = np.sum(a * b) / max(np.linalg.norm(a) * np.linalg.norm(b), 1e-30)
            rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
            assert cos >= 0.998 and rel <= 6e-2, (name + s, cos, rel)


def test_training_step_gradient_matches_directional_difference():
    """d/dh of the L1 loss of FLR(FLNR(x)) along the normalised gradient equals |grad|."""
    import synth
    B, c = 4, 32
    flr = flrmod.FLR(q=8, radius=8, eps=1e-3)
    net = flnr.FLNR(B * c * c, flnr.init_weights(5))
    xs, refs = [], []
    for b in range(B):
        g, y, r = synth.render(50 + b, c, c, ref_spp=64)
        xs.append(np.concatenate([g, y]))
        refs.append(r)
    x, ref = to_dev(np.stack(xs)), to_dev(np.stack(refs))
    guides = torch.empty((B, 8, c, c), device="cuda")
    out = torch.empty((B, 3, c, c), device="cuda")
    w0 = net.get_weights()

    def loss_at(w):
        net.set_weights(w)
        net.forward(x, out=guides)
        for b in range(B):
            flr.denoise(guides[b], x[b, 8:11], out=out[b])
        return flnr.l1_loss(out, ref)

    loss, g_out = loss_at(w0)
    g_guides = torch.empty_like(guides)
    for b in range(B):
        flr.backward(guides[b], x[b, 8:11], g_out[b], grad_guide=g_guides[b])
    net.zero_grads(x)
    net.backward(g_guides)
    torch.cuda.synchronize()
    g = net.grads().astype(np.float64)
    d = g / np.linalg.norm(g)
    h = 1e-2
    fd = (float(loss_at(w0 + h * d)[0].item()) - float(loss_at(w0 - h * d)[0].item())) / (2 * h)
    assert abs(fd - np.linalg.norm(g)) <= 0.05 * np.linalg.norm(g), (fd, np.linalg.norm(g))


def test_adam_and_l1_match_their_formulas():
    rng = np.random.default_rng(9)
    p = params_with_bias(4)
    net = flnr.FLNR(16 * 16, p)
    x, G = network_case(1, 16, 16, 2)
    w = net.get_weights().astype(np.float64)
    m = np.zeros_like(w)
    v = np.zeros_like(w)
    lr, b1, b2, eps = 1e-3, 0.9, 0.999, 1e-8
    for t in (1, 2, 3):
        net.forward(to_dev(x))
        net.zero_grads(to_dev(x))
        net.backward(to_dev(G * t))
        torch.cuda.synchronize()
        g = net.grads().astype(np.float64)
        net.adam_step(t, lr=lr, beta1=b1, beta2=b2, eps=eps)
        torch.cuda.synchronize()
        m = b1 * m + (1 - b1) * g
        v = b2 * v + (1 - b2) * g * g
        w = w - lr * (m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps)
        got = net.get_weights()
        assert np.max(np.abs(got - w)) <= 1e-6 * max(1.0, np.abs(w).max()) + 1e-3 * lr
    pred = rng.normal(size=(2, 3, 17, 19)).astype(np.float32)
    ref = rng.normal(size=(2, 3, 17, 19)).astype(np.float32)
    pred.ravel()[:7] = ref.ravel()[:7]  # zero differences give a zero gradient
    loss, grad = flnr.l1_loss(to_dev(pred), to_dev(ref))
    d = pred.astype(np.float64) - ref
    assert abs(float(loss.item()) - np.abs(d).mean()) <= 1e-5
    assert np.array_equal(grad.cpu().numpy(), (np.sign(d) / d.size).astype(np.float32))


def test_smape_matches_its_formula():
    """Sec. 3.3's SMAPE loss mean |p - r| / (|p| + |r| + eps) and its gradient, against numpy;
    the gradient formula itself against central differences of the loss."""
    rng = np.random.default_rng(21)
    pred = rng.normal(size=(2, 3, 17, 19)).astype(np.float32)
    ref = rng.normal(size=(2, 3, 17, 19)).astype(np.float32)
    pred.ravel()[:5] = ref.ravel()[:5]  # zero differences
    pred.ravel()[5:9] = 0.0             # zero predictions
    eps = 1e-2
    loss, grad = flnr.smape_loss(to_dev(pred), to_dev(ref), eps=eps)
    p, r = pred.astype(np.float64), ref.astype(np.float64)
    D = np.abs(p) + np.abs(r) + eps
    L = np.mean(np.abs(p - r) / D)
    G = (np.sign(p - r) / D - np.abs(p - r) * np.sign(p) / D ** 2) / p.size
    assert abs(float(loss.item()) - L) <= 1e-5 * L
    assert np.max(np.abs(grad.cpu().numpy() - G)) <= 1e-6 * np.max(np.abs(G))
    f = lambda q: np.mean(np.abs(q - r) / (np.abs(q) + np.abs(r) + eps))
    for idx in [(0, 1, 3, 4), (1, 2, 16, 0), (0, 0, 8, 8)]:
        e = np.zeros_like(p)
        e[idx] = 1e-6
        assert abs((f(p + e) - f(p - e)) / 2e-6 - G[idx]) <= 1e-6 * max(1.0, abs(G[idx]) * p.size) / p.size
