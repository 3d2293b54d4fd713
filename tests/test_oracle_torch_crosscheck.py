"""A second, independent formulation of FLR pins the C oracle at sizes brute force cannot
reach: PyTorch CPU float64, in the shape of the paper's Fig. 3 (outer products of the guide
vector with itself and with the radiance, a window filter over each product plane, one
batched linear solve per pixel, the model applied to the guides), with the clipped box
window of the oracle instead of the figure's Gaussian, and the oracle's regulariser (eps on
the centred guide covariance of window means, the bias unpenalised).

The bias is a guide column of ones, so each pixel solves the augmented (Q + 1) x (Q + 1)
system of window means
    [ E[x x^T] + eps I   E[x] ] [ a ]   [ E[x y^T] ]
    [ E[x]^T             1    ] [ b ] = [ E[y]^T   ]
(eps on the guide rows only, bias unpenalised; Sec. 3.1's closed form with the Appendix's
centring eliminated: its Schur complement is the oracle's centred system).  Window means
are box sums of the zero-padded planes divided by the box sum of the ones plane (clipped
windows); torch.linalg.solve is an LU solve, the oracle a Cholesky of the centred system.
Coefficient averaging (rc > 0) averages a and b over the clipped radius-rc window.  The
formulation's reverse-mode automatic derivative pins the oracle's analytic adjoint too, and
the paper's fast FLR (Sec. 3.2, 3.2.1) written the same way pins the fast-FLR oracle."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")


def box_sum(planes, r):
    """Sum of each [C, H, W] plane over the clipped (2r + 1)^2 window (zero padding)."""
    c = planes.shape[0]
    k = torch.ones((c, 1, 2 * r + 1, 2 * r + 1), dtype=planes.dtype)
    return torch.nn.functional.conv2d(planes[None], k, padding=r, groups=c)[0]


def flr_torch(g, y, r, eps, rc):
    x = torch.from_numpy(np.asarray(g, np.float64))
    yy = torch.from_numpy(np.asarray(y, np.float64))
    q, H, W = x.shape
    xa = torch.cat([x, torch.ones((1, H, W), dtype=torch.float64)])  # guides and the bias column
    n = box_sum(torch.ones((1, H, W), dtype=torch.float64), r)[0]
    xx = box_sum(torch.einsum("ihw,jhw->ijhw", xa, xa).reshape(-1, H, W), r).reshape(q + 1, q + 1, H, W) / n
    xy = box_sum(torch.einsum("ihw,jhw->ijhw", xa, yy).reshape(-1, H, W), r).reshape(q + 1, 3, H, W) / n
    reg = torch.zeros((q + 1, q + 1), dtype=torch.float64)
    reg[:q, :q] = eps * torch.eye(q, dtype=torch.float64)
    A = torch.linalg.solve(xx.permute(2, 3, 0, 1) + reg, xy.permute(2, 3, 0, 1))  # [H, W, q+1, 3]
    if rc > 0:
        m = box_sum(torch.ones((1, H, W), dtype=torch.float64), rc)[0]
        A = (box_sum(A.permute(2, 3, 0, 1).reshape(-1, H, W), rc) / m).reshape(q + 1, 3, H, W).permute(2, 3, 0, 1)
    return torch.einsum("ihw,hwic->chw", xa, A).numpy()


@pytest.mark.parametrize("kind,H,W,r,rc", [
    ("random", 40, 52, 3, 2), ("random", 33, 47, 5, 0), ("rendered", 64, 64, 5, 5), ("rendered", 48, 80, 8, 0),
])
def test_oracle_matches_an_independent_torch_formulation(kind, H, W, r, rc):
    if kind == "random":
        g, y = synth.random_frame(17 + H, H, W, 8)
    else:
        g, y = synth.render(4, H, W)
    ref = oracle.flr_forward(g, y, r, 1e-3, coef_radius=rc)
    got = flr_torch(g, y, r, 1e-3, rc)
    scale = np.sqrt(np.mean(ref ** 2))
    assert np.max(np.abs(got - ref)) <= 1e-9 * scale


def flr_torch_t(x, yy, r, eps, rc, z=None):
    """flr_torch on tensors (differentiable in x, yy, eps and the map guide z, default x)."""
    q, H, W = x.shape
    xa = torch.cat([x, torch.ones((1, H, W), dtype=torch.float64)])
    n = box_sum(torch.ones((1, H, W), dtype=torch.float64), r)[0]
    xx = box_sum(torch.einsum("ihw,jhw->ijhw", xa, xa).reshape(-1, H, W), r).reshape(q + 1, q + 1, H, W) / n
    xy = box_sum(torch.einsum("ihw,jhw->ijhw", xa, yy).reshape(-1, H, W), r).reshape(q + 1, 3, H, W) / n
    mask = torch.zeros((q + 1, q + 1), dtype=torch.float64)
    mask[:q, :q] = torch.eye(q, dtype=torch.float64)
    A = torch.linalg.solve(xx.permute(2, 3, 0, 1) + eps * mask, xy.permute(2, 3, 0, 1))
    if rc > 0:
        m = box_sum(torch.ones((1, H, W), dtype=torch.float64), rc)[0]
        A = (box_sum(A.permute(2, 3, 0, 1).reshape(-1, H, W), rc) / m).reshape(q + 1, 3, H, W).permute(2, 3, 0, 1)
    za = xa if z is None else torch.cat([z, torch.ones((1, H, W), dtype=torch.float64)])
    return torch.einsum("ihw,hwic->chw", za, A)


@pytest.mark.parametrize("rc", [0, 3])
def test_oracle_map_guide_adjoint_matches_autograd(rc):
    """With a separate map guide z (Sec. 3.3's second guide set) the oracle returns the
    gradients of the model guides and of the map guide apart; both against autograd."""
    H, W, r = 26, 34, 3
    g, y = synth.random_frame(71, H, W, 8)
    z, _ = synth.random_frame(72, H, W, 8)
    G = np.random.default_rng(5).normal(size=(3, H, W))
    x = torch.tensor(np.asarray(g, np.float64), requires_grad=True)
    yy = torch.tensor(np.asarray(y, np.float64), requires_grad=True)
    zt = torch.tensor(np.asarray(z, np.float64), requires_grad=True)
    (flr_torch_t(x, yy, r, 1e-3, rc, z=zt) * torch.from_numpy(G)).sum().backward()
    ref = oracle.flr_backward(g, y, G, r, 1e-3, coef_radius=rc, map_guide=z)
    for name, got in (("guide", x.grad.numpy()), ("radiance", yy.grad.numpy()), ("map_guide", zt.grad.numpy())):
        scale = np.sqrt(np.mean(ref[name] ** 2))
        assert np.max(np.abs(got - ref[name])) <= 1e-11 * scale, name


@pytest.mark.parametrize("kind,H,W,r,rc", [("random", 24, 30, 3, 2), ("rendered", 32, 40, 4, 4)])
def test_oracle_adjoint_matches_autograd_of_the_torch_formulation(kind, H, W, r, rc):
    """The oracle's analytic adjoint (reverse mode through centring, Cholesky, bias and the
    average) against reverse-mode automatic differentiation of the independent formulation:
    gradients of <G, I> with respect to the guides (model and map guide alike), the radiance
    and eps."""
    if kind == "random":
        g, y = synth.random_frame(40 + H, H, W, 8)
    else:
        g, y = synth.render(6, H, W)
    G = np.random.default_rng(H).normal(size=(3, H, W))
    x = torch.tensor(np.asarray(g, np.float64), requires_grad=True)
    yy = torch.tensor(np.asarray(y, np.float64), requires_grad=True)
    e = torch.tensor(1e-3, dtype=torch.float64, requires_grad=True)
    (flr_torch_t(x, yy, r, e, rc) * torch.from_numpy(G)).sum().backward()
    ref = oracle.flr_backward(g, y, G, r, 1e-3, coef_radius=rc)
    for name, got in (("guide", x.grad.numpy()), ("radiance", yy.grad.numpy())):
        scale = np.sqrt(np.mean(ref[name] ** 2))
        assert np.max(np.abs(got - ref[name])) <= 1e-11 * scale, name
    assert abs(float(e.grad) - ref["eps"]) <= 1e-11 * abs(ref["eps"])


def fast_torch(g, y, F, sigma, taps, eps, z=None, s=1):
    """The paper's fast FLR (Sec. 3.2, 3.2.1) as array operations: block sums of the outer
    products of (1, x) with itself and with y over F x F blocks, a separable Gaussian over the
    block grid (weights exp(-d^2 / 2 sigma^2), |d| <= taps, clipped at the grid edge), the
    augmented ridge system of each block's weighted sums solved by LU, and the block models
    interpolated bilinearly between block centres ((i + 1/2) F s - 1/2 in output pixels,
    clamped to the outermost centres) and applied to the map guide."""
    x = torch.from_numpy(np.asarray(g, np.float64))
    yy = torch.from_numpy(np.asarray(y, np.float64))
    q, Hi, Wi = x.shape
    Hb, Wb = -(-Hi // F), -(-Wi // F)
    xa = torch.cat([torch.ones((1, Hi, Wi), dtype=torch.float64), x])

    def blocks(p):  # [C, Hi, Wi] -> block sums [C, Hb, Wb] (zero padding to whole blocks)
        pp = torch.nn.functional.pad(p, (0, Wb * F - Wi, 0, Hb * F - Hi))
        return pp.reshape(p.shape[0], Hb, F, Wb, F).sum(dim=(2, 4))

    S = blocks(torch.einsum("ihw,jhw->ijhw", xa, xa).reshape(-1, Hi, Wi)).reshape(q + 1, q + 1, Hb, Wb)
    T = blocks(torch.einsum("ihw,jhw->ijhw", xa, yy).reshape(-1, Hi, Wi)).reshape(q + 1, 3, Hb, Wb)
    d = torch.arange(-taps, taps + 1, dtype=torch.float64)
    w = torch.exp(-d * d / (2.0 * sigma * sigma))  # sigma may be a tensor (autograd)

    def blur(p):  # [C, Hb, Wb], separable, clipped (zero padding)
        c = p.shape[0]
        kx = w.reshape(1, 1, 1, -1).repeat(c, 1, 1, 1)
        ky = w.reshape(1, 1, -1, 1).repeat(c, 1, 1, 1)
        p = torch.nn.functional.conv2d(p[None], kx, padding=(0, taps), groups=c)
        return torch.nn.functional.conv2d(p, ky, padding=(taps, 0), groups=c)[0]

    S = blur(S.reshape(-1, Hb, Wb)).reshape(q + 1, q + 1, Hb, Wb)
    T = blur(T.reshape(-1, Hb, Wb)).reshape(q + 1, 3, Hb, Wb)
    n = S[0, 0]
    mask = torch.zeros((q + 1, q + 1), dtype=torch.float64)
    mask[1:, 1:] = torch.eye(q, dtype=torch.float64)
    A = torch.linalg.solve((S / n).permute(2, 3, 0, 1) + eps * mask, (T / n).permute(2, 3, 0, 1))  # [Hb, Wb, q+1, 3]
    zz = x if z is None else torch.from_numpy(np.asarray(z, np.float64))
    Ho, Wo = zz.shape[1:]
    P = F * s

    def axis(nout, nb):  # lower block index and weight per output coordinate
        u = ((torch.arange(nout, dtype=torch.float64) + 0.5) / P - 0.5).clamp(0, nb - 1)
        i0 = torch.floor(u).long().clamp(max=max(nb - 2, 0))
        i1 = (i0 + 1).clamp(max=nb - 1)
        return i0, i1, u - i0
    i0, i1, fy = axis(Ho, Hb)
    j0, j1, fx = axis(Wo, Wb)
    fy, fx = fy[:, None, None, None], fx[None, :, None, None]
    Ai = (1 - fy) * ((1 - fx) * A[i0][:, j0] + fx * A[i0][:, j1]) + fy * ((1 - fx) * A[i1][:, j0] + fx * A[i1][:, j1])
    za = torch.cat([torch.ones((1, Ho, Wo), dtype=torch.float64), zz])
    out = torch.einsum("ihw,hwic->chw", za, Ai)
    return out if torch.is_tensor(sigma) or torch.is_tensor(eps) else out.numpy()


@pytest.mark.parametrize("H,W,F,s,taps", [(64, 80, 8, 1, 3), (50, 70, 4, 1, 2), (40, 56, 4, 2, 3)])
def test_fast_oracle_matches_an_independent_torch_formulation(H, W, F, s, taps):
    g, y = synth.render(8, H, W)
    if s == 1:
        z = None
        ref = oracle.flr_fast(g, y, factor=F, sigma_blocks=1.25, taps=taps, eps=1e-3)
    else:  # joint upsampling: model guides and radiance at H x W, the map guide s times finer
        z = synth.render(8, H * s, W * s)[0]
        ref = oracle.flr_fast(g, y, factor=F, sigma_blocks=1.25, taps=taps, eps=1e-3, map_guide=z, scale=s)
    got = fast_torch(g, y, F, 1.25, taps, 1e-3, z=z, s=s)
    assert np.max(np.abs(got - ref)) <= 1e-10 * np.sqrt(np.mean(ref ** 2))


def test_fast_parameter_gradients_match_autograd():
    """Sec. 3.2 learns the blur's sigma and the regulariser by backpropagation; the oracle
    takes those derivatives by Richardson-extrapolated central differences of its FP64
    forward pass.  Reverse-mode automatic differentiation of the independent formulation
    gives them exactly."""
    H, W = 48, 64
    g, y = synth.render(9, H, W)
    G = np.random.default_rng(9).normal(size=(3, H, W))
    sig = torch.tensor(1.25, dtype=torch.float64, requires_grad=True)
    e = torch.tensor(1e-3, dtype=torch.float64, requires_grad=True)
    (fast_torch(g, y, 4, sig, 2, e) * torch.from_numpy(G)).sum().backward()
    ref = oracle.flr_fast_param_grads(g, y, G, factor=4, sigma_blocks=1.25, taps=2, eps=1e-3)
    assert abs(float(sig.grad) - ref["sigma"]) <= 1e-9 * abs(ref["sigma"])
    assert abs(float(e.grad) - ref["eps"]) <= 1e-9 * abs(ref["eps"])


def fast_appendix_torch(g, y, F, sigma, taps, eps_add, eps_mul):
    """Fast FLR with the Appendix's regularised normalised solve, through the un-normalised
    form it reduces to: per block a = (Wh + eps_add diag(Wh))^-1 D with
    Wh = W + eps_mul (m m^T + diag(m^2)) + eps_add I (W the centred guide covariance of the
    blurred window means, m the absolute guide means, D the centred guide-radiance
    covariance), b = mean(y) - a^T m; the oracle follows the printed steps (normalise by the
    standard deviations, solve with eps_add added, un-normalise)."""
    x = torch.from_numpy(np.asarray(g, np.float64))
    yy = torch.from_numpy(np.asarray(y, np.float64))
    q, Hi, Wi = x.shape
    Hb, Wb = -(-Hi // F), -(-Wi // F)
    xa = torch.cat([torch.ones((1, Hi, Wi), dtype=torch.float64), x])

    def blocks(p):
        pp = torch.nn.functional.pad(p, (0, Wb * F - Wi, 0, Hb * F - Hi))
        return pp.reshape(p.shape[0], Hb, F, Wb, F).sum(dim=(2, 4))

    d = torch.arange(-taps, taps + 1, dtype=torch.float64)
    w = torch.exp(-d * d / (2.0 * sigma * sigma))

    def blur(p):
        c = p.shape[0]
        p = torch.nn.functional.conv2d(p[None], w.reshape(1, 1, 1, -1).repeat(c, 1, 1, 1), padding=(0, taps), groups=c)
        return torch.nn.functional.conv2d(p, w.reshape(1, 1, -1, 1).repeat(c, 1, 1, 1), padding=(taps, 0), groups=c)[0]

    S = blur(blocks(torch.einsum("ihw,jhw->ijhw", xa, xa).reshape(-1, Hi, Wi))).reshape(q + 1, q + 1, Hb, Wb)
    T = blur(blocks(torch.einsum("ihw,jhw->ijhw", xa, yy).reshape(-1, Hi, Wi))).reshape(q + 1, 3, Hb, Wb)
    n = S[0, 0]
    m = (S[0, 1:] / n).permute(1, 2, 0)                     # [Hb, Wb, q] absolute guide means
    my = (T[0] / n).permute(1, 2, 0)                        # [Hb, Wb, 3]
    Wc = (S[1:, 1:] / n).permute(2, 3, 0, 1) - m[..., :, None] * m[..., None, :]
    D = (T[1:] / n).permute(2, 3, 0, 1) - m[..., :, None] * my[..., None, :]
    eye = torch.eye(q, dtype=torch.float64)
    Wh = Wc + eps_mul * (m[..., :, None] * m[..., None, :] + torch.diag_embed(m * m)) + eps_add * eye
    M = Wh + eps_add * torch.diag_embed(torch.diagonal(Wh, dim1=-2, dim2=-1))
    a = torch.linalg.solve(M, D)                            # [Hb, Wb, q, 3]
    b = my - torch.einsum("hwic,hwi->hwc", a, m)
    A = torch.cat([b[..., None, :], a], dim=-2)             # [Hb, Wb, q + 1, 3], bias first
    P = F

    def axis(nout, nb):
        u = ((torch.arange(nout, dtype=torch.float64) + 0.5) / P - 0.5).clamp(0, nb - 1)
        j0 = torch.floor(u).long().clamp(max=max(nb - 2, 0))
        return j0, (j0 + 1).clamp(max=nb - 1), u - j0
    i0, i1, fy = axis(Hi, Hb)
    j0, j1, fx = axis(Wi, Wb)
    fy, fx = fy[:, None, None, None], fx[None, :, None, None]
    Ai = (1 - fy) * ((1 - fx) * A[i0][:, j0] + fx * A[i0][:, j1]) + fy * ((1 - fx) * A[i1][:, j0] + fx * A[i1][:, j1])
    return torch.einsum("ihw,hwic->chw", xa, Ai).numpy()


@pytest.mark.parametrize("eps_add,eps_mul", [(1e-4, 0.0), (1e-5, 0.2), (1e-3, 1.0)])
def test_fast_appendix_oracle_matches_its_unnormalised_form(eps_add, eps_mul):
    g, y = synth.render(10, 48, 64)
    ref = oracle.flr_fast(g, y, factor=4, sigma_blocks=1.25, taps=2, appendix=(eps_add, eps_mul))
    got = fast_appendix_torch(g, y, 4, 1.25, 2, eps_add, eps_mul)
    assert np.max(np.abs(got - ref)) <= 1e-9 * np.sqrt(np.mean(ref ** 2))
