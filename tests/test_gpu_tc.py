"""tcgen05 BF16 GEMM core against a plain FP32 matmul of the same BF16 inputs (needs a B300)."""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2607_24059_b300 as v  # noqa: E402
import math  # noqa: E402


@pytest.mark.parametrize("M,N,K", [(128, 64, 64), (256, 16, 128), (384, 128, 576), (128, 256, 64), (128, 48, 192)])
def test_tc_gemm_matches_matmul(M, N, K):
    g = torch.Generator(device="cuda").manual_seed(M + N + K)
    A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
    D = torch.full((M, N), float("nan"), device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    v.vlbm_tc_gemm_bf16(A, B, D, err)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    ref = A.double() @ B.double().T           # products of BF16 values are exact in FP32
    scale = (A.double().abs() @ B.double().abs().T).max().item()
    assert torch.isfinite(D).all()
    assert (D.double() - ref).abs().max().item() <= 1e-6 * scale


def torch_conv_periodic(X, W, bias, act):
    """Reference: X (B, H, W, cin) bf16 NHWC, W (cout, 9, cin) -> FP64 NHWC via conv2d with circular
    padding (the BF16 inputs are exact in FP64), and GELU in its tanh form."""
    import torch.nn.functional as F
    cout, _, cin = W.shape
    w = W.double().reshape(cout, 3, 3, cin).permute(0, 3, 1, 2)          # (cout, cin, kh, kw)
    x = X.double().permute(0, 3, 1, 2)
    z = F.conv2d(F.pad(x, (1, 1, 1, 1), mode="circular"), w) + bias.double().view(1, -1, 1, 1)
    y = F.gelu(z, approximate="tanh") if act else z
    return y.permute(0, 2, 3, 1), z.permute(0, 2, 3, 1)


@pytest.mark.parametrize("cin,cout", [(16, 64), (64, 64), (64, 16), (16, 16)])
@pytest.mark.parametrize("shape", [(2, 16, 32), (1, 8, 24), (3, 5, 7), (1, 37, 200), (2, 64, 256), (1, 1, 130)])
def test_conv3x3_periodic_matches_torch(cin, cout, shape):
    B, H, Wd = shape
    g = torch.Generator(device="cuda").manual_seed(cin * 7 + cout + H)
    X = torch.randn(B, H, Wd, cin, device="cuda", generator=g).to(torch.bfloat16)
    W = (torch.randn(cout, 9, cin, device="cuda", generator=g) * 0.1).to(torch.bfloat16)
    bias = torch.randn(cout, device="cuda", generator=g)
    for act in (True, False):
        Y = torch.empty(B, H, Wd, cout, device="cuda", dtype=torch.bfloat16)
        Z = torch.empty_like(Y) if act else None
        err = torch.zeros(1, dtype=torch.int32, device="cuda")
        v.vlbm_sur_conv3x3(X, W, bias, Y, err, act=act, Z=Z)
        torch.cuda.synchronize()
        assert int(err.item()) == 0
        ry, rz = torch_conv_periodic(X, W, bias, act)
        # element by element: the kernel accumulates the 9 cin exact BF16 products in FP32 (an
        # error of a few 1e-6 of the largest output; 1e-4 allowed) and rounds once to BF16 (half an
        # ulp, 2^-9 of the value; 2^-8 allowed); GELU adds the tanh approximation's error, at most
        # 2^-11 in tanh, which is 2^-12 |z| in 0.5 z (1 + tanh) (2^-11 |z| allowed)
        acc = 1e-4 * rz.abs().max().item()
        bound_y = 2.0 ** -8 * ry.abs() + (2.0 ** -11 * rz.abs() if act else 0.0) + acc
        assert torch.all((Y.double() - ry).abs() <= bound_y), float(((Y.double() - ry).abs() - bound_y).max())
        if act:
            bound_z = 2.0 ** -8 * rz.abs() + acc
            assert torch.all((Z.double() - rz).abs() <= bound_z), float(((Z.double() - rz).abs() - bound_z).max())


def ref_wgrad(X, dZ):
    """FP64 CPU weight and bias gradients of the periodic conv: G[co][tap][ci] = sum_p dZ[p][co] X[p + tap][ci]."""
    x, dz = X.double().cpu(), dZ.double().cpu()
    cin, cout = x.shape[3], dz.shape[3]
    G = torch.zeros(cout, 9, cin, dtype=torch.float64)
    for tap in range(9):
        dy, dx = tap // 3 - 1, tap % 3 - 1
        xs = torch.roll(x, shifts=(-dy, -dx), dims=(1, 2))          # xs[y][x] = x[y + dy][x + dx]
        G[:, tap, :] = dz.reshape(-1, cout).T @ xs.reshape(-1, cin)
    return G, dz.reshape(-1, cout).sum(0)


@pytest.mark.parametrize("cin,cout", [(16, 64), (64, 64), (64, 16)])
@pytest.mark.parametrize("shape", [(2, 16, 32), (3, 40, 72), (1, 5, 7), (3, 97, 131)])
def test_conv3x3_wgrad_matches_fp64(cin, cout, shape):
    B, H, Wd = shape
    g = torch.Generator(device="cuda").manual_seed(cin + cout * 3 + H * Wd)
    X = torch.randn(B, H, Wd, cin, device="cuda", generator=g).to(torch.bfloat16)
    dZ = torch.randn(B, H, Wd, cout, device="cuda", generator=g).to(torch.bfloat16)
    G = torch.zeros(cout, 9, cin, device="cuda")
    Gb = torch.zeros(cout, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    v.vlbm_sur_conv3x3_wgrad(X, dZ, G, Gb, err)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    rG, rGb = ref_wgrad(X, dZ)
    scale = float(B * H * Wd) * 16.0                                # bound of sum |dZ||X| for these draws
    assert (G.double().cpu() - rG).abs().max().item() <= 1e-6 * scale
    assert (Gb.double().cpu() - rGb).abs().max().item() <= 1e-6 * scale


def ste_bf16(t):
    """Round to BF16 in the forward pass, identity in the backward pass."""
    return t + (t.to(torch.bfloat16).float() - t).detach()


def torch_surrogate(params, u, channels=2):
    """FP32 reference of the surrogate network with the kernels' BF16 roundings of weights and activations;
    returns the first `channels` output channels."""
    import torch.nn.functional as F
    B, C, H, W = u.shape
    x = torch.zeros(B, 16, H, W, device=u.device)
    x = torch.cat([u, x[:, C:]], dim=1)
    x = ste_bf16(x)
    layers = v.Surrogate.split_params(params)
    for l, (Wl, bl) in enumerate(layers):
        cout, _, cin = Wl.shape
        w = ste_bf16(Wl).reshape(cout, 3, 3, cin).permute(0, 3, 1, 2)
        z = F.conv2d(F.pad(x, (1, 1, 1, 1), mode="circular"), w) + bl.view(1, -1, 1, 1)
        x = ste_bf16(F.gelu(z, approximate="tanh") if l < len(layers) - 1 else z)
    return x[:, :channels]


def smooth_fields(B, H, W, seed):
    g = torch.Generator(device="cuda").manual_seed(seed)
    u = torch.randn(B, 2, H, W, device="cuda", generator=g)
    for _ in range(3):                                               # a few box filters: smooth random flow
        u = (u + u.roll(1, 2) + u.roll(-1, 2) + u.roll(1, 3) + u.roll(-1, 3)) / 5.0
    return (u / u.abs().max()).contiguous()


def laplacian(u):
    return u.roll(1, 2) + u.roll(-1, 2) + u.roll(1, 3) + u.roll(-1, 3) - 4 * u


# ------------------------------------------------------------ element-wise gradient check
#
# The kernels round to BF16 at fixed points: the input, every activation and pre-activation
# (forward), the loss gradient, every data gradient and every GELU-backward product
# (backward); the weight gradients accumulate exact BF16 products in FP32.  The reference
# below rounds at the same points (FP32 torch arithmetic in between), so kernel and reference
# differ only by FP32 accumulation order and the hardware tanh of the GELU, which now and then
# flip one BF16 rounding by one unit (at most 2u relative, u = 2^-8).  Treating each term
# dZ[p] X[p + tap] of a weight gradient as perturbed independently by at most 4u of itself
# (a flip in either factor), the error of G has a standard deviation of at most 4u S with
# S = sqrt(sum_p (dZ[p] X[p + tap])^2); the check allows 6 of those (24u S) plus 1e-5 of the
# absolute sum for FP32 accumulation.  A wrong tap, channel or sign changes an element by
# the order of |G| itself.
BF16_U = 2.0 ** -8


def bf16(t):
    return t.to(torch.bfloat16).float()


def conv_periodic_nchw(x, Wt):
    """x (B, cin, H, W), Wt (cout, 9, cin) -> (B, cout, H, W), periodic 3x3 conv, FP32."""
    import torch.nn.functional as F
    cout, _, cin = Wt.shape
    return F.conv2d(F.pad(x, (1, 1, 1, 1), mode="circular"), Wt.reshape(cout, 3, 3, cin).permute(0, 3, 1, 2))


def gelu_tanh_grad(z):
    k, a = math.sqrt(2.0 / math.pi), 0.044715
    t = torch.tanh(k * (z + a * z ** 3))
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * k * (1.0 + 3.0 * a * z * z)


def wgrad_fp64(X, dZ):
    """G[co][tap][ci] = sum_p dZ[p][co] X[p + tap][ci] in FP64 (X, dZ as NCHW)."""
    G = torch.empty(dZ.shape[1], 9, X.shape[1], dtype=torch.float64, device=X.device)
    for tap in range(9):
        dy, dx = tap // 3 - 1, tap % 3 - 1
        xs = torch.roll(X, shifts=(-dy, -dx), dims=(2, 3)).double()
        G[:, tap, :] = torch.einsum("bohw,bihw->oi", dZ.double(), xs)
    return G


def replicated_gradients(params, u, target, channels, curl=False):
    """Per layer (G, Gb, bound_G, bound_Gb) with the kernels' BF16 rounding points, and the loss."""
    import torch.nn.functional as F
    B, C, H, W = u.shape
    layers = v.Surrogate.split_params(params)
    X = torch.zeros(B, 16, H, W, device=u.device)
    X[:, :C] = u
    X = bf16(X)
    xs, zb = [], []
    for l, (Wl, bl) in enumerate(layers):
        xs.append(X)
        z = conv_periodic_nchw(X, bf16(Wl)) + bl.view(1, -1, 1, 1)
        if l < len(layers) - 1:
            zb.append(bf16(z))
            X = bf16(F.gelu(z, approximate="tanh"))
        else:
            Y = bf16(z)
    npix = B * H * W
    inv = 1.0 / (C * npix)
    dY = torch.zeros_like(Y)
    if curl:
        psi = Y[:, 0]
        ddy = 0.5 * (psi.roll(-1, 1) - psi.roll(1, 1))
        ddx = 0.5 * (psi.roll(-1, 2) - psi.roll(1, 2))
        rx, ry = ddy - target[:, 0], -ddx - target[:, 1]
        rc = Y[:, 2:C] - target[:, 2:C]
        loss = float(((rx.double() ** 2).sum() + (ry.double() ** 2).sum() + (rc.double() ** 2).sum()) * inv)
        g = rx.roll(1, 1) - rx.roll(-1, 1) + ry.roll(-1, 2) - ry.roll(1, 2)
        dY[:, 0] = bf16(g * inv)
        dY[:, 2:C] = bf16(2.0 * rc * inv)
    else:
        d = Y[:, :C] - target
        loss = float((d.double() ** 2).sum() * inv)
        dY[:, :C] = bf16(2.0 * d * inv)
    out = [None] * len(layers)
    dZ = dY
    for l in range(len(layers) - 1, -1, -1):
        G = wgrad_fp64(xs[l], dZ)
        Gb = dZ.double().sum(dim=(0, 2, 3))
        S = wgrad_fp64(xs[l] ** 2, dZ ** 2).sqrt()
        A = wgrad_fp64(xs[l].abs(), dZ.abs())
        Sb = (dZ.double() ** 2).sum(dim=(0, 2, 3)).sqrt()
        Ab = dZ.double().abs().sum(dim=(0, 2, 3))
        out[l] = (G, Gb, 24 * BF16_U * S + 1e-5 * A, 24 * BF16_U * Sb + 1e-5 * Ab)
        if l == 0:
            break
        Wflip = bf16(layers[l][0]).flip(1).permute(2, 1, 0).contiguous()   # [ci][8 - tap][co]
        dYp = bf16(conv_periodic_nchw(dZ, Wflip))
        dZ = bf16(dYp * gelu_tanh_grad(zb[l - 1]))
    return out, loss


def assert_gradients_elementwise(grads, ref):
    for l, ((gk, bk), (G, Gb, bound, bound_b)) in enumerate(zip(v.Surrogate.split_params(grads), ref)):
        err = (gk.double() - G).abs()
        assert torch.all(err <= bound + 1e-30), (l, float((err - bound).max()), int((err > bound).sum()))
        errb = (bk.double() - Gb).abs()
        assert torch.all(errb <= bound_b + 1e-30), (l, "bias", float((errb - bound_b).max()))


@pytest.fixture
def no_tf32():
    old = torch.backends.cudnn.allow_tf32, torch.backends.cuda.matmul.allow_tf32
    torch.backends.cudnn.allow_tf32 = False
    torch.backends.cuda.matmul.allow_tf32 = False
    yield
    torch.backends.cudnn.allow_tf32, torch.backends.cuda.matmul.allow_tf32 = old


@pytest.mark.parametrize("shape", [(2, 32, 48), (1, 20, 12)])
def test_surrogate_forward_matches_torch(shape, no_tf32):
    B, H, W = shape
    net = v.Surrogate(H, W, max_batch=B, seed=7)
    # larger last layer than the initialisation so that the output is not tiny
    p = net.params()
    layers = v.Surrogate.split_params(p)
    layers[4][0].mul_(10.0)
    layers[4][0][2:].zero_()
    net.load_params(p)
    u = smooth_fields(B, H, W, seed=H)
    du = net.forward(u)
    net.status()
    ref = torch_surrogate(p, u)
    assert torch.isfinite(du).all()
    assert (du - ref).abs().max().item() <= 2e-2 * ref.abs().max().item()
    net.close()


def test_surrogate_gradients_match_autograd(no_tf32):
    B, H, W = 2, 24, 32
    net = v.Surrogate(H, W, max_batch=B, seed=3)
    p0 = net.params()
    u = smooth_fields(B, H, W, seed=1)
    target = (0.05 * laplacian(u)).contiguous()
    loss = net.train_step(u, target, lr=0.0)
    grads = net.grads()
    w = p0.clone().requires_grad_(True)
    out = torch_surrogate(w, u)
    ref_loss = ((out - target) ** 2).mean()
    ref_loss.backward()
    assert abs(loss - ref_loss.item()) <= 1e-2 * ref_loss.item()
    # the replicated-rounding reference is the gradient: against autograd of the FP32 network
    # (norm, per tensor: they differ by the backward roundings only)
    rep, rep_loss = replicated_gradients(p0, u, target, 2)
    for l, ((G, Gb, _, _), (gr, br)) in enumerate(zip(rep, v.Surrogate.split_params(w.grad))):
        for a, b in ((G, gr), (Gb, br)):
            nb = b.norm().item()
            assert (a.float() - b).norm().item() <= 5e-2 * nb + 1e-30, f"reference layer {l}"
    # the kernels element by element against the replicated reference
    assert abs(loss - rep_loss) <= 1e-3 * rep_loss
    assert_gradients_elementwise(grads, rep)
    # padding stays exactly zero: layer 1 inputs 2..15, layer 5 outputs 2..15
    g = v.Surrogate.split_params(grads)
    assert g[0][0][:, :, 2:].abs().max().item() == 0.0
    assert g[4][0][2:].abs().max().item() == 0.0 and g[4][1][2:].abs().max().item() == 0.0
    net.close()


def test_surrogate_training_reduces_loss():
    B, H, W = 4, 32, 32
    net = v.Surrogate(H, W, max_batch=B, seed=11)
    u = smooth_fields(B, H, W, seed=5)
    target = (0.05 * laplacian(u)).contiguous()
    losses = [net.train_step(u, target, lr=2e-3) for _ in range(150)]
    net.status()
    assert all(map(lambda x: x == x, losses))
    assert losses[-1] < 0.1 * losses[0]
    p = net.params()
    layers = v.Surrogate.split_params(p)
    assert layers[0][0][:, :, 2:].abs().max().item() == 0.0
    assert layers[4][0][2:].abs().max().item() == 0.0
    # parameters round-trip through load_params
    net2 = v.Surrogate(H, W, max_batch=B, seed=99)
    net2.load_params(p)
    assert torch.equal(net2.forward(u), net.forward(u))
    net.close()
    net2.close()


def curl_increment(y, s0=1.0):
    """(D_y psi, -D_x psi) of psi = y[:, 0] with periodic central differences; channels >= 2 unchanged."""
    psi = y[:, 0]
    dx = 0.5 * (psi.roll(-1, 2) - psi.roll(1, 2))
    dy = 0.5 * (psi.roll(-1, 1) - psi.roll(1, 1))
    return torch.cat([(s0 * dy)[:, None], (-s0 * dx)[:, None], y[:, 2:]], 1)


def test_curl_increment_matches_torch_and_is_divergence_free():
    B, H, W = 2, 24, 40
    net = v.Surrogate(H, W, max_batch=B, channels=3, curl_output=True, seed=8)
    net.set_scaling([1.0, 1.0, 0.5], [0.3, 0.3, 0.2])
    u = smooth_fields(B, H, W, seed=2)
    u = torch.cat([u, 0.5 * u[:, :1]], 1).contiguous()
    y = net.forward(u)
    du = net.increment(u)
    ref = curl_increment(y, 0.3)
    ref[:, 2] *= 0.2
    assert torch.allclose(du, ref, rtol=1e-6, atol=1e-7)
    nxt = net.advance(u)
    assert torch.allclose(nxt, u + ref, rtol=1e-6, atol=1e-6)
    st = torch.empty(B, 3, dtype=torch.float64, device="cuda")
    v.vlbm_field_stats(du, st)
    assert (st[:, 1] / st[:, 2]).max().item() <= 1e-10      # central-difference divergence vanishes
    net.close()


def test_curl_gradients_match_autograd(no_tf32):
    B, H, W = 2, 24, 32
    net = v.Surrogate(H, W, max_batch=B, channels=3, curl_output=True, seed=4)
    p0 = net.params()
    u = smooth_fields(B, H, W, seed=6)
    u = torch.cat([u, 0.5 * u[:, 1:2]], 1).contiguous()
    target = torch.cat([0.05 * laplacian(u[:, :2]), 0.1 * u[:, 2:3]], 1).contiguous()
    loss = net.train_step(u, target, lr=0.0)
    grads = net.grads()
    w = p0.clone().requires_grad_(True)
    pred = curl_increment(torch_surrogate(w, u, channels=3))
    ref_loss = ((pred - target) ** 2).mean()
    ref_loss.backward()
    assert abs(loss - ref_loss.item()) <= 1e-2 * ref_loss.item()
    rep, rep_loss = replicated_gradients(p0, u, target, 3, curl=True)
    for l, ((G, Gb, _, _), (gr, br)) in enumerate(zip(rep, v.Surrogate.split_params(w.grad))):
        for a, b in ((G, gr), (Gb, br)):
            nb = b.norm().item()
            assert (a.float() - b).norm().item() <= 5e-2 * nb + 1e-30, f"reference layer {l}"
    assert abs(loss - rep_loss) <= 1e-3 * rep_loss
    assert_gradients_elementwise(grads, rep)
    g = v.Surrogate.split_params(grads)
    assert g[4][0][1].abs().max().item() == 0.0 and g[4][1][1].item() == 0.0     # channel 1 unused
    net.close()
