"""Warm-start network kernels (include/lbm_nn.h) against the FP64 oracle (oracle/nn_oracle.py)
and numpy, through the C ABI.

Tolerances follow the arithmetic: the GEMM accumulates exact BF16 x BF16 products in FP32, so
against an FP64 product of the same BF16-rounded operands it agrees to a few FP32 ulps of the
accumulated magnitude (1e-5 relative L2); a BF16 output adds one BF16 rounding (2^-8 relative per
element).  A whole layer rounds its input, weights and output to BF16 (3e-3 relative L2 against
FP64).  The network compounds that over its layers and is held to 3e-2 on the output and 5e-2 on
every parameter gradient, the error measured against the magnitudes of the terms the gradient
sums (sum_v |dL/dy| |x| for a weight, sum_v |dL/dy| for a bias): the first layer's weight gradient
over a white-noise input cancels to a twelfth of those magnitudes, so its plain relative error is
twelve times its rounding.  An index, flip or wiring mistake is off by order one either way.
"""
import numpy as np
import pytest

from oracle import nn_oracle as orc

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
from paper_2502_12955_gb300 import surrogate as sg  # noqa: E402


def _bf(x):
    """numpy FP64 copy of x rounded to BF16."""
    return torch.tensor(np.asarray(x, np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)


def _dev(x, dtype=torch.bfloat16):
    return torch.tensor(np.ascontiguousarray(x, np.float32)).to(device="cuda", dtype=dtype)


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("M,N,K,splits", [(128, 16, 64, 1), (256, 32, 192, 1), (384, 64, 576, 1),
                                          (512, 128, 1024, 1), (128, 48, 128, 1), (256, 16, 4096, 7),
                                          (128, 128, 2048, 16), (256, 256, 512, 1), (384, 768, 256, 1),
                                          (256, 512, 1024, 3)])
def test_gemm_fp32_against_fp64_product(M, N, K, splits):
    rng = np.random.default_rng(M + N + K)
    A, B = _bf(rng.standard_normal((M, K))), _bf(rng.standard_normal((N, K)))
    ns = sg.lbm_nn_gemm_splits(K, splits)
    out = torch.zeros((ns, M, N), dtype=torch.float32, device="cuda")
    sg.lbm_nn_gemm_tn(_dev(A), _dev(B), out, N, M, N, K, splits, sg.OUT_F32)
    red = torch.empty((M, N), dtype=torch.float32, device="cuda")
    sg.lbm_nn_reduce_splits(out, red, M * N, ns, M * N)
    sg.lbm_nn_status()
    assert _rel(red.cpu().numpy(), A @ B.T) < 1e-5


@pytest.mark.parametrize("relu", [False, True])
def test_gemm_bf16_epilogue_bias_relu(relu):
    rng = np.random.default_rng(7)
    M, N, K = 256, 64, 320
    A, B = _bf(rng.standard_normal((M, K))), _bf(rng.standard_normal((N, K)))
    bias = rng.standard_normal(N).astype(np.float32)
    out = torch.empty((M, N), dtype=torch.bfloat16, device="cuda")
    sg.lbm_nn_gemm_tn(_dev(A), _dev(B), out, N, M, N, K, 1, sg.OUT_BF16_RELU if relu else sg.OUT_BF16,
                      _dev(bias, torch.float32))
    sg.lbm_nn_status()
    want = A @ B.T + bias
    if relu:
        want = np.maximum(want, 0.0)
    got = out.float().cpu().numpy()
    assert np.all(np.abs(got - want) <= 2.0 ** -8 * np.abs(want) + 1e-6)


def test_gemm_rejects_bad_shapes():
    a = torch.zeros((128, 64), dtype=torch.bfloat16, device="cuda")
    c = torch.zeros((128, 16), dtype=torch.float32, device="cuda")
    for M, N, K in [(100, 16, 64), (128, 12, 64), (128, 16, 60)]:
        with pytest.raises(Exception):
            sg.lbm_nn_gemm_tn(a, a, c, 16, M, N, K)


def _conv_case(ci, co, shape=(8, 8, 16), seed=0):
    rng = np.random.default_rng(seed)
    D, H, W = shape
    x = _bf(rng.standard_normal((ci, D, H, W)))
    w = rng.standard_normal((co, ci, 3, 3, 3)) * np.sqrt(2.0 / (27 * ci))
    b = rng.standard_normal(co) * 0.1
    return x, w, b


def _chlast(x):
    """[C, D, H, W] -> channel-last [V][C] on the device."""
    return _dev(np.moveaxis(x, 0, -1).reshape(-1, x.shape[0]))


@pytest.mark.parametrize("ci,co", [(4, 16), (16, 32), (48, 16)])
def test_conv3_forward_against_oracle(ci, co):
    x, w, b = _conv_case(ci, co)
    D, H, W = x.shape[1:]
    V = D * H * W
    kp = sg.kpad(27 * ci)
    wk = torch.empty((co, kp), dtype=torch.bfloat16, device="cuda")
    sg.lbm_nn_pack_weights(_dev(w.reshape(co, ci, 27), torch.float32), wk, None, co, ci, kp, 0)
    col = torch.empty((V, kp), dtype=torch.bfloat16, device="cuda")
    sg.lbm_nn_im2col(_chlast(x), col, D, H, W, ci, kp, 0)
    y = torch.empty((V, co), dtype=torch.bfloat16, device="cuda")
    sg.lbm_nn_gemm_tn(col, wk, y, co, V, co, kp, 1, sg.OUT_BF16, _dev(b, torch.float32))
    sg.lbm_nn_status()
    want = orc.conv3d(x, w, b)
    got = np.moveaxis(y.float().cpu().numpy().reshape(D, H, W, co), -1, 0)
    assert _rel(got, want) < 3e-3
    # the same with BF16-rounded weights is exact up to FP32 accumulation and one output rounding
    want_bf = orc.conv3d(x, _bf(w), b)
    assert np.all(np.abs(got - want_bf) <= 2.0 ** -8 * np.abs(want_bf) + 1e-5)


@pytest.mark.parametrize("ci,co", [(16, 32), (32, 16), (4, 16)])
def test_conv3_gradients_against_oracle(ci, co):
    x, w, _ = _conv_case(ci, co, seed=1)
    D, H, W = x.shape[1:]
    V = D * H * W
    dy = _bf(np.random.default_rng(2).standard_normal((co, D, H, W)))
    kp, kpt = sg.kpad(27 * ci), sg.kpad(27 * co)
    wk = torch.empty((co, kp), dtype=torch.bfloat16, device="cuda")
    wt = torch.empty((ci, kpt), dtype=torch.bfloat16, device="cuda")
    sg.lbm_nn_pack_weights(_dev(w.reshape(co, ci, 27), torch.float32), wk, wt, co, ci, kp, kpt)
    # input gradient: convolution of dy with the flipped, transposed kernel (not taken for the
    # network's first layer, whose 4 input channels are no GEMM N tile)
    col = torch.empty((V * max(kp, kpt),), dtype=torch.bfloat16, device="cuda")
    dyd = _chlast(dy)
    dx = None
    if ci % 16 == 0:
        sg.lbm_nn_im2col(dyd, col, D, H, W, co, kpt, 0)
        dx = torch.empty((V, ci), dtype=torch.bfloat16, device="cuda")
        sg.lbm_nn_gemm_tn(col, wt, dx, ci, V, ci, kpt, 1, sg.OUT_BF16, None)
    # weight gradient: transposed im2col, split over voxels; the channel-major route builds the same
    # transposed columns bit for bit
    xd = _chlast(x)
    xT = torch.empty((ci, V), dtype=torch.bfloat16, device="cuda")
    sg.lbm_nn_transpose(xd, xT, V, ci)
    col2 = torch.empty((kp * V,), dtype=torch.bfloat16, device="cuda")
    sg.lbm_nn_im2col_cv(xT, col2, D, H, W, ci, kp)
    sg.lbm_nn_im2col(xd, col, D, H, W, ci, kp, 1)
    assert torch.equal(col[:kp * V], col2)
    # and the row layout's vector route equals the generic one (C % 8 == 0)
    if ci % 8 == 0:
        r1 = torch.empty((V * kp,), dtype=torch.bfloat16, device="cuda")
        sg.lbm_nn_im2col(xd, r1, D, H, W, ci, kp, 0)
        r2 = torch.zeros((V, kp), dtype=torch.float32)
        xh = np.moveaxis(x, 0, -1)
        for tap in range(27):
            dz, dy_, dx_ = tap // 9 - 1, (tap // 3) % 3 - 1, tap % 3 - 1
            sh = np.zeros_like(xh)
            zs = slice(max(0, -dz), D - max(0, dz)); zt = slice(max(0, dz), D - max(0, -dz))
            ys = slice(max(0, -dy_), H - max(0, dy_)); yt = slice(max(0, dy_), H - max(0, -dy_))
            xs = slice(max(0, -dx_), W - max(0, dx_)); xt = slice(max(0, dx_), W - max(0, -dx_))
            sh[zs, ys, xs] = xh[zt, yt, xt]
            r2[:, tap * ci:(tap + 1) * ci] = torch.tensor(sh.reshape(V, ci), dtype=torch.float32)
        assert torch.equal(r1.view(V, kp).float().cpu(), r2)
    dyT = torch.empty((co, V), dtype=torch.bfloat16, device="cuda")
    sg.lbm_nn_transpose(dyd, dyT, V, co)
    ns = sg.lbm_nn_gemm_splits(V, 8)
    part = torch.empty((ns, kp, co), dtype=torch.float32, device="cuda")
    sg.lbm_nn_gemm_tn(col, dyT, part, co, kp, co, V, 8, sg.OUT_F32)
    dwcol = torch.empty((kp, co), dtype=torch.float32, device="cuda")
    sg.lbm_nn_reduce_splits(part, dwcol, kp * co, ns, kp * co)
    dw = torch.empty((co, ci, 27), dtype=torch.float32, device="cuda")
    sg.lbm_nn_unpack_wgrad(dwcol, dw, co, ci)
    db = torch.empty(co, dtype=torch.float32, device="cuda")
    sg.lbm_nn_colsum(dyd, db, V, co)
    sg.lbm_nn_status()
    if dx is not None:
        want_dx = orc.conv3d_grad_input(dy, _bf(w))
        got_dx = np.moveaxis(dx.float().cpu().numpy().reshape(D, H, W, ci), -1, 0)
        assert _rel(got_dx, want_dx) < 5e-3
    want_dw, want_db = orc.conv3d_grad_weight(x, dy)
    assert _rel(dw.cpu().numpy().reshape(co, ci, 3, 3, 3), want_dw) < 1e-5
    assert _rel(db.cpu().numpy(), want_db) < 1e-5


def test_pool_upsample_concat_against_oracle():
    rng = np.random.default_rng(3)
    C1, C2, D, H, W = 16, 32, 4, 8, 8
    x = _bf(rng.standard_normal((C1, D, H, W)))
    V = D * H * W
    p = torch.empty((V // 8, C1), dtype=torch.bfloat16, device="cuda")
    sg.lbm_nn_pool2(_chlast(x), p, D, H, W, C1, 0)
    got = np.moveaxis(p.float().cpu().numpy().reshape(D // 2, H // 2, W // 2, C1), -1, 0)
    assert _rel(got, orc.avgpool2(x)) < 4e-3
    u = torch.empty((V, C1), dtype=torch.bfloat16, device="cuda")
    sg.lbm_nn_up2(p, u, D // 2, H // 2, W // 2, C1, 0)
    assert _rel(np.moveaxis(u.float().cpu().numpy().reshape(D, H, W, C1), -1, 0), orc.upsample2(got)) == 0.0
    y = _bf(rng.standard_normal((C2, D, H, W)))
    cat = torch.empty((V, C1 + C2), dtype=torch.bfloat16, device="cuda")
    a, b = _chlast(x), _chlast(y)
    sg.lbm_nn_concat(a, C1, b, C2, cat, V, 0)
    got = np.moveaxis(cat.float().cpu().numpy().reshape(D, H, W, C1 + C2), -1, 0)
    assert np.array_equal(got, np.concatenate([x, y]))
    a2, b2 = torch.zeros_like(a), torch.zeros_like(b)
    sg.lbm_nn_concat(a2, C1, b2, C2, cat, V, 1)
    assert torch.equal(a2, a) and torch.equal(b2, b)


def test_network_forward_and_gradients_against_oracle():
    """Two-level encoder-decoder (widths 16 / 16 / 32) on a 32 x 16 x 16 input: the output, the
    masked loss and every parameter gradient of the CUDA network against the FP64 oracle network
    with the same (BF16-rounded) weights."""
    width = (16, 16, 32)
    shape = (16, 16, 32)
    plan = orc.layer_plan(c_in=4, c_out=4, width=width)
    params = orc.init_params(plan, seed=5)
    rng = np.random.default_rng(6)
    for k in params:
        if k.endswith(".b"):
            params[k] = rng.uniform(0.0, 0.1, params[k].shape)
        elif k != "head.w":
            params[k] = _bf(params[k])
    x = _bf(rng.standard_normal((4,) + shape))
    t = rng.standard_normal((4,) + shape)
    fluid = rng.random(shape) > 0.4
    y_o, acts = orc.forward(params, x, plan, width)
    loss_o, dy_o = orc.masked_mse(y_o, t, fluid)
    # the oracle's backward, recording the term magnitudes of every 3^3 layer's gradient sums
    calls = []
    grad_w = orc.conv3d_grad_weight

    def recording(xx, dd):
        calls.append(grad_w(np.abs(xx), np.abs(dd)))
        return grad_w(xx, dd)

    orc.conv3d_grad_weight = recording
    try:
        g_o = orc.backward(params, acts, dy_o, plan, width)
    finally:
        orc.conv3d_grad_weight = grad_w
    L = len(width) - 1
    order = [f"dec{l}" for l in range(L)] + ["mid_b", "mid_a"] + \
        [f"enc{l}{s}" for l in reversed(range(L)) for s in "ba"]
    scale = {k: np.linalg.norm(v) for k, v in g_o.items()}
    for n, (mw, mb) in zip(order, calls):
        scale[n + ".w"], scale[n + ".b"] = np.linalg.norm(mw), np.linalg.norm(mb)

    net = sg.WarmStartNet(width=width, c_in=4)
    net.set_params(params)
    y = net.forward(_chlast(x), shape)
    td = torch.tensor(np.moveaxis(t, 0, -1).reshape(-1, 4), dtype=torch.float32, device="cuda")
    fl = torch.tensor(fluid.reshape(-1).astype(np.uint8), device="cuda")
    loss, dy = net.loss_and_grad(y, td, fl, int(fluid.sum()))
    net.backward(dy)
    net.check()
    got_y = np.moveaxis(y.cpu().numpy().reshape(shape + (4,)), -1, 0)
    assert _rel(got_y, y_o) < 3e-2
    assert abs(float(loss.item()) - loss_o) < 3e-2 * loss_o
    g = net.grads_numpy()
    errs = {k: float(np.linalg.norm(g[k].reshape(v.shape) - v) / scale[k]) for k, v in g_o.items()}
    print("gradient error / term magnitudes, by parameter:", {k: f"{e:.2e}" for k, e in errs.items()})
    for k, e in errs.items():
        assert e < 5e-2, f"gradient {k}: error {e:.3e} of its term magnitudes (all: {errs})"


def test_training_steps_reduce_the_loss():
    width = (16, 16, 32)
    shape = (16, 16, 32)
    rng = np.random.default_rng(8)
    x = _chlast(_bf(rng.standard_normal((4,) + shape)))
    tgt = np.stack([np.sin(np.linspace(0, 3, shape[2]))[None, None, :] * np.ones(shape)] * 4)
    td = torch.tensor(np.moveaxis(tgt, 0, -1).reshape(-1, 4), dtype=torch.float32, device="cuda")
    fl = torch.ones(int(np.prod(shape)), dtype=torch.uint8, device="cuda")
    net = sg.WarmStartNet(width=width, c_in=4, seed=1)
    losses = [float(net.train_step(x, td, fl, int(np.prod(shape)), shape, lr=3e-3).item()) for _ in range(30)]
    net.check()
    assert losses[-1] < 0.5 * losses[0], losses
