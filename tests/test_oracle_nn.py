"""Pins of the surrogate network's FP64 oracle (oracle/nn_oracle.py) against what its definitions
fix: closed forms of single-tap kernels, a brute-force loop nest, the adjoint identities that tie
each gradient to its forward operation (a flipped tap, transposed channel pair or dropped term
breaks them), and central finite differences of the whole encoder-decoder's loss."""
import numpy as np
import pytest

from oracle import nn_oracle as nn


def _rand(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


def test_centre_tap_is_identity_plus_bias():
    x = _rand((3, 4, 5, 6), 1)
    w = np.zeros((3, 3, 3, 3, 3))
    for c in range(3):
        w[c, c, 1, 1, 1] = 1.0
    b = np.array([0.5, -1.0, 2.0])
    np.testing.assert_array_equal(nn.conv3d(x, w, b), x + b[:, None, None, None])


@pytest.mark.parametrize("tap", [(1, 0, 0), (0, -1, 1), (-1, 1, -1)])
def test_single_tap_is_a_shift_with_zero_fill(tap):
    dz, dy, dx = tap
    x = _rand((2, 5, 4, 6), 2)
    w = np.zeros((2, 2, 3, 3, 3))
    w[0, 1, dz + 1, dy + 1, dx + 1] = 3.0
    y = nn.conv3d(x, w)
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (1, 1)))
    D, H, W = x.shape[1:]
    want = 3.0 * xp[1, 1 + dz:1 + dz + D, 1 + dy:1 + dy + H, 1 + dx:1 + dx + W]
    np.testing.assert_array_equal(y[0], want)
    np.testing.assert_array_equal(y[1], 0.0)


def test_conv_against_brute_force_loop_nest():
    x = _rand((2, 3, 4, 5), 3)
    w = _rand((3, 2, 3, 3, 3), 4)
    b = _rand((3,), 5)
    C, D, H, W = x.shape
    want = np.zeros((3, D, H, W))
    for o in range(3):
        for z in range(D):
            for y in range(H):
                for xx in range(W):
                    s = b[o]
                    for c in range(C):
                        for a in range(3):
                            for bb in range(3):
                                for cc in range(3):
                                    zz, yy, x2 = z + a - 1, y + bb - 1, xx + cc - 1
                                    if 0 <= zz < D and 0 <= yy < H and 0 <= x2 < W:
                                        s += w[o, c, a, bb, cc] * x[c, zz, yy, x2]
                    want[o, z, y, xx] = s
    np.testing.assert_allclose(nn.conv3d(x, w, b), want, rtol=1e-13, atol=1e-13)


def test_input_gradient_is_the_adjoint():
    x, w, dy = _rand((3, 4, 5, 6), 6), _rand((4, 3, 3, 3, 3), 7), _rand((4, 4, 5, 6), 8)
    lhs = (dy * nn.conv3d(x, w)).sum()
    rhs = (x * nn.conv3d_grad_input(dy, w)).sum()
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_weight_gradient_is_the_adjoint():
    x, w, dy = _rand((3, 4, 5, 6), 9), _rand((4, 3, 3, 3, 3), 10), _rand((4, 4, 5, 6), 11)
    dw, db = nn.conv3d_grad_weight(x, dy)
    lhs = (dy * nn.conv3d(x, w)).sum()
    assert abs(lhs - (w * dw).sum()) <= 1e-12 * abs(lhs)
    np.testing.assert_allclose(db, dy.sum(axis=(1, 2, 3)), rtol=1e-14)
    # the bias enters every node once
    b = _rand((4,), 12)
    assert abs((dy * nn.conv3d(x, w, b)).sum() - lhs - (b * db).sum()) <= 1e-12 * abs(lhs)


def test_pool_and_upsample_adjoints():
    x, y = _rand((2, 4, 6, 8), 13), _rand((2, 2, 3, 4), 14)
    assert abs((nn.avgpool2(x) * y).sum() - (x * nn.avgpool2_grad(y)).sum()) < 1e-12
    assert abs((nn.upsample2(y) * x).sum() - (y * nn.upsample2_grad(x)).sum()) < 1e-12
    np.testing.assert_allclose(nn.avgpool2(nn.upsample2(y)), y, rtol=1e-15)
    # the pool of a block-constant field is that constant
    np.testing.assert_allclose(nn.avgpool2(np.ones((1, 4, 4, 4)) * 2.5), 2.5)


def test_conv1x1_and_loss_gradients_by_finite_differences():
    rng = np.random.default_rng(15)
    x, w, b = rng.standard_normal((3, 2, 2, 2)), rng.standard_normal((2, 3)), rng.standard_normal(2)
    t = rng.standard_normal((2, 2, 2, 2))
    fl = rng.random((2, 2, 2)) > 0.3

    def loss(w_, x_):
        return nn.masked_mse(nn.conv1x1(x_, w_, b), t, fl)[0]

    _, dy = nn.masked_mse(nn.conv1x1(x, w, b), t, fl)
    dx, dw, _ = nn.conv1x1_grads(x, w, dy)
    h = 1e-6
    for idx in [(0, 0), (1, 2)]:
        e = np.zeros_like(w)
        e[idx] = h
        assert abs((loss(w + e, x) - loss(w - e, x)) / (2 * h) - dw[idx]) < 1e-7
    for idx in [(0, 1, 0, 1), (2, 0, 1, 1)]:
        e = np.zeros_like(x)
        e[idx] = h
        assert abs((loss(w, x + e) - loss(w, x - e)) / (2 * h) - dx[idx]) < 1e-7


def test_network_gradients_by_finite_differences():
    """The whole encoder-decoder (two levels, widths 3 / 4 / 5) on an 8^3 input: every parameter
    group's analytic gradient against central differences of the masked loss."""
    width = (3, 4, 5)
    plan = nn.layer_plan(c_in=2, c_out=2, width=width)
    p = nn.init_params(plan, seed=3)
    for k in p:
        if k.endswith(".b"):
            p[k] = np.random.default_rng(hash(k) % 1000).uniform(0.05, 0.2, p[k].shape)
    rng = np.random.default_rng(16)
    x = rng.standard_normal((2, 8, 8, 8))
    t = rng.standard_normal((2, 8, 8, 8))
    fl = rng.random((8, 8, 8)) > 0.4

    def loss(pp):
        y, _ = nn.forward(pp, x, plan, width)
        return nn.masked_mse(y, t, fl)[0]

    y, acts = nn.forward(p, x, plan, width)
    _, dy = nn.masked_mse(y, t, fl)
    g = nn.backward(p, acts, dy, plan, width)
    assert set(g) == set(p)
    h = 1e-6
    checked = 0
    for k in sorted(p):
        flat = p[k].reshape(-1)
        for j in np.random.default_rng(len(k)).choice(flat.size, size=min(2, flat.size), replace=False):
            pp = {kk: v.copy() for kk, v in p.items()}
            pm = {kk: v.copy() for kk, v in p.items()}
            pp[k].reshape(-1)[j] += h
            pm[k].reshape(-1)[j] -= h
            fd = (loss(pp) - loss(pm)) / (2 * h)
            an = g[k].reshape(-1)[j]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)) + 1e-8, (k, j, fd, an)
            checked += 1
    assert checked >= 2 * len(plan)


def test_layer_plan_counts():
    plan = nn.layer_plan()
    p = nn.init_params(plan)
    n = sum(v.size for v in p.values())
    assert 1.0e6 < n < 2.5e6   # the ~2M-parameter encoder-decoder of the warm-start workload
    names = [q[0] for q in plan]
    assert names[0] == "enc0a" and names[-1] == "head"
