"""FP64 CPU oracle of the surrogate network (learned warm start of the steady state).

TEST INFRASTRUCTURE ONLY: this module is the independent definition the CUDA network kernels are
checked against.  Only tests, the smoke entry point and the benchmark's CPU baseline may import
it; the product path never does.

The warm start maps a binary geometry (plus the transport numbers) to the steady velocity and
concentration fields, which the lattice Boltzmann step then relaxes to its own steady state
(the convergence criterion is the residual of the step, not the network).  The paper has no
network: its steady states come from running the method (Sec. 3.4); the network is the
acceleration pattern of learned initial conditions and is defined here by its plain operations:

  conv3d        y[o, p] = b[o] + sum_c sum_t w[o, c, t] x[c, p + t]  (cross-correlation over the
                27 taps t in {-1, 0, 1}^3, zero outside the domain: "same" padding)
  conv1x1       y[o, p] = b[o] + sum_c w[o, c] x[c, p]
  relu          max(x, 0)
  avgpool2      mean over non-overlapping 2 x 2 x 2 blocks
  upsample2     nearest-neighbour copy of every value into a 2 x 2 x 2 block
  concat        along channels
  loss          L = sum_{p fluid} sum_k (y[k, p] - t[k, p])^2 / (n_fluid * n_out)

and their gradients, written out from the definitions (the gradient of a sum over taps is the
same sum with the tap reversed).  Arrays are channel-first [C, D, H, W]; D, H, W are z, y, x.
Parity pins: tests/test_oracle_nn.py (closed forms, adjointness, brute force, finite
differences).
"""
from __future__ import annotations

import numpy as np

TAPS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def _shifted(x, dz, dy, dx):
    """s[c, p] = x[c, p + (dz, dy, dx)], zero where p + t leaves the domain."""
    out = np.zeros_like(x)
    D, H, W = x.shape[1:]

    def rng(d, n):
        # destination indices p with 0 <= p + d < n
        return slice(max(0, -d), n - max(0, d)), slice(max(0, d), n - max(0, -d))

    (zd, zs), (yd, ys), (xd, xs) = rng(dz, D), rng(dy, H), rng(dx, W)
    out[:, zd, yd, xd] = x[:, zs, ys, xs]
    return out


def conv3d(x, w, b=None):
    """x [C_in, D, H, W], w [C_out, C_in, 3, 3, 3] (tap index dz+1, dy+1, dx+1), b [C_out]."""
    x = np.asarray(x, np.float64)
    w = np.asarray(w, np.float64)
    y = np.zeros((w.shape[0],) + x.shape[1:])
    for dz, dy, dx in TAPS:
        xs = _shifted(x, dz, dy, dx)
        y += np.einsum("oc,cdhw->odhw", w[:, :, dz + 1, dy + 1, dx + 1], xs)
    if b is not None:
        y += np.asarray(b, np.float64)[:, None, None, None]
    return y


def conv3d_grad_input(dy, w):
    """dL/dx of conv3d: dx[c, p] = sum_o sum_t w[o, c, t] dy[o, p - t]."""
    dy = np.asarray(dy, np.float64)
    w = np.asarray(w, np.float64)
    dx = np.zeros((w.shape[1],) + dy.shape[1:])
    for dz, dy_, dx_ in TAPS:
        ds = _shifted(dy, -dz, -dy_, -dx_)
        dx += np.einsum("oc,odhw->cdhw", w[:, :, dz + 1, dy_ + 1, dx_ + 1], ds)
    return dx


def conv3d_grad_weight(x, dy):
    """dL/dw of conv3d: dw[o, c, t] = sum_p dy[o, p] x[c, p + t]; dL/db[o] = sum_p dy[o, p]."""
    x = np.asarray(x, np.float64)
    dy = np.asarray(dy, np.float64)
    dw = np.zeros((dy.shape[0], x.shape[0], 3, 3, 3))
    for dz, dy_, dx_ in TAPS:
        xs = _shifted(x, dz, dy_, dx_)
        dw[:, :, dz + 1, dy_ + 1, dx_ + 1] = np.einsum("odhw,cdhw->oc", dy, xs)
    return dw, dy.sum(axis=(1, 2, 3))


def conv1x1(x, w, b=None):
    y = np.einsum("oc,cdhw->odhw", np.asarray(w, np.float64), np.asarray(x, np.float64))
    if b is not None:
        y += np.asarray(b, np.float64)[:, None, None, None]
    return y


def conv1x1_grads(x, w, dy):
    """(dx, dw, db) of conv1x1."""
    dx = np.einsum("oc,odhw->cdhw", np.asarray(w, np.float64), dy)
    dw = np.einsum("odhw,cdhw->oc", dy, np.asarray(x, np.float64))
    return dx, dw, dy.sum(axis=(1, 2, 3))


def relu(x):
    return np.maximum(x, 0.0)


def relu_grad(y, dy):
    """dL/dx of y = relu(x), given y (the gradient is 0 where y == 0)."""
    return np.where(y > 0.0, dy, 0.0)


def avgpool2(x):
    C, D, H, W = x.shape
    return x.reshape(C, D // 2, 2, H // 2, 2, W // 2, 2).mean(axis=(2, 4, 6))


def avgpool2_grad(dy):
    return np.repeat(np.repeat(np.repeat(dy, 2, axis=1), 2, axis=2), 2, axis=3) / 8.0


def upsample2(x):
    return np.repeat(np.repeat(np.repeat(x, 2, axis=1), 2, axis=2), 2, axis=3)


def upsample2_grad(dy):
    C, D, H, W = dy.shape
    return dy.reshape(C, D // 2, 2, H // 2, 2, W // 2, 2).sum(axis=(2, 4, 6))


def masked_mse(y, t, fluid):
    """Loss and its gradient over fluid nodes (fluid [D, H, W] boolean)."""
    m = np.asarray(fluid, np.float64)[None]
    n = max(1.0, float(m.sum())) * y.shape[0]
    d = (y - t) * m
    return float((d * d).sum() / n), 2.0 * d / n


# ---------------------------------------------------------------- the encoder-decoder

def layer_plan(c_in=4, c_out=4, width=(16, 32, 64, 128)):
    """Convolutions of the U-shaped encoder-decoder, in order: (name, kind, C_in, C_out).
    Encoder level l: two 3^3 convolutions (ReLU), then 2x average pooling; bottleneck: two
    3^3 convolutions; decoder level l: 2x nearest upsampling, concatenation with the encoder's
    level-l output, one 3^3 convolution (ReLU); head: 1x1 convolution (linear)."""
    plan, c = [], c_in
    for l, wd in enumerate(width[:-1]):
        plan += [(f"enc{l}a", "conv3", c, wd), (f"enc{l}b", "conv3", wd, wd)]
        c = wd
    plan += [("mid_a", "conv3", c, width[-1]), ("mid_b", "conv3", width[-1], width[-1])]
    c = width[-1]
    for l in reversed(range(len(width) - 1)):
        plan.append((f"dec{l}", "conv3", c + width[l], width[l]))
        c = width[l]
    plan.append(("head", "conv1", c, c_out))
    return plan


def init_params(plan, seed=0):
    """He-normal weights (fan-in), zero biases."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, kind, ci, co in plan:
        fan = ci * (27 if kind == "conv3" else 1)
        shape = (co, ci, 3, 3, 3) if kind == "conv3" else (co, ci)
        p[name + ".w"] = rng.standard_normal(shape) * np.sqrt(2.0 / fan)
        p[name + ".b"] = np.zeros(co)
    return p


def forward(params, x, plan, width=(16, 32, 64, 128)):
    """Network output and the activations the backward pass needs."""
    acts = {"in": x}
    h = x
    L = len(width) - 1
    skips = []
    for l in range(L):
        for s in "ab":
            n = f"enc{l}{s}"
            h = relu(conv3d(h, params[n + ".w"], params[n + ".b"]))
            acts[n] = h
        skips.append(h)
        h = avgpool2(h)
        acts[f"pool{l}"] = h
    for s in ("mid_a", "mid_b"):
        h = relu(conv3d(h, params[s + ".w"], params[s + ".b"]))
        acts[s] = h
    for l in reversed(range(L)):
        u = upsample2(h)
        cat = np.concatenate([u, skips[l]], axis=0)
        acts[f"cat{l}"] = cat
        n = f"dec{l}"
        h = relu(conv3d(cat, params[n + ".w"], params[n + ".b"]))
        acts[n] = h
    y = conv1x1(h, params["head.w"], params["head.b"])
    return y, acts


def backward(params, acts, dy, plan, width=(16, 32, 64, 128)):
    """Gradients of every parameter given dL/dy of the output."""
    g = {}
    L = len(width) - 1
    h = acts[f"dec0"]
    dh, g["head.w"], g["head.b"] = conv1x1_grads(h, params["head.w"], dy)
    dskip = {}
    for l in range(L):
        n = f"dec{l}"
        dpre = relu_grad(acts[n], dh)
        g[n + ".w"], g[n + ".b"] = conv3d_grad_weight(acts[f"cat{l}"], dpre)
        dcat = conv3d_grad_input(dpre, params[n + ".w"])
        cu = acts[f"cat{l}"].shape[0] - width[l]
        dskip[l] = dcat[cu:]
        dh = upsample2_grad(dcat[:cu])
    for s, prev in (("mid_b", "mid_a"), ("mid_a", f"pool{L - 1}")):
        dpre = relu_grad(acts[s], dh)
        g[s + ".w"], g[s + ".b"] = conv3d_grad_weight(acts[prev], dpre)
        dh = conv3d_grad_input(dpre, params[s + ".w"])
    for l in reversed(range(L)):
        dh = avgpool2_grad(dh) + dskip[l]
        for s, prev in (("b", f"enc{l}a"), ("a", f"pool{l - 1}" if l > 0 else "in")):
            n = f"enc{l}{s}"
            dpre = relu_grad(acts[n], dh)
            g[n + ".w"], g[n + ".b"] = conv3d_grad_weight(acts[prev], dpre)
            if not (l == 0 and s == "a"):
                dh = conv3d_grad_input(dpre, params[n + ".w"])
    return g
