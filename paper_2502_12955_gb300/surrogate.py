"""Learned warm start: a 3D convolutional encoder-decoder that predicts the steady velocity and
concentration of the reactive porous-media workload from its geometry and transport numbers.

The lattice Boltzmann step (lbm.py) then starts from the prediction instead of from rest and
relaxes it to its own steady state; its residual, not the network, decides convergence, so a
poor prediction costs steps but never accuracy.  Plain LBM from rest stays the fallback and the
arbiter of the network's error.

Binding: the `lbm_nn_*` functions below carry the C ABI's names (include/lbm_nn.h) and only
marshal torch tensors into device pointers; every operation runs in liblbm.so's sm_103a kernels
(the 3^3 convolutions as im2col + tcgen05 GEMMs, BF16 storage, FP32 accumulation).  PyTorch is
used for device memory and the stream only.

Network (the same plan as the FP64 reference of the test suite): encoder levels of two 3^3
convolutions (ReLU) and 2x average pooling, a bottleneck of two 3^3 convolutions, decoder levels
of 2x nearest upsampling, concatenation with the encoder output of that level and one 3^3
convolution (ReLU), and a 1x1 head to 4 outputs.  Inputs (5 channels): solid indicator,
x / (nx - 1), ln(Pe / 10), ln(Da / 0.1) and the distance to the nearest solid over the mean sphere
radius (pore size, which sets how far a pore's concentration is depleted).  Outputs: u / 0.005 (3 channels) and 2 (C - 1/2), which
weights the concentration, the field whose error sets the relaxation time, above the velocity.
Training: masked mean squared error over fluid voxels, Adam.
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np

from . import lbm as _lbm

U_SCALE = 0.005      # velocity scale of the targets (of the order of the packings' mean fluid speed)
C_OFF, C_SCALE = 0.5, 2.0   # concentration target 2 (C - 1/2): order one, and weighted above u
PE0, DA0 = 10.0, 0.1
OUT_F32, OUT_BF16, OUT_BF16_RELU = 0, 1, 2
PORE_SCALE = 9.0     # length scale of the pore-size channel (the packings' mean sphere radius)
N_FEATURES = 5

_NN = None


def nn_lib():
    """liblbm.so with the lbm_nn_* signatures declared (raises if the library is missing)."""
    global _NN
    if _NN is not None:
        return _NN
    lib = _lbm.load()
    vp, i32, i64, f32 = C.c_void_p, C.c_int32, C.c_int64, C.c_float
    sig = {
        "lbm_nn_gemm_tn": [vp, vp, vp, i64, i32, i32, i32, i32, i32, vp, vp],
        "lbm_nn_status": [vp],
        "lbm_nn_im2col": [vp, vp, i32, i32, i32, i32, i32, i32, vp],
        "lbm_nn_im2col_cv": [vp, vp, i32, i32, i32, i32, i32, vp],
        "lbm_nn_transpose": [vp, vp, i64, i32, vp],
        "lbm_nn_reduce_splits": [vp, vp, i64, i32, i64, vp],
        "lbm_nn_relu_grad": [vp, vp, vp, i64, vp],
        "lbm_nn_pool2": [vp, vp, i32, i32, i32, i32, i32, vp],
        "lbm_nn_up2": [vp, vp, i32, i32, i32, i32, i32, vp],
        "lbm_nn_concat": [vp, i32, vp, i32, vp, i64, i32, vp],
        "lbm_nn_colsum": [vp, vp, i64, i32, vp],
        "lbm_nn_head_fwd": [vp, vp, vp, vp, i64, i32, i32, vp],
        "lbm_nn_head_bwd": [vp, vp, vp, vp, vp, vp, i64, i32, i32, vp],
        "lbm_nn_mse": [vp, vp, vp, vp, vp, i64, i32, i64, vp],
        "lbm_nn_adam": [vp, vp, vp, vp, i64, f32, f32, f32, f32, i32, vp],
        "lbm_nn_pack_weights": [vp, vp, vp, i32, i32, i32, i32, vp],
        "lbm_nn_unpack_wgrad": [vp, vp, i32, i32, vp],
        "lbm_nn_add": [vp, vp, vp, i64, vp],
        "lbm_nn_cast_bf16": [vp, vp, i64, vp],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = C.c_int
    lib.lbm_nn_gemm_splits.argtypes = [i32, i32]
    lib.lbm_nn_gemm_splits.restype = i32
    _NN = lib
    return lib


def _p(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ck(name, st):
    if st != 0:
        raise _lbm.LbmError(st, f"{name} failed")


def _call(name, *args):
    _ck(name, getattr(nn_lib(), name)(*args, _stream()))


# ------------------------------------------------------------------ the C ABI, marshalled

def lbm_nn_gemm_tn(A, B, Cout, ldc, M, N, K, splits=1, out_kind=OUT_F32, bias=None):
    _call("lbm_nn_gemm_tn", _p(A), _p(B), _p(Cout), ldc, M, N, K, splits, out_kind, _p(bias))


def lbm_nn_gemm_splits(K, splits):
    return int(nn_lib().lbm_nn_gemm_splits(K, splits))


def lbm_nn_status():
    _ck("lbm_nn_status", nn_lib().lbm_nn_status(_stream()))


def lbm_nn_im2col(x, col, D, H, W, Cc, Kp, transposed=0):
    _call("lbm_nn_im2col", _p(x), _p(col), D, H, W, Cc, Kp, transposed)


def lbm_nn_im2col_cv(xT, colT, D, H, W, Cc, Kp):
    _call("lbm_nn_im2col_cv", _p(xT), _p(colT), D, H, W, Cc, Kp)


def lbm_nn_transpose(x, y, R, Cc):
    _call("lbm_nn_transpose", _p(x), _p(y), R, Cc)


def lbm_nn_reduce_splits(part, out, n, splits, stride):
    _call("lbm_nn_reduce_splits", _p(part), _p(out), n, splits, stride)


def lbm_nn_relu_grad(y, dy, dx, n):
    _call("lbm_nn_relu_grad", _p(y), _p(dy), _p(dx), n)


def lbm_nn_pool2(i, o, D, H, W, Cc, backward=0):
    _call("lbm_nn_pool2", _p(i), _p(o), D, H, W, Cc, backward)


def lbm_nn_up2(i, o, D, H, W, Cc, backward=0):
    _call("lbm_nn_up2", _p(i), _p(o), D, H, W, Cc, backward)


def lbm_nn_concat(a, Ca, b, Cb, out, V, backward=0):
    _call("lbm_nn_concat", _p(a), Ca, _p(b), Cb, _p(out), V, backward)


def lbm_nn_colsum(x, out, V, Cc):
    _call("lbm_nn_colsum", _p(x), _p(out), V, Cc)


def lbm_nn_head_fwd(h, w, b, y, V, Cc, Co):
    _call("lbm_nn_head_fwd", _p(h), _p(w), _p(b), _p(y), V, Cc, Co)


def lbm_nn_head_bwd(h, w, dy, dh, dw, db, V, Cc, Co):
    _call("lbm_nn_head_bwd", _p(h), _p(w), _p(dy), _p(dh), _p(dw), _p(db), V, Cc, Co)


def lbm_nn_mse(y, t, fluid, dy, loss, V, Co, n_fluid):
    _call("lbm_nn_mse", _p(y), _p(t), _p(fluid), _p(dy), _p(loss), V, Co, n_fluid)


def lbm_nn_adam(w, g, m, v, n, lr, b1, b2, eps, step):
    _call("lbm_nn_adam", _p(w), _p(g), _p(m), _p(v), n, lr, b1, b2, eps, step)


def lbm_nn_pack_weights(w, wk, wt, Co, Ci, Kp, Kpt):
    _call("lbm_nn_pack_weights", _p(w), _p(wk), _p(wt), Co, Ci, Kp, Kpt)


def lbm_nn_unpack_wgrad(dwcol, dw, Co, Ci):
    _call("lbm_nn_unpack_wgrad", _p(dwcol), _p(dw), Co, Ci)


def lbm_nn_add(a, b, y, n):
    _call("lbm_nn_add", _p(a), _p(b), _p(y), n)


def lbm_nn_cast_bf16(x, y, n):
    _call("lbm_nn_cast_bf16", _p(x), _p(y), n)


# ------------------------------------------------------------------ network

def kpad(k):
    """K of a 3^3 convolution padded to the GEMM's 128-row tiles."""
    return ((k + 127) // 128) * 128


def layer_plan(c_in=4, c_out=4, width=(16, 32, 64, 160)):
    """(name, kind, C_in, C_out) of every convolution, in forward order."""
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


class WarmStartNet:
    """The encoder-decoder on one GPU: FP32 master weights with Adam, BF16 copies for the
    tensor-core GEMMs, channel-last BF16 activations."""

    def __init__(self, width=(16, 32, 64, 160), c_in=N_FEATURES, c_out=4, seed=0, device=0):
        import torch
        if width[0] != 16 or c_out != 4:
            raise ValueError("the head kernel takes 16 input and 4 output channels")
        if any(w % 16 for w in width):
            raise ValueError("channel widths must be multiples of 16 (GEMM N tiles)")
        self.torch = torch
        self.dev = torch.device("cuda", device)
        self.width, self.c_in, self.c_out = tuple(width), c_in, c_out
        self.plan = layer_plan(c_in, c_out, width)
        self.L = len(width) - 1
        # one flat FP32 buffer of parameters (views per tensor), gradients and Adam moments
        shapes = {}
        for name, kind, ci, co in self.plan:
            shapes[name + ".w"] = (co, ci, 27) if kind == "conv3" else (co, ci)
            shapes[name + ".b"] = (co,)
        self.shapes = shapes
        n = sum(int(np.prod(s)) for s in shapes.values())
        self.n_params = n
        f32 = dict(dtype=torch.float32, device=self.dev)
        self.flat = torch.zeros(n, **f32)
        self.gflat = torch.zeros(n, **f32)
        self.m = torch.zeros(n, **f32)
        self.v = torch.zeros(n, **f32)
        self.p, self.g, off = {}, {}, 0
        for k, s in shapes.items():
            sz = int(np.prod(s))
            self.p[k] = self.flat[off:off + sz].view(s)
            self.g[k] = self.gflat[off:off + sz].view(s)
            off += sz
        rng = np.random.default_rng(seed)
        init = {}
        for name, kind, ci, co in self.plan:
            fan = ci * (27 if kind == "conv3" else 1)
            init[name + ".w"] = rng.standard_normal(shapes[name + ".w"]) * math.sqrt(2.0 / fan)
            init[name + ".b"] = np.zeros(co)
        self.set_params(init)
        self.step_count = 0
        self._scratch = None

    # -------------------------------------------------------------- parameters

    def set_params(self, params):
        """Load parameters given as numpy arrays (conv weights [Co, Ci, 3, 3, 3] or [Co, Ci, 27],
        head [Co, Ci], biases [Co]) and repack the BF16 GEMM copies."""
        for k, v in params.items():
            self.p[k].copy_(self.torch.from_numpy(np.asarray(v, np.float32).reshape(self.shapes[k])))
        self._pack()

    def params_numpy(self):
        return {k: v.detach().cpu().numpy().copy() for k, v in self.p.items()}

    def grads_numpy(self):
        return {k: v.detach().cpu().numpy().copy() for k, v in self.g.items()}

    def _pack(self):
        """BF16 GEMM copies of the 3^3 kernels: wk [Co][Kp] and the flipped transpose wt [Ci][Kpt]."""
        torch = self.torch
        if not hasattr(self, "wk"):
            self.wk, self.wt = {}, {}
            for name, kind, ci, co in self.plan:
                if kind == "conv3":
                    self.wk[name] = torch.empty((co, kpad(27 * ci)), dtype=torch.bfloat16, device=self.dev)
                    self.wt[name] = torch.empty((ci, kpad(27 * co)), dtype=torch.bfloat16, device=self.dev)
        for name, kind, ci, co in self.plan:
            if kind == "conv3":
                lbm_nn_pack_weights(self.p[name + ".w"], self.wk[name], self.wt[name], co, ci, kpad(27 * ci),
                                    kpad(27 * co))

    # -------------------------------------------------------------- buffers

    def _scratch_for(self, shape):
        """BF16 im2col scratch and FP32 split-K partials sized for an input of this shape."""
        D, H, W = shape
        need, part = 0, 0
        for l, (name, kind, ci, co) in enumerate(self.plan):
            if kind != "conv3":
                continue
            V = self._level_volume(name, shape)
            need = max(need, V * kpad(27 * ci), V * kpad(27 * co))
            part = max(part, kpad(27 * ci) * co * 64)
        if self._scratch is None or self._scratch[0] < need or self._scratch[2] < part:
            torch = self.torch
            self._scratch = (need, torch.empty(need, dtype=torch.bfloat16, device=self.dev), part,
                             torch.empty(part, dtype=torch.float32, device=self.dev))
        return self._scratch[1], self._scratch[3]

    def _level_volume(self, name, shape):
        D, H, W = shape
        if name.startswith("enc"):
            lv = int(name[3])
        elif name.startswith("dec"):
            lv = int(name[3])
        else:
            lv = self.L
        return (D >> lv) * (H >> lv) * (W >> lv)

    # -------------------------------------------------------------- layers

    def _conv3(self, name, x, shape, ci, co):
        torch = self.torch
        D, H, W = shape
        V = D * H * W
        kp = kpad(27 * ci)
        col, _ = self._scratch_for(self._in_shape)
        lbm_nn_im2col(x, col, D, H, W, ci, kp, 0)
        y = torch.empty((V, co), dtype=torch.bfloat16, device=self.dev)
        lbm_nn_gemm_tn(col, self.wk[name], y, co, V, co, kp, 1, OUT_BF16_RELU, self.p[name + ".b"])
        return y

    def _conv3_backward(self, name, xin, yout, dy, shape, ci, co, need_dx=True):
        torch = self.torch
        D, H, W = shape
        V = D * H * W
        kp, kpt = kpad(27 * ci), kpad(27 * co)
        col, part = self._scratch_for(self._in_shape)
        dpre = torch.empty_like(dy)
        lbm_nn_relu_grad(yout, dy, dpre, V * co)
        lbm_nn_colsum(dpre, self.g[name + ".b"], V, co)
        # weight gradient: dW[k][o] = sum_v colT[k][v] dpreT[o][v], split over v; colT is built
        # from a channel-major copy of the input when the rows allow 8-voxel vectors
        if W % 8 == 0:
            xT = torch.empty((ci, V), dtype=torch.bfloat16, device=self.dev)
            lbm_nn_transpose(xin, xT, V, ci)
            lbm_nn_im2col_cv(xT, col, D, H, W, ci, kp)
        else:
            lbm_nn_im2col(xin, col, D, H, W, ci, kp, 1)
        dpreT = torch.empty((co, V), dtype=torch.bfloat16, device=self.dev)
        lbm_nn_transpose(dpre, dpreT, V, co)
        tiles = (kp // 128) * max(1, co // 128)
        want = max(1, min(64, (4 * 152) // max(1, tiles), V // 64))
        splits = lbm_nn_gemm_splits(V, want)
        lbm_nn_gemm_tn(col, dpreT, part, co, kp, co, V, splits, OUT_F32, None)
        dwcol = torch.empty((kp, co), dtype=torch.float32, device=self.dev)
        lbm_nn_reduce_splits(part, dwcol, kp * co, splits, kp * co)
        lbm_nn_unpack_wgrad(dwcol, self.g[name + ".w"], co, ci)
        if not need_dx:
            return None
        # input gradient: a convolution of dpre with the flipped, transposed kernel
        lbm_nn_im2col(dpre, col, D, H, W, co, kpt, 0)
        dx = torch.empty((V, ci), dtype=torch.bfloat16, device=self.dev)
        lbm_nn_gemm_tn(col, self.wt[name], dx, ci, V, ci, kpt, 1, OUT_BF16, None)
        return dx

    # -------------------------------------------------------------- passes

    def forward(self, x, shape):
        """x: BF16 [V][c_in] channel-last; returns FP32 [V][c_out] and keeps the activations."""
        torch = self.torch
        self._in_shape = tuple(shape)
        acts = {"in": (x, tuple(shape), self.c_in)}
        h, shp, c = x, tuple(shape), self.c_in
        skips = []
        for l, wd in enumerate(self.width[:-1]):
            for s in "ab":
                n = f"enc{l}{s}"
                h = self._conv3(n, h, shp, c, wd)
                c = wd
                acts[n] = (h, shp, c)
            skips.append((h, shp, c))
            D, H, W = shp
            nxt = (D // 2, H // 2, W // 2)
            pooled = torch.empty((nxt[0] * nxt[1] * nxt[2], c), dtype=torch.bfloat16, device=self.dev)
            lbm_nn_pool2(h, pooled, D, H, W, c, 0)
            h, shp = pooled, nxt
            acts[f"pool{l}"] = (h, shp, c)
        for n in ("mid_a", "mid_b"):
            h = self._conv3(n, h, shp, c, self.width[-1])
            c = self.width[-1]
            acts[n] = (h, shp, c)
        for l in reversed(range(self.L)):
            sk, sshp, sc = skips[l]
            D, H, W = shp
            up = torch.empty((8 * D * H * W, c), dtype=torch.bfloat16, device=self.dev)
            lbm_nn_up2(h, up, D, H, W, c, 0)
            V = sshp[0] * sshp[1] * sshp[2]
            cat = torch.empty((V, c + sc), dtype=torch.bfloat16, device=self.dev)
            lbm_nn_concat(up, c, sk, sc, cat, V, 0)
            acts[f"cat{l}"] = (cat, sshp, c + sc)
            n = f"dec{l}"
            h = self._conv3(n, cat, sshp, c + sc, self.width[l])
            shp, c = sshp, self.width[l]
            acts[n] = (h, shp, c)
        V = shp[0] * shp[1] * shp[2]
        y = torch.empty((V, self.c_out), dtype=torch.float32, device=self.dev)
        lbm_nn_head_fwd(h, self.p["head.w"], self.p["head.b"], y, V, c, self.c_out)
        self._acts = acts
        return y

    def backward(self, dy):
        """dy: FP32 [V][c_out] = dL/dy of the last forward; fills the gradients."""
        torch = self.torch
        acts = self._acts
        h, shp, c = acts["dec0"]
        V = shp[0] * shp[1] * shp[2]
        dh = torch.empty((V, c), dtype=torch.bfloat16, device=self.dev)
        lbm_nn_head_bwd(h, self.p["head.w"], dy, dh, self.g["head.w"], self.g["head.b"], V, c, self.c_out)
        dskip = {}
        for l in range(self.L):
            n = f"dec{l}"
            cat, cshp, cc = acts[f"cat{l}"]
            y, _, co = acts[n]
            dcat = self._conv3_backward(n, cat, y, dh, cshp, cc, co)
            sc = self.width[l]
            cu = cc - sc
            Vf = cshp[0] * cshp[1] * cshp[2]
            du = torch.empty((Vf, cu), dtype=torch.bfloat16, device=self.dev)
            ds = torch.empty((Vf, sc), dtype=torch.bfloat16, device=self.dev)
            lbm_nn_concat(du, cu, ds, sc, dcat, Vf, 1)
            dskip[l] = ds
            D, H, W = cshp
            dh = torch.empty((Vf // 8, cu), dtype=torch.bfloat16, device=self.dev)
            lbm_nn_up2(du, dh, D // 2, H // 2, W // 2, cu, 1)
        for n, prev in (("mid_b", "mid_a"), ("mid_a", f"pool{self.L - 1}")):
            xin, xshp, ci = acts[prev]
            y, _, co = acts[n]
            dh = self._conv3_backward(n, xin, y, dh, xshp, ci, co)
        for l in reversed(range(self.L)):
            sk, sshp, sc = acts[f"enc{l}b"]
            D, H, W = sshp
            Vf = D * H * W
            up = torch.empty((Vf, sc), dtype=torch.bfloat16, device=self.dev)
            lbm_nn_pool2(dh, up, D, H, W, sc, 1)
            dh = torch.empty_like(up)
            lbm_nn_add(up, dskip[l], dh, Vf * sc)
            for s, prev in (("b", f"enc{l}a"), ("a", f"pool{l - 1}" if l > 0 else "in")):
                n = f"enc{l}{s}"
                xin, xshp, ci = acts[prev]
                y, _, co = acts[n]
                dh = self._conv3_backward(n, xin, y, dh, xshp, ci, co, need_dx=not (l == 0 and s == "a"))

    def loss_and_grad(self, y, t, fluid, n_fluid):
        torch = self.torch
        V = y.shape[0]
        dy = torch.empty_like(y)
        loss = torch.zeros(1, dtype=torch.float64, device=self.dev)
        lbm_nn_mse(y, t, fluid, dy, loss, V, self.c_out, n_fluid)
        return loss, dy

    def adam(self, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.step_count += 1
        lbm_nn_adam(self.flat, self.gflat, self.m, self.v, self.n_params, lr, b1, b2, eps, self.step_count)
        self._pack()

    def train_step(self, x, t, fluid, n_fluid, shape, lr=1e-3):
        y = self.forward(x, shape)
        loss, dy = self.loss_and_grad(y, t, fluid, n_fluid)
        self.backward(dy)
        self.adam(lr)
        return loss

    def check(self):
        """Raises if a GEMM gave up waiting on its copies since the last check."""
        lbm_nn_status()


# ------------------------------------------------------------------ data

def pore_distance(geom, pad=16):
    """Euclidean distance of every fluid node to the nearest solid node (0 on solids), with the
    domain wrapped periodically in y and z and open in x (inlet and outlet faces)."""
    from scipy.ndimage import distance_transform_edt
    fl = geom == 0
    p = min(pad, geom.shape[0], geom.shape[1])
    big = np.pad(fl, ((p, p), (p, p), (0, 0)), mode="wrap")
    d = distance_transform_edt(big)
    return d[p:p + geom.shape[0], p:p + geom.shape[1], :]


def features(geom, Pe=PE0, Da=DA0, device=0):
    """Input channels (channel-last BF16 [V][5]) of a geometry [nz, ny, nx] of flags: solid
    indicator, x / (nx - 1), ln(Pe / 10), ln(Da / 0.1), distance to the nearest solid / 9."""
    import torch
    nz, ny, nx = geom.shape
    f = np.empty((nz, ny, nx, N_FEATURES), np.float32)
    f[..., 0] = (geom != 0)
    f[..., 1] = (np.arange(nx) / max(1, nx - 1))[None, None, :]
    f[..., 2] = math.log(Pe / PE0)
    f[..., 3] = math.log(Da / DA0)
    f[..., 4] = pore_distance(geom) / PORE_SCALE
    return torch.from_numpy(f.reshape(-1, N_FEATURES)).to(device=torch.device("cuda", device), dtype=torch.bfloat16)


def targets(u, Cf, device=0):
    """Training targets (FP32 [V][4]): u / U_SCALE and C_SCALE (C - C_OFF)."""
    import torch
    nz, ny, nx = Cf.shape[-3:]
    t = np.empty((nz, ny, nx, 4), np.float32)
    for a in range(3):
        t[..., a] = u[a] / U_SCALE
    t[..., 3] = C_SCALE * (Cf.reshape(nz, ny, nx) - C_OFF)
    return torch.from_numpy(t.reshape(-1, 4)).to(torch.device("cuda", device))


def predict_fields(net, geom, Pe=PE0, Da=DA0):
    """(rho, u, C) for lbm Solver.set_fields from the network's prediction: rho = 1, u and C
    from the outputs on fluid nodes (solid nodes: u = 0, C = 1)."""
    import torch
    nz, ny, nx = geom.shape
    with torch.no_grad():
        y = net.forward(features(geom, Pe, Da, net.dev.index), geom.shape)
    net.check()
    y = y.cpu().numpy().reshape(nz, ny, nx, 4)
    fl = geom == 0
    u = np.stack([np.where(fl, y[..., a] * U_SCALE, 0.0) for a in range(3)])
    Cf = np.where(fl, y[..., 3] / C_SCALE + C_OFF, 1.0)[None]
    rho = np.ones((1, nz, ny, nx))
    return rho, u, Cf
