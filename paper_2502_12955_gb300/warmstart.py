"""Warm start of the steady state by the learned encoder-decoder (surrogate.py), end to end.

  generate()  solver-generated training data: seeded random-sphere packings (the dissolution
              workload's recipe at the given size, seeds from 10^4), transport numbers Pe, Da
              drawn log-uniform in [5, 10] and [0.05, 0.2], each run by the lattice Boltzmann step from
              rest to its steady state (residual <= tol, geometry update frozen);
  train()     Adam on the masked squared error of the fields, one sample per step;
  compare()   on held-out geometries: steps and wall time to residual <= tol from rest and from
              the network's prediction (inference time included), the same solver and stream.

The residual is the step's own (relative L2 change of u and C over 100 steps, the larger of the
two), so the network only moves the starting point: a wrong prediction costs steps, never
accuracy, and plain LBM from rest is the fallback.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import inputs
from . import surrogate as sg
from .lbm import Solver

L_CHAR = 9.0        # characteristic length: mean sphere radius of the packing
U_DESIGN = 0.0185   # design speed the dissolution workload's transport numbers are built on
CS2_D3Q7 = 0.25     # c_s^2 of the D3Q7 lattice at J0 = 1/4


def transport(Pe, Da):
    """tau_c and k of the dissolution workload for the given Peclet and Damkohler numbers
    (D = U L / Pe, tau_c = D / c_s^2 + 1/2, k = Da D / L)."""
    D = U_DESIGN * L_CHAR / Pe
    return D / CS2_D3Q7 + 0.5, Da * D / L_CHAR


def case(seed, n, Pe=sg.PE0, Da=sg.DA0, precision="fp32"):
    cfg, geom, fields = inputs.dissolution_3d(n=n, seed=seed, precision=precision)
    tau_c, k = transport(Pe, Da)
    cfg = dict(cfg, tau_c=[tau_c], k_react=k, geo_mode="none", N_mon=100)
    return cfg, geom, fields


def run_to_steady(cfg, geom, fields, tol, max_steps, stream=None):
    """Steps the solver from the given fields until the residual is <= tol; returns
    (steps, seconds, converged, solver).  Seconds are CUDA-event time on the solver's stream,
    including the host reads of the residual.  A run whose populations turn non-finite stops
    there and is not converged (its residual would read zero)."""
    import torch
    s = Solver(cfg, stream=stream.cuda_stream if stream is not None else None)
    s.set_geometry(geom)
    rho, u, C = fields
    s.set_fields(rho, u, C)
    s.sync()
    st = stream or torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    steps, r = 0, float("inf")
    finite = True
    while steps < max_steps:
        s.step(100)
        steps += 100
        m = s.monitors()
        r = m["residual"]
        # a diverging run: non-finite populations, a residual that grows past 5 % per 100 steps,
        # or a species total beyond twice that of a domain filled at the inlet value
        if (m["nonfinite"] != 0 or not math.isfinite(r) or (steps > 1000 and r > 0.05)
                or abs(m["species0"]) > 2.0 * max(1.0, m["nfluid"])):
            finite = False
            break
        if 0.0 <= r <= tol:
            break
    e1.record(st)
    torch.cuda.synchronize()
    return steps, e0.elapsed_time(e1) * 1e-3, bool(finite and 0.0 <= r <= tol), s


class Sample:
    """One training or test case held on the device: features, targets and fluid mask."""

    def __init__(self, seed, n, Pe, Da, geom, u=None, Cf=None, device=0):
        import torch
        self.seed, self.n, self.Pe, self.Da, self.geom = seed, n, Pe, Da, geom
        self.x = sg.features(geom, Pe, Da, device)
        fl = (geom == 0).reshape(-1).astype(np.uint8)
        self.fluid = torch.from_numpy(fl).to(torch.device("cuda", device))
        self.n_fluid = int(fl.sum())
        self.t = sg.targets(u, Cf, device) if u is not None else None


PE_RANGE = (5.0, 10.0)   # the recipe's scalar lattice (tau_c = 1/2 + 0.67 / Pe) is stable below ~Pe 10
DA_RANGE = (0.05, 0.2)


def draw_transport(rng):
    """Pe and Da log-uniform in PE_RANGE and DA_RANGE.  At Pe = 10 (tau_c = 0.567) the scalar
    lattice of some packings grows an unstable concentration mode; below it the recipe is stable."""
    lp = rng.uniform(math.log(PE_RANGE[0]), math.log(PE_RANGE[1]))
    ld = rng.uniform(math.log(DA_RANGE[0]), math.log(DA_RANGE[1]))
    return math.exp(lp), math.exp(ld)


def generate(count, n=128, seed0=10_000, tol=1e-5, max_steps=400_000, device=0, log=None):
    """count solver-generated samples (cases that do not converge are skipped and recorded, up to
    count more draws); returns (samples, per-case steps, seconds and outcome)."""
    rng = np.random.default_rng(seed0)
    out, stats = [], []
    seed = seed0
    while len(out) < count and seed < seed0 + 2 * count:
        Pe, Da = draw_transport(rng)
        cfg, geom, fields = case(seed, n, Pe, Da)
        cfg = dict(cfg, device=device)
        steps, sec, ok, s = run_to_steady(cfg, geom, fields, tol, max_steps)
        f = s.fields() if ok else None
        s.close()
        if ok:
            out.append(Sample(seed, n, Pe, Da, geom, f["u"], f["C"][0], device))
        stats.append({"seed": seed, "Pe": Pe, "Da": Da, "steps": steps, "seconds": sec, "converged": ok})
        if log:
            log(f"case seed {seed}: Pe {Pe:.2f} Da {Da:.3f} steps {steps} {sec:.2f} s converged {ok}")
        seed += 1
    return out, stats


def symmetric_copy(s, k):
    """Sample s under symmetry k (0..7) of the y-z plane: bit 0 mirrors y, bit 1 mirrors z, bit 2
    exchanges y and z (cubic cross-sections only).  The flow is driven along x and y, z are
    periodic, so the D3Q19 / D3Q7 step commutes with these maps: the mapped steady state is the
    steady state of the mapped packing, with u_y, u_z mirrored or exchanged alike.  Returns
    (features, targets, fluid mask) as device tensors in the layout of Sample."""
    nz, ny, nx = s.geom.shape
    if k == 0:
        return s.x, s.t, s.fluid
    x = s.x.view(nz, ny, nx, -1)
    t = s.t.view(nz, ny, nx, 4)
    f = s.fluid.view(nz, ny, nx)
    sign = [1.0, 1.0, 1.0, 1.0]
    if k & 1:
        x, t, f = x.flip(1), t.flip(1), f.flip(1)
        sign[1] = -1.0
    if k & 2:
        x, t, f = x.flip(0), t.flip(0), f.flip(0)
        sign[2] = -1.0
    if (k & 4) and ny == nz:
        x, t, f = x.transpose(0, 1), t.transpose(0, 1), f.transpose(0, 1)
        t = t[..., [0, 2, 1, 3]]
        sign[1], sign[2] = sign[2], sign[1]
    t = t * t.new_tensor(sign)
    return x.contiguous().view(-1, x.shape[-1]), t.contiguous().view(-1, 4), f.contiguous().view(-1)


def train(net, samples, epochs, lr=1e-3, lr_final=1e-4, seed=0, log=None, augment=True):
    """Adam over the samples in a seeded random order each epoch, cosine-decayed learning rate;
    with augment, each visit takes one of the eight y-z symmetric copies of the sample (drawn
    from the same seeded generator).  Returns the mean loss of each epoch."""
    rng = np.random.default_rng(seed)
    total = epochs * len(samples)
    hist, it = [], 0
    for ep in range(epochs):
        acc = []
        for j in rng.permutation(len(samples)):
            s = samples[j]
            a = lr_final + 0.5 * (lr - lr_final) * (1 + math.cos(math.pi * it / max(1, total - 1)))
            x, t, fl = symmetric_copy(s, int(rng.integers(8))) if augment else (s.x, s.t, s.fluid)
            loss = net.train_step(x, t, fl, s.n_fluid, s.geom.shape, lr=a)
            acc.append(loss)
            it += 1
        net.check()
        m = float(sum(float(v.item()) for v in acc) / len(acc))
        hist.append(m)
        if log:
            log(f"epoch {ep}: loss {m:.4e}")
    return hist


def compare(net, seeds, n=128, tol=1e-6, max_steps=400_000, device=0, rng_seed=99):
    """Time to steady state from rest and from the network's prediction on held-out seeds."""
    import torch
    rng = np.random.default_rng(rng_seed)
    rows = []
    for seed in seeds:
        Pe, Da = draw_transport(rng)
        cfg, geom, fields = case(seed, n, Pe, Da)
        cfg = dict(cfg, device=device)
        steps0, sec0, ok0, s0 = run_to_steady(cfg, geom, fields, tol, max_steps)
        f_ref = s0.fields()
        s0.close()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        warm = sg.predict_fields(net, geom, Pe, Da)
        torch.cuda.synchronize()
        t_inf = time.perf_counter() - t0
        steps1, sec1, ok1, s1 = run_to_steady(cfg, geom, warm, tol, max_steps)
        f_w = s1.fields()
        s1.close()
        fl = geom == 0
        if not (np.all(np.isfinite(warm[1])) and np.all(np.isfinite(warm[2]))):
            ok1 = False
        eC = float(np.linalg.norm((warm[2][0] - f_ref["C"][0])[fl]) / np.linalg.norm(f_ref["C"][0][fl]))
        eu = float(np.linalg.norm((warm[1] - f_ref["u"])[:, fl]) / np.linalg.norm(f_ref["u"][:, fl]))
        # both runs end at the same steady state (to the tolerance): the network changes the path only
        dC = float(np.linalg.norm((f_w["C"][0] - f_ref["C"][0])[fl]) / np.linalg.norm(f_ref["C"][0][fl]))
        # the warm run counts only if it reached the rest run's steady state
        ok1 = ok1 and math.isfinite(dC) and dC <= 1e-2
        rows.append({"seed": seed, "Pe": Pe, "Da": Da, "rest_steps": steps0, "rest_s": sec0,
                     "warm_steps": steps1, "warm_s": sec1 + t_inf, "inference_s": t_inf,
                     "converged_rest": ok0, "converged_warm": ok1, "converged": ok0 and ok1,
                     "pred_err_C": eC, "pred_err_u": eu,
                     "final_fields_rel_diff_C": dC,
                     "speedup_steps": steps0 / max(1, steps1), "speedup_time": sec0 / (sec1 + t_inf)})
    return rows
