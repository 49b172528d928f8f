"""Write tests/golden/droplet64_R*.npz: the FP64 oracle's two-component static droplet at 64^3.

The droplet workload (D3Q19 per component, psi = rho, cross-cohesion G = 2.7, tau 1, fully
periodic, a sharp sphere of densities 1.0 / 0.05 centred in the box; Sec. 3.2.2 with the
readings of the two-component psi convention and of the initial droplet) is the 128^3 workload
at half scale: radii 8, 12 and 16 instead of 16, 24 and 32.  The oracle needs about two hours
per radius for 10,000 steps, so its results are stored here, sampled, and the GPU test compares
its own FP64 run against them at the same nodes.

Stored per checkpoint (steps 2000 and 10000):
  rho, u   densities (2) and velocity (3) at the sample nodes: every node of the central plane
           z = 32 and 1024 seeded random nodes elsewhere (node index n = x + 64 (y + 64 z));
  mass     the total mass of each component (conserved exactly by the method);
  dp       p(centre) - p(corner) with p = c_s^2 (rho_1 + rho_2 + G rho_1 rho_2);
  umax     the largest |u| over the whole domain (spurious currents);
  rho2sum  sum over all nodes of rho_1^2 and rho_2^2 (a whole-field check).

Only oracle/ and the seeded input generators are used: no value comes from the CUDA path.
Run from the repository root:  python tests/golden/make_droplet_golden.py [R ...]
"""
from __future__ import annotations

import multiprocessing as mp
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))

N = 64
G = 2.7
RADII = (8.0, 12.0, 16.0)
CHECKPOINTS = (2000, 10000)


def sample_nodes(n=N, extra=1024, seed=64):
    plane = np.arange(n * n, dtype=np.int64) + (n // 2) * n * n
    rng = np.random.default_rng(seed)
    others = rng.choice(np.setdiff1d(np.arange(n ** 3, dtype=np.int64), plane), size=extra, replace=False)
    return np.sort(np.concatenate([plane, others]))


def summarise(rho, u, nodes):
    cs2 = 1.0 / 3.0
    p = cs2 * (rho[0] + rho[1]) + cs2 * G * rho[0] * rho[1]
    c = N // 2
    return dict(
        rho=rho.reshape(2, -1)[:, nodes], u=u.reshape(3, -1)[:, nodes],
        mass=rho.reshape(2, -1).sum(axis=1), dp=np.array(p[c, c, c] - p[0, 0, 0]),
        umax=np.array(np.sqrt((u ** 2).sum(axis=0)).max()),
        rho2sum=(rho.reshape(2, -1) ** 2).sum(axis=1))


def run(R):
    sys.path.insert(0, ROOT)
    from oracle.oracle import Oracle
    from paper_2502_12955_gb300 import inputs

    cfg, geom, _ = inputs.droplet_3d(n=N, radius=R, precision="fp64", G=G)
    rho, u = inputs.droplet_fields((N, N, N), R)
    o = Oracle(cfg)
    o.set_geometry(geom)
    o.set_fields(rho, u, None)
    nodes = sample_nodes()
    out, done = {"nodes": nodes, "R": np.array(R), "G": np.array(G)}, 0
    for t in CHECKPOINTS:
        o.step(t - done)
        done = t
        f = o.fields()
        for k, v in summarise(f["rho"], f["u"], nodes).items():
            out[f"{k}_{t}"] = v
    path = os.path.join(HERE, f"droplet64_R{int(R)}.npz")
    np.savez_compressed(path, **out)
    return path


if __name__ == "__main__":
    radii = [float(r) for r in sys.argv[1:]] or list(RADII)
    with mp.get_context("spawn").Pool(len(radii)) as pool:
        for p in pool.imap_unordered(run, radii):
            print("wrote", p, flush=True)
