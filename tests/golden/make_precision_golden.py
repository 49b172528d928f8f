"""Write tests/golden/precision64_pe{Pe}.npz: the FP64 oracle on a 64^3 crop of the dissolution
workload, the reference against which the 16-bit storage modes state their error per field.

Case: the corner 64^3 crop of the seeded 256^3 random-sphere packing (radius 6-12, porosity 0.4),
D3Q19 MRT flow by body force + D3Q7 solute with the wet-node reaction (Sec. 2.1.1, 2.1.5), the
transport numbers of the workload (tau_c from Pe, k from Da), geometry update frozen, run for the
workload's 20,000 steps.  Stored at steps 2,000 and 20,000, at every 4th fluid node (node index
n = x + 64 (y + 64 z)): rho - 1, u, C - 1 (the deviations from the rest state that 16-bit storage
keeps), as float32 (their own rounding, ~6e-8 relative, is far below the errors being measured).

Only oracle/ and the seeded input generator are used: no value comes from the CUDA path.
Run from the repository root:  python tests/golden/make_precision_golden.py [Pe ...]
"""
from __future__ import annotations

import multiprocessing as mp
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
N = 64
CHECKPOINTS = (2000, 20000)


def crop_case(Pe=10.0, Da=0.1):
    sys.path.insert(0, ROOT)
    from paper_2502_12955_gb300 import inputs

    cfg, geom, _ = inputs.dissolution_3d(n=256)
    geom = np.ascontiguousarray(geom[:N, :N, :N])
    # transport numbers: D = U L / Pe (U = 0.0185, L = 9), tau_c = D / c_s^2 + 1/2 (c_s^2 = 1/4), k = Da D / L
    D = 0.0185 * 9.0 / Pe
    cfg = dict(cfg, nx=N, ny=N, nz=N, tau_c=[D / 0.25 + 0.5], k_react=Da * D / 9.0, geo_mode="none")
    rho, u, C = inputs.uniform_fields((N, N, N), 1, 1, rho=1.0, C=1.0)
    return cfg, geom, (rho, u, C)


def sample_nodes(geom):
    fl = np.flatnonzero(geom.reshape(-1) == 0)
    return fl[::4]


def run(Pe):
    sys.path.insert(0, ROOT)
    from oracle.oracle import Oracle

    cfg, geom, fields = crop_case(Pe)
    o = Oracle(dict(cfg, precision="fp64"))
    o.set_geometry(geom)
    o.set_fields(*fields)
    nodes = sample_nodes(geom)
    out, done = {"nodes": nodes, "Pe": np.array(Pe), "tau_c": np.array(cfg["tau_c"][0]),
                 "k_react": np.array(cfg["k_react"])}, 0
    for t in CHECKPOINTS:
        o.step(t - done)
        done = t
        f = o.fields()
        out[f"drho_{t}"] = (f["rho"][0].reshape(-1)[nodes] - 1.0).astype(np.float32)
        out[f"u_{t}"] = f["u"].reshape(3, -1)[:, nodes].astype(np.float32)
        out[f"dC_{t}"] = (f["C"][0].reshape(-1)[nodes] - 1.0).astype(np.float32)
        out[f"Cmin_{t}"] = np.array(f["C"][0][geom == 0].min())
    path = os.path.join(HERE, f"precision64_pe{int(round(Pe))}.npz")
    np.savez_compressed(path, **out)
    return path


if __name__ == "__main__":
    pes = [float(p) for p in sys.argv[1:]] or [10.0]
    with mp.get_context("spawn").Pool(len(pes)) as pool:
        for p in pool.imap_unordered(run, pes):
            print("wrote", p, flush=True)
