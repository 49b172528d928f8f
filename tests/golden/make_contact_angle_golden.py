"""Write tests/golden/sessile200_g*.npz: the FP64 oracle's sessile droplet (contact-angle case of
Sec. 3.2) after 60,000 steps, for adhesion G_ads = (g, -g), g = -0.15, 0, 0.15.

Case (inputs.sessile_droplet_2d): 200 x 80 D2Q9, two components, psi = rho, cross cohesion
G = 2.7, tau 1, a half disc of radius 30 of component 0 (1.0 / 0.05) on the closed bottom face,
periodic x.  Stored: the final densities of both components (float64, node order) and the
step count.  The GPU test runs the same case in FP64, compares the fields, and measures the
angle on both.

Only oracle/ and the seeded input generators are used: no value comes from the CUDA path.
Run from the repository root:  python tests/golden/make_contact_angle_golden.py [g ...]
"""
from __future__ import annotations

import multiprocessing as mp
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
STEPS = 60000


def path_of(g):
    return os.path.join(HERE, f"sessile200_g{g:+.2f}.npz")


def run(g):
    sys.path.insert(0, ROOT)
    from oracle.oracle import Oracle
    from paper_2502_12955_gb300 import inputs

    cfg, geom, fields = inputs.sessile_droplet_2d(g_ads=g, precision="fp64")
    o = Oracle(cfg)
    o.set_geometry(geom)
    o.set_fields(*fields)
    o.step(STEPS)
    rho = o.fields()["rho"]
    np.savez_compressed(path_of(g), rho=rho, steps=np.array(STEPS), g_ads=np.array(g))
    return path_of(g)


if __name__ == "__main__":
    gs = [float(v) for v in sys.argv[1:]] or [-0.15, 0.0, 0.15]
    with mp.get_context("spawn").Pool(len(gs)) as pool:
        for p in pool.imap_unordered(run, gs):
            print("wrote", p, flush=True)
