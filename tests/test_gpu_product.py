"""The reaction product (CO2) lattice on the GPU against the FP64 oracle (Sec. 2.1.5, Eq. react,
reactCO2): at each reactive link the product gains the rate the reaction takes from scalar 0
there, h_P,i = h_P,opp(i) + r tau_p / (tau_p - 1/2).  Every field, population array (the product's
included) and monitor (species_p, inflow_p, outflow_p, inj_spec_p, produced) within 1e-10, flags
exact, at both layout parities."""
import numpy as np
import pytest

from paper_2502_12955_gb300 import inputs
from tests.gpu_common import compare, make_pair

pytestmark = pytest.mark.gpu


def _fields(shape, n_lat, seed, C0=0.9):
    rho, u, C = inputs.perturbed_fields(shape, 1, n_lat, seed=seed, amp_rho=0.01, amp_u=0.01, C0=C0)
    return rho, u, C


@pytest.mark.parametrize("steps", [7, 40])
def test_product_2d_open_faces(steps):
    """D2Q9 BGK + D2Q5 species and product, inlet / outlet on both, reactive and inert solids."""
    shape = (1, 19, 27)
    geom = inputs.random_solids(shape, 0.2, seed=70, reactive_fraction=0.7)
    geom[0, :, 0] = 0
    geom[0, :, -1] = 0
    cfg = dict(dim=2, nx=27, ny=19, tau=[0.8], g=[3e-5, -1e-5, 0], n_scal=1, tau_c=[0.7], J0=0.4,
               k_react=0.06, ade_open_x=True, C_in=[1.0], product=True, tau_p=1.1, C_in_p=0.05,
               periodic=[1, 1, 1])
    o, g = make_pair(cfg, geom, _fields(shape, 2, 71))
    o.step(steps)
    g.step(steps)
    compare(o, g, what=f"product 2d {steps}")
    assert o.monitors()["produced"] > 0


@pytest.mark.parametrize("steps", [60, 61])
def test_product_3d_mrt_with_dissolution(steps):
    """D3Q19 MRT + D3Q7 species and product, dissolution flips: a new fluid node takes its
    neighbours' mean product like any scalar."""
    cfg, geom, (rho, u, C) = inputs.dissolution_3d(shape=(11, 14, 20), g=5e-4, radius=(2.0, 4.0),
                                                   precision="fp64")
    cfg.update(k_react=0.05, V_m=25.0, product=True, tau_p=0.8, C_in_p=0.0)
    Cp = np.concatenate([C, 0.02 * np.ones_like(C)])
    o, g = make_pair(cfg, geom, (rho, u, Cp))
    o.step(steps)
    g.step(steps)
    assert o.monitors()["inj_spec_p"] != 0.0, "the case should dissolve solids"
    compare(o, g, what=f"product 3d mrt {steps}")


@pytest.mark.parametrize("dim,steps", [(2, 41), (3, 30)])
def test_product_with_temperature_dependent_rate(dim, steps):
    """Three scalar lattices: species, temperature with k(T_b) and reaction heat, and the
    product of the same link rates (the paper's O2, T, CO2)."""
    if dim == 2:
        shape = (1, 14, 18)
        cfg = dict(dim=2, nx=18, ny=14, tau=[0.8], g=[2e-4, 0, 0], n_scal=2, tau_c=[0.7, 0.9], J0=0.4,
                   arrhenius=True, arr_A=0.4, arr_Ta=1.0, heat_release=0.02, n_it=24,
                   ade_open_x=True, C_in=[1.0, 0.6], product=True, tau_p=0.75, C_in_p=0.0,
                   periodic=[1, 1, 1])
    else:
        shape = (8, 10, 12)
        cfg = dict(dim=3, nx=12, ny=10, nz=8, tau=[0.9], collision="mrt", g=[1e-4, 0, 0], n_scal=2,
                   tau_c=[0.6, 0.8], J0=0.25, arrhenius=True, arr_A=0.3, arr_Ta=0.8, heat_release=0.03,
                   n_it=24, periodic=[1, 0, 1], geo_mode="dissolve", V_m=40.0, m_s0=1.0, product=True,
                   tau_p=0.9)
    geom = inputs.random_solids(shape, 0.18, seed=72 + dim, reactive_fraction=0.7)
    o, g = make_pair(cfg, geom, _fields(shape, 3, 73))
    o.step(steps)
    g.step(steps)
    compare(o, g, what=f"product thermal {dim}d")


def test_product_with_two_plain_scalars():
    """Two scalars with the constant-rate closure on scalar 0, plus the product (three lattices,
    the plain kernel variant), 3D BGK with walls on a closed axis."""
    shape = (9, 13, 18)
    geom = inputs.random_solids(shape, 0.15, seed=74, reactive_fraction=0.6)
    cfg = dict(dim=3, nx=18, ny=13, nz=9, tau=[0.9], g=[1e-5, 2e-6, -3e-6], n_scal=2, tau_c=[0.8, 0.6],
               J0=0.25, k_react=0.02, product=True, tau_p=0.7, periodic=[1, 0, 1])
    o, g = make_pair(cfg, geom, _fields(shape, 3, 75))
    o.step(33)
    g.step(33)
    compare(o, g, what="product with two scalars")
