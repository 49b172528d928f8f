"""Pins of the oracle's reaction product (CO2) lattice (Sec. 2.1.5, Eq. react, reactCO2).

At each reactive link the product enters the fluid at the rate the reaction takes the species.
The pins: with equal diffusivities the sum species + product does not react at all, so it equals
a run without reaction; in a 1D channel at steady state the product leaves through the inlet
with a linear profile whose flux is the reaction rate; and the product's budget closes exactly
per step.
"""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2502_12955_gb300 import inputs


def make(cfg, geom, fields):
    o = Oracle(cfg)
    o.set_geometry(geom)
    o.set_fields(*fields)
    return o


@pytest.mark.parametrize("mode", ["constant", "arrhenius", "conjugate"])
def test_species_plus_product_does_not_react(mode):
    """With tau_p = tau_c, the closures of species and product add up, link by link, to the
    wet node with k = 0 (h_i = h_opp(i)): species + product follows the same flow, the same
    inlet (C_in + C_in_p) and outlet, and no reaction. It must equal, on every node and to
    round-off, a single scalar started from the sum with k = 0."""
    shape = (1, 12, 14)
    geom = inputs.random_solids(shape, 0.25, seed=71, reactive_fraction=0.7)
    ns = 1 if mode == "constant" else 2
    rho, u, C = inputs.perturbed_fields(shape, 1, ns + 1, seed=72, amp_rho=0.01, amp_u=0.01, C0=0.9)
    base = dict(dim=2, nx=14, ny=12, tau=[0.8], g=[2e-4, 0, 0], J0=0.4, ade_open_x=True,
                periodic=[1, 0, 1])
    tau0 = 0.7
    if mode == "constant":
        cfg = dict(base, n_scal=1, tau_c=[tau0], k_react=0.08, C_in=[1.0])
    else:
        cfg = dict(base, n_scal=2, tau_c=[tau0, 0.9], C_in=[1.0, 0.8], arrhenius=True, arr_A=0.5,
                   arr_Ta=0.6, heat_release=0.05, n_it=32)
        if mode == "conjugate":
            cfg.update(conjugate=True, tau_s=0.65, c_fs=2.0)
    a = make(dict(cfg, product=True, tau_p=tau0, C_in_p=0.2), geom, (rho, u, C))
    b = make(dict(base, n_scal=1, tau_c=[tau0], k_react=0.0, C_in=[1.2]), geom,
             (rho, u, C[0] + C[ns]))
    a.step(60)
    b.step(60)
    fa, fb = a.fields(), b.fields()
    total = fa["C"][0] + fa["C"][ns]
    fluid = fa["flags"] == 0
    assert np.abs(total - fb["C"][0])[fluid].max() < 1e-13
    assert a.monitors()["produced"] > 0
    assert np.abs(fa["C"][ns] - C[ns])[fluid].max() > 1e-3     # the product did change


@pytest.mark.parametrize("tau_p", [0.7, 1.3])
def test_steady_product_flux_is_the_reaction_rate(tau_p):
    """1D channel at rest: the species enters at the inlet and reacts at the far wall, the
    product (inlet value 0) is made there and leaves through the inlet. At steady state both
    profiles are linear, and the product's flux through every link,
    D_p (C_p(x+1) - C_p(x)) with D_p = c_s^2 (tau_p - 1/2), equals the reaction per step."""
    nx = 16
    geom = np.zeros((1, 1, nx), np.uint8)
    geom[0, 0, nx - 1] = 2
    cfg = dict(dim=2, nx=nx, ny=1, tau=[1.0], n_scal=1, tau_c=[0.8], J0=0.4, k_react=0.02,
               ade_open_x=True, C_in=[1.0], product=True, tau_p=tau_p, C_in_p=0.0, periodic=[1, 1, 1])
    shape = (1, 1, nx)
    rho, u = np.ones((1,) + shape), np.zeros((3,) + shape)
    o = make(cfg, geom, (rho, u, np.zeros((2,) + shape)))
    o.step(60000)
    m0 = o.monitors()
    o.step(1)
    m1 = o.monitors()
    reaction = m1["reacted"] - m0["reacted"]
    P = o.fields()["C"][1, 0, 0, : nx - 1]
    D = 0.3 * (tau_p - 0.5)
    np.testing.assert_allclose(P[1:-2] - 2 * P[2:-1] + P[3:], 0, atol=1e-12)
    np.testing.assert_allclose(D * (P[2:-1] - P[1:-2]), reaction, rtol=1e-9)
    # what is made leaves through the inlet
    np.testing.assert_allclose(-(m1["inflow_p"] - m0["inflow_p"]), reaction, rtol=1e-9)
    assert reaction > 0


def test_product_budget_per_step():
    """With flow, open faces, walls and dissolution flips, the product lattice changes each step
    by exactly what the reactive links add, what the inlet and outlet carry, and what the new
    fluid nodes bring."""
    shape = (1, 12, 14)
    geom = inputs.random_solids(shape, 0.25, seed=73, reactive_fraction=0.7)
    rho, u, C = inputs.perturbed_fields(shape, 1, 2, seed=74, amp_rho=0.01, amp_u=0.01, C0=0.9)
    cfg = dict(dim=2, nx=14, ny=12, tau=[0.8], g=[3e-4, 0, 0], n_scal=1, tau_c=[0.7], J0=0.4,
               k_react=0.1, ade_open_x=True, C_in=[1.0], product=True, tau_p=1.1, C_in_p=0.05,
               geo_mode="dissolve", V_m=60.0, periodic=[1, 0, 1])
    o = make(cfg, geom, (rho, u, C))
    for _ in range(40):
        m0 = o.monitors()
        o.step(1)
        m1 = o.monitors()
        d = {k: m1[k] - m0[k] for k in ("species_p", "produced", "inflow_p", "outflow_p", "inj_spec_p")}
        rhs = d["produced"] + d["inflow_p"] - d["outflow_p"] + d["inj_spec_p"]
        assert abs(d["species_p"] - rhs) < 1e-12 * m0["species_p"]
    assert m1["produced"] > 0 and m1["inj_spec_p"] > 0


def test_product_needs_the_reacting_species():
    ok = dict(dim=2, nx=8, ny=8, n_scal=1, k_react=0.1, product=True, tau_p=0.8)
    Oracle(ok)
    for bad in (dict(n_scal=0), dict(tau_p=0.5), dict(geo_mode="deposit", DP=0.1)):
        with pytest.raises(Exception):
            Oracle(dict(ok, **bad))
