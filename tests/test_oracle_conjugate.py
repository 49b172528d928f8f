"""Pins of the oracle's heat conduction in the solid and its exchange with the fluid temperature
(Sec. 2.1.5, Eq. therpop_solid, macroreacb_solid, tempCon, fluxCon, reacRate).

The exchange is checked against what the physics fixes without it: two identical media must
behave as one medium, two half-spaces put in contact must reach the contact temperature of the
erf solution of the heat equation, the energy of both lattices must change by exactly the
reaction heat and what the open faces and the flips carry, and the heat of each link must match
the reaction that the species closure books for it.
"""
from math import erf, sqrt

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2502_12955_gb300 import inputs


def make(cfg, geom, fields):
    o = Oracle(cfg)
    o.set_geometry(geom)
    rho, u, C = fields
    o.set_fields(rho, u, C)
    return o


def _at_rest(shape, seed, T_lo=0.5, T_hi=0.8):
    """Uniform density, zero velocity (so the flow stays exactly at rest) and random
    species and temperature on every node, solids included."""
    rng = np.random.default_rng(seed)
    rho = np.ones((1,) + shape)
    u = np.zeros((3,) + shape)
    C = np.stack([1.0 + 0.1 * rng.random(shape), T_lo + (T_hi - T_lo) * rng.random(shape)])
    return rho, u, C


@pytest.mark.parametrize("dim", [2, 3])
def test_identical_media_are_one_medium(dim):
    """With c_fs = 1, tau_s = tau_T and no reaction heat, the solid conducts exactly as the fluid
    at rest: the temperature of a domain with solids equals that of the same domain without
    them, on every node, to round-off."""
    shape = (1, 12, 16) if dim == 2 else (6, 8, 10)
    nz, ny, nx = shape
    geom = inputs.random_solids(shape, 0.3, seed=3 + dim, reactive_fraction=0.6)
    fields = _at_rest(shape, 11 + dim)
    base = dict(dim=dim, nx=nx, ny=ny, nz=nz, tau=[0.8], n_scal=2, tau_c=[0.7, 0.9],
                J0=0.4 if dim == 2 else 0.25, periodic=[1, 0, 1])
    a = make(dict(base, arrhenius=True, arr_A=0.3, arr_Ta=0.8, heat_release=0.0, n_it=8,
                  conjugate=True, tau_s=0.9, c_fs=1.0), geom, fields)
    b = make(base, np.zeros_like(geom), fields)
    a.step(25)
    b.step(25)
    Ta, Tb = a.fields()["C"][1], b.fields()["C"][1]
    assert np.abs(Ta - Tb).max() < 1e-14
    assert np.ptp(Tb) > 0.005         # the field has not flattened: the comparison has content
    assert a.monitors()["reacted"] > 0


def _contact(dim, t_steps, tau_T=0.9, tau_s=0.7, c_fs=2.0, Tf0=1.0, Ts0=0.5):
    n = 160
    shape = (1, 2, n) if dim == 2 else (2, 2, n)
    geom = np.zeros(shape, np.uint8)
    geom[..., : n // 2] = 1
    rho, u = np.ones((1,) + shape), np.zeros((3,) + shape)
    C = np.stack([np.ones(shape), np.where(geom == 1, Ts0, Tf0)])
    J0 = 0.4 if dim == 2 else 0.25
    cfg = dict(dim=dim, nx=n, ny=2, nz=shape[0], tau=[0.8], n_scal=2, tau_c=[0.7, tau_T], J0=J0,
               periodic=[0, 1, 1], arrhenius=True, arr_A=0.0, arr_Ta=0.0, heat_release=0.0,
               conjugate=True, tau_s=tau_s, c_fs=c_fs)
    o = make(cfg, geom, (rho, u, C))
    cs2 = (1.0 - J0) / dim               # the scalar lattice's c_s^2; alpha = c_s^2 (tau - 1/2)
    a_f, a_s = cs2 * (tau_T - 0.5), cs2 * (tau_s - 0.5)
    # contact temperature of two semi-infinite bodies: effusivities e = rho c_p sqrt(alpha),
    # in units of the solid's rho c_p
    e_f, e_s = c_fs * sqrt(a_f), sqrt(a_s)
    Tc = (e_f * Tf0 + e_s * Ts0) / (e_f + e_s)
    errs = []
    xi = n // 2 - 0.5                    # the interface lies halfway between the two nodes
    for t in t_steps:
        o.step(t - int(o.monitors()["step"]))
        T = o.fields()["C"][1][0, 0]
        ex = np.array([Tc + (Tf0 - Tc) * erf((x - xi) / (2 * sqrt(a_f * t))) if x > xi else
                       Tc + (Ts0 - Tc) * erf((xi - x) / (2 * sqrt(a_s * t))) for x in range(n)])
        errs.append(np.abs(T - ex).max() / (Tf0 - Ts0))
    return errs


@pytest.mark.parametrize("dim", [2, 3])
def test_two_half_spaces_reach_the_contact_temperature(dim):
    """A fluid half-space at T_f and a solid one at T_s, put in contact at t = 0, follow the erf
    solutions of the heat equation on each side about the contact temperature
    (e_f T_f + e_s T_s) / (e_f + e_s), e = rho c_p sqrt(alpha): the error falls as 1/t (second
    order in the lattice spacing over the diffusion length).  Swapping c_fs, or the two
    relaxation times, moves the contact temperature by tens of percent of T_f - T_s."""
    e200, e400 = _contact(dim, (200, 400))
    assert e400 < 1.5e-3
    assert 1.7 < e200 / e400 < 2.3


def _energy(m, c_fs):
    """Heat in both lattices, in units of the fluid's rho c_p."""
    return m["species1"] + m["tsolid"] / c_fs


@pytest.mark.parametrize("geo", [dict(), dict(geo_mode="dissolve", V_m=60.0)])
def test_energy_budget_per_step(geo):
    """With flow, reaction heat, c_fs != 1 and tau_s != tau_T, the heat in both lattices changes
    each step by exactly the reaction heat put into the exchanges, plus what the dissolution
    flips move from the solid into the fluid (the node keeps its temperature, so the fluid gains
    T_s while the solid loses T_s / c_fs)."""
    c_fs = 2.5
    shape = (1, 12, 14)
    geom = inputs.random_solids(shape, 0.25, seed=61, reactive_fraction=0.7)
    rho, u, C = inputs.perturbed_fields(shape, 1, 2, seed=62, amp_rho=0.01, amp_u=0.01, C0=0.9)
    cfg = dict(dim=2, nx=14, ny=12, tau=[0.8], g=[3e-4, 0, 0], n_scal=2, tau_c=[0.7, 0.9], J0=0.4,
               periodic=[1, 0, 1], arrhenius=True, arr_A=0.4, arr_Ta=0.8, heat_release=0.05, n_it=24,
               conjugate=True, tau_s=0.65, c_fs=c_fs, **geo)
    o = make(cfg, geom, (rho, u, C))
    for _ in range(40):
        m0 = o.monitors()
        o.step(1)
        m1 = o.monitors()
        d = {k: m1[k] - m0[k] for k in ("heat_src", "heat", "heat_s", "inj_spec1", "solid_rem")}
        dE = _energy(m1, c_fs) - _energy(m0, c_fs)
        assert abs(dE - (d["heat_src"] + d["inj_spec1"] - d["solid_rem"] / c_fs)) < 1e-12 * _energy(m0, c_fs)
        assert abs(d["heat"] + d["heat_s"] / c_fs - d["heat_src"]) < 1e-13
        assert d["inj_spec1"] == d["solid_rem"]
    assert m1["heat_src"] > 0
    if geo:
        assert m1["solid_rem"] > 0, "no flip happened"


def test_reaction_heat_matches_the_booked_reaction():
    """The exchange of step t solves C_b and T_b together and keeps k(T_b); the species closure
    of step t + 1 books k C_b for the same link.  So the heat of steps 1..K equals h_r times
    the reaction booked by the closures of steps 2..K+1 (Eq. reacRate)."""
    shape = (1, 12, 14)
    geom = inputs.random_solids(shape, 0.25, seed=63, reactive_fraction=0.7)
    fields = inputs.perturbed_fields(shape, 1, 2, seed=64, amp_rho=0.01, amp_u=0.01, C0=0.9)
    hr, tau_T = 0.05, 0.9
    cfg = dict(dim=2, nx=14, ny=12, tau=[0.8], g=[2e-4, 0, 0], n_scal=2, tau_c=[0.7, tau_T], J0=0.4,
               periodic=[1, 0, 1], arrhenius=True, arr_A=0.4, arr_Ta=0.8, heat_release=hr, n_it=32,
               conjugate=True, tau_s=0.65, c_fs=2.5)
    first = make(cfg, geom, fields)
    first.step(1)
    o = make(cfg, geom, fields)
    K = 20
    o.step(K)
    heat = o.monitors()["heat_src"]
    o.step(1)
    booked = o.monitors()["reacted"] - first.monitors()["reacted"]
    assert heat > 0
    assert abs(heat - hr * booked) < 1e-12 * heat


def test_uniform_temperature_gives_the_rate_at_that_temperature():
    """Fluid at rest and solid at one temperature T0, no reaction heat: every link's T_b is T0
    whatever c_fs and tau_s, so the species equal those of the constant rate A exp(-Ta / T0) and
    the temperature stays T0 on every node."""
    shape = (1, 12, 14)
    geom = inputs.random_solids(shape, 0.25, seed=65, reactive_fraction=0.7)
    T0, A, Ta = 1.3, 0.2, 0.9
    rho, u, C = _at_rest(shape, 66)
    C[1] = T0
    cfg = dict(dim=2, nx=14, ny=12, tau=[0.8], n_scal=2, tau_c=[0.7, 0.9], J0=0.4, periodic=[1, 0, 1])
    a = make(dict(cfg, arrhenius=True, arr_A=A, arr_Ta=Ta, heat_release=0.0, conjugate=True,
                  tau_s=0.6, c_fs=3.0), geom, (rho, u, C))
    b = make(dict(cfg, k_react=A * np.exp(-Ta / T0)), geom, (rho, u, C))
    a.step(30)
    b.step(30)
    fa, fb = a.fields(), b.fields()
    assert np.abs(fa["C"][0] - fb["C"][0]).max() < 1e-13
    assert np.abs(fa["C"][1] - T0).max() < 1e-13
    assert abs(a.monitors()["reacted"] - b.monitors()["reacted"]) < 1e-12 * b.monitors()["reacted"]


def test_coupling_converges_in_the_iterations():
    """The fixed-point iterations of the C_b - T_b coupling converge: 40 and 80 iterations give
    the same fields to round-off, while a single one does not."""
    shape = (1, 12, 14)
    geom = inputs.random_solids(shape, 0.25, seed=67, reactive_fraction=0.7)
    fields = inputs.perturbed_fields(shape, 1, 2, seed=68, amp_rho=0.01, amp_u=0.01, C0=0.9)
    cfg = dict(dim=2, nx=14, ny=12, tau=[0.8], n_scal=2, tau_c=[0.7, 0.9], J0=0.4, periodic=[1, 0, 1],
               arrhenius=True, arr_A=0.6, arr_Ta=1.5, heat_release=0.3, conjugate=True, tau_s=0.65, c_fs=2.5)
    runs = {}
    for n_it in (0, 40, 64):
        o = make(dict(cfg, n_it=n_it), geom, fields)
        o.step(10)
        runs[n_it] = o.fields()["C"]
    assert np.abs(runs[40] - runs[64]).max() < 1e-13
    assert np.abs(runs[0] - runs[64]).max() > 1e-8


def test_conduction_needs_the_temperature_rate_and_valid_media():
    ok = dict(dim=2, nx=8, ny=8, n_scal=2, arrhenius=True, arr_A=0.1, arr_Ta=1.0, conjugate=True,
              tau_s=0.8, c_fs=1.0)
    Oracle(ok)
    for bad in (dict(arrhenius=False), dict(tau_s=0.5), dict(c_fs=0.0), dict(geo_mode="deposit")):
        with pytest.raises(Exception):
            Oracle(dict(ok, **bad))


def test_reactive_channel_budgets():
    """The reactive porous channel of Sec. 3.4 in small (84 x 16, four carbon discs): velocity
    inlet, O2, temperature and CO2 entering at x = 0, the temperature-dependent rate, heat
    release, conduction in the discs and the CO2 product, all at once. Each step the O2, the CO2
    and the heat of both lattices change by exactly what the links and the open faces carry; the
    fields stay within the bounds the inlet and the initial state set (O2 below its inlet value,
    CO2 non-negative, the temperature not below its initial value under an exothermic
    reaction)."""
    cfg, geom, fields = inputs.combustion_channel_2d(nx=84, ny=16)
    o = make(cfg, geom, fields)
    c_fs = cfg["c_fs"]
    for _ in range(600):
        m0 = o.monitors()
        o.step(1)
        m1 = o.monitors()

        def d(k):
            return m1[k] - m0[k]

        o2 = d("species0") - (d("inflow0") - d("outflow0") - d("wallx"))
        co2 = d("species_p") - (d("produced") + d("inflow_p") - d("outflow_p"))
        heat = (_energy(m1, c_fs) - _energy(m0, c_fs)) - (d("heat_src") + d("inflow1") - d("outflow1"))
        assert abs(o2) < 1e-13 * max(m1["species0"], 1.0)
        assert abs(co2) < 1e-13 * max(m1["species_p"], 1.0)
        assert abs(heat) < 1e-13 * _energy(m1, c_fs)
    f = o.fields()
    assert m1["nonfinite"] == 0
    assert m1["heat_src"] > 0 and m1["produced"] > 0
    assert f["C"][0].max() <= cfg["C_in"][0]
    assert f["C"][2].min() >= 0.0
    assert f["C"][1].min() >= 1.0 - 1e-12
    assert f["C"][1][geom == 2].max() > 1.0      # the discs heat up


@pytest.mark.parametrize("dim,J0", [(2, 0.4), (3, 0.25)])
def test_steady_front_fluxes_and_interface_temperature(dim, J0):
    """1D burning front at steady state: O2 enters at x = 0 and reacts at the face of a carbon
    slab whose far end is adiabatic; heat and CO2 flow back to the inlet. Then (Eq. reactO2,
    reactCO2, fluxCon, tempCon):
    - the O2 and CO2 profiles are linear with link fluxes D ΔC equal to the reaction per step,
    - the fluid temperature is linear, with link flux D_T ΔT equal to the heat released per step,
      which is h_r times the reaction (Eq. reacRate, the same flux the adiabatic closure gives),
    - the slab is isothermal (no heat leaves through its far end), at the temperature the fluid
      profile takes at the halfway face: temperature continuity,
    - and all of it equals the closed-form steady state, up to one bracketed root for T_b."""
    nx, nf = 16, 10
    geom = np.zeros((1, 1, nx), np.uint8)
    geom[0, 0, nf:] = 2
    tau_O, tau_T, tau_P, hr = 0.8, 0.9, 0.75, 0.5
    cfg = dict(dim=dim, nx=nx, ny=1, nz=1, tau=[1.0], n_scal=2, tau_c=[tau_O, tau_T], J0=J0, ade_open_x=True,
               C_in=[1.0, 1.0], arrhenius=True, arr_A=0.5, arr_Ta=1.0, heat_release=hr, n_it=40,
               conjugate=True, tau_s=0.7, c_fs=0.5, product=True, tau_p=tau_P, C_in_p=0.0,
               periodic=[1, 1, 1])
    shape = (1, 1, nx)
    C = np.zeros((3,) + shape)
    C[1] = 1.0
    o = make(cfg, geom, (np.ones((1,) + shape), np.zeros((3,) + shape), C))
    o.step(80000)
    m0 = o.monitors()
    o.step(1)
    m1 = o.monitors()
    reaction = m1["reacted"] - m0["reacted"]
    heat = m1["heat_src"] - m0["heat_src"]
    f = o.fields()["C"][:, 0, 0]
    O2, T, P = f[0, :nf], f[1, :nf], f[2, :nf]
    D = {k: (1.0 - J0) / dim * (t - 0.5) for k, t in (("O", tau_O), ("T", tau_T), ("P", tau_P))}
    inner = slice(1, nf - 2)
    for prof in (O2, T, P):
        np.testing.assert_allclose(prof[:-2] - 2 * prof[1:-1] + prof[2:], 0, atol=1e-12)
    np.testing.assert_allclose(D["O"] * (O2[:-1] - O2[1:])[inner], reaction, rtol=1e-9)
    np.testing.assert_allclose(D["P"] * (P[1:] - P[:-1])[inner], reaction, rtol=1e-9)
    np.testing.assert_allclose(D["T"] * (T[1:] - T[:-1])[inner], heat, rtol=1e-9)
    np.testing.assert_allclose(heat, hr * reaction, rtol=1e-9)
    Ts = f[1, nf:]
    assert np.ptp(Ts) < 1e-11
    assert abs(T[-1] + 0.5 * (T[-1] - T[-2]) - Ts[0]) < 1e-11
    assert reaction > 0 and Ts[0] > 1.2
    # The same state in closed form. A linear profile phi(x) = phi_in + b (tau + x) carries the
    # populations w (phi -/+ b tau), so each inlet ghost sets phi(0) = phi_in + b tau. At the slab
    # face the species closure gives k C_b = -D_O b_O with C_b = O2(nf - 1); the product gains r
    # there, D_P b_P = r; the fluid carries the whole heat to the inlet, D_T b_T = h_r r; and
    # the face temperature is the fluid profile at the halfway point, T_b = T(nf - 1/2). With
    # k = A exp(-Ta / T_b) this leaves one equation in T_b, solved here by bracketing.
    from scipy.optimize import brentq
    A, Ta = cfg["arr_A"], cfg["arr_Ta"]

    def rate(Tb):
        k = A * np.exp(-Ta / Tb)
        return D["O"] * 1.0 * k / (k * (nf - 1 + tau_O) + D["O"])

    Tb = brentq(lambda t: t - (1.0 + hr * rate(t) / D["T"] * (tau_T + nf - 0.5)), 1.0, 10.0,
                xtol=1e-15, rtol=1e-15)
    r = rate(Tb)
    x = np.arange(nf)
    np.testing.assert_allclose(reaction, r, rtol=1e-10)
    np.testing.assert_allclose(Ts, Tb, rtol=1e-11)
    np.testing.assert_allclose(O2, 1.0 - r / D["O"] * (tau_O + x), atol=1e-11)
    np.testing.assert_allclose(P, 0.0 + r / D["P"] * (tau_P + x), atol=1e-11)
    np.testing.assert_allclose(T, 1.0 + hr * r / D["T"] * (tau_T + x), atol=1e-11)


def test_reactive_channel_recipe_uses_the_printed_values():
    """The channel recipe takes the printed inlet values, Pe and Da of Sec. 3.4
    (tests/golden/reactive_channel.json): Pe = U L / D and Da = k(T_in) L / D with L the disc
    diameter, U the mean inlet velocity and D the O2 diffusivity of the scalar lattice; and the
    inlet profile 6 U s (1 - s) has mean U and peak 1.5 U."""
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "reactive_channel.json")))
    cfg, geom, _ = inputs.combustion_channel_2d()
    assert (cfg["nx"], cfg["ny"]) == (gold["nx"], gold["ny"])
    assert cfg["C_in"][0] == gold["C_O2_inlet"] and cfg["C_in_p"] == gold["C_CO2_inlet"]
    # the disc diameter 2 (ny // 8), and the discs in the geometry are that wide
    L = 2.0 * (cfg["ny"] // 8)
    widths = [np.diff(np.nonzero(np.diff(np.r_[0, row != 0, 0]))[0])[::2].max()
              for row in geom[0] if (row != 0).any()]
    assert abs(max(widths) - L) <= 1
    D = (1.0 - cfg["J0"]) / 2.0 * (cfg["tau_c"][0] - 0.5)
    k_in = cfg["arr_A"] * np.exp(-cfg["arr_Ta"] / cfg["C_in"][1])
    assert abs(cfg["u_in"] * L / D / gold["Pe"] - 1) < 1e-12
    assert abs(k_in * L / D / gold["Da"] - 1) < 1e-12
    s = (np.arange(cfg["ny"]) + 0.5) / cfg["ny"]
    prof = 6.0 * s * (1.0 - s)
    assert abs(prof.mean() - 1.0) < 1e-3
    assert abs(prof.mean() / prof.max() - gold["inlet_profile_mean_over_peak"]) < 1e-3
