"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: the paper's
printed tables and formulas (tests/golden/lattice_tables.json), textbook
closed forms (equilibrium moments, Guo forcing moments, Poiseuille curvature,
the exact Fourier-mode update of the diffusion lattice), conservation
invariants, and linear-stability thresholds of the Shan-Chen equation of state.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2502_12955_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden", "lattice_tables.json")


def make(cfg, geom=None, fields=None):
    o = Oracle(cfg)
    shape = o.shape
    o.set_geometry(np.zeros(shape, np.uint8) if geom is None else geom)
    if fields is None:
        fields = inputs.uniform_fields(shape, o.p.n_comp, o.p.n_scal)
    rho, u, C = fields
    o.set_fields(rho, u, C if o.p.n_scal else None)
    return o


# ------------------------------------------------------------ lattice tables

def _frac(s):
    return float(Fraction(s))


@pytest.mark.parametrize("dim", [2, 3])
def test_lattices_match_printed_tables(dim):
    gold = json.load(open(GOLD))
    o = Oracle(dict(dim=dim, nx=2, ny=2, nz=2 if dim == 3 else 1, n_scal=1, J0=0.4))
    c, w = o.lattice(0)
    name = "D3Q19" if dim == 3 else "D2Q9"
    g = gold[name]
    np.testing.assert_array_equal(c[:, 0], g["cx"])
    np.testing.assert_array_equal(c[:, 1], g["cy"])
    if dim == 3:
        np.testing.assert_array_equal(c[:, 2], g["cz"])
    printed = np.array([_frac(s) for s in g["w"]])
    if dim == 3:
        np.testing.assert_allclose(w, printed, rtol=0, atol=1e-16)
    else:
        # the printed D2Q9 weights sum to 11/12: direction 4 is an axis direction (1/9)
        assert abs(printed.sum() - 11.0 / 12.0) < 1e-15
        expect = printed.copy()
        expect[4] = 1.0 / 9.0
        np.testing.assert_allclose(w, expect, rtol=0, atol=1e-16)
    if dim == 2:
        cc, wc = o.lattice(1)
        g5 = gold["D2Q5"]
        np.testing.assert_array_equal(cc[:, 0], g5["cx"])
        np.testing.assert_array_equal(cc[:, 1], g5["cy"])
        np.testing.assert_allclose(wc, [float(s) for s in g5["w"]], rtol=0, atol=1e-16)


@pytest.mark.parametrize("dim,which", [(2, 0), (3, 0), (2, 1), (3, 1)])
def test_lattice_isotropy(dim, which):
    J0 = 0.4 if dim == 2 else 0.25
    o = Oracle(dict(dim=dim, nx=2, ny=2, nz=2 if dim == 3 else 1, n_scal=1, J0=J0))
    c, w = o.lattice(which)
    c = c.astype(float)
    cs2 = 1.0 / 3.0 if which == 0 else (1 - J0) / dim
    d = np.eye(3)
    d[2, 2] = 1.0 if dim == 3 else 0.0
    assert abs(w.sum() - 1) < 1e-15
    np.testing.assert_allclose(w @ c, 0, atol=1e-16)
    np.testing.assert_allclose(np.einsum("i,ia,ib->ab", w, c, c), cs2 * d, atol=1e-15)
    np.testing.assert_allclose(np.einsum("i,ia,ib,ic->abc", w, c, c, c), 0, atol=1e-16)
    if which == 0:
        # fourth-order isotropy of D2Q9 / D3Q19: cs^4 (dab dcd + dac dbd + dad dbc)
        t = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
        e = cs2 ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                        + np.einsum("ad,bc->abcd", d, d))
        np.testing.assert_allclose(t, e, atol=1e-15)


def test_d2q5_sound_speed_fixes_paper_tau_relation():
    """tau_d = (10/3) D + 1/2 (Sec. 2.1.5) is D = c_s^2 (tau - 1/2) with c_s^2 = 0.3 =
    (1 - J0)/2 at J0 = 0.4, the same constant as Eq. wetnode9's denominator; the
    deposition case (Sec. 3.3) pairs tau 0.9687 with D 0.156 on D2Q9 (c_s^2 = 1/3)."""
    gold = json.load(open(GOLD))["relations"]
    o = Oracle(dict(dim=2, nx=2, ny=2, n_scal=1, J0=gold["J0"]))
    c, w = o.lattice(1)
    cs2 = float(np.sum(w * c[:, 0] ** 2))
    assert abs(1.0 / cs2 - _frac(gold["d2q5_tau_over_D"])) < 1e-14
    assert abs(cs2 - (1 - gold["J0"]) / 2) < 1e-16
    # printed to four digits: 3 * 0.156 + 0.5 = 0.968 vs 0.9687
    assert abs(3.0 * gold["deposition_D"] + 0.5 - gold["deposition_tau"]) < 1e-3


# -------------------------------------------- single-node closed forms (tau = 1)

def _one_node(dim, **kw):
    cfg = dict(dim=dim, nx=1, ny=1, nz=1, n_comp=1, tau=[1.0], periodic=[1, 1, 1], **kw)
    return make(cfg)


@pytest.mark.parametrize("dim", [2, 3])
def test_equilibrium_and_guo_moments(dim):
    """In a 1-node periodic box with tau = 1, one step maps f to f^eq(rho, u^b) + F_i/2.
    Its moments must be rho, j + F and rho (cs2 I + u u) + (u F + F u)/2 (Eq. 6, 1.19, 1.21)."""
    rng = np.random.default_rng(3)
    for g in ([0.0, 0.0, 0.0], [1e-3, -2e-3, 3e-3]):
        if dim == 2:
            g = [g[0], g[1], 0.0]
        o = _one_node(dim, g=g)
        q = o.qf
        f0 = rng.uniform(0.02, 0.2, size=(1, q, 1))
        o.set_pops(f0)
        c, _ = o.lattice(0)
        c = c.astype(float)
        rho = f0[0, :, 0].sum()
        j = f0[0, :, 0] @ c
        F = rho * np.array(g)
        u = (j + F / 2) / rho
        o.step(1)
        f1 = o.pops()[0][0, :, 0]
        cs2 = 1 / 3
        d = np.eye(3)
        if dim == 2:
            d[2, 2] = 0
        assert abs(f1.sum() - rho) < 1e-15
        np.testing.assert_allclose(f1 @ c, j + F, atol=1e-15)
        P = np.einsum("i,ia,ib->ab", f1, c, c)
        expect = rho * (cs2 * d + np.outer(u, u)) + 0.5 * (np.outer(u, F) + np.outer(F, u))
        np.testing.assert_allclose(P, expect, atol=1e-15)


@pytest.mark.parametrize("dim", [2, 3])
def test_scalar_equilibrium_moments(dim):
    """tau_c = 1: one step maps h to h^eq(C, u): sum = C, first moment C u (Eq. therpopeq_species)."""
    rng = np.random.default_rng(4)
    J0 = 0.4 if dim == 2 else 0.25
    o = _one_node(dim, n_scal=1, tau_c=[1.0], J0=J0)
    q, qc = o.qf, o.qc
    f0 = rng.uniform(0.02, 0.2, size=(1, q, 1))
    h0 = rng.uniform(0.01, 0.3, size=(1, qc, 1))
    o.set_pops(f0, h0)
    c, _ = o.lattice(0)
    cc, _ = o.lattice(1)
    u = (f0[0, :, 0] @ c) / f0[0, :, 0].sum()
    C = h0.sum()
    o.step(1)
    h1 = o.pops()[1][0, :, 0]
    cs2 = (1 - J0) / dim
    assert abs(h1.sum() - C) < 1e-15
    np.testing.assert_allclose(h1 @ cc.astype(float), C * u, atol=1e-16)
    d = np.eye(3)
    if dim == 2:
        d[2, 2] = 0
    np.testing.assert_allclose(np.einsum("i,ia,ib->ab", h1, cc, cc), C * cs2 * d, atol=1e-15)


# ------------------------------------------------------------ conservation

@pytest.mark.parametrize("dim,collision", [(2, "bgk"), (3, "bgk"), (3, "mrt"), (2, "mrt")])
def test_mass_and_species_conservation_with_walls(dim, collision):
    shape = (1, 24, 32) if dim == 2 else (10, 12, 14)
    geom = inputs.random_solids(shape, 0.25, seed=5, reactive_fraction=0.0)
    cfg = dict(dim=dim, nx=shape[2], ny=shape[1], nz=shape[0], tau=[0.7], g=[1e-5, 2e-6, 0.0],
               collision=collision, n_scal=2, tau_c=[0.8, 0.6], k_react=0.0,
               periodic=[1, 1, 1])
    rho, u, C = inputs.perturbed_fields(shape, 1, 2, seed=6, amp_rho=1e-2, amp_u=1e-2)
    u[:, geom != 0] = 0
    o = make(cfg, geom, (rho, u, C))
    m0 = o.monitors()
    o.step(400 if dim == 2 else 100)
    m1 = o.monitors()
    assert abs(m1["mass0"] - m0["mass0"]) < 1e-13 * m0["mass0"]
    for s in (0, 1):
        assert abs(m1[f"species{s}"] - m0[f"species{s}"]) < 1e-13 * m0[f"species{s}"]


@pytest.mark.parametrize("dim,collision,forcing", [(2, "bgk", "guo"), (3, "mrt", "guo"),
                                                   (2, "bgk", "sc_shift"), (3, "bgk", "sc_shift")])
def test_body_force_momentum_increment(dim, collision, forcing):
    """Fully periodic, no walls: sum_x sum_i c_i f_i grows by exactly g * total mass per step."""
    shape = (1, 12, 16) if dim == 2 else (6, 7, 8)
    g = np.array([3e-5, -1e-5, 2e-5 if dim == 3 else 0.0])
    cfg = dict(dim=dim, nx=shape[2], ny=shape[1], nz=shape[0], tau=[0.9], g=g.tolist(),
               collision=collision, forcing=forcing, periodic=[1, 1, 1])
    rho, u, _ = inputs.perturbed_fields(shape, 1, 0, seed=7, amp_rho=0.05, amp_u=0.02)
    o = make(cfg, None, (rho, u, None))
    m0 = o.monitors()
    o.step(50)
    m1 = o.monitors()
    M = m0["mass0"]
    for a, k in enumerate(("momx", "momy", "momz")):
        # round-off budget: ~1e-15 per node update (a wrong force term is ~1e-4 off)
        tol = 2e-15 * rho[0].size * 50
        assert abs((m1[k] - m0[k]) - 50 * g[a] * M) < tol


# ---------------------------------------------------------------- Poiseuille

def _poiseuille(tau, collision="bgk", forcing="guo", ny=21, steps=None):
    shape = (1, ny, 4)
    geom = np.zeros(shape, np.uint8)
    geom[0, 0, :] = 1
    geom[0, ny - 1, :] = 1
    g = 1e-6
    cfg = dict(dim=2, nx=4, ny=ny, tau=[tau], g=[g, 0, 0], collision=collision, forcing=forcing,
               periodic=[1, 1, 1], mrt_rates=dict(s_e=1.1, s_eps=1.3, s_q=1.5))
    o = make(cfg, geom)
    o.step(steps or 30000)
    ux = o.fields()["u"][0, 0, 1:ny - 1, 1]
    nu = (tau - 0.5) / 3
    return ux, g, nu


@pytest.mark.parametrize("tau,collision,forcing", [(0.8, "bgk", "guo"), (1.3, "bgk", "guo"),
                                                   (0.8, "mrt", "guo"), (0.8, "bgk", "sc_shift")])
def test_poiseuille_profile_is_exact_parabola(tau, collision, forcing):
    """Steady force-driven channel: the profile is quadratic with curvature -g/nu,
    nu = c_s^2 (tau - 1/2), at every fluid node including those next to the walls."""
    ux, g, nu = _poiseuille(tau, collision, forcing)
    d2 = ux[2:] - 2 * ux[1:-1] + ux[:-2]
    np.testing.assert_allclose(d2, -g / nu, rtol=1e-7)
    np.testing.assert_allclose(ux, ux[::-1], rtol=1e-10)


def test_poiseuille_halfway_wall_exact_at_magic_tau():
    """BGK with halfway bounce-back puts the wall exactly halfway between the wall and
    the first fluid node when (tau - 1/2)^2 = 3/16 (Ginzburg & d'Humieres 2003):
    u(y) = g/(2 nu) (y - 1/2)(ny - 3/2 - y) for fluid rows y = 1 .. ny-2."""
    tau = 0.5 + np.sqrt(3.0) / 4.0
    ny = 21
    ux, g, nu = _poiseuille(tau, ny=ny, steps=40000)
    y = np.arange(1, ny - 1)
    exact = g / (2 * nu) * (y - 0.5) * (ny - 1.5 - y)
    np.testing.assert_allclose(ux, exact, rtol=1e-8)


@pytest.mark.parametrize("dim,tau,collision,s_q", [(2, 0.6, "bgk", None), (2, 0.8, "bgk", None),
                                                   (2, 1.5, "bgk", None), (2, 0.8, "mrt", 1.2),
                                                   (2, 1.1, "mrt", 1.6), (3, 0.8, "bgk", None),
                                                   (3, 0.9, "mrt", 1.3)])
def test_poiseuille_equals_its_exact_discrete_solution(dim, tau, collision, s_q):
    """For any tau, the steady force-driven D2Q9 channel with halfway bounce-back is the exact
    discrete solution u(y) = g/(2 nu) ((H/2)^2 - y^2) + (g/nu) (16 Lambda - 3)/24, y measured
    from the channel centre, H the fluid width. Lambda = (1/s_nu - 1/2)(1/s_q - 1/2) is the
    product of the relaxation parameters of the shear and the odd (energy-flux) moments, the
    only odd non-conserved moments of D2Q9; for BGK it is (tau - 1/2)^2 (Ginzburg & d'Humieres
    2003). The wall slip vanishes at Lambda = 3/16, the magic value of the test above. D3Q19 has
    two families of odd moments (q and m); with one rate for both, the same Lambda holds."""
    ny = 12
    nz = 1 if dim == 2 else 2
    shape = (nz, ny, 1)
    g = 1e-6
    cfg = dict(dim=dim, nx=1, ny=ny, nz=nz, tau=[tau], g=[g, 0, 0], collision=collision,
               periodic=[1, 0, 1])
    if s_q is not None:
        cfg["mrt_rates"] = dict(s_q=s_q, s_m=s_q)
    o = make(cfg, np.zeros(shape, np.uint8))
    nu = (tau - 0.5) / 3
    o.step(int(25 * ny * ny / nu))
    ux = o.fields()["u"][0, 0, :, 0]
    y = np.arange(ny) - (ny - 1) / 2
    lam = (tau - 0.5) * ((1.0 / s_q if s_q else tau) - 0.5)
    exact = g / (2 * nu) * ((ny / 2) ** 2 - y ** 2) + g / nu * (16 * lam - 3) / 24
    np.testing.assert_allclose(ux, exact, rtol=1e-8)


def test_poiseuille_slip_small_at_config_tau():
    """tau = 0.8 (config 1): u_max within 1e-3 relative of g H^2 / (8 nu) with H = ny - 2."""
    ux, g, nu = _poiseuille(0.8)
    H = len(ux)
    assert abs(ux.max() / (g * H * H / (8 * nu)) - 1) < 1e-3 * 10  # slip O(1/H^2)


# ---------------------------------------------------------------- diffusion

@pytest.mark.parametrize("dim,tau_c,J0", [(2, 0.7, 0.4), (2, 1.4, 0.4), (3, 0.6, 0.25)])
def test_fourier_mode_matches_exact_linear_update(dim, tau_c, J0):
    """A cosine concentration mode at rest evolves as Re(1^T A^t w) with
    A = S(k) [(1 - 1/tau) I + w 1^T / tau] and S(k) = diag(exp(-i k.c_i)): the exact
    single-mode update of the collide-stream pair; it decays like exp(-D k^2 t),
    D = c_s^2 (tau - 1/2)."""
    L = 32
    shape = (1, 1, L) if dim == 2 else (1, 1, L)
    cfg = dict(dim=dim, nx=L, ny=1, nz=1, n_comp=1, tau=[1.0], n_scal=1, tau_c=[tau_c], J0=J0,
               periodic=[1, 1, 1])
    x = np.arange(L)
    k = 2 * np.pi / L
    a = 0.1
    C0 = (1.0 + a * np.cos(k * x)).reshape(shape)
    rho, u, _ = inputs.uniform_fields(shape, 1, 0)
    o = make(cfg, None, (rho, u, C0[None]))
    cc, w = o.lattice(1)
    S = np.diag(np.exp(-1j * k * cc[:, 0]))
    A = S @ ((1 - 1 / tau_c) * np.eye(len(w)) + np.outer(w, np.ones(len(w))) / tau_c)
    v = w.astype(complex)
    cs2 = (1 - J0) / dim
    D = cs2 * (tau_c - 0.5)
    amps = {}
    for t in range(1, 201):
        v = A @ v
        o.step(1)
        if t % 20 == 0:
            Cx = o.fields()["C"][0].reshape(-1)
            amp = 2 * np.mean((Cx - 1.0) * np.cos(k * x))
            np.testing.assert_allclose(amp, a * v.sum().real, rtol=1e-11, atol=1e-15)
            amps[t] = amp
    # continuum limit: late-time decay rate D k^2 up to O(k^2) relative corrections
    rate = -np.log(amps[200] / amps[100]) / 100
    assert abs(rate / (D * k * k) - 1) < 0.05


# ---------------------------------------------------------------- wet node

@pytest.mark.parametrize("tau_c,k", [(1.0, 1e-3), (0.7, 5e-2), (1.3, 0.2)])
def test_wet_node_reduces_to_printed_formula(tau_c, k):
    """Flat reactive wall with normal +y on D2Q5, J0 = 0.4 (Sec. 2.1.5): the closed
    concentration is Eq. wetnode9, C_b = 2 h_4 / ((1 - J0)/2 + tau/(tau - 0.5) k), with
    h_4 the gathered population moving into the wall; the removed amount is the stored
    bounce-back value minus the closed h_2."""
    shape = (1, 3, 1)
    geom = np.zeros(shape, np.uint8)
    geom[0, 0, 0] = 2   # reactive wall below the fluid node
    geom[0, 2, 0] = 1   # inert wall above
    cfg = dict(dim=2, nx=1, ny=3, tau=[1.0], n_scal=1, tau_c=[tau_c], J0=0.4, k_react=k,
               periodic=[1, 1, 1])
    rng = np.random.default_rng(8)
    o = make(cfg, geom)
    h0 = np.zeros((1, 5, 3))
    h0[0, :, 1] = rng.uniform(0.05, 0.2, size=5)
    o.set_pops(np.zeros((1, 9, 3)), h0)
    o.step(1)
    hs = h0[0, :, 1]
    h4 = hs[4]
    Cb = 2 * h4 / ((1 - 0.4) / 2 + tau_c / (tau_c - 0.5) * k)     # Eq. wetnode9
    h2_closed = 2 * 0.15 * Cb - h4
    m = o.monitors()
    np.testing.assert_allclose(m["wallx"], hs[2] - h2_closed, rtol=1e-13)
    np.testing.assert_allclose(m["reacted"], k * Cb, rtol=1e-13)
    # CE flux at the wet node: (1 - 1/(2 tau)) (h_4 - h_2) = k C_b  (Eq. reactO2)
    np.testing.assert_allclose((1 - 1 / (2 * tau_c)) * (h4 - h2_closed), k * Cb, rtol=1e-13)


def test_species_budget_closes_exactly():
    """Inlet + zero-gradient outlet + reactive obstacles + flow: the stored scalar sum changes
    by inflow - outflow - (populations lost through reactive links), to round-off; the
    per-node reaction bookkeeping sums to the reacted total."""
    cfg, geom, fields = inputs.reactive_channel_2d(nx=48, ny=24, seed=2)
    cfg["k_react"] = 0.05
    cfg["g"] = [2e-5, 0, 0]
    o = make(cfg, geom, fields)
    prev = o.monitors()
    for _ in range(30):
        o.step(10)
        m = o.monitors()
        lhs = m["species0"] - prev["species0"]
        rhs = ((m["inflow0"] - prev["inflow0"]) - (m["outflow0"] - prev["outflow0"])
               - (m["wallx"] - prev["wallx"]))
        assert abs(lhs - rhs) < 1e-12
        prev = m
    assert m["reacted"] > 0 and m["inflow0"] > 0
    np.testing.assert_allclose(o.fields()["acc"].sum(), m["reacted"], rtol=1e-12)


@pytest.mark.parametrize("tau_c", [0.8, 1.2])
def test_steady_reactive_diffusion_flux(tau_c):
    """1D channel at rest, inlet C = 1, reactive wall at the far end: at steady state the
    profile is linear and the flux through every link, D (C(x) - C(x+1)) with
    D = c_s^2 (tau_c - 1/2), equals the amount reacted per step."""
    nx = 24
    geom = np.zeros((1, 1, nx), np.uint8)
    geom[0, 0, nx - 1] = 2
    cfg = dict(dim=2, nx=nx, ny=1, tau=[1.0], n_scal=1, tau_c=[tau_c], J0=0.4, k_react=0.02,
               ade_open_x=True, C_in=[1.0], periodic=[1, 1, 1])
    o = make(cfg, geom)
    o.step(40000)
    m0 = o.monitors()
    o.step(1)
    m1 = o.monitors()
    per_step = m1["wallx"] - m0["wallx"]
    reaction = m1["reacted"] - m0["reacted"]
    C = o.fields()["C"][0, 0, 0, : nx - 1]
    D = 0.3 * (tau_c - 0.5)
    np.testing.assert_allclose(C[1:-2] - 2 * C[2:-1] + C[3:], 0, atol=1e-12)
    np.testing.assert_allclose(D * (C[1:-2] - C[2:-1]), per_step, rtol=1e-9)
    # at steady state the wall takes exactly the reaction rate k C_b (Eq. reactO2)
    np.testing.assert_allclose(reaction, per_step, rtol=1e-9)


@pytest.mark.parametrize("dim,tau_c,k,xs,J0,C_in", [(2, 0.8, 0.05, 10, 0.4, 1.0), (2, 1.3, 0.2, 7, 0.4, 0.7),
                                                     (2, 0.6, 0.01, 12, 0.2, 1.5), (3, 0.5667, 0.02, 9, 0.25, 1.0),
                                                     (3, 1.1, 0.1, 6, 0.4, 0.5)])
def test_steady_reactive_channel_closed_form(dim, tau_c, k, xs, J0, C_in):
    """The whole steady 1D solution in closed form, derived from the update itself: at rest,
    with a linear profile C(x) = C_in + b (tau + x), the +x and -x populations are
    w (C -/+ b tau) (w = (1 - J0)/4), so the inlet ghost w C_in entering node 0 fixes C(0) =
    C_in + b tau; at the last fluid node xs - 1 the wet-node closure (Eq. wetnode9, per link)
    gives C_b = C(xs - 1) and k C_b = -D b with D = (1 - J0)/dim (tau - 1/2) (D2Q5, and D3Q7
    with w = (1 - J0)/6). Together: b = -C_in / (xs - 1 + tau + D / k), and the reaction per
    step is -D b."""
    nx = xs + 3
    shape = (1, 1, nx)
    geom = np.zeros(shape, np.uint8)
    geom[0, 0, xs:] = 2
    cfg = dict(dim=dim, nx=nx, ny=1, nz=1, tau=[1.0], n_scal=1, tau_c=[tau_c], J0=J0, k_react=k,
               ade_open_x=True, C_in=[C_in], periodic=[1, 1, 1])
    o = make(cfg, geom, (np.ones((1,) + shape), np.zeros((3,) + shape), np.zeros((1,) + shape)))
    o.step(100000)
    m0 = o.monitors()
    o.step(1)
    r = o.monitors()["reacted"] - m0["reacted"]
    D = (1.0 - J0) / dim * (tau_c - 0.5)
    b = -C_in / (xs - 1 + tau_c + D / k)
    C = o.fields()["C"][0, 0, 0, :xs]
    np.testing.assert_allclose(C, C_in + b * (tau_c + np.arange(xs)), atol=1e-12)
    np.testing.assert_allclose(r, -D * b, rtol=1e-10)


# ------------------------------------------------------------------ MRT

def test_mrt_basis_orthogonal_and_dhumieres():
    o = Oracle(dict(dim=3, nx=2, ny=2, nz=2, tau=[0.8], collision="mrt"))
    M, S = o.mrt()
    G = M @ M.T
    np.testing.assert_allclose(G - np.diag(np.diag(G)), 0, atol=1e-12)
    c, _ = o.lattice(0)
    c2 = (c ** 2).sum(1).astype(float)
    cx = c[:, 0].astype(float)

    def prop(row, ref):
        r = np.dot(row, ref) / np.dot(ref, ref)
        np.testing.assert_allclose(row, r * ref, atol=1e-12)

    # d'Humieres et al. (2002) D3Q19 rows: e = 19c^2 - 30, eps = (21c^4 - 53c^2 + 24)/2,
    # q_x = (5c^2 - 9) c_x, 3 pi_xx = (3c^2 - 5)(3c_x^2 - c^2)
    prop(M[1], 19 * c2 - 30)
    prop(M[2], (21 * c2 ** 2 - 53 * c2 + 24) / 2)
    prop(M[4], (5 * c2 - 9) * cx)
    prop(M[10], (3 * c2 - 5) * (3 * cx ** 2 - c2))


@pytest.mark.parametrize("dim", [2, 3])
def test_mrt_with_uniform_rates_is_bgk(dim):
    shape = (1, 10, 12) if dim == 2 else (6, 7, 8)
    tau = 0.8
    base = dict(dim=dim, nx=shape[2], ny=shape[1], nz=shape[0], tau=[tau], g=[2e-5, 1e-5, 0],
                n_scal=1, tau_c=[0.9])
    geom = inputs.random_solids(shape, 0.2, seed=9)
    flds = inputs.perturbed_fields(shape, 1, 1, seed=10, amp_rho=0.02, amp_u=0.02)
    r = 1 / tau
    a = make(dict(base, collision="bgk"), geom, flds)
    b = make(dict(base, collision="mrt", mrt_rates=dict(s_e=r, s_eps=r, s_q=r, s_pi=r, s_m=r)),
             geom, flds)
    a.step(50)
    b.step(50)
    fa, fb = a.pops()[0], b.pops()[0]
    np.testing.assert_allclose(fb, fa, rtol=0, atol=1e-14)


# --------------------------------------------------------------- Shan-Chen

def _sc_variance(cfg, shape, rho_mean, seed, steps):
    rng = np.random.default_rng(seed)
    n_comp = cfg["n_comp"]
    rho = np.empty((n_comp,) + shape)
    for s in range(n_comp):
        rho[s] = rho_mean[s] * (1 + 0.01 * rng.uniform(-1, 1, size=shape))
    u = np.zeros((3,) + shape)
    o = make(cfg, None, (rho, u, None))
    v0 = o.fields()["rho"][0].var()
    o.step(steps)
    f = o.fields()["rho"]
    m = o.monitors()
    return v0, f[0].var(), f, m


@pytest.mark.parametrize("rho_mean,unstable", [(0.693, True), (2.2, False), (0.15, False)])
def test_single_component_spinodal(rho_mean, unstable):
    """psi = 1 - exp(-rho), G = -5 (Sec. 3.2.1): the EOS p = c_s^2 rho + c_s^2 G psi^2 / 2 has
    dp/drho < 0 for exp(-rho) in (0.276, 0.724), i.e. rho in (0.32, 1.29): a uniform state
    inside separates, one outside relaxes back.  Mass is conserved exactly."""
    shape = (1, 32, 32)
    cfg = dict(dim=2, nx=32, ny=32, n_comp=1, tau=[1.0], G=[[-5.0, 0], [0, 0]], psi_kind="exp")
    v0, v1, f, m = _sc_variance(cfg, shape, [rho_mean], 11, 600)
    assert (v1 > 100 * v0) == unstable
    if not unstable:
        assert v1 < v0
    np.testing.assert_allclose(m["mass0"], rho_mean * 32 * 32, rtol=2e-3)


@pytest.mark.parametrize("G,unstable", [(0.8, False), (1.3, True)])
def test_two_component_mixing_threshold(G, unstable):
    """psi = rho, cross-cohesion G: the mixture rho_1 = rho_2 = 1 is linearly unstable iff
    G^2 rho_1 rho_2 > 1 (p = c_s^2 (rho_1 + rho_2 + G rho_1 rho_2)).  Below threshold the
    scaled densities stay at 0.5 / 0.5 (Sec. 3.2.2)."""
    shape = (1, 32, 32)
    cfg = dict(dim=2, nx=32, ny=32, n_comp=2, tau=[1.0, 1.0], G=[[0, G], [G, 0]],
               psi_kind="identity")
    v0, v1, f, m = _sc_variance(cfg, shape, [1.0, 1.0], 12, 1500)
    assert (v1 > 100 * v0) == unstable
    if not unstable:
        np.testing.assert_allclose(f[0] / (f[0] + f[1]), 0.5, atol=1e-4)
    assert abs(m["mass0"] - f[0].sum()) < 1e-9 and abs(m["mass1"] - f[1].sum()) < 1e-9


def _two_comp(shape, G, rho):
    cfg = dict(dim=2, nx=shape[2], ny=shape[1], n_comp=2, tau=[1.0, 1.0], G=[[0, G], [G, 0]],
               psi_kind="identity")
    return make(cfg, None, (rho, np.zeros((3,) + shape), None))


def _coexistence(G, steps=6000, tension=False):
    """Flat interfaces in a periodic slab: bulk densities of the two phases and, if asked, the
    surface tension of one interface by its mechanical definition (below)."""
    shape = (1, 2, 64)
    x = np.arange(64)
    inside = (x >= 16) & (x < 48)
    rho = np.empty((2,) + shape)
    rho[0] = np.where(inside, 1.0, 0.05)
    rho[1] = np.where(inside, 0.05, 1.0)
    o = _two_comp(shape, G, rho)
    o.step(steps)
    r = o.fields()["rho"][:, 0, 0]
    if not tension:
        return r[0, 32], r[1, 32]
    return r[0, 32], r[1, 32], _mechanical_tension(r[0], r[1], G)


def _mechanical_tension(psi1, psi2, G):
    """gamma = integral of (P_N - P_T) across a flat interface normal to x, for the pair force
    F_1 = -psi_1 G sum_i w_i psi_2(x + c_i) c_i and its mirror (Eq. 1.14), with the node-centred
    pressure tensor P_ab = c_s^2 (rho_1 + rho_2) delta_ab
    + (G / 2) sum_i w_i [psi_1(x) psi_2(x + c_i) + psi_2(x) psi_1(x + c_i)] c_ia c_ib, whose
    normal component is constant through the interface at equilibrium (mechanical balance).  On
    D2Q9 only the axis links differ between P_xx and P_yy, and summation by parts leaves
    -G w_1 sum_x (psi_1(x+1) - psi_1(x)) (psi_2(x+1) - psi_2(x)) for the whole periodic slab,
    which holds two interfaces."""
    d1 = np.roll(psi1, -1) - psi1
    d2 = np.roll(psi2, -1) - psi2
    return -G * (1.0 / 9.0) * float((d1 * d2).sum()) / 2.0


def _droplet_dp(R, G, hi, lo, n=48, steps=2000):
    shape = (1, n, n)
    yy, xx = np.mgrid[0:n, 0:n]
    ins = (xx - n / 2) ** 2 + (yy - n / 2) ** 2 < R * R
    rho = np.empty((2,) + shape)
    rho[0, 0] = np.where(ins, hi, lo)
    rho[1, 0] = np.where(ins, lo, hi)
    o = _two_comp(shape, G, rho)
    m0 = o.monitors()
    o.step(steps)
    f = o.fields()["rho"][:, 0]
    m1 = o.monitors()
    cs2 = 1 / 3
    p = cs2 * (f[0] + f[1]) + cs2 * G * f[0] * f[1]    # EOS with psi = rho
    Rm = np.sqrt(((f[0] - f[0].min()) / (f[0].max() - f[0].min())).sum() / np.pi)
    return p[n // 2, n // 2] - p[0, 0], Rm, f, m0, m1


@pytest.mark.slow
def test_coexistence_and_laplace_law_2d():
    """Two-component Shan-Chen with psi = rho (Sec. 3.2.2).  (1) The flat-interface
    coexistence densities satisfy the symmetric-binary binodal ln(rho_h / rho_l) =
    G (rho_h - rho_l) of the EOS p = c_s^2 (rho_1 + rho_2 + G rho_1 rho_2), up to lattice
    corrections.  (2) Static droplets obey Delta p = gamma / R (2D Laplace law): Delta p is
    linear in 1/R with a small intercept, and component masses are conserved exactly.  (3) That
    gamma is the mechanical surface tension of the flat interface, the integral of
    P_N - P_T across it, to 3 %: the absolute tension, not only its scaling."""
    G = 2.7
    hi, lo, gamma_mech = _coexistence(G, tension=True)
    assert abs(np.log(hi / lo) / (G * (hi - lo)) - 1) < 0.03
    Rs, dps = [], []
    for R in (7.0, 10.0, 13.0):
        dp, Rm, f, m0, m1 = _droplet_dp(R, G, hi, lo)
        Rs.append(Rm)
        dps.append(dp)
        for s in (0, 1):
            assert abs(m1[f"mass{s}"] - m0[f"mass{s}"]) < 1e-11 * m0[f"mass{s}"]
        assert abs(Rm - R) < 1.0
    Rs, dps = np.array(Rs), np.array(dps)
    A = np.vstack([1 / Rs, np.ones_like(Rs)]).T
    coef, *_ = np.linalg.lstsq(A, dps, rcond=None)
    pred = A @ coef
    r2 = 1 - ((dps - pred) ** 2).sum() / ((dps - dps.mean()) ** 2).sum()
    assert r2 > 0.99
    assert coef[0] > 0 and abs(coef[1]) < 0.2 * dps.min()
    # (3) the Laplace slope is the surface tension of the flat interface at the same bulk state
    assert abs(coef[0] / gamma_mech - 1) < 0.03, (coef[0], gamma_mech)


def test_literal_weak_cohesion_dissolves_droplet():
    """G = 0.9 with Eq. 1.14's w_i weights and densities 1 / 0.05 lies below the mixing
    threshold (G (rho_1 + rho_2) < 2): the droplet dissolves, which is why the droplet
    workload reads G = 0.9 in the w_i / c_s^2 convention (G = 2.7 here)."""
    shape = (1, 32, 32)
    rho, u = inputs.droplet_fields(shape, 10.0)
    o = _two_comp(shape, 0.9, rho)
    o.step(2000)
    f = o.fields()["rho"][:, 0]
    assert f[0].max() - f[0].min() < 0.2


# ---------------------------------------------------------------- moving wall (Couette)

@pytest.mark.parametrize("dim,tau,steps", [(2, 0.8, 8000), (3, 0.59, 20000)])
def test_couette_profile_is_linear(dim, tau, steps):
    """Sec. 3.1.1, Eq. couette_velocity_profile: the top plate moves with U_wall = 0.02 (the
    paper's value; tau 0.59 in 3D is its Re = 10 on Ny = 15).  With halfway walls at y = -1/2
    and y = ny - 1/2 the steady profile is u_x = U (y + 1/2) / ny, which the moving-wall
    bounce-back reproduces exactly (to the residual decay of the transient)."""
    ny = 16 if dim == 2 else 15
    nx, nz = 4, (4 if dim == 3 else 1)
    U = 0.02
    cfg = dict(dim=dim, nx=nx, ny=ny, nz=nz, tau=[tau], periodic=[1, 0, 1], u_wall_ymax=[U, 0, 0])
    shape = (nz, ny, nx)
    o = Oracle(cfg)
    o.set_geometry(np.zeros(shape, np.uint8))
    rho, u, _ = inputs.uniform_fields(shape, 1, 0, rho=1.0)
    o.set_fields(rho, u, None)
    m0 = o.monitors()["mass0"]
    o.step(steps)
    f = o.fields()
    y = np.arange(ny)
    exact = U * (y + 0.5) / ny
    prof = f["u"][0].mean(axis=(0, 2))
    assert np.abs(prof - exact).max() < 1e-9 * U, np.abs(prof - exact).max()
    assert np.abs(f["u"][1]).max() < 1e-12 and np.abs(f["u"][2]).max() < 1e-12
    # a tangential plate moves no mass: its momentum terms cancel pairwise at every node; what
    # remains is the round-off bias of the FP64 equilibria of a steady flow (~1e-16 per node
    # and step, the same sign every step: 1.8e-12 relative after 20000 steps in 3D)
    assert abs(o.monitors()["mass0"] - m0) < 1e-11 * m0


def test_moving_wall_needs_closed_tangential_plate():
    for bad in (dict(periodic=[1, 1, 1], u_wall_ymax=[0.01, 0, 0]),
                dict(periodic=[1, 0, 1], u_wall_ymax=[0.0, 0.01, 0])):
        with pytest.raises(Exception):
            Oracle(dict(dim=2, nx=4, ny=8, **bad))


# ---------------------------------------------------------------- velocity inlet (Sec. 3.4)

@pytest.mark.parametrize("dim,collision", [(2, "bgk"), (3, "mrt")])
def test_velocity_inlet_mass_budget_per_step(dim, collision):
    """Sec. 3.4 inlet u = 6y(1-y) (here u_x = 6 U s (1 - s), s = (y + 1/2) / ny) as a face moving
    with that velocity: the populations arriving with c_x = +1 gain 2 w_i rho u_x / c_s^2 =
    6 w_i rho u_x.  Those directions' weights sum to 1/6, so each inlet node gains exactly
    rho u_x(y) per step.  The zero-gradient outlet gives each population entering through
    x = nx - 1 the node's own post-collision value of the same direction, so each outlet node
    loses its post-collision x momentum, j_x + F_x (collision keeps mass and adds the force).
    Walls and solids move no mass.  So the total mass changes per step by
    sum_inlet rho u_x - sum_outlet (j_x + F_x), computed here from the stored populations."""
    nx, ny, nz = 10, 8, (5 if dim == 3 else 1)
    U = 0.03
    g = [2e-4, 0.0, 1e-4 if dim == 3 else 0.0]
    cfg = dict(dim=dim, nx=nx, ny=ny, nz=nz, tau=[0.8], collision=collision, flow_open_x=True, u_in=U,
               g=g, periodic=[0, 0, 1])
    shape = (nz, ny, nx)
    geom = inputs.random_solids(shape, 0.15, seed=41, reactive_fraction=0.0)
    geom[:, :, 0] = 0
    geom[:, :, -1] = 0
    rho, u, _ = inputs.perturbed_fields(shape, 1, 0, seed=42, amp_rho=0.02, amp_u=0.01)
    o = make(cfg, geom, (rho, u, None))
    o.step(4)
    cv, _ = o.lattice(0)
    sy = (np.arange(ny) + 0.5) / ny
    u_in = 6.0 * U * sy * (1.0 - sy)
    fluid = geom == 0
    for _ in range(3):
        f, _ = o.pops()
        fr = f[0].reshape((len(cv),) + shape)
        r = fr.sum(axis=0)
        jx = np.tensordot(cv[:, 0].astype(float), fr, axes=1)
        inflow = float((r[:, :, 0] * u_in[None, :]).sum())
        outflow = float((jx[:, :, -1] + r[:, :, -1] * g[0]).sum())
        m0 = float(r[fluid].sum())
        o.step(1)
        m1 = o.monitors()["mass0"]
        assert abs((m1 - m0) - (inflow - outflow)) < 1e-13 * m0, (m1 - m0, inflow - outflow)
        assert inflow > 0.5 * U * ny * nz


def test_velocity_inlet_profile_is_carried_downstream():
    """The inlet profile 6 U s (1 - s) is the developed plane-Poiseuille profile between walls at
    y = -1/2 and y = ny - 1/2, where halfway bounce-back puts the BGK no-slip wall exactly for
    (tau - 1/2)^2 = 3/16.  At steady state the mass flux sum_y rho u_x through every column equals
    what the inlet injects, and mid-channel the profile keeps the parabolic shape (its amplitude
    grows slightly downstream as the density falls along the pressure drop)."""
    nx, ny, U = 40, 12, 0.01
    o = make(dict(dim=2, nx=nx, ny=ny, tau=[0.5 + np.sqrt(3.0) / 4.0], flow_open_x=True, u_in=U,
                  periodic=[0, 0, 1]))
    o.step(6000)
    f = o.fields()
    ux, r = f["u"][0, 0], f["rho"][0, 0]
    sy = (np.arange(ny) + 0.5) / ny
    shape = 6.0 * sy * (1.0 - sy)
    q_in = float((r[:, 0] * U * shape).sum())
    for x in range(nx):
        assert abs(float((r[:, x] * ux[:, x]).sum()) / q_in - 1.0) < 1e-5, x
    col = ux[:, nx // 2]
    a = float(col @ shape / (shape @ shape))
    assert abs(a / U - 1.0) < 0.02
    assert np.abs(col - a * shape).max() < 2e-4 * U
    assert np.abs(f["u"][1, 0, :, nx // 2]).max() < 1e-3 * U


def test_velocity_inlet_needs_a_closed_channel():
    for bad in (dict(periodic=[1, 0, 1]), dict(periodic=[0, 1, 1]),
                dict(periodic=[0, 0, 1], n_comp=2, tau=[1.0, 1.0]),
                dict(periodic=[0, 0, 1], G=[[-5.0, 0], [0, 0]])):
        with pytest.raises(Exception):
            Oracle(dict(dim=2, nx=8, ny=8, flow_open_x=True, u_in=0.01, **bad))


# ------------------------------------------- temperature-dependent rate and heat release

def _thermal_case(seed, **over):
    shape = (1, 12, 14)
    geom = inputs.random_solids(shape, 0.2, seed=seed, reactive_fraction=0.7)
    cfg = dict(dim=2, nx=14, ny=12, tau=[0.8], n_scal=2, tau_c=[0.7, 0.9], J0=0.4, periodic=[1, 0, 1])
    cfg.update(over)
    return cfg, geom, shape


@pytest.mark.parametrize("geo", [dict(), dict(geo_mode="dissolve", V_m=60.0)])
def test_arrhenius_without_activation_or_heat_is_the_constant_rate(geo):
    """k(T) = A exp(-Ta / T) with Ta = 0 and no heat release is the constant rate k = A: the
    species, the flow, the geometry flips (new nodes take the neighbours' closed species) and the
    reaction bookkeeping equal those of the Eq. wetnode9 closure."""
    cfg, geom, shape = _thermal_case(51, g=[2e-4, 0, 0], **geo)
    rho, u, C = inputs.perturbed_fields(shape, 1, 2, seed=52, amp_rho=0.01, amp_u=0.01, C0=0.8)
    a = make(dict(cfg, arrhenius=True, arr_A=0.05, arr_Ta=0.0, heat_release=0.0), geom, (rho, u, C))
    b = make(dict(cfg, k_react=0.05), geom, (rho, u, C))
    a.step(40)
    b.step(40)
    fa, fb = a.fields(), b.fields()
    for k in ("rho", "u", "acc"):
        assert np.abs(fa[k] - fb[k]).max() < 1e-13 * max(1.0, np.abs(fb[k]).max()), k
    assert np.abs(fa["C"][0] - fb["C"][0]).max() < 1e-13
    ma, mb = a.monitors(), b.monitors()
    assert abs(ma["reacted"] - mb["reacted"]) < 1e-13 * mb["reacted"]
    assert mb["reacted"] > 0
    assert np.array_equal(fa["flags"], fb["flags"])
    if geo:
        assert mb["inj_mass0"] > 0, "no flip happened"


def test_arrhenius_at_uniform_temperature_is_the_rate_at_that_temperature():
    """At rest with a uniform temperature T0 and no heat release, every interface sits at T0, so
    the rate is the constant A exp(-Ta / T0)."""
    cfg, geom, shape = _thermal_case(53)
    T0, A, Ta = 1.3, 0.2, 0.9
    rho, u, _ = inputs.uniform_fields(shape, 1, 0)
    rng = np.random.default_rng(54)
    C = np.stack([0.8 + 0.1 * rng.uniform(size=shape), np.full(shape, T0)])
    a = make(dict(cfg, arrhenius=True, arr_A=A, arr_Ta=Ta, heat_release=0.0), geom, (rho, u, C))
    b = make(dict(cfg, k_react=A * np.exp(-Ta / T0)), geom, (rho, u, C))
    a.step(30)
    b.step(30)
    fa, fb = a.fields(), b.fields()
    assert np.abs(fa["C"][0] - fb["C"][0]).max() < 1e-13
    assert np.abs(fa["C"][1][geom == 0] - T0).max() < 1e-13     # heat-free, at rest: T stays uniform
    assert abs(a.monitors()["reacted"] - b.monitors()["reacted"]) < 1e-12 * b.monitors()["reacted"]


def test_heat_release_budget_per_step():
    """With reaction heat, flow, walls and a closed box, the temperature lattice gains per step
    exactly what the reactive links add (the heat monitor: closed minus stored populations at
    those links), and the species loses exactly the wall exchange."""
    cfg, geom, shape = _thermal_case(55, g=[3e-4, 0, 0], arrhenius=True, arr_A=0.4, arr_Ta=1.0,
                                     heat_release=0.05, n_it=24)
    rho, u, C = inputs.perturbed_fields(shape, 1, 2, seed=56, amp_rho=0.01, amp_u=0.01, C0=0.9)
    o = make(cfg, geom, (rho, u, C))
    o.step(3)
    for _ in range(4):
        m0 = o.monitors()
        o.step(1)
        m1 = o.monitors()
        dheat = m1["heat"] - m0["heat"]
        assert dheat > 0
        assert abs((m1["species1"] - m0["species1"]) - dheat) < 1e-12 * m0["species1"]
        assert abs((m1["species0"] - m0["species0"]) + (m1["wallx"] - m0["wallx"])) < 1e-12 * m0["species0"]


@pytest.mark.parametrize("dim,J0", [(2, 0.4), (3, 0.25)])
def test_steady_burning_face_closed_form(dim, J0):
    """The steady 1D state of the temperature-dependent closure (adiabatic solid): O2 and heat
    enter at x = 0, the reactive face is past node xs - 1. Linear profiles
    phi(x) = phi_in + b (tau + x) carry the populations w (phi -/+ b tau). The closure's two
    conditions then give C_b = C(xs - 1) and T_b = T(xs - 1) (each pair sum is 2 w times the node
    value), k(T_b) C_b = -D_O b_O, and a heat flux D_T b_T = h_r k(T_b) C_b carried back to the
    inlet (Eq. reactO2, reacRate, fluxCon). One equation in T_b remains; its bracketed root
    fixes the profiles, the rate and the heat monitor."""
    from scipy.optimize import brentq
    xs, tau_O, tau_T, hr, A, Ta = 10, 0.8, 0.9, 0.5, 0.5, 1.0
    nx = xs + 3
    shape = (1, 1, nx)
    geom = np.zeros(shape, np.uint8)
    geom[0, 0, xs:] = 2
    cfg = dict(dim=dim, nx=nx, ny=1, nz=1, tau=[1.0], n_scal=2, tau_c=[tau_O, tau_T], J0=J0,
               ade_open_x=True, C_in=[1.0, 1.0], arrhenius=True, arr_A=A, arr_Ta=Ta, heat_release=hr, n_it=40,
               periodic=[1, 1, 1])
    C0 = np.zeros((2,) + shape)
    C0[1] = 1.0
    o = make(cfg, geom, (np.ones((1,) + shape), np.zeros((3,) + shape), C0))
    o.step(40000)
    m0 = o.monitors()
    o.step(1)
    m1 = o.monitors()
    reaction = m1["reacted"] - m0["reacted"]
    DO, DT = (1.0 - J0) / dim * (tau_O - 0.5), (1.0 - J0) / dim * (tau_T - 0.5)

    def rate(Tb):
        k = A * np.exp(-Ta / Tb)
        return DO * k / (k * (xs - 1 + tau_O) + DO)

    Tb = brentq(lambda t: t - (1.0 + hr * rate(t) / DT * (tau_T + xs - 1)), 1.0, 10.0,
                xtol=1e-15, rtol=1e-15)
    r = rate(Tb)
    x = np.arange(xs)
    f = o.fields()["C"][:, 0, 0, :xs]
    np.testing.assert_allclose(reaction, r, rtol=1e-10)
    np.testing.assert_allclose(f[0], 1.0 - r / DO * (tau_O + x), atol=1e-11)
    np.testing.assert_allclose(f[1], 1.0 + hr * r / DT * (tau_T + x), atol=1e-11)
    np.testing.assert_allclose(f[1][-1], Tb, rtol=1e-11)
    assert Tb > 1.2


def test_thermal_closure_needs_the_temperature_scalar():
    for bad in (dict(n_scal=1), dict(n_scal=2, arr_A=-1.0), dict(n_scal=2, n_it=65)):
        with pytest.raises(Exception):
            Oracle(dict(dim=2, nx=8, ny=8, arrhenius=True, arr_A=0.1, arr_Ta=1.0, **bad))


# ---------------------------------------------------------------- residual (reading 16)

def test_residual_of_a_decaying_mode_is_its_closed_form():
    """The steady-state residual r is the relative L2 change of u and C over the fluid nodes
    between two evaluations.  For a cosine concentration mode at rest the field at step t is
    exactly C = 1 + a Re(1^T A^t w) cos(k x) (the single-mode update of the Fourier pin) and u = 0,
    so r between steps t0 and t1 is |c(t1) - c(t0)| |cos| / |1 + a c(t1) cos| in closed form;
    a field at rest that does not change has r = 0."""
    L, tau_c, J0, a = 32, 0.8, 0.4, 0.1
    shape = (1, 1, L)
    cfg = dict(dim=2, nx=L, ny=1, nz=1, n_comp=1, tau=[1.0], n_scal=1, tau_c=[tau_c], J0=J0,
               periodic=[1, 1, 1])
    x = np.arange(L)
    k = 2 * np.pi / L
    C0 = (1.0 + a * np.cos(k * x)).reshape(shape)
    rho, u, _ = inputs.uniform_fields(shape, 1, 0)
    o = make(cfg, None, (rho, u, C0[None]))
    cc, w = o.lattice(1)
    A = np.diag(np.exp(-1j * k * cc[:, 0])) @ ((1 - 1 / tau_c) * np.eye(len(w)) + np.outer(w, np.ones(len(w))) / tau_c)

    def mode(t):
        return (np.linalg.matrix_power(A, t) @ w.astype(complex)).sum().real

    o.step(40)
    assert o.residual() == -1.0          # the first evaluation only takes the snapshot
    o.step(30)
    r = o.residual()
    c0, c1 = mode(40), mode(70)
    cosx = np.cos(k * x)
    expect = np.linalg.norm(a * (c1 - c0) * cosx) / np.linalg.norm(1.0 + a * c1 * cosx)
    assert abs(r - expect) < 1e-10 * expect, (r, expect)
    # uniform fields at rest do not change: r = 0
    q = make(cfg, None, (rho, u, np.ones((1,) + shape)))
    q.residual()
    q.step(25)
    assert q.residual() == 0.0
