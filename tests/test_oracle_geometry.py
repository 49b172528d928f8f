"""Pins of the oracle's wall forces and geometry updates.

Flat-wall closed forms of the Shan-Chen solid and adhesion terms (Eq. 1.13,
1.15), exact first-step values of the wet-node reaction and of deposition
(Eq. wetnode9, Eq. surface_deposition), and the mass / species budgets that
dissolution and deposition flips must close to round-off.
"""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2502_12955_gb300 import inputs


def make(cfg, geom, fields=None):
    o = Oracle(cfg)
    o.set_geometry(geom)
    if fields is None:
        fields = inputs.uniform_fields(o.shape, o.p.n_comp, o.p.n_scal, rho=1.0, C=1.0)
    rho, u, C = fields
    o.set_fields(rho, u, C if o.p.n_scal else None)
    return o


@pytest.mark.parametrize("dim", [2, 3])
def test_flat_wall_adhesion_and_solid_psi_force(dim):
    """Uniform fluid above a flat wall at rest: the wall-normal force on the first fluid
    layer is G_ads rho / 6 (Eq. 1.15) and -G psi(rho) (psi(rho) - psi(rho_s)) / 6 (Eq. 1.13),
    because sum over wall-pointing directions of w_i c_i = -c_s^2 / 2 = -1/6 on D2Q9 and
    D3Q19; it vanishes in the bulk.  The reported velocity at rest is F / (2 rho)."""
    axis = 1 if dim == 2 else 0               # y in 2D, z in 3D (array axis)
    shape = (1, 12, 6) if dim == 2 else (12, 5, 6)
    geom = np.zeros(shape, np.uint8)
    if dim == 2:
        geom[0, 0, :] = 1
    else:
        geom[0, :, :] = 1
    rho0, G, Gads, rs = 0.8, -2.0, 0.3, 0.5
    cfg = dict(dim=dim, nx=shape[2], ny=shape[1], nz=shape[0], tau=[1.0],
               G=[[G, 0], [0, 0]], G_ads=[Gads, 0], rho_solid=rs, psi_kind="exp")
    o = make(cfg, geom, inputs.uniform_fields(shape, 1, 0, rho=rho0))
    u = o.fields()["u"]
    comp = 1 if dim == 2 else 2
    psi = lambda r: 1 - np.exp(-r)
    F = Gads * rho0 / 6 - G * psi(rho0) * (psi(rho0) - psi(rs)) / 6
    first = u[comp, 0, 1, :] if dim == 2 else u[comp, 1, :, :]
    np.testing.assert_allclose(first, F / (2 * rho0), rtol=1e-13)
    bulk = u[comp, 0, 5, :] if dim == 2 else u[comp, 5, :, :]
    np.testing.assert_allclose(bulk, 0, atol=1e-17)


def _single_solid(k, V_m, m_s0, geo="dissolve", tau_c=1.0):
    shape = (1, 9, 9)
    geom = np.zeros(shape, np.uint8)
    geom[0, 4, 4] = 2
    cfg = dict(dim=2, nx=9, ny=9, tau=[1.0], n_scal=1, tau_c=[tau_c], J0=0.4, k_react=k,
               geo_mode=geo, V_m=V_m, m_s0=m_s0, periodic=[1, 1, 1])
    return make(cfg, geom)


def test_dissolution_first_step_closed_form_and_flip():
    """C = 1 at rest around one reactive node: the first closure gives each of its four links
    C_b = 2 * 0.15 / (0.3 + K), K = k tau/(tau - 1/2) (Eq. wetnode9), so the node has reacted
    4 k C_b.  With m_s0 just below V_m times that it dissolves after the first step and is
    re-initialised at rest with the mean density and concentration of its fluid neighbours."""
    k, tau_c = 0.01, 1.0
    K = k * tau_c / (tau_c - 0.5)
    r1 = 4 * k * 2 * 0.15 / (0.3 + K)
    # just above: no flip; its neighbour values are those the flip below averages
    o = _single_solid(k, 1.0, r1 * (1 + 1e-9))
    o.step(1)
    f0 = o.fields()
    assert f0["flags"][0, 4, 4] == 2
    np.testing.assert_allclose(f0["acc"][0, 4, 4], r1, rtol=1e-14)
    nb = [(3, 3), (3, 4), (3, 5), (4, 3), (4, 5), (5, 3), (5, 4), (5, 5)]
    rho_nb = np.mean([f0["rho"][0, 0, y, x] for y, x in nb])
    C_nb = np.mean([f0["C"][0, 0, y, x] for y, x in nb])
    # just below: flips after the first step
    o = _single_solid(k, 1.0, r1 * (1 - 1e-9))
    o.step(1)
    f = o.fields()
    assert f["flags"][0, 4, 4] == 0
    m = o.monitors()
    np.testing.assert_allclose(f["rho"][0, 0, 4, 4], rho_nb, rtol=1e-14)
    np.testing.assert_allclose(f["C"][0, 0, 4, 4], C_nb, rtol=1e-14)
    np.testing.assert_allclose(m["inj_mass0"], rho_nb, rtol=1e-14)
    np.testing.assert_allclose(m["inj_spec0"], C_nb, rtol=1e-14)
    fp, hp = o.pops()
    w9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    np.testing.assert_allclose(fp[0, :, 4 * 9 + 4], w9 * rho_nb, rtol=1e-14)
    assert m["nsolid"] == 0


def test_dissolution_budgets_close():
    """Channel with reactive circles, strong consumption: solids dissolve over time; fluid
    mass changes only by what flips inject, the stored scalar sum by inflow - outflow -
    wall exchange + injected, and the per-node reaction bookkeeping sums to the total."""
    cfg, geom, fields = inputs.reactive_channel_2d(nx=64, ny=32, seed=1)
    cfg.update(k_react=0.05, geo_mode="dissolve", V_m=40.0, m_s0=1.0, g=[5e-5, 0, 0])
    fields[2][:] = 1.0
    o = make(cfg, geom, fields)
    m0 = o.monitors()
    o.step(400)
    m = o.monitors()
    assert m["nsolid"] < m0["nsolid"] - 10, "expected some solids to dissolve"
    np.testing.assert_allclose(m["mass0"], m0["mass0"] + m["inj_mass0"], rtol=1e-13)
    lhs = m["species0"] - m0["species0"]
    rhs = m["inflow0"] - m["outflow0"] - m["wallx"] + m["inj_spec0"]
    assert abs(lhs - rhs) < 1e-12 * m0["species0"]
    f = o.fields()
    np.testing.assert_allclose(f["acc"].sum(), m["reacted"], rtol=1e-12)
    # every node that flipped has consumed at least m_s0 / V_m; none still solid has
    flipped = (geom[0] == 2) & (f["flags"][0] == 0)
    assert np.all(cfg["V_m"] * f["acc"][0][flipped] >= 1.0)
    still = f["flags"][0] == 2
    assert np.all(cfg["V_m"] * f["acc"][0][still] < 1.0)


def test_deposition_first_step_closed_form():
    """Eq. surface_deposition: after one step every near-substrate fluid node holds
    C_p,s = DP * sum_i h_p,i = DP * C; other nodes hold 0."""
    shape = (1, 8, 8)
    geom = np.zeros(shape, np.uint8)
    geom[0, 3, 3] = 1
    cfg = dict(dim=2, nx=8, ny=8, tau=[1.0], n_scal=1, tau_c=[0.8], J0=0.4, geo_mode="deposit",
               DP=0.002, periodic=[1, 1, 1])
    C0 = 0.7
    o = make(cfg, geom, inputs.uniform_fields(shape, 1, 1, rho=1.0, C=C0))
    o.step(1)
    acc = o.fields()["acc"][0]
    near = np.zeros((8, 8), bool)
    for y, x in [(2, 3), (4, 3), (3, 2), (3, 4)]:
        near[y, x] = True
    np.testing.assert_allclose(acc[near], 0.002 * C0, rtol=1e-14)
    assert np.all(acc[~near] == 0)


@pytest.mark.parametrize("conservative", [True, False])
def test_deposition_budget_and_flips(conservative):
    """Particles carried through a channel with inert obstacles deposit on the obstacles;
    nodes whose deposit exceeds 1 turn solid.  Conservative mode: stored particle sum +
    deposited + removed-by-flips is constant in a closed box."""
    cfg, geom, fields = inputs.reactive_channel_2d(nx=48, ny=24, seed=3)
    geom[geom != 0] = 1
    cfg.update(k_react=0.0, geo_mode="deposit", DP=0.2, deposit_conservative=conservative,
               ade_open_x=False, g=[5e-5, 0, 0])
    fields[2][:] = 2.0
    o = make(cfg, geom, fields)
    m0 = o.monitors()
    o.step(150)
    m = o.monitors()
    f = o.fields()
    grown = (geom[0] == 0) & (f["flags"][0] == 1)
    assert grown.sum() > 0
    assert np.all(f["acc"][0][grown] > 1.0)
    assert np.all(f["acc"][0][f["flags"][0] == 0] <= 1.0)
    np.testing.assert_allclose(m["mass0"] + m["rem_mass0"], m0["mass0"], rtol=1e-13)
    if conservative:
        np.testing.assert_allclose(m["species0"] + m["deposited"] + m["rem_spec0"],
                                   m0["species0"], rtol=1e-13)
    else:
        np.testing.assert_allclose(m["species0"] + m["rem_spec0"], m0["species0"], rtol=1e-13)
    np.testing.assert_allclose(f["acc"].sum(), m["deposited"], rtol=1e-12)


def _front_channel(xs, **geo):
    """1D channel at rest: inlet C = 1 at x = 0, reactive solid from node xs to the end."""
    nx = 24
    shape = (1, 1, nx)
    g = np.zeros(shape, np.uint8)
    g[0, 0, xs:] = 2
    cfg = dict(dim=2, nx=nx, ny=1, tau=[1.0], n_scal=1, tau_c=[0.8], J0=0.4, k_react=0.05,
               ade_open_x=True, C_in=[1.0], periodic=[1, 1, 1], **geo)
    return make(cfg, g, (np.ones((1,) + shape), np.zeros((3,) + shape), np.zeros((1,) + shape)))


def test_dissolution_front_advances_at_the_quasi_steady_rate():
    """A slowly dissolving slab (Sec. 2.1.5 solid consumption): each front node takes
    m_s0 / V_m of reaction to dissolve, and while the front is slow the reaction at it is the
    steady rate for the current front position (whose link flux the steady-diffusion pin ties
    to k C_b). So the time between two flips is (m_s0 / V_m) / r(front), to 0.5 %: the
    threshold, the booking of each link's reaction on its own solid node, and the closure of
    the links the new fluid node opens all enter it. The steady rate with the front at node xs
    is D C_in / (xs - 1 + tau_c + D / k), D = 0.3 (tau_c - 1/2) (the closed form of the steady
    reactive channel)."""
    D, tau_c, k = 0.3 * (0.8 - 0.5), 0.8, 0.05
    rates = {xs: D / (xs - 1 + tau_c + D / k) for xs in (11, 12, 13)}
    thr = 300.0
    o = _front_channel(10, geo_mode="dissolve", V_m=1.0 / thr, m_s0=1.0)
    flips, step, n_solid = [], 0, o.monitors()["nsolid"]
    while len(flips) < 4 and step < 400000:
        o.step(20)
        step += 20
        ns = o.monitors()["nsolid"]
        if ns < n_solid:
            assert ns == n_solid - 1, "one node per flip"
            flips.append(step)
            n_solid = ns
    assert len(flips) == 4
    for k, xs in enumerate((11, 12, 13), start=1):
        interval = flips[k] - flips[k - 1]
        assert abs(interval / (thr / rates[xs]) - 1) < 5e-3, (xs, interval, thr / rates[xs])


@pytest.mark.parametrize("tau_c,DP,xs,J0,C_in,conservative", [(0.8, 0.01, 10, 0.4, 1.0, True),
                                                               (1.2, 0.05, 7, 0.2, 0.6, True),
                                                               (0.9, 0.02, 8, 0.4, 0.8, False)])
def test_steady_deposition_channel_closed_form(tau_c, DP, xs, J0, C_in, conservative):
    """Particles enter a 1D channel at x = 0 and deposit at the node next to an inert wall
    (Sec. 3.3, Eq. surface_deposition), with the flips held off. The steady state follows from
    the update itself. Before the last node the profile is linear, C(x) = C_in + b (tau + x),
    with populations w (C -/+ b tau). At the last node n = xs - 1 every population is scaled by
    s = 1 - DP (by 1 without removal), relaxed, and the +x one comes back by bounce-back. Three
    linear equations in b, C(n) and the returning population give the whole state, and the
    deposit per step is DP C(n)."""
    nx = xs + 3
    shape = (1, 1, nx)
    geom = np.zeros(shape, np.uint8)
    geom[0, 0, xs:] = 1
    cfg = dict(dim=2, nx=nx, ny=1, tau=[1.0], n_scal=1, tau_c=[tau_c], J0=J0, ade_open_x=True,
               C_in=[C_in], geo_mode="deposit", DP=DP, deposit_conservative=conservative,
               N_geo=10 ** 9, periodic=[1, 1, 1])
    o = make(cfg, geom, (np.ones((1,) + shape), np.zeros((3,) + shape), np.zeros((1,) + shape)))
    o.step(60000)
    m0 = o.monitors()
    o.step(1)
    dep = o.monitors()["deposited"] - m0["deposited"]
    C = o.fields()["C"][0, 0, 0, :xs]
    w, om, n = (1.0 - J0) / 4.0, 1.0 / tau_c, xs - 1
    s = 1.0 - DP if conservative else 1.0
    q = om * (J0 + 2 * w) * s / (1.0 - (1.0 - om) * s)      # rest + y populations over C(n)
    # unknowns (b, C(n), m): the -x population m* leaving n is the linear profile's at n - 1;
    # m at n is the bounced-back +x population; C(n) sums all populations of n
    M = np.array([[-w * (2 * tau_c + n - 1), om * w * s, (1 - om) * s],
                  [-(1 - om) * s * w * n, -om * w * s, 1.0],
                  [-w * n, 1.0 - q, -1.0]])
    rhs = np.array([w * C_in, (1 - om) * s * w * C_in, w * C_in])
    b, Cn, _ = np.linalg.solve(M, rhs)
    np.testing.assert_allclose(C[:n], C_in + b * (tau_c + np.arange(n)), atol=1e-12)
    np.testing.assert_allclose(C[n], Cn, rtol=1e-11)
    np.testing.assert_allclose(dep, DP * Cn, rtol=1e-10)
