"""Brute force on tiny lattices: the oracle against a second, naive formulation of the step
(tests/naive_lbm.py: push streaming, full-matrix MRT from the printed polynomials, plain
loops), written independently of oracle/.  A dropped term, a wrong sign or index, a transposed
operand or a misread boundary rule in either shows up as a difference far above round-off."""
import zlib

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2502_12955_gb300 import inputs
from tests.naive_lbm import NaiveLBM

CASES = {
    "2d_bgk_reactive_open": dict(dim=2, nx=8, ny=8, tau=[0.8], g=[2e-4, -1e-4, 0], n_scal=1, tau_c=[0.7],
                                 J0=0.4, k_react=0.05, ade_open_x=True, C_in=[1.3], periodic=[1, 1, 1]),
    "2d_mrt_walls_two_scalars": dict(dim=2, nx=8, ny=8, tau=[0.9], g=[1e-4, 0, 0], collision="mrt", n_scal=2,
                                     tau_c=[0.7, 1.1], J0=0.25, k_react=0.03, periodic=[1, 0, 1]),
    "2d_two_component_sc": dict(dim=2, nx=8, ny=8, n_comp=2, tau=[1.0, 0.8], G=[[0, 2.5], [2.5, 0]],
                                psi_kind="identity", g=[0, -1e-4, 0], periodic=[1, 1, 1]),
    "2d_sc_shift_adhesion": dict(dim=2, nx=8, ny=8, n_comp=2, tau=[1.0, 0.9], G=[[0, 1.8], [1.8, 0]],
                                 psi_kind="exp", forcing="sc_shift", G_ads=[0.2, -0.1], periodic=[1, 0, 1]),
    "3d_mrt_reactive_open": dict(dim=3, nx=8, ny=8, nz=8, tau=[1.0], g=[3e-4, 1e-4, 0], collision="mrt",
                                 n_scal=1, tau_c=[0.5667], J0=0.25, k_react=0.02, ade_open_x=True,
                                 C_in=[1.0], periodic=[1, 1, 0]),
    "2d_couette_moving_plate_scalar": dict(dim=2, nx=8, ny=8, tau=[0.7], u_wall_ymax=[0.03, 0, 0], n_scal=1,
                                          tau_c=[0.8], J0=0.4, k_react=0.04, periodic=[1, 0, 1]),
    "3d_mrt_moving_plate": dict(dim=3, nx=8, ny=8, nz=8, tau=[0.9], collision="mrt", g=[1e-4, 0, 0],
                                u_wall_ymax=[0.02, 0, -0.01], periodic=[1, 0, 1]),
    "3d_bgk_single_sc_walls": dict(dim=3, nx=8, ny=8, nz=8, tau=[1.0], G=[[-4.5, 0], [0, 0]], psi_kind="exp",
                                   rho_solid=0.3, periodic=[0, 1, 1]),
    "2d_velocity_inlet_reactive": dict(dim=2, nx=8, ny=8, tau=[0.8], flow_open_x=True, u_in=0.03, n_scal=1,
                                       tau_c=[0.7], J0=0.4, k_react=0.05, ade_open_x=True, C_in=[1.0],
                                       periodic=[0, 0, 1]),
    "2d_arrhenius_heat_open": dict(dim=2, nx=8, ny=8, tau=[0.8], g=[2e-4, 0, 0], n_scal=2, tau_c=[0.7, 0.9],
                                   J0=0.4, arrhenius=True, arr_A=0.4, arr_Ta=1.0, heat_release=0.02, n_it=24,
                                   ade_open_x=True, C_in=[1.0, 0.6], periodic=[1, 1, 1]),
    "3d_mrt_arrhenius_heat_walls": dict(dim=3, nx=8, ny=8, nz=8, tau=[0.9], collision="mrt", g=[1e-4, 0, 0],
                                        n_scal=2, tau_c=[0.6, 0.8], J0=0.25, arrhenius=True, arr_A=0.3,
                                        arr_Ta=0.8, heat_release=0.03, n_it=24, periodic=[1, 0, 1]),
    "2d_dissolution_flips": dict(dim=2, nx=8, ny=8, tau=[0.8], g=[2e-4, 0, 0], n_scal=1, tau_c=[0.7], J0=0.4,
                                 k_react=0.08, geo_mode="dissolve", V_m=25.0, periodic=[1, 1, 1]),
    "3d_mrt_deposition_flips": dict(dim=3, nx=8, ny=8, nz=8, tau=[0.9], collision="mrt", g=[1e-4, 0, 0],
                                    n_scal=1, tau_c=[0.6], J0=0.25, geo_mode="deposit", DP=0.7,
                                    deposit_conservative=False, periodic=[1, 0, 1]),
    "2d_deposition_conservative": dict(dim=2, nx=8, ny=8, tau=[0.8], n_scal=1, tau_c=[0.8], J0=0.4,
                                       geo_mode="deposit", DP=0.4, ade_open_x=True, C_in=[1.5],
                                       periodic=[1, 0, 1]),
    "3d_arrhenius_dissolution_flips": dict(dim=3, nx=8, ny=8, nz=8, tau=[1.0], g=[1e-4, 0, 0], n_scal=2,
                                           tau_c=[0.6, 0.8], J0=0.25, arrhenius=True, arr_A=0.3,
                                           arr_Ta=0.8, heat_release=0.03, n_it=24, geo_mode="dissolve",
                                           V_m=40.0, N_geo=2, periodic=[1, 1, 1]),
    "2d_conjugate_heat_walls": dict(dim=2, nx=8, ny=8, tau=[0.8], g=[2e-4, 0, 0], n_scal=2, tau_c=[0.7, 0.9],
                                    J0=0.4, arrhenius=True, arr_A=0.4, arr_Ta=1.0, heat_release=0.05, n_it=40,
                                    conjugate=True, tau_s=0.65, c_fs=2.5, periodic=[1, 0, 1]),
    "2d_conjugate_open": dict(dim=2, nx=8, ny=8, tau=[0.9], g=[1e-4, 0, 0], n_scal=2, tau_c=[0.8, 0.7], J0=0.4,
                              arrhenius=True, arr_A=0.3, arr_Ta=0.6, heat_release=0.04, n_it=40, conjugate=True,
                              tau_s=1.1, c_fs=0.7, ade_open_x=True, C_in=[1.0, 0.9], periodic=[1, 1, 1]),
    "3d_mrt_conjugate_dissolution": dict(dim=3, nx=8, ny=8, nz=8, tau=[1.0], collision="mrt", g=[1e-4, 0, 0],
                                         n_scal=2, tau_c=[0.6, 0.8], J0=0.25, arrhenius=True, arr_A=0.3,
                                         arr_Ta=0.8, heat_release=0.03, n_it=40, conjugate=True, tau_s=0.7,
                                         c_fs=0.6, geo_mode="dissolve", V_m=40.0, N_geo=2, periodic=[1, 1, 1]),
    "2d_product_open": dict(dim=2, nx=8, ny=8, tau=[0.8], g=[2e-4, -1e-4, 0], n_scal=1, tau_c=[0.7], J0=0.4,
                            k_react=0.05, product=True, tau_p=0.9, ade_open_x=True, C_in=[1.0], C_in_p=0.1,
                            periodic=[1, 1, 1]),
    "3d_mrt_arrhenius_product_dissolution": dict(dim=3, nx=8, ny=8, nz=8, tau=[1.0], collision="mrt",
                                                 g=[1e-4, 0, 0], n_scal=2, tau_c=[0.6, 0.8], J0=0.25,
                                                 arrhenius=True, arr_A=0.3, arr_Ta=0.8, heat_release=0.03,
                                                 n_it=24, product=True, tau_p=0.75, geo_mode="dissolve",
                                                 V_m=40.0, N_geo=2, periodic=[1, 1, 1]),
    "2d_conjugate_product_walls": dict(dim=2, nx=8, ny=8, tau=[0.8], g=[2e-4, 0, 0], n_scal=2, tau_c=[0.7, 0.9],
                                       J0=0.4, arrhenius=True, arr_A=0.4, arr_Ta=1.0, heat_release=0.05,
                                       n_it=40, conjugate=True, tau_s=0.65, c_fs=2.5, product=True, tau_p=1.2,
                                       periodic=[1, 0, 1]),
    "3d_conjugate_product_open": dict(dim=3, nx=8, ny=8, nz=8, tau=[0.9], g=[1e-4, 0, 1e-4], n_scal=2,
                                      tau_c=[0.7, 0.6], J0=0.25, arrhenius=True, arr_A=0.5, arr_Ta=0.7,
                                      heat_release=0.08, n_it=40, conjugate=True, tau_s=0.9, c_fs=1.7,
                                      product=True, tau_p=0.65, ade_open_x=True, C_in=[1.0, 1.1], C_in_p=0.05,
                                      periodic=[1, 0, 1]),
    "2d_burning_channel": dict(dim=2, nx=8, ny=8, tau=[0.8], flow_open_x=True, u_in=0.03, n_scal=2,
                               tau_c=[0.8, 0.9], J0=0.4, ade_open_x=True, C_in=[0.22, 1.0], arrhenius=True,
                               arr_A=2.0, arr_Ta=1.5, heat_release=0.5, n_it=40, conjugate=True, tau_s=0.7,
                               c_fs=0.5, product=True, tau_p=0.75, C_in_p=0.0, geo_mode="dissolve", V_m=200.0,
                               periodic=[0, 0, 1]),
    "3d_mrt_velocity_inlet": dict(dim=3, nx=8, ny=8, nz=8, tau=[0.9], collision="mrt", flow_open_x=True,
                                  u_in=0.02, g=[0, 0, 1e-4], u_wall_ymax=[0.01, 0, 0], periodic=[0, 0, 1]),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_oracle_matches_naive_formulation(name):
    cfg = dict(CASES[name], precision="fp64")
    dim = cfg["dim"]
    shape = (cfg.get("nz", 1), cfg["ny"], cfg["nx"])
    geom = inputs.random_solids(shape, 0.2, seed=zlib.crc32(name.encode()) % 1000)
    nc, ns = cfg.get("n_comp", 1), cfg.get("n_scal", 0) + int(cfg.get("product", False))
    rho, u, C = inputs.perturbed_fields(shape, nc, ns, seed=7, amp_rho=0.02, amp_u=0.02,
                                        rho0=[0.9, 0.4] if nc == 2 else 1.0)
    if dim == 2:
        u[2] = 0.0
    o = Oracle(cfg)
    o.set_geometry(geom)
    o.set_fields(rho, u, C if ns else None)
    f0, h0 = o.pops()
    nv = NaiveLBM(cfg, geom, f0, h0, T_solid=C[1] if cfg.get("conjugate") else None)
    for step in range(4):
        o.step(1)
        nv.step()
        f, h = o.pops()
        flags = o.fields()["flags"]
        assert np.array_equal(flags, nv.flags), f"{name} step {step + 1}: geometry flips differ"
        fl = (geom == 0) | (flags == 0)
        df = np.abs(f.reshape(nv.f.shape) - nv.f)[..., fl].max()
        assert df < 1e-13, f"{name} step {step + 1}: flow populations differ by {df:.3e}"
        if ns:
            dh = np.abs(h.reshape(nv.h.shape) - nv.h)[..., fl].max()
            assert dh < 1e-13, f"{name} step {step + 1}: scalar populations differ by {dh:.3e}"
            acc = o.fields()["acc"]
            assert np.abs(acc - nv.acc).max() < 1e-13, f"{name} step {step + 1}: reaction bookkeeping"
        if cfg.get("conjugate"):
            sol = flags != 0
            dT = np.abs(o.fields()["C"][1][sol] - nv.g.sum(axis=0)[sol]).max()
            assert dT < 1e-13, f"{name} step {step + 1}: solid temperatures differ by {dT:.3e}"


def _vectorised_channel(dim, tau, rates, g, H, steps):
    """Plane channel u_x(y) stepped with whole-array numpy operations: the naive formulation's
    velocity sets and printed MRT polynomials (tests/naive_lbm.py), Guo forcing in moment
    space, halfway bounce-back at y = -1/2 and H - 1/2, uniform in x and z."""
    from tests.naive_lbm import moment_matrix, opposite, velocity_sets
    cf, wf, _, _ = velocity_sets(dim, 0.25)
    opp = np.array(opposite(cf))
    M, grp = moment_matrix(dim, cf)
    Minv = np.linalg.inv(M)
    S = np.array([1.0 / tau if k in ("c", "nu") else rates[k] for k in grp])
    c = cf.astype(float)
    F = np.array([g, 0.0, 0.0])
    f = wf[:, None] * np.ones((1, H))
    cy = cf[:, 1]
    for _ in range(steps):
        rho = f.sum(0)
        u = (c.T @ f + F[:, None] / 2) / rho                       # [3, H]
        cu = c @ u
        feq = wf[:, None] * rho * (1 + 3 * cu + 4.5 * cu ** 2 - 1.5 * (u ** 2).sum(0))
        Fi = wf[:, None] * (3 * ((c @ F)[:, None] - (F @ u)[None, :]) + 9 * cu * (c @ F)[:, None])
        m = M @ f
        post = Minv @ (m - S[:, None] * (m - M @ feq) + (1 - S[:, None] / 2) * (M @ Fi))
        new = np.empty_like(f)
        for i in range(len(cf)):
            dst = np.arange(H) + cy[i]
            ok = (dst >= 0) & (dst < H)
            new[i, dst[ok]] = post[i, ok]
            new[opp[i], np.nonzero(~ok)[0]] = post[i, ~ok]          # halfway bounce-back
        f = new
    rho = f.sum(0)
    return ((c.T @ f)[0] + g / 2) / rho


def test_mrt_channel_steady_state_matches_vectorised_formulation():
    """D3Q19 MRT with the default rates of the full-size workload, driven to steady state in a
    plane channel: the oracle's profile equals, to 1e-10, that of the same update written with
    whole-array operations on the naive formulation's printed polynomials. The four-step brute
    force above cannot see slow long-time drifts; this comparison runs 20,000 steps."""
    tau, H, g = 0.9, 10, 1e-5
    rates = {"e": 1.19, "eps": 1.4, "q": 1.2, "pi": 1.0 / tau, "m": 1.98}
    steps = 20000
    ref = _vectorised_channel(3, tau, rates, g, H, steps)
    cfg = dict(dim=3, nx=1, ny=H, nz=1, tau=[tau], g=[g, 0, 0], collision="mrt", periodic=[1, 0, 1],
               mrt_rates=dict(s_e=1.19, s_eps=1.4, s_q=1.2, s_pi=1.0 / tau, s_m=1.98))
    o = Oracle(cfg)
    shape = (1, H, 1)
    o.set_geometry(np.zeros(shape, np.uint8))
    o.set_fields(np.ones((1,) + shape), np.zeros((3,) + shape), None)
    o.step(steps)
    ux = o.fields()["u"][0, 0, :, 0]
    assert ux.max() > 1e-4
    np.testing.assert_allclose(ux, ref, rtol=1e-10)


def _vectorised_slab(G, tau, H, steps, rho0):
    """Two-component Shan-Chen (psi = rho, Eq. 1.14) flat interfaces, uniform in x and periodic
    in y, stepped with whole-array operations on the naive formulation's D2Q9 set: Guo forcing
    with the barycentric velocity (Eq. 1.19-1.21), BGK."""
    from tests.naive_lbm import velocity_sets
    cf, wf, _, _ = velocity_sets(2, 0.4)
    c = cf.astype(float)
    cy = cf[:, 1]
    f = np.stack([wf[:, None] * r[None, :] for r in rho0])           # [2, 9, H]
    for _ in range(steps):
        rho = f.sum(1)                                               # [2, H]
        j = np.einsum("ia,sih->sah", c, f)                           # [2, 3, H]
        F = np.zeros((2, 3, H))
        for s, t in ((0, 1), (1, 0)):
            acc = sum(wf[i] * np.roll(rho[t], -cy[i]) * c[i, 1] for i in range(9))
            F[s, 1] = -rho[s] * G * acc
        u = (j + F / 2).sum(0) / rho.sum(0)                          # [3, H]
        cu = c @ u
        new = np.empty_like(f)
        for s in range(2):
            feq = wf[:, None] * rho[s] * (1 + 3 * cu + 4.5 * cu ** 2 - 1.5 * (u ** 2).sum(0))
            cF = c @ F[s]
            Fi = wf[:, None] * (3 * (cF - (F[s] * u).sum(0)) + 9 * cu * cF)
            post = f[s] - (f[s] - feq) / tau + (1 - 1 / (2 * tau)) * Fi
            for i in range(9):
                new[s, i] = np.roll(post[i], cy[i])
        f = new
    return f.sum(1)


def test_shan_chen_slab_matches_vectorised_formulation():
    """Two-component Shan-Chen flat interfaces relaxed over 6,000 steps: the oracle's density
    profiles equal those of a whole-array formulation to 1e-10. The four-step brute force cannot
    see the slow approach to coexistence; this comparison does."""
    G, tau, H, steps = 2.7, 1.0, 48, 6000
    y = np.arange(H)
    inside = (y >= 12) & (y < 36)
    rho0 = [np.where(inside, 1.0, 0.05), np.where(inside, 0.05, 1.0)]
    ref = _vectorised_slab(G, tau, H, steps, rho0)
    cfg = dict(dim=2, nx=1, ny=H, n_comp=2, tau=[tau, tau], G=[[0, G], [G, 0]], psi_kind="identity",
               periodic=[1, 1, 1])
    o = Oracle(cfg)
    shape = (1, H, 1)
    o.set_geometry(np.zeros(shape, np.uint8))
    o.set_fields(np.stack([r.reshape(shape) for r in rho0]), np.zeros((3,) + shape), None)
    o.step(steps)
    rho = o.fields()["rho"][:, 0, :, 0]
    assert rho[0].max() > 0.9 and rho[0].min() < 0.1
    np.testing.assert_allclose(rho, ref, rtol=1e-10, atol=1e-12)
