"""GPU (CUDA path through the C ABI) against the FP64 oracle, element by element.

FP64 mode must match within 1e-10 relative L2 on every field, population array and monitor,
with integer flags bit-exact, after the stated number of steps.  Cases cover both in-place
layout parities (odd and even step counts), ragged sizes, walls on closed axes, inlet /
outlet, the wet-node closure, dissolution and deposition flips, MRT, Shan-Chen multi-
component and single-component forces, adhesion and the velocity-shift scheme.
"""
import numpy as np
import pytest

from paper_2502_12955_gb300 import inputs
from paper_2502_12955_gb300.lbm import Solver
from tests.gpu_common import FP64_TOL, compare, make_pair, rel_l2

pytestmark = pytest.mark.gpu


def test_reactive_channel_2d_full_workload():
    """128x64 D2Q9 BGK + D2Q5 reactive channel, 2000 steps (checked at 1, 2 and 2000)."""
    cfg, geom, fields = inputs.reactive_channel_2d()
    o, g = make_pair(cfg, geom, fields)
    done = 0
    for target in (1, 2, 2000):
        o.step(target - done)
        g.step(target - done)
        done = target
        compare(o, g, what=f"channel step {target}")


@pytest.mark.parametrize("steps", [7, 40])
def test_2d_all_scalar_features(steps):
    """Ragged 37x23, inert + reactive solids, two scalars, inlet / outlet, body force."""
    shape = (1, 23, 37)
    geom = inputs.random_solids(shape, 0.2, seed=21)
    geom[0, :, 0] = 0
    geom[0, :, -1] = 0
    cfg = dict(dim=2, nx=37, ny=23, tau=[0.8], g=[3e-5, -1e-5, 0], n_scal=2, tau_c=[0.7, 1.1],
               J0=0.4, k_react=0.05, ade_open_x=True, C_in=[1.0, 0.3], periodic=[1, 1, 1])
    fields = inputs.perturbed_fields(shape, 1, 2, seed=22, amp_rho=0.01, amp_u=0.01)
    o, g = make_pair(cfg, geom, fields)
    o.step(steps)
    g.step(steps)
    compare(o, g, what=f"2d scalars {steps}")


@pytest.mark.parametrize("periodic", [[1, 1, 1], [1, 0, 1], [0, 0, 0]])
def test_3d_bgk_walls_and_scalars(periodic):
    shape = (9, 13, 18)
    geom = inputs.random_solids(shape, 0.15, seed=23)
    cfg = dict(dim=3, nx=18, ny=13, nz=9, tau=[0.9], g=[1e-5, 2e-6, -3e-6], n_scal=2,
               tau_c=[0.8, 0.6], J0=0.25, k_react=0.02, periodic=periodic)
    fields = inputs.perturbed_fields(shape, 1, 2, seed=24, amp_rho=0.01, amp_u=0.01)
    o, g = make_pair(cfg, geom, fields)
    o.step(31)
    g.step(31)
    compare(o, g, what=f"3d bgk {periodic}")


@pytest.mark.parametrize("steps", [60, 61])
def test_3d_mrt_dissolution_with_flips(steps):
    """D3Q19 MRT + D3Q7, ragged 20x14x11 packing, fast consumption so solids dissolve."""
    cfg, geom, fields = inputs.dissolution_3d(shape=(11, 14, 20), g=5e-4, radius=(2.0, 4.0))
    cfg.update(k_react=0.05, V_m=25.0)
    o, g = make_pair(cfg, geom, fields)
    o.step(steps)
    g.step(steps)
    m = o.monitors()
    assert m["inj_mass0"] > 0, "the case should dissolve some solids"
    compare(o, g, what=f"mrt dissolution {steps}")


def test_dissolution_every_n_geo():
    cfg, geom, fields = inputs.dissolution_3d(shape=(8, 12, 16), g=5e-4, radius=(2.0, 4.0))
    cfg.update(k_react=0.05, V_m=25.0, N_geo=3, collision="bgk")
    o, g = make_pair(cfg, geom, fields)
    o.step(47)
    g.step(47)
    assert o.monitors()["inj_mass0"] > 0
    compare(o, g, what="n_geo 3")


@pytest.mark.parametrize("conservative,steps", [(True, 150), (True, 151), (False, 120)])
def test_2d_deposition_with_flips(conservative, steps):
    cfg, geom, fields = inputs.reactive_channel_2d(nx=48, ny=24, seed=3)
    geom[geom != 0] = 1
    cfg.update(k_react=0.0, geo_mode="deposit", DP=0.2, deposit_conservative=conservative,
               ade_open_x=False, g=[5e-5, 0, 0])
    fields[2][:] = 2.0
    o, g = make_pair(cfg, geom, fields)
    o.step(steps)
    g.step(steps)
    assert o.monitors()["rem_mass0"] > 0, "the case should grow deposits"
    compare(o, g, what=f"deposition {conservative} {steps}")


def test_3d_deposition_inlet():
    cfg, geom, fields = inputs.dissolution_3d(shape=(10, 12, 22), g=5e-4, radius=(2.0, 4.0))
    geom[geom != 0] = 1
    cfg.update(geo_mode="deposit", DP=0.3, k_react=0.0, C_in=[3.0])
    o, g = make_pair(cfg, geom, fields)
    o.step(45)
    g.step(45)
    compare(o, g, what="3d deposition")


def test_two_component_droplet_3d():
    cfg, geom, fields = inputs.droplet_3d(n=24, radius=7.0, precision="fp64")
    o, g = make_pair(cfg, geom, fields)
    o.step(101)
    g.step(101)
    compare(o, g, what="droplet 3d")


@pytest.mark.parametrize("forcing", ["guo", "sc_shift"])
def test_two_component_2d_forcing_schemes(forcing):
    shape = (1, 30, 34)
    cfg = dict(dim=2, nx=34, ny=30, n_comp=2, tau=[1.0, 0.8], G=[[0, 2.5], [2.5, 0]],
               psi_kind="identity", forcing=forcing, g=[0, -1e-5, 0], periodic=[1, 1, 1])
    rho, u = inputs.droplet_fields(shape, 9.0)
    o, g = make_pair(cfg, np.zeros(shape, np.uint8), (rho, u, None))
    o.step(150)
    g.step(150)
    compare(o, g, what=f"two component {forcing}")


def test_single_component_sc_with_walls_adhesion():
    """Eq. 1.13 / 1.15: exp pseudopotential, G = -5, solid psi and adhesion on closed walls."""
    shape = (1, 28, 40)
    geom = np.zeros(shape, np.uint8)
    geom[0, 10:14, 15:22] = 1
    cfg = dict(dim=2, nx=40, ny=28, n_comp=1, tau=[1.0], G=[[-5.0, 0], [0, 0]], psi_kind="exp",
               G_ads=[-0.3, 0], rho_solid=0.4, periodic=[1, 0, 1])
    rng = np.random.default_rng(25)
    rho = (0.7 * (1 + 0.05 * rng.uniform(-1, 1, size=shape)))[None]
    u = np.zeros((3,) + shape)
    o, g = make_pair(cfg, geom, (rho, u, None))
    o.step(120)
    g.step(120)
    compare(o, g, what="sc single")


def test_two_component_3d_with_solid_and_adhesion():
    shape = (10, 12, 14)
    geom = inputs.random_solids(shape, 0.1, seed=26, reactive_fraction=0.0)
    cfg = dict(dim=3, nx=14, ny=12, nz=10, n_comp=2, tau=[1.0, 1.0], G=[[0, 2.2], [2.2, 0]],
               psi_kind="identity", G_ads=[0.1, -0.1], rho_solid=0.5, periodic=[1, 1, 0])
    rng = np.random.default_rng(27)
    rho = np.stack([0.5 + 0.1 * rng.uniform(size=shape), 0.5 + 0.1 * rng.uniform(size=shape)])
    u = np.zeros((3,) + shape)
    o, g = make_pair(cfg, geom, (rho, u, None))
    o.step(33)
    g.step(33)
    compare(o, g, what="sc 3d walls")


def test_pops_roundtrip_and_odd_layout():
    cfg, geom, fields = inputs.dissolution_3d(shape=(6, 7, 9), g=1e-4, radius=(1.5, 2.5))
    _, g = make_pair(cfg, geom, fields)
    g.step(3)
    f, h = g.pops()
    g.set_pops(f, h)
    f2, h2 = g.pops()
    assert np.array_equal(f, f2) and np.array_equal(h, h2)


def test_checkpoint_resume_is_bitwise():
    cfg, geom, fields = inputs.dissolution_3d(shape=(10, 12, 16), g=5e-4, radius=(2.0, 4.0))
    cfg.update(geo_mode="none", precision="fp32")
    _, g = make_pair(cfg, geom, fields, precision="fp32")
    g.step(31)
    blob = g.get_state()
    g.step(20)
    fa, ha = g.pops()
    g.set_state(blob)
    g.step(20)
    fb, hb = g.pops()
    assert np.array_equal(fa, fb) and np.array_equal(ha, hb)


# Relative L2 tolerances per field of the reduced-precision modes against the FP64 oracle on
# the dissolution workload's transport parameters (velocity ~ 1e-2), 200 steps.
REDUCED_TOL = {"fp32": {"rho": 1e-6, "u": 1e-4, "C": 1e-5},
               "fp16": {"rho": 1e-4, "u": 1e-2, "C": 2e-3},
               "bf16": {"rho": 1e-3, "u": 5e-2, "C": 1e-2}}
# the mixed modes store the flow as the 16-bit modes do and the scalars in FP32: flow bounds
# of the 16-bit mode, scalar bound of FP32 arithmetic carried by a 16-bit flow
REDUCED_TOL["fp16s32"] = dict(REDUCED_TOL["fp16"])
REDUCED_TOL["bf16s32"] = dict(REDUCED_TOL["bf16"])


@pytest.mark.parametrize("precision", ["fp32", "fp16", "bf16", "fp16s32", "bf16s32"])
def test_reduced_precision_against_fp64_oracle(precision):
    cfg, geom, fields = inputs.dissolution_3d(shape=(16, 18, 24), radius=(2.0, 4.0), g=2e-3)
    cfg.update(geo_mode="none")
    o, g = make_pair(cfg, geom, fields, precision=precision)
    o.step(200)
    g.step(200)
    fo, fg = o.fields(), g.fields()
    errs = {k: rel_l2(fo[k], fg[k]) for k in ("rho", "u", "C")}
    print(precision, {k: f"{e:.2e}" for k, e in errs.items()})
    for k, e in errs.items():
        assert e < REDUCED_TOL[precision][k], f"{precision} {k}: {e:.3e}"


def test_state_errors():
    from paper_2502_12955_gb300.lbm import LbmError, Solver
    s = Solver(dict(dim=2, nx=8, ny=8, precision="fp64"))
    with pytest.raises(LbmError) as e:
        s.step(1)
    assert e.value.status == -6
    with pytest.raises(LbmError) as e:
        s.set_geometry(np.full((1, 8, 8), 3, np.uint8))
    assert e.value.status == -1


def test_nonfinite_initial_field_is_reported():
    """A NaN in a host-prepared initial field must surface as LBM_ERR_NONFINITE at the next
    monitor evaluation (no device fault involved)."""
    from paper_2502_12955_gb300.lbm import LbmError, Solver
    cfg, geom, fields = inputs.dissolution_3d(shape=(6, 8, 10), g=1e-4, radius=(1.5, 2.5))
    rho, u, C = fields
    rho = rho.copy()
    z, y, x = np.argwhere(geom == 0)[3]
    rho[0, z, y, x] = np.nan
    s = Solver(dict(cfg, precision="fp32", N_mon=2))
    s.set_geometry(geom)
    s.set_fields(rho, u, C)
    s.step(2)
    with pytest.raises(LbmError) as e:
        s.sync()
    assert e.value.status == -4
    assert s.monitors()["nonfinite"] >= 1


def test_allocation_failure_is_reported_and_cleaned_up():
    """A domain larger than device memory fails with LBM_ERR_OOM and leaves nothing allocated
    (a second, small context still works)."""
    from paper_2502_12955_gb300.lbm import LbmError, Solver
    with pytest.raises(LbmError) as e:
        Solver(dict(dim=3, nx=1280, ny=1280, nz=1280, precision="fp64", n_scal=2))
    assert e.value.status == -2
    s = Solver(dict(dim=2, nx=16, ny=16, precision="fp64"))
    s.set_geometry(np.zeros((1, 16, 16), np.uint8))
    s.set_fields(np.ones((1, 1, 16, 16)), np.zeros((3, 1, 16, 16)), None)
    s.step(3)
    s.sync()


@pytest.mark.parametrize("dim,steps", [(2, 3000), (3, 1500)])
def test_couette_moving_plate(dim, steps):
    """Sec. 3.1.1: top plate at U_wall = 0.02, Re = 10 on Ny = 15 (tau 0.59), periodic x and z;
    the plate's Ladd bounce-back against the oracle in FP64, then the converged FP32 profile
    against Eq. couette_velocity_profile."""
    ny, U = 15, 0.02
    nx, nz = 15, (15 if dim == 3 else 1)
    cfg = dict(dim=dim, nx=nx, ny=ny, nz=nz, tau=[0.59], periodic=[1, 0, 1], u_wall_ymax=[U, 0, 0])
    shape = (nz, ny, nx)
    rho, u, _ = inputs.perturbed_fields(shape, 1, 0, seed=31, amp_rho=0.01, amp_u=0.005)
    o, g = make_pair(cfg, np.zeros(shape, np.uint8), (rho, u, None))
    o.step(steps)
    g.step(steps)
    compare(o, g, what=f"couette {dim}d")
    s = Solver(dict(cfg, precision="fp32"))
    s.set_geometry(np.zeros(shape, np.uint8))
    s.set_fields(*inputs.uniform_fields(shape, 1, 0, rho=1.0)[:2], None)
    s.step(40000)
    prof = s.fields()["u"][0].mean(axis=(0, 2))
    exact = U * (np.arange(ny) + 0.5) / ny
    assert np.abs(prof - exact).max() < 1e-4 * U, np.abs(prof - exact).max()   # FP32 storage of O(1) values


@pytest.mark.parametrize("dim,steps", [(2, 61), (2, 60), (3, 41)])
def test_velocity_inlet_channel(dim, steps):
    """Sec. 3.4: flow velocity inlet u_x = 6 U s (1 - s) at x = 0 and zero-gradient outlet at
    x = nx - 1.  2D: BGK with the reactive scalar's inlet / outlet on the same faces and random
    solids (reactive and inert).  3D: MRT with a moving top plate meeting the inlet at the
    corner links, a body force and two scalars."""
    if dim == 2:
        nx, ny, nz = 26, 14, 1
        cfg = dict(dim=2, nx=nx, ny=ny, tau=[0.8], flow_open_x=True, u_in=0.03, n_scal=1, tau_c=[0.7],
                   J0=0.4, k_react=0.05, ade_open_x=True, C_in=[1.0], periodic=[0, 0, 1])
    else:
        nx, ny, nz = 16, 10, 8
        cfg = dict(dim=3, nx=nx, ny=ny, nz=nz, tau=[0.9], collision="mrt", flow_open_x=True, u_in=0.02,
                   u_wall_ymax=[0.01, 0, 0.005], g=[0, 0, 1e-4], n_scal=2, tau_c=[0.6, 0.9], J0=0.25,
                   k_react=0.03, periodic=[0, 0, 1])
    shape = (nz, ny, nx)
    geom = inputs.random_solids(shape, 0.12, seed=33 + dim)
    rho, u, C = inputs.perturbed_fields(shape, 1, cfg["n_scal"], seed=34, amp_rho=0.01, amp_u=0.01)
    o, g = make_pair(cfg, geom, (rho, u, C))
    o.step(steps)
    g.step(steps)
    compare(o, g, what=f"velocity inlet {dim}d")


def test_velocity_inlet_steady_channel_fp32():
    """The converged FP32 channel against the converged FP64 oracle: the inlet parabola carried to
    the outlet with the mass flux of the inlet in every column."""
    nx, ny, U = 40, 12, 0.01
    cfg = dict(dim=2, nx=nx, ny=ny, tau=[0.5 + np.sqrt(3.0) / 4.0], flow_open_x=True, u_in=U,
               periodic=[0, 0, 1])
    shape = (1, ny, nx)
    fields = inputs.uniform_fields(shape, 1, 0)
    o, g = make_pair(cfg, np.zeros(shape, np.uint8), fields, precision="fp32")
    o.step(6000)
    g.step(6000)
    fo, fg = o.fields(), g.fields()
    assert rel_l2(fo["rho"], fg["rho"]) < 1e-6
    assert rel_l2(fo["u"], fg["u"]) < 1e-4


@pytest.mark.parametrize("dim,steps", [(2, 61), (2, 60), (3, 47)])
def test_temperature_dependent_reaction_with_heat(dim, steps):
    """Sec. 2.1.5: rate k(T_b) = A exp(-Ta / T_b) at each reactive link's interface temperature,
    reaction heat into the temperature scalar, C_b - T_b solved per link.  2D: BGK with open
    faces for both scalars; 3D: MRT with closed walls and dissolution flips (new nodes take the
    neighbours' closed species and temperature)."""
    if dim == 2:
        shape = (1, 14, 18)
        cfg = dict(dim=2, nx=18, ny=14, tau=[0.8], g=[2e-4, 0, 0], n_scal=2, tau_c=[0.7, 0.9], J0=0.4,
                   arrhenius=True, arr_A=0.4, arr_Ta=1.0, heat_release=0.02, n_it=24,
                   ade_open_x=True, C_in=[1.0, 0.6], periodic=[1, 1, 1])
    else:
        shape = (8, 10, 12)
        cfg = dict(dim=3, nx=12, ny=10, nz=8, tau=[0.9], collision="mrt", g=[1e-4, 0, 0], n_scal=2,
                   tau_c=[0.6, 0.8], J0=0.25, arrhenius=True, arr_A=0.3, arr_Ta=0.8, heat_release=0.03,
                   n_it=24, periodic=[1, 0, 1], geo_mode="dissolve", V_m=40.0, m_s0=1.0)
    geom = inputs.random_solids(shape, 0.18, seed=60 + dim, reactive_fraction=0.7)
    rho, u, C = inputs.perturbed_fields(shape, 1, 2, seed=61, amp_rho=0.01, amp_u=0.01, C0=0.9)
    o, g = make_pair(cfg, geom, (rho, u, C))
    o.step(steps)
    g.step(steps)
    compare(o, g, what=f"thermal reaction {dim}d")
    if dim == 3:
        assert o.monitors()["inj_mass0"] > 0, "no dissolution flip happened"


def test_temperature_dependent_reaction_fp32():
    """The FP32 kernel variant of the coupled closure (single-precision exponential and
    iteration) against the FP64 oracle after 200 steps."""
    shape = (1, 14, 18)
    cfg = dict(dim=2, nx=18, ny=14, tau=[0.8], g=[2e-4, 0, 0], n_scal=2, tau_c=[0.7, 0.9], J0=0.4,
               arrhenius=True, arr_A=0.4, arr_Ta=1.0, heat_release=0.02, n_it=24,
               ade_open_x=True, C_in=[1.0, 0.6], periodic=[1, 1, 1])
    geom = inputs.random_solids(shape, 0.18, seed=62, reactive_fraction=0.7)
    rho, u, C = inputs.perturbed_fields(shape, 1, 2, seed=61, amp_rho=0.01, amp_u=0.01, C0=0.9)
    o, g = make_pair(cfg, geom, (rho, u, C), precision="fp32")
    o.step(200)
    g.step(200)
    fo, fg = o.fields(), g.fields()
    for k, tol in (("rho", 1e-6), ("u", 1e-4), ("C", 1e-5), ("acc", 1e-5)):
        e = rel_l2(fo[k], fg[k])
        assert e < tol, (k, e)
    mo, mg = o.monitors(), g.monitors()
    assert abs(mg["heat"] - mo["heat"]) < 1e-4 * abs(mo["heat"])
