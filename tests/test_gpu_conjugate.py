"""Heat conduction in the solid on the GPU against the FP64 oracle (Sec. 2.1.5, Eq. therpop_solid,
macroreacb_solid, tempCon, fluxCon, reacRate): the solid thermal lattice, the per-link exchange
with the fluid temperature at T_b = (c_fs ho + go + c_fs Qp / 2) / (w (c_fs + 1)), the species
closure with the exchange's k(T_b), and the reaction product on top.  Every field (the solid
temperature in row 1 at solid nodes included), population array and monitor (tsolid, heat,
heat_s, heat_src, solid_rem) within 1e-10, flags exact, at both layout parities."""
import numpy as np
import pytest

from paper_2502_12955_gb300 import inputs
from paper_2502_12955_gb300.lbm import Solver
from tests.gpu_common import compare, make_pair, rel_l2

pytestmark = pytest.mark.gpu


def _fields(shape, n_lat, seed, C0=0.9, T_solid=None):
    rho, u, C = inputs.perturbed_fields(shape, 1, n_lat, seed=seed, amp_rho=0.01, amp_u=0.01, C0=C0)
    if T_solid is not None:
        C[1] = T_solid + 0.05 * np.sin(np.arange(C[1].size).reshape(C[1].shape) * 0.37)
    return rho, u, C


WALLS_2D = dict(dim=2, nx=18, ny=14, tau=[0.8], g=[2e-4, 0, 0], n_scal=2, tau_c=[0.7, 0.9], J0=0.4,
                arrhenius=True, arr_A=0.4, arr_Ta=1.0, heat_release=0.05, n_it=40, conjugate=True,
                tau_s=0.65, c_fs=2.5, periodic=[1, 0, 1])


@pytest.mark.parametrize("steps", [7, 40])
def test_conjugate_2d_closed_walls(steps):
    """D2Q9 + two D2Q5 scalars, closed y faces (the solid reflects there), inert and reactive
    discs of random solid nodes, a solid starting hotter than the fluid."""
    shape = (1, 14, 18)
    geom = inputs.random_solids(shape, 0.22, seed=80, reactive_fraction=0.6)
    o, g = make_pair(WALLS_2D, geom, _fields(shape, 2, 81, T_solid=1.3))
    o.step(steps)
    g.step(steps)
    compare(o, g, what=f"conjugate 2d walls {steps}")
    m = o.monitors()
    assert m["heat_src"] > 0 and m["heat_s"] != 0 and m["tsolid"] > 0


@pytest.mark.parametrize("steps", [6, 33])
def test_conjugate_2d_open_faces(steps):
    """Inlet / outlet on the scalars' x faces: solid nodes on those faces reflect."""
    shape = (1, 12, 20)
    geom = inputs.random_solids(shape, 0.2, seed=82, reactive_fraction=0.7)
    cfg = dict(dim=2, nx=20, ny=12, tau=[0.9], g=[1e-4, 0, 0], n_scal=2, tau_c=[0.8, 0.7], J0=0.4,
               arrhenius=True, arr_A=0.3, arr_Ta=0.6, heat_release=0.04, n_it=40, conjugate=True,
               tau_s=1.1, c_fs=0.7, ade_open_x=True, C_in=[1.0, 0.9], periodic=[1, 1, 1])
    o, g = make_pair(cfg, geom, _fields(shape, 2, 83, T_solid=0.8))
    o.step(steps)
    g.step(steps)
    compare(o, g, what=f"conjugate 2d open {steps}")


@pytest.mark.parametrize("steps", [10, 31])
def test_conjugate_3d_mrt(steps):
    """D3Q19 MRT + two D3Q7 scalars with conduction in the solid, y walls closed."""
    shape = (9, 11, 13)
    geom = inputs.random_solids(shape, 0.2, seed=84, reactive_fraction=0.6)
    cfg = dict(dim=3, nx=13, ny=11, nz=9, tau=[1.0], collision="mrt", g=[1e-4, 0, 0], n_scal=2,
               tau_c=[0.6, 0.8], J0=0.25, arrhenius=True, arr_A=0.3, arr_Ta=0.8, heat_release=0.03,
               n_it=40, conjugate=True, tau_s=0.7, c_fs=0.6, periodic=[1, 0, 1])
    o, g = make_pair(cfg, geom, _fields(shape, 2, 85, T_solid=1.2))
    o.step(steps)
    g.step(steps)
    compare(o, g, what=f"conjugate 3d mrt {steps}")


@pytest.mark.parametrize("steps", [60, 61])
def test_conjugate_3d_with_dissolution(steps):
    """Dissolution with conduction in the solid: a dissolved node keeps its own temperature (its
    solid populations leave the solid lattice, monitor solid_rem) and its new reactive links
    start from the heat-capacity-weighted mean temperature."""
    shape = (8, 10, 12)
    geom = inputs.random_solids(shape, 0.25, seed=86, reactive_fraction=0.8)
    cfg = dict(dim=3, nx=12, ny=10, nz=8, tau=[1.0], collision="mrt", g=[1e-4, 0, 0], n_scal=2,
               tau_c=[0.6, 0.8], J0=0.25, arrhenius=True, arr_A=0.3, arr_Ta=0.8, heat_release=0.03,
               n_it=40, conjugate=True, tau_s=0.7, c_fs=0.6, geo_mode="dissolve", V_m=40.0, N_geo=2,
               periodic=[1, 1, 1])
    o, g = make_pair(cfg, geom, _fields(shape, 2, 87, T_solid=1.1))
    o.step(steps)
    g.step(steps)
    m = o.monitors()
    assert m["solid_rem"] != 0.0, "the case should dissolve solids"
    compare(o, g, what=f"conjugate dissolution {steps}")


@pytest.mark.parametrize("dim,steps", [(2, 41), (3, 30)])
def test_conjugate_with_product(dim, steps):
    """Three scalar lattices with conduction in the solid: species, temperature, product."""
    if dim == 2:
        shape = (1, 14, 18)
        cfg = dict(WALLS_2D, product=True, tau_p=1.2)
    else:
        shape = (8, 10, 12)
        cfg = dict(dim=3, nx=12, ny=10, nz=8, tau=[0.9], g=[1e-4, 0, 1e-4], n_scal=2, tau_c=[0.7, 0.6],
                   J0=0.25, arrhenius=True, arr_A=0.5, arr_Ta=0.7, heat_release=0.08, n_it=40,
                   conjugate=True, tau_s=0.9, c_fs=1.7, product=True, tau_p=0.65, ade_open_x=True,
                   C_in=[1.0, 1.1], C_in_p=0.05, periodic=[1, 0, 1])
    geom = inputs.random_solids(shape, 0.2, seed=88 + dim, reactive_fraction=0.7)
    o, g = make_pair(cfg, geom, _fields(shape, 3, 89, T_solid=1.15))
    o.step(steps)
    g.step(steps)
    compare(o, g, what=f"conjugate product {dim}d")
    assert o.monitors()["produced"] > 0


def test_burning_channel():
    """The reactive porous channel recipe (Sec. 3.4 stand-in) at 90 x 24: velocity inlet,
    zero-gradient outlets, O2 / T / CO2, conduction in the carbon discs, 300 steps."""
    cfg, geom, fields = inputs.combustion_channel_2d(nx=90, ny=24, n_obstacles=3, precision="fp64")
    o, g = make_pair(cfg, geom, fields)
    for target in (1, 150, 300):
        done = int(o.monitors()["step"])
        o.step(target - done)
        g.step(target - done)
        compare(o, g, what=f"burning channel step {target}")
    m = o.monitors()
    assert m["produced"] > 0 and m["heat_src"] > 0


def test_burning_channel_with_dissolution():
    """The same channel small enough to burn through: discs dissolve under the exchange's
    heat release."""
    shape = (1, 8, 8)
    geom = np.zeros(shape, dtype=np.uint8)
    geom[0, 3:5, 3:5] = inputs.REACTIVE
    cfg = dict(dim=2, nx=8, ny=8, tau=[0.8], flow_open_x=True, u_in=0.03, n_scal=2, tau_c=[0.8, 0.9], J0=0.4,
               ade_open_x=True, C_in=[0.22, 1.0], arrhenius=True, arr_A=2.0, arr_Ta=1.5, heat_release=0.5,
               n_it=40, conjugate=True, tau_s=0.7, c_fs=0.5, product=True, tau_p=0.75, C_in_p=0.0,
               geo_mode="dissolve", V_m=200.0, periodic=[0, 0, 1])
    rho, u, _ = inputs.uniform_fields(shape, 1, 0)
    C = np.zeros((3,) + shape)
    C[0] = 0.22
    C[1] = 1.0
    o, g = make_pair(cfg, geom, (rho, u, C))
    for target in (40, 121):
        done = int(o.monitors()["step"])
        o.step(target - done)
        g.step(target - done)
        compare(o, g, what=f"small burning channel {target}")
    assert o.monitors()["solid_rem"] != 0.0, "a disc node should burn away"


# relative L2 bounds of the storage modes on the closed-wall case after 200 steps: FP32 round-off;
# 16-bit flow storage of deviations (2^-11 of the O(1e-2) deviations per step); FP16 scalars round
# the O(1) temperature and species deviations at 2^-11 every step
STORAGE_BOUND = {"fp32": 1e-5, "fp16s32": 2e-3, "fp16": 1e-2}


@pytest.mark.parametrize("precision", ["fp32", "fp16s32", "fp16"])
def test_conjugate_storage_modes_track_fp64(precision):
    """The closed-wall case in the reduced storage modes against the oracle over 200 steps (the
    solid lattice is held in the compute type, FP32)."""
    shape = (1, 14, 18)
    geom = inputs.random_solids(shape, 0.22, seed=80, reactive_fraction=0.6)
    o, g = make_pair(WALLS_2D, geom, _fields(shape, 2, 81, T_solid=1.3), precision=precision)
    o.step(200)
    g.step(200)
    fo, fg = o.fields(), g.fields()
    errs = {k: rel_l2(fo[k], fg[k]) for k in ("rho", "u", "C", "acc")}
    print(precision, {k: f"{v:.2e}" for k, v in errs.items()})
    for k, v in errs.items():
        assert v <= STORAGE_BOUND[precision], (k, v)
    assert abs(g.monitors()["tsolid"] - o.monitors()["tsolid"]) <= STORAGE_BOUND[precision] * abs(o.monitors()["tsolid"])


def test_conjugate_checkpoint_resume_is_bitwise():
    """The checkpoint carries the solid thermal lattice (both copies), the exchange's rate
    constants and the heat monitors: resuming reproduces the uninterrupted run bit for bit, at
    both layout parities."""
    shape = (1, 14, 18)
    geom = inputs.random_solids(shape, 0.22, seed=80, reactive_fraction=0.6)
    s = Solver(dict(WALLS_2D, precision="fp32", product=True, tau_p=1.2))
    s.set_geometry(geom)
    s.set_fields(*_fields(shape, 3, 81, T_solid=1.3))
    for first in (30, 2):   # checkpoints at steps 30 and 53
        s.step(first)
        blob = s.get_state()
        s.step(21)
        fa, ma = s.fields(), s.monitors()
        s.set_state(blob)
        s.step(21)
        fb, mb = s.fields(), s.monitors()
        for k in fa:
            assert np.array_equal(fa[k], fb[k]), (first, k)
        for k in ("tsolid", "heat", "heat_s", "heat_src", "produced", "wallx"):
            assert ma[k] == mb[k], (first, k)
    s.close()


def test_conjugate_sphere_packing_400_steps():
    """A 32^3 sphere packing of the dissolution recipe with the temperature-dependent rate, heat
    release and conduction in the solid, MRT, dissolving (V_m = 1: 40 % of the solid nodes turn
    fluid within the 400 steps): every field, population and monitor at steps 200 and 400."""
    cfg, geom, (rho, u, C) = inputs.dissolution_3d(shape=(32, 32, 32), g=2e-4, radius=(3.0, 6.0), precision="fp64")
    cfg.update(n_scal=2, tau_c=[0.6, 0.8], C_in=[1.0, 1.0], C_ref=[1.0, 1.0], arrhenius=True, arr_A=0.3,
               arr_Ta=0.8, heat_release=0.03, n_it=24, conjugate=True, tau_s=0.7, c_fs=0.6, V_m=1.0)
    T = np.ones_like(C) + 0.1 * (geom[None] != 0)
    o, g = make_pair(cfg, geom, (rho, u, np.concatenate([C, T])))
    done = 0
    for target in (200, 400):
        o.step(target - done)
        g.step(target - done)
        done = target
        compare(o, g, what=f"conjugate packing step {target}")
    m = o.monitors()
    assert m["heat_src"] > 0 and m["tsolid"] > 0
