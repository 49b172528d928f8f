"""Ensembles of uneven domains: the tile-list kernel must update every member exactly as the
single-domain path does (bitwise populations), match the FP64 oracle, stop converged members
and autotune its tile size."""
import numpy as np
import pytest

from paper_2502_12955_gb300 import inputs
from paper_2502_12955_gb300.lbm import Ensemble, Solver
from tests.gpu_common import FP64_TOL, compare, make_pair

pytestmark = pytest.mark.gpu


def _members_3d(precision):
    out = []
    for k, shape in enumerate([(11, 14, 20), (16, 16, 16), (9, 10, 24)]):
        cfg, geom, fields = inputs.dissolution_3d(shape=shape, g=5e-4 * (1 + k), radius=(2.0, 4.0), seed=k)
        cfg = dict(cfg, geo_mode="none", precision=precision, tau=[0.8 + 0.1 * k], N_mon=10)
        out.append((cfg, geom, fields))
    return out


def _load(s, geom, fields):
    s.set_geometry(geom)
    rho, u, C = fields
    s.set_fields(rho, u, C if s.n_scal else None)


@pytest.mark.parametrize("precision", ["fp32", "fp16", "fp64", "fp16s32"])
def test_ensemble_matches_single_domains_bitwise(precision):
    mem = _members_3d(precision)
    ens = Ensemble([c for c, _, _ in mem])
    singles = []
    for (cfg, geom, fields), m in zip(mem, ens.members):
        _load(m, geom, fields)
        s = Solver(cfg)
        _load(s, geom, fields)
        singles.append(s)
    ens.step(37)
    for s in singles:
        s.step(37)
    for k, (m, s) in enumerate(zip(ens.members, singles)):
        fm, hm = m.pops()
        fs, hs = s.pops()
        assert np.array_equal(fm, fs) and np.array_equal(hm, hs), f"member {k} differs"
        assert m.monitors()["step"] == 37
    ens.close()


def test_ensemble_2d_against_oracle():
    cfgs, data = [], []
    for k, (nx, ny) in enumerate([(48, 24), (37, 23), (64, 32)]):
        cfg, geom, fields = inputs.reactive_channel_2d(nx=nx, ny=ny, seed=10 + k)
        # body force large enough that u is not a difference of round-off (|u| ~ 1e-3)
        cfg = dict(cfg, precision="fp64", tau=[0.7 + 0.1 * k], k_react=0.02 * (k + 1), g=[5e-5 * (k + 1), 0, 0])
        cfgs.append(cfg)
        data.append((geom, fields))
    ens = Ensemble(cfgs)
    oracles = []
    for cfg, (geom, fields), m in zip(cfgs, data, ens.members):
        _load(m, geom, fields)
        o, _ = make_pair(cfg, geom, fields)
        oracles.append(o)
    ens.step(41)
    for o, m in zip(oracles, ens.members):
        o.step(41)
        compare(o, m, tol=FP64_TOL, what="ensemble 2d member")
    ens.close()


def test_run_to_steady_stops_members_and_autotune():
    cfgs, data = [], []
    for k, n in enumerate([12, 16, 20]):
        cfg, geom, fields = inputs.dissolution_3d(shape=(n, n, n), g=2e-4, radius=(2.0, 3.0), seed=20 + k)
        cfg = dict(cfg, geo_mode="none", precision="fp32", k_react=0.0, N_mon=50)
        cfgs.append(cfg)
        data.append((geom, fields))
    ens = Ensemble(cfgs)
    for (geom, fields), m in zip(data, ens.members):
        _load(m, geom, fields)
    t = ens.autotune(steps=4)
    assert t in (64, 128, 256)
    start = ens.members[0].monitors()["step"]
    steps, conv = ens.run_to_steady(1e-4, 20000)
    assert conv == len(cfgs), (steps, conv)
    done = [m.monitors()["step"] for m in ens.members]
    res = [m.monitors()["residual"] for m in ens.members]
    assert all(0 <= r <= 1e-4 for r in res), res
    # members stop at residual evaluations (multiples of N_mon); the last one ends the run
    assert all(d % 50 == 0 for d in done) and max(done) == start + steps
    assert ens.launch_count() > 0
    ens.close()
