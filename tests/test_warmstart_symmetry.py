"""The y-z symmetric copies used to augment the warm-start training set are exact symmetries of the
method: the FP64 oracle run on a mirrored or transposed packing equals the mirrored or
transposed run of the original packing, with the velocity components mapped alike (D3Q19 MRT
flow driven along x, D3Q7 solute with the x inlet and outlet, periodic y and z).  Checked for all
eight maps on a small packing, and symmetric_copy applied to the original run reproduces the
mapped run's targets."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.oracle import Oracle  # noqa: E402
from paper_2502_12955_gb300 import inputs  # noqa: E402
from paper_2502_12955_gb300.warmstart import symmetric_copy  # noqa: E402


def _map_geom(g, k):
    if k & 1:
        g = g[:, ::-1, :]
    if k & 2:
        g = g[::-1, :, :]
    if k & 4:
        g = g.transpose(1, 0, 2)
    return np.ascontiguousarray(g)


def _run(geom, steps=25):
    shp = geom.shape
    cfg, _, fields = inputs.dissolution_3d(shape=shp, g=2e-4, radius=(1.0, 2.0), precision="fp64")
    cfg = dict(cfg, geo_mode="none", k_react=0.02)
    o = Oracle(cfg)
    o.set_geometry(geom)
    o.set_fields(*fields)
    o.step(steps)
    f = o.fields()
    t = np.empty(shp + (4,))
    for a in range(3):
        t[..., a] = f["u"][a]
    t[..., 3] = f["C"][0]
    return t


class _Sample:
    def __init__(self, geom, t):
        self.geom = geom
        self.x = torch.from_numpy((geom != 0).astype(np.float32).reshape(-1, 1))
        self.t = torch.from_numpy(t.reshape(-1, 4))
        self.fluid = torch.from_numpy((geom == 0).astype(np.uint8).reshape(-1))


def test_symmetric_copies_are_runs_of_the_mapped_packing():
    shp = (6, 6, 9)
    geom = inputs.random_solids(shp, 0.2, seed=5, reactive_fraction=0.6)
    t0 = _run(geom)
    s = _Sample(geom, t0)
    for k in range(8):
        gk = _map_geom(geom, k)
        tk = _run(gk)
        x, t, fl = symmetric_copy(s, k)
        assert np.array_equal(x.numpy().reshape(shp)[..., None].squeeze(-1), (gk != 0).astype(np.float32)), k
        assert np.array_equal(fl.numpy().reshape(shp), (gk == 0).astype(np.uint8)), k
        err = np.abs(t.numpy().reshape(shp + (4,)) - tk).max()
        assert err <= 1e-12 * max(1.0, np.abs(tk).max()), (k, err)
    assert np.abs(t0[..., 1]).max() > 1e-6 and np.abs(t0[..., 2]).max() > 1e-6, "transverse flow must be nonzero"
