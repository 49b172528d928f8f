"""lbm_get_fields_device: the macroscopic fields left in device memory (CUDA array interface
views from Solver.fields_device) equal the host read-back of lbm_get_fields element by element,
for one and two components, with and without scalars, at both layout parities."""
import numpy as np
import pytest

from paper_2502_12955_gb300 import inputs
from paper_2502_12955_gb300.lbm import Solver

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _check(s):
    host = s.fields()
    dev = s.fields_device()
    assert set(dev) == {k for k in host if host[k].size}
    for k, v in dev.items():
        t = torch.as_tensor(v, device="cuda")
        assert tuple(t.shape) == host[k].shape
        np.testing.assert_array_equal(t.cpu().numpy(), host[k])


@pytest.mark.parametrize("steps", [6, 7])
def test_device_fields_dissolution(steps):
    cfg, geom, fields = inputs.dissolution_3d(shape=(10, 12, 14), g=5e-4, radius=(2.0, 4.0), precision="fp32")
    s = Solver(cfg)
    s.set_geometry(geom)
    s.set_fields(*fields)
    s.step(steps)
    _check(s)
    s.close()


def test_device_fields_two_components_without_scalars():
    n = 12
    cfg, geom, _ = inputs.droplet_3d(n=n, radius=3.5, precision="fp64")
    rho, u = inputs.droplet_fields((n, n, n), 3.5)
    s = Solver(cfg)
    s.set_geometry(geom)
    s.set_fields(rho, u, None)
    s.step(5)
    _check(s)
    assert "C" not in s.fields_device()
    s.close()
