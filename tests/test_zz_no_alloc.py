"""lbm_get_pops_noalloc: the populations read back through a fixed device scratch array, for
callers that cannot allocate device memory (their memory is fully reserved by another
allocator, or they must not trigger the device-wide synchronisation of cudaMalloc / cudaFree).
Its output must equal lbm_get_pops on consecutive calls, for every combination of flow
components, scalars and requested outputs that changes the size and offset arithmetic of the
staging, and requests too large for the fixed 16 MiB array must be rejected without harming
the context.

The file name sorts last so that a run stopping at its first failure has already run every
other test: the entry point is an extra, and a failure here must not hide one in the step."""
import numpy as np
import pytest

from paper_2502_12955_gb300 import inputs
from paper_2502_12955_gb300.lbm import LbmError, Solver

pytestmark = pytest.mark.gpu


def _solver(shape, precision, n_scal=1):
    cfg, geom, fields = inputs.dissolution_3d(shape=shape, g=5e-4, radius=(2.0, 4.0))
    cfg.update(precision=precision, k_react=0.05)
    rho, u, C = fields
    if n_scal != 1:
        cfg.update(n_scal=n_scal, tau_c=[0.5667, 0.8][:max(n_scal, 1)], C_in=[1.0, 0.5][:max(n_scal, 1)],
                   C_ref=[1.0, 0.5][:max(n_scal, 1)])
        if n_scal == 0:
            cfg.update(geo_mode="none", ade_open_x=False)
        C = np.concatenate([C, 0.5 * np.ones_like(C)])[:n_scal]
    s = Solver(cfg)
    s.set_geometry(geom)
    s.set_fields(rho, u, C if n_scal else None)
    return s


def _droplet(precision):
    n = 12
    cfg, geom, _ = inputs.droplet_3d(n=n, radius=3.5, precision=precision)
    rho, u = inputs.droplet_fields((n, n, n), 3.5)
    s = Solver(cfg)
    s.set_geometry(geom)
    s.set_fields(rho, u, None)
    return s


def _same_as_allocating_read(s):
    f_ref, h_ref = s.pops()
    f_na, h_na = s.pops_noalloc()
    np.testing.assert_array_equal(f_na, f_ref)
    np.testing.assert_array_equal(h_na, h_ref)
    # one output at a time: the other pointer is NULL and stages nothing
    f_only, h_none = s.pops_noalloc(want_h=False)
    assert h_none is None
    np.testing.assert_array_equal(f_only, f_ref)
    f_none, h_only = s.pops_noalloc(want_f=False)
    assert f_none is None
    np.testing.assert_array_equal(h_only, h_ref)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16", "fp16s32"])
def test_noalloc_matches_allocating_read_on_consecutive_calls(precision):
    s = _solver((10, 12, 16), precision)
    for steps in (3, 8):                      # odd then even layout parity
        s.step(steps)
        _same_as_allocating_read(s)
    s.close()


@pytest.mark.parametrize("n_scal", [0, 2])
def test_noalloc_scalar_counts(n_scal):
    s = _solver((9, 10, 13), "fp32", n_scal=n_scal)
    for steps in (5, 2):
        s.step(steps)
        _same_as_allocating_read(s)
    s.close()


def test_noalloc_two_components():
    s = _droplet("fp64")
    for steps in (7, 4):
        s.step(steps)
        _same_as_allocating_read(s)
    s.close()


def test_noalloc_two_contexts_in_a_row():
    a = _solver((8, 9, 11), "fp32")
    b = _solver((9, 10, 12), "fp64")
    a.step(5)
    b.step(4)
    for s in (a, b, a):
        _same_as_allocating_read(s)


def test_noalloc_rejects_requests_beyond_the_scratch():
    s = _solver((40, 40, 40), "fp32")     # 64000 nodes x 26 x 8 B = 13.3 MB fits
    s.pops_noalloc()
    big = _solver((48, 48, 48), "fp32")   # 110592 nodes x 26 x 8 B = 23 MB does not
    with pytest.raises(LbmError) as e:
        big.pops_noalloc()
    assert e.value.status == -7
    # the flow populations alone (110592 x 19 x 8 B = 16.8 MB) still do not fit; the scalar
    # ones alone (6.2 MB) do, and the rejected calls left the context usable
    with pytest.raises(LbmError):
        big.pops_noalloc(want_h=False)
    _, h_ref = big.pops()
    _, h_na = big.pops_noalloc(want_f=False)
    np.testing.assert_array_equal(h_na, h_ref)
    big.step(2)
    big.sync()
