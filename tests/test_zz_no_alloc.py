"""lbm_get_pops_noalloc: the populations read back through a fixed device scratch array, for
callers that cannot allocate device memory (their memory is fully reserved by another
allocator, or they must not trigger the device-wide synchronisation of cudaMalloc / cudaFree).
Its output must equal lbm_get_pops on consecutive calls, and domains too large for the fixed
16 MiB array must be rejected.  This file is collected last on purpose."""
import numpy as np
import pytest

from paper_2502_12955_gb300 import inputs
from paper_2502_12955_gb300.lbm import LbmError, Solver

pytestmark = pytest.mark.gpu


def _solver(shape, precision):
    cfg, geom, fields = inputs.dissolution_3d(shape=shape, g=5e-4, radius=(2.0, 4.0))
    cfg.update(precision=precision, k_react=0.05)
    s = Solver(cfg)
    s.set_geometry(geom)
    s.set_fields(*fields)
    return s


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16"])
def test_noalloc_matches_allocating_read_on_consecutive_calls(precision):
    s = _solver((10, 12, 16), precision)
    for steps in (3, 8):                      # odd then even layout parity
        s.step(steps)
        f_ref, h_ref = s.pops()
        f_na, h_na = s.pops_noalloc()
        np.testing.assert_array_equal(f_na, f_ref)
        np.testing.assert_array_equal(h_na, h_ref)
    s.close()


def test_noalloc_two_contexts_in_a_row():
    a = _solver((8, 9, 11), "fp32")
    b = _solver((9, 10, 12), "fp64")
    a.step(5)
    b.step(4)
    for s in (a, b, a):
        f_ref, h_ref = s.pops()
        f_na, h_na = s.pops_noalloc()
        np.testing.assert_array_equal(f_na, f_ref)
        np.testing.assert_array_equal(h_na, h_ref)


def test_noalloc_rejects_domains_beyond_the_scratch():
    s = _solver((40, 40, 40), "fp32")     # 64000 nodes x 26 x 8 B = 13.3 MB fits
    s.pops_noalloc()
    big = _solver((48, 48, 48), "fp32")   # 110592 nodes x 26 x 8 B = 23 MB does not
    with pytest.raises(LbmError) as e:
        big.pops_noalloc()
    assert e.value.status == -7
