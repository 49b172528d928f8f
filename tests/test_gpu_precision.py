"""Storage precision on the dissolution workload's recipe (64^3 sphere packing, D3Q19 MRT +
D3Q7, transport numbers of the 256^3 case, geometry held fixed): FP32, FP16 and BF16 storage
against the FP64 path (itself within 1e-10 of the oracle) after 500 steps, per field.  The
bounds are the stated tolerance of 16-bit storage, 1e-3 relative L2 per field, for FP16 and the
FP16 flow modes; ten times that for BF16 (8 bits of mantissa against FP16's 11, 8x coarser);
and 1e-5 for FP32 (13 bits finer than FP16).  The same rule bounds the oracle comparisons of the
long runs.  FP16 stays within 1e-3 on every field; BF16 does not on u."""
import numpy as np
import pytest

from paper_2502_12955_gb300 import inputs
from paper_2502_12955_gb300.lbm import Solver
from tests.gpu_common import rel_l2

pytestmark = pytest.mark.gpu

# relative L2 of the full fields over the fluid nodes (measured: FP32 2.8e-8 / 5.7e-7 / 8.7e-8,
# FP16 2.4e-6 / 3.9e-4 / 8.1e-5, BF16 1.6e-5 / 2.9e-3 / 8.0e-4 for rho / u / C)
BOUND = {"fp32": dict.fromkeys(("rho", "u", "C"), 1e-5),
         "fp16": dict.fromkeys(("rho", "u", "C"), 1e-3),
         "bf16": dict.fromkeys(("rho", "u", "C"), 1e-2)}
# mixed storage (16-bit flow, FP32 scalars): the bounds of its flow format
BOUND["fp16s32"] = dict(BOUND["fp16"])
BOUND["bf16s32"] = dict(BOUND["bf16"])


@pytest.fixture(scope="module")
def fp64_reference():
    cfg, geom, fields = inputs.dissolution_3d(64, precision="fp64")
    cfg = dict(cfg, geo_mode="none")
    s = Solver(cfg)
    s.set_geometry(geom)
    s.set_fields(*fields)
    s.step(500)
    ref = s.fields()
    s.close()
    return cfg, geom, fields, ref


@pytest.mark.parametrize("precision", ["fp32", "fp16", "bf16", "fp16s32", "bf16s32"])
def test_storage_precision_errors_per_field(fp64_reference, precision):
    cfg, geom, fields, ref = fp64_reference
    s = Solver(dict(cfg, precision=precision))
    s.set_geometry(geom)
    s.set_fields(*fields)
    s.step(500)
    out = s.fields()
    s.close()
    fl = geom.reshape(-1) == 0
    errs = {}
    for k in ("rho", "u", "C"):
        a = ref[k].reshape(ref[k].shape[0], -1)[:, fl]
        b = out[k].reshape(out[k].shape[0], -1)[:, fl]
        errs[k] = rel_l2(a, b)
    print(precision, {k: f"{v:.2e}" for k, v in errs.items()})
    for k, v in errs.items():
        assert v <= BOUND[precision][k], f"{precision} {k}: {v:.3e}"
