"""Shared helpers of the GPU parity tests: run the CUDA path (through the C ABI) and the
FP64 oracle on identical seeded inputs and compare them element by element."""
import numpy as np

from oracle.oracle import Oracle
from paper_2502_12955_gb300.lbm import Solver

FP64_TOL = 1e-10   # relative L2 per field for the FP64 path after the stated steps


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    na = np.linalg.norm(a)
    d = np.linalg.norm(a - b)
    return d / na if na > 0 else d


def make_pair(cfg, geom, fields, precision="fp64"):
    o = Oracle(cfg)
    g = Solver(dict(cfg, precision=precision))
    for s in (o, g):
        s.set_geometry(geom)
        rho, u, C = fields
        s.set_fields(rho, u, C if s.p.n_scal else None)
    return o, g


def compare(o, g, tol=FP64_TOL, pops=True, mon=True, flags_exact=True, what=""):
    g.sync()   # raises if a kernel set a device error flag (capacity, retry limit, bounds)
    fo, fg = o.fields(), g.fields()
    report = {}
    if flags_exact:
        bad = np.argwhere(fo["flags"] != fg["flags"])
        assert bad.size == 0, f"{what}: flags differ at {bad[:5].tolist()}"
    for k in ("rho", "u", "C", "acc"):
        e = rel_l2(fo[k], fg[k])
        report[k] = e
        assert e <= tol, f"{what}: field {k} rel L2 {e:.3e} > {tol:.1e}"
    if pops:
        (f_o, h_o), (f_g, h_g) = o.pops(), g.pops()
        e = rel_l2(f_o, f_g)
        report["f"] = e
        assert e <= tol, f"{what}: populations f rel L2 {e:.3e}"
        if o.p.n_scal:
            e = rel_l2(h_o, h_g)
            report["h"] = e
            assert e <= tol, f"{what}: populations h rel L2 {e:.3e}"
    if mon:
        mo, mg = o.monitors(), g.monitors()
        scale = max(1.0, abs(mo["mass0"]))
        for k, v in mo.items():
            if k not in mg:
                # oracle-only monitors (features the CUDA path does not have) must be idle
                assert v == 0.0, f"{what}: monitor {k} = {v!r} has no CUDA counterpart"
                continue
            if k in ("step",):
                assert mg[k] == v
                continue
            assert abs(mg[k] - v) <= tol * max(abs(v), scale) * 10, \
                f"{what}: monitor {k}: gpu {mg[k]!r} oracle {v!r}"
    return report
