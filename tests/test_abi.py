"""Host-side checks of the C ABI (no GPU needed): the library loads, exports every entry point
include/lbm.h declares, the ctypes mirrors match the C layouts, and invalid arguments are
rejected before any CUDA call."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2502_12955_gb300 import lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "include", "lbm.h")


def declared_functions():
    text = open(HDR).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_]+)\s*\(", text)))


NN_HDR = os.path.join(ROOT, "include", "lbm_nn.h")


def declared_nn_functions():
    text = open(NN_HDR).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_nn_[a-z0-9_]+)\s*\(", text)))


def test_network_library_exports_every_declared_symbol():
    """include/lbm_nn.h: every declared call is exported by liblbm.so and bound by the Python
    binding under the same name."""
    from paper_2502_12955_gb300 import surrogate

    names = declared_nn_functions()
    assert len(names) >= 18
    lib = surrogate.nn_lib()
    nm = subprocess.run(["nm", "-D", "--defined-only", lbm.library_path()], capture_output=True,
                        text=True).stdout
    for name in names:
        assert hasattr(lib, name), name
        assert hasattr(surrogate, name), f"{name} has no binding"
        assert re.search(rf"\bT {name}$", nm, re.M), f"{name} not exported"


def test_library_exports_every_declared_symbol():
    lib = lbm.load()
    names = declared_functions()
    assert set(names) == set(lbm.EXPORTS)
    for name in names:
        assert hasattr(lib, name), name
    nm = subprocess.run(["nm", "-D", "--defined-only", lbm.library_path()], capture_output=True,
                        text=True).stdout
    for name in names:
        assert re.search(rf"\bT {name}$", nm, re.M), f"{name} not exported"


def _c_layout(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "lbm.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(lbm_params),
         offsetof(lbm_params, l2_fetch_bytes), offsetof(lbm_params, u_wall_ymax), offsetof(lbm_params, u_in),
         offsetof(lbm_params, stream),
         offsetof(lbm_params, N_mon), offsetof(lbm_params, C_ref), sizeof(lbm_monitors),
         offsetof(lbm_monitors, wall_exchange), offsetof(lbm_monitors, residual),
         offsetof(lbm_params, product), offsetof(lbm_params, C_in_p), offsetof(lbm_monitors, produced),
         offsetof(lbm_params, conjugate), offsetof(lbm_params, c_fs), offsetof(lbm_monitors, t_solid),
         offsetof(lbm_monitors, solid_removed));
  return 0;
}
''')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.dirname(HDR), str(src), "-o", str(exe)], check=True)
    return [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]


def test_ctypes_layout_matches_c(tmp_path):
    c = _c_layout(tmp_path)
    P, M = lbm.LbmParams, lbm.LbmMonitors
    assert c == [C.sizeof(P), P.l2_fetch_bytes.offset, P.u_wall_ymax.offset, P.u_in.offset, P.stream.offset, P.N_mon.offset, P.C_ref.offset, C.sizeof(M),
                 M.wall_exchange.offset, M.residual.offset, P.product.offset, P.C_in_p.offset, M.produced.offset,
                 P.conjugate.offset, P.c_fs.offset, M.t_solid.offset, M.solid_removed.offset]


def test_params_default():
    lib = lbm.load()
    p = lbm.LbmParams()
    assert lib.lbm_params_default(C.byref(p)) == 0
    assert p.precision == 1 and p.n_comp == 1 and p.tau[0] == 1.0 and p.N_geo == 1
    assert list(p.periodic) == [1, 1, 1] and p.deposit_conservative == 1
    assert p.n_it == 16 and p.arrhenius == 0
    assert p.conjugate == 0 and p.tau_s == 1.0 and p.c_fs == 1.0 and p.tau_p == 1.0


@pytest.mark.parametrize("bad", [
    dict(tau=[0.5]), dict(n_comp=3), dict(n_scal=3), dict(collision="mrt", n_comp=2, tau=[1, 1]),
    dict(collision="mrt", forcing="sc_shift"), dict(N_geo=0), dict(block_x=48),
    dict(n_scal=1, tau_c=[0.4]), dict(geo_mode="dissolve", n_scal=0), dict(J0=1.0, n_scal=1),
    dict(product=True, n_scal=0), dict(product=True, n_scal=1, tau_p=0.5),
    dict(product=True, n_scal=1, geo_mode="deposit", DP=0.1),
    dict(l2_fetch_bytes=48), dict(u_wall_ymax=[0.01, 0, 0]), dict(u_wall_ymax=[0, 0.01, 0], periodic=[1, 0, 1]),
    dict(flow_open_x=True, u_in=0.01), dict(flow_open_x=True, periodic=[0, 1, 1]),
    dict(flow_open_x=True, periodic=[0, 0, 1], n_comp=2, tau=[1, 1]),
    dict(flow_open_x=True, periodic=[0, 0, 1], G=[[-5, 0], [0, 0]]),
    dict(flow_open_x=True, periodic=[0, 0, 1], G_ads=[0.1, 0]),
    dict(arrhenius=True, n_scal=1, arr_A=0.1), dict(arrhenius=True, n_scal=2, arr_A=-0.1),
    dict(arrhenius=True, n_scal=2, arr_A=0.1, n_it=65),
    dict(conjugate=True, n_scal=2, tau_s=0.8), dict(conjugate=True, n_scal=2, arrhenius=True, tau_s=0.5),
    dict(conjugate=True, n_scal=2, arrhenius=True, c_fs=0.0),
    dict(conjugate=True, n_scal=2, arrhenius=True, geo_mode="deposit", DP=0.1),
])
def test_create_rejects_invalid_parameters(bad):
    lib = lbm.load()
    cfg = dict(dim=2, nx=8, ny=8, precision="fp64")
    cfg.update(bad)
    p = lbm.make_params(cfg, lib)
    h = C.c_void_p()
    st = lib.lbm_create(lbm.LBM_D2Q9_D2Q5, 8, 8, 1, C.byref(p), C.byref(h))
    assert st == -1 and not h.value
    assert lib.lbm_last_error(None)


def test_create_rejects_bad_shapes():
    lib = lbm.load()
    p = lbm.make_params(dict(dim=2, nx=8, ny=8), lib)
    h = C.c_void_p()
    assert lib.lbm_create(lbm.LBM_D2Q9_D2Q5, 8, 8, 2, C.byref(p), C.byref(h)) == -1
    assert lib.lbm_create(lbm.LBM_D3Q19_D3Q7, 0, 8, 8, C.byref(p), C.byref(h)) == -1
    assert lib.lbm_create(7, 8, 8, 1, C.byref(p), C.byref(h)) == -1


def test_null_context_calls_fail_cleanly():
    lib = lbm.load()
    assert lib.lbm_step(None, 1) == -1
    assert lib.lbm_sync(None) == -1
    m = lbm.LbmMonitors()
    assert lib.lbm_get_monitors(None, C.byref(m)) == -1
    lib.lbm_destroy(None)


@pytest.mark.parametrize("bad", [dict(precision="fp16"), dict(geo_mode="dissolve", n_scal=1),
                                 dict(G=[[-5.0, 0], [0, 0]]), dict(forcing="sc_shift"), dict(collision="mrt")])
def test_ensemble_create_rejects_mixed_or_unsupported_members(bad):
    lib = lbm.load()
    base = dict(dim=2, nx=8, ny=8, precision="fp32")
    ps = (lbm.LbmParams * 2)()
    ps[0] = lbm.make_params(base, lib)
    ps[1] = lbm.make_params(dict(base, **bad), lib)
    dims = (C.c_int32 * 6)(8, 8, 1, 8, 8, 1)
    h = C.c_void_p()
    assert lib.lbm_ensemble_create(lbm.LBM_D2Q9_D2Q5, 2, dims, ps, C.byref(h)) == -1 and not h.value
    assert b"member 1" in lib.lbm_ensemble_last_error(None)
    assert lib.lbm_ensemble_create(lbm.LBM_D2Q9_D2Q5, 0, dims, ps, C.byref(h)) == -1


def test_save_fields_round_trip(tmp_path):
    """Fields are exported as arrays for offline plotting (no graphics stack)."""
    rng = np.random.default_rng(3)
    fields = {"rho": rng.uniform(size=(1, 1, 4, 5)), "u": rng.uniform(size=(3, 1, 4, 5)),
              "C": rng.uniform(size=(1, 1, 4, 5)), "flags": rng.integers(0, 3, size=(1, 4, 5)).astype(np.uint8),
              "acc": np.zeros((1, 4, 5))}
    path = lbm.save_fields(fields, tmp_path / "state")
    back = np.load(path)
    for k, v in fields.items():
        assert np.array_equal(back[k], v) and back[k].dtype == v.dtype


def test_missing_library_fails_loudly(tmp_path):
    """Without the CUDA library there is no fallback: loading it, and so constructing a
    Solver, raises."""
    import subprocess
    import sys
    code = ("import sys\n"
            "from paper_2502_12955_gb300 import lbm\n"
            "try:\n"
            "    lbm.Solver(dict(dim=2, nx=8, ny=8))\n"
            "except RuntimeError as e:\n"
            "    print('raised:', e)\n"
            "    sys.exit(0)\n"
            "sys.exit(1)\n")
    env = dict(os.environ, LBM_LIBRARY=str(tmp_path / "absent" / "liblbm.so"))
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", code], cwd=root, env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "not found" in r.stdout


@pytest.mark.parametrize("extra", [dict(conjugate=True), dict(product=True)])
def test_ensemble_rejects_conduction_in_the_solid_and_the_product(extra):
    lib = lbm.load()
    base = dict(dim=2, nx=8, ny=8, precision="fp32", n_scal=2, tau_c=[0.7, 0.8], arrhenius=True, arr_A=0.1)
    ps = (lbm.LbmParams * 2)()
    ps[0] = lbm.make_params(base, lib)
    ps[1] = lbm.make_params(dict(base, **extra), lib)
    dims = (C.c_int32 * 6)(8, 8, 1, 8, 8, 1)
    h = C.c_void_p()
    assert lib.lbm_ensemble_create(lbm.LBM_D2Q9_D2Q5, 2, dims, ps, C.byref(h)) == -1 and not h.value
    msg = lib.lbm_ensemble_last_error(None)
    assert b"member 1" in msg and (b"solid" in msg or b"product" in msg), msg
