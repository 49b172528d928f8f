"""ctypes wrapper of the FP64 CPU oracle (lbm_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
cpu_baseline / reference leg of bench.py.  The product path never imports it.

The oracle follows the paper's per-step update (CooLBM, arXiv 2502.12955,
Sec. 2.1-2.1.5 and Sec. 3.3); see lbm_oracle.c for the equation map.

Configuration keys are the fields of orc_params (lbm_oracle.h).  Scalar fields and
populations come as [n_scal + product] rows: the given scalars, then the CO2 product
lattice when `product` is set.  With `conjugate`, fields()["C"][1] holds the solid
temperature on solid nodes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    hdr = os.path.join(_HERE, "lbm_oracle.h")
    fresh = os.path.exists(_LIB) and os.path.getmtime(_LIB) >= max(
        os.path.getmtime(_SRC), os.path.getmtime(hdr))
    if fresh and not force:
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-Wall", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class OrcParams(C.Structure):
    _fields_ = [
        ("dim", C.c_int32), ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
        ("n_comp", C.c_int32), ("tau", C.c_double * 2), ("G", (C.c_double * 2) * 2),
        ("G_ads", C.c_double * 2), ("rho_solid", C.c_double), ("psi_kind", C.c_int32),
        ("rho0", C.c_double), ("forcing", C.c_int32), ("g", C.c_double * 3),
        ("collision", C.c_int32), ("s_e", C.c_double), ("s_eps", C.c_double),
        ("s_q", C.c_double), ("s_pi", C.c_double), ("s_m", C.c_double),
        ("n_scal", C.c_int32), ("tau_c", C.c_double * 2), ("J0", C.c_double),
        ("k_react", C.c_double), ("ade_open_x", C.c_int32), ("C_in", C.c_double * 2),
        ("periodic", C.c_int32 * 3), ("geo_mode", C.c_int32), ("V_m", C.c_double),
        ("m_s0", C.c_double), ("DP", C.c_double), ("deposit_conservative", C.c_int32),
        ("N_geo", C.c_int32), ("u_wall_ymax", C.c_double * 3), ("flow_open_x", C.c_int32),
        ("u_in", C.c_double), ("arrhenius", C.c_int32), ("arr_A", C.c_double), ("arr_Ta", C.c_double),
        ("heat_release", C.c_double), ("n_it", C.c_int32), ("conjugate", C.c_int32),
        ("tau_s", C.c_double), ("c_fs", C.c_double), ("product", C.c_int32), ("tau_p", C.c_double),
        ("C_in_p", C.c_double),
    ]


MON_NAMES = [
    "step", "mass0", "mass1", "momx", "momy", "momz", "species0", "species1", "reacted",
    "inflow0", "inflow1", "outflow0", "outflow1", "inj_mass0", "inj_mass1", "inj_spec0",
    "inj_spec1", "rem_mass0", "rem_mass1", "rem_spec0", "rem_spec1", "deposited", "nsolid",
    "nfluid", "nonfinite", "wallx", "heat", "tsolid", "heat_s", "heat_src", "solid_rem",
    "species_p", "inflow_p", "outflow_p", "inj_spec_p", "rem_spec_p", "produced",
]

_ENUMS = {
    "forcing": {"guo": 0, "sc_shift": 1},
    "collision": {"bgk": 0, "mrt": 1},
    "psi_kind": {"exp": 0, "identity": 1},
    "geo_mode": {"none": 0, "dissolve": 1, "deposit": 2},
}


def _lib_handle():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.POINTER
            dp = P(C.c_double)
            lib.orc_create.restype = C.c_void_p
            lib.orc_create.argtypes = [P(OrcParams), P(C.c_int)]
            lib.orc_destroy.argtypes = [C.c_void_p]
            lib.orc_set_geometry.argtypes = [C.c_void_p, P(C.c_uint8)]
            lib.orc_set_fields.argtypes = [C.c_void_p, dp, dp, dp]
            lib.orc_step.argtypes = [C.c_void_p, C.c_int64]
            lib.orc_get_fields.argtypes = [C.c_void_p, dp, dp, dp, P(C.c_uint8), dp]
            lib.orc_get_pops.argtypes = [C.c_void_p, dp, dp]
            lib.orc_set_pops.argtypes = [C.c_void_p, dp, dp]
            lib.orc_get_monitors.argtypes = [C.c_void_p, dp]
            lib.orc_residual.restype = C.c_double
            lib.orc_residual.argtypes = [C.c_void_p]
            lib.orc_get_mrt.argtypes = [C.c_void_p, dp, dp]
            lib.orc_lattice.argtypes = [C.c_void_p, C.c_int, P(C.c_int), P(C.c_int), dp]
            _lib = lib
    return _lib


def make_params(cfg: dict) -> OrcParams:
    """Fill the oracle's own parameter struct from a plain configuration dict."""
    p = OrcParams()
    d = dict(cfg)
    p.dim = int(d["dim"])
    p.nx, p.ny, p.nz = int(d["nx"]), int(d["ny"]), int(d.get("nz", 1))
    p.n_comp = int(d.get("n_comp", 1))
    tau = d.get("tau", [1.0, 1.0])
    p.tau[0], p.tau[1] = float(tau[0]), float(tau[1] if len(tau) > 1 else tau[0])
    G = d.get("G", [[0.0, 0.0], [0.0, 0.0]])
    for a in range(2):
        for b in range(2):
            p.G[a][b] = float(G[a][b])
    ga = d.get("G_ads", [0.0, 0.0])
    p.G_ads[0], p.G_ads[1] = float(ga[0]), float(ga[1])
    p.rho_solid = float(d.get("rho_solid", 0.0))
    p.psi_kind = _ENUMS["psi_kind"][d.get("psi_kind", "exp")]
    p.rho0 = float(d.get("rho0", 1.0))
    p.forcing = _ENUMS["forcing"][d.get("forcing", "guo")]
    g = d.get("g", [0.0, 0.0, 0.0])
    for a in range(3):
        p.g[a] = float(g[a])
    p.collision = _ENUMS["collision"][d.get("collision", "bgk")]
    rates = d.get("mrt_rates", {})
    p.s_e = float(rates.get("s_e", 1.19))
    p.s_eps = float(rates.get("s_eps", 1.4))
    p.s_q = float(rates.get("s_q", 1.2))
    p.s_pi = float(rates.get("s_pi", 1.0 / p.tau[0]))
    p.s_m = float(rates.get("s_m", 1.98))
    p.n_scal = int(d.get("n_scal", 0))
    tc = d.get("tau_c", [1.0, 1.0])
    p.tau_c[0], p.tau_c[1] = float(tc[0]), float(tc[1] if len(tc) > 1 else tc[0])
    p.J0 = float(d.get("J0", 0.4 if p.dim == 2 else 0.25))
    p.k_react = float(d.get("k_react", 0.0))
    p.ade_open_x = int(bool(d.get("ade_open_x", False)))
    ci = d.get("C_in", [0.0, 0.0])
    p.C_in[0], p.C_in[1] = float(ci[0]), float(ci[1] if len(ci) > 1 else 0.0)
    per = d.get("periodic", [1, 1, 1])
    for a in range(3):
        p.periodic[a] = int(per[a])
    p.geo_mode = _ENUMS["geo_mode"][d.get("geo_mode", "none")]
    p.V_m = float(d.get("V_m", 1.0))
    p.m_s0 = float(d.get("m_s0", 1.0))
    p.DP = float(d.get("DP", 0.0))
    p.deposit_conservative = int(bool(d.get("deposit_conservative", True)))
    p.N_geo = int(d.get("N_geo", 1))
    uw = d.get("u_wall_ymax", [0.0, 0.0, 0.0])
    for a in range(3):
        p.u_wall_ymax[a] = float(uw[a])
    p.flow_open_x = int(bool(d.get("flow_open_x", False)))
    p.u_in = float(d.get("u_in", 0.0))
    p.arrhenius = int(bool(d.get("arrhenius", False)))
    p.arr_A = float(d.get("arr_A", 0.0))
    p.arr_Ta = float(d.get("arr_Ta", 0.0))
    p.heat_release = float(d.get("heat_release", 0.0))
    p.n_it = int(d.get("n_it", 16))
    p.conjugate = int(bool(d.get("conjugate", False)))
    p.tau_s = float(d.get("tau_s", 1.0))
    p.c_fs = float(d.get("c_fs", 1.0))
    p.product = int(bool(d.get("product", False)))
    p.tau_p = float(d.get("tau_p", 1.0))
    p.C_in_p = float(d.get("C_in_p", 0.0))
    return p


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double)) if a is not None else None


class Oracle:
    """FP64 reference solver; all arrays are numpy, node index x fastest."""

    def __init__(self, cfg: dict):
        self.lib = _lib_handle()
        self.cfg = dict(cfg)
        self.p = make_params(cfg)
        st = C.c_int(0)
        self.h = self.lib.orc_create(C.byref(self.p), C.byref(st))
        if not self.h:
            raise ValueError(f"oracle rejected the configuration (status {st.value})")
        self.dim = self.p.dim
        self.n_lat = self.p.n_scal + self.p.product    # scalar lattices, the product last
        self.shape = (self.p.nz, self.p.ny, self.p.nx)
        self.N = self.p.nx * self.p.ny * self.p.nz
        self.qf = 19 if self.dim == 3 else 9
        self.qc = 7 if self.dim == 3 else 5

    def close(self):
        if getattr(self, "h", None):
            self.lib.orc_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def set_geometry(self, flags):
        fl = np.ascontiguousarray(flags, dtype=np.uint8).reshape(-1)
        assert fl.size == self.N
        if self.lib.orc_set_geometry(self.h, fl.ctypes.data_as(C.POINTER(C.c_uint8))) != 0:
            raise ValueError("bad flag value")

    def set_fields(self, rho, u, Cs=None):
        nc, ns = self.p.n_comp, self.n_lat
        r = np.ascontiguousarray(rho, dtype=np.float64).reshape(nc, self.N)
        uu = np.ascontiguousarray(u, dtype=np.float64).reshape(3, self.N)
        cc = np.ascontiguousarray(Cs, dtype=np.float64).reshape(ns, self.N) if ns else None
        self.lib.orc_set_fields(self.h, _dp(r), _dp(uu), _dp(cc))

    def step(self, n=1):
        self.lib.orc_step(self.h, int(n))

    def fields(self):
        nc, ns, N = self.p.n_comp, self.n_lat, self.N
        rho = np.zeros((nc, N))
        u = np.zeros((3, N))
        Cs = np.zeros((max(ns, 1), N))
        flags = np.zeros(N, dtype=np.uint8)
        acc = np.zeros(N)
        self.lib.orc_get_fields(self.h, _dp(rho), _dp(u), _dp(Cs),
                                flags.ctypes.data_as(C.POINTER(C.c_uint8)), _dp(acc))
        sh = self.shape
        return {"rho": rho.reshape((nc,) + sh), "u": u.reshape((3,) + sh),
                "C": Cs[:ns].reshape((ns,) + sh), "flags": flags.reshape(sh),
                "acc": acc.reshape(sh)}

    def pops(self):
        nc, ns, N = self.p.n_comp, self.n_lat, self.N
        f = np.zeros((nc, self.qf, N))
        h = np.zeros((max(ns, 1), self.qc, N))
        self.lib.orc_get_pops(self.h, _dp(f), _dp(h))
        return f, h[:ns]

    def set_pops(self, f, h=None):
        f = np.ascontiguousarray(f, dtype=np.float64)
        hh = np.ascontiguousarray(h, dtype=np.float64) if h is not None and self.n_lat else None
        self.lib.orc_set_pops(self.h, _dp(f), _dp(hh))

    def monitors(self):
        out = np.zeros(len(MON_NAMES))
        self.lib.orc_get_monitors(self.h, _dp(out))
        return dict(zip(MON_NAMES, out.tolist()))

    def residual(self):
        return float(self.lib.orc_residual(self.h))

    def mrt(self):
        q = self.qf
        M = np.zeros(q * q)
        S = np.zeros(q)
        if self.lib.orc_get_mrt(self.h, _dp(M), _dp(S)) != 0:
            raise ValueError("not an MRT configuration")
        return M.reshape(q, q), S

    def lattice(self, which=0):
        q = C.c_int(0)
        cv = np.zeros(19 * 3, dtype=np.int32)
        w = np.zeros(19)
        self.lib.orc_lattice(self.h, which, C.byref(q), cv.ctypes.data_as(C.POINTER(C.c_int)), _dp(w))
        n = q.value
        return cv[: 3 * n].reshape(n, 3).astype(np.int64), w[:n].copy()
