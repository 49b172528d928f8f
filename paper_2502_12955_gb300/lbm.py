"""Python binding of the C ABI in include/lbm.h (ctypes marshalling only).

Every step of the lattice Boltzmann update runs in liblbm.so's sm_103a kernels; this module
only converts numpy arrays and parameter dictionaries into the C structures.  There is no
host fallback: if the library cannot be loaded, constructing a Solver raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

LBM_D2Q9_D2Q5 = 2
LBM_D3Q19_D3Q7 = 3
PRECISION = {"fp64": 0, "fp32": 1, "fp16": 2, "bf16": 3, "fp16s32": 4, "bf16s32": 5}   # *s32: FP32 scalars
FORCING = {"guo": 0, "sc_shift": 1}
COLLISION = {"bgk": 0, "mrt": 1}
PSI = {"exp": 0, "identity": 1}
GEO = {"none": 0, "dissolve": 1, "deposit": 2}
STATUS = {0: "LBM_OK", -1: "LBM_ERR_INVALID_ARG", -2: "LBM_ERR_OOM", -3: "LBM_ERR_CUDA",
          -4: "LBM_ERR_NONFINITE", -5: "LBM_ERR_TIMEOUT", -6: "LBM_ERR_STATE", -7: "LBM_ERR_CAPACITY",
          -8: "LBM_ERR_BOUNDS"}

# Names of every entry point declared in include/lbm.h.
EXPORTS = ["lbm_params_default", "lbm_create", "lbm_set_geometry", "lbm_set_fields", "lbm_step",
           "lbm_sync", "lbm_get_fields", "lbm_get_fields_device", "lbm_get_pops", "lbm_set_pops", "lbm_get_monitors",
           "lbm_residual", "lbm_get_state", "lbm_set_state", "lbm_profile_enable",
           "lbm_profile_read", "lbm_launch_count", "lbm_last_error", "lbm_destroy",
           "lbm_get_pops_noalloc", "lbm_ensemble_create", "lbm_ensemble_member", "lbm_ensemble_step",
           "lbm_ensemble_run_to_steady", "lbm_ensemble_autotune", "lbm_ensemble_launch_count",
           "lbm_ensemble_last_error", "lbm_ensemble_destroy"]


class LbmParams(C.Structure):
    _fields_ = [
        ("precision", C.c_int32), ("n_comp", C.c_int32), ("tau", C.c_double * 2),
        ("G", (C.c_double * 2) * 2), ("G_ads", C.c_double * 2), ("rho_solid", C.c_double),
        ("psi_kind", C.c_int32), ("rho0", C.c_double), ("forcing", C.c_int32),
        ("g", C.c_double * 3), ("collision", C.c_int32), ("s_e", C.c_double),
        ("s_eps", C.c_double), ("s_q", C.c_double), ("s_pi", C.c_double), ("s_m", C.c_double),
        ("n_scal", C.c_int32), ("tau_c", C.c_double * 2), ("J0", C.c_double),
        ("k_react", C.c_double), ("ade_open_x", C.c_int32), ("C_in", C.c_double * 2),
        ("periodic", C.c_int32 * 3), ("geo_mode", C.c_int32), ("V_m", C.c_double),
        ("m_s0", C.c_double), ("DP", C.c_double), ("deposit_conservative", C.c_int32),
        ("N_geo", C.c_int32), ("N_mon", C.c_int32), ("rho_ref", C.c_double * 2),
        ("C_ref", C.c_double * 2), ("stream", C.c_void_p), ("block_x", C.c_int32),
        ("device", C.c_int32), ("l2_fetch_bytes", C.c_int32), ("u_wall_ymax", C.c_double * 3),
        ("flow_open_x", C.c_int32), ("u_in", C.c_double), ("arrhenius", C.c_int32),
        ("arr_A", C.c_double), ("arr_Ta", C.c_double), ("heat_release", C.c_double), ("n_it", C.c_int32),
        ("product", C.c_int32), ("tau_p", C.c_double), ("C_in_p", C.c_double),
        ("conjugate", C.c_int32), ("tau_s", C.c_double), ("c_fs", C.c_double),
    ]


class LbmMonitors(C.Structure):
    _fields_ = [
        ("step", C.c_double), ("mass", C.c_double * 2), ("momentum", C.c_double * 3),
        ("species", C.c_double * 2), ("reacted", C.c_double), ("inflow", C.c_double * 2),
        ("outflow", C.c_double * 2), ("injected_mass", C.c_double * 2),
        ("injected_species", C.c_double * 2), ("removed_mass", C.c_double * 2),
        ("removed_species", C.c_double * 2), ("deposited", C.c_double), ("n_solid", C.c_double),
        ("n_fluid", C.c_double), ("nonfinite", C.c_double), ("wall_exchange", C.c_double),
        ("residual", C.c_double), ("heat", C.c_double), ("species_p", C.c_double),
        ("inflow_p", C.c_double), ("outflow_p", C.c_double), ("injected_species_p", C.c_double),
        ("removed_species_p", C.c_double), ("produced", C.c_double),
        ("t_solid", C.c_double), ("heat_solid", C.c_double), ("heat_source", C.c_double),
        ("solid_removed", C.c_double),
    ]


class LbmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load liblbm.so (building it first when absent or stale and nvcc is available).
    The environment variable LBM_LIBRARY selects another build of the same ABI."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = os.environ.get("LBM_LIBRARY") or _build.LIB
        if build_if_missing and not os.environ.get("LBM_LIBRARY"):
            path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"liblbm.so not found at {path}; build it with "
                               "paper_2502_12955_gb300.build.build()")
        lib = C.CDLL(path)
        P = C.POINTER
        dp = P(C.c_double)
        vp = C.c_void_p
        lib.lbm_params_default.argtypes = [P(LbmParams)]
        lib.lbm_create.argtypes = [C.c_int, C.c_int32, C.c_int32, C.c_int32, P(LbmParams), P(vp)]
        lib.lbm_set_geometry.argtypes = [vp, P(C.c_uint8), C.c_size_t]
        lib.lbm_set_fields.argtypes = [vp, dp, dp, dp, C.c_size_t]
        lib.lbm_step.argtypes = [vp, C.c_int64]
        lib.lbm_sync.argtypes = [vp]
        lib.lbm_get_fields.argtypes = [vp, dp, dp, dp, P(C.c_uint8), dp]
        lib.lbm_get_fields_device.argtypes = [vp, P(vp), P(vp), P(vp), P(vp), P(vp)]
        lib.lbm_get_pops.argtypes = [vp, dp, dp]
        lib.lbm_set_pops.argtypes = [vp, dp, dp]
        lib.lbm_get_pops_noalloc.argtypes = [vp, dp, dp]
        lib.lbm_get_monitors.argtypes = [vp, P(LbmMonitors)]
        lib.lbm_residual.argtypes = [vp, dp]
        lib.lbm_get_state.argtypes = [vp, vp, P(C.c_size_t)]
        lib.lbm_set_state.argtypes = [vp, vp, C.c_size_t]
        lib.lbm_profile_enable.argtypes = [vp, C.c_int32]
        lib.lbm_profile_read.argtypes = [vp, dp, P(C.c_int64)]
        lib.lbm_launch_count.argtypes = [vp, P(C.c_int64)]
        lib.lbm_last_error.argtypes = [vp]
        lib.lbm_last_error.restype = C.c_char_p
        lib.lbm_destroy.argtypes = [vp]
        lib.lbm_ensemble_create.argtypes = [C.c_int, C.c_int32, P(C.c_int32), P(LbmParams), P(vp)]
        lib.lbm_ensemble_member.argtypes = [vp, C.c_int32, P(vp)]
        lib.lbm_ensemble_step.argtypes = [vp, C.c_int64]
        lib.lbm_ensemble_run_to_steady.argtypes = [vp, C.c_double, C.c_int64, P(C.c_int64), P(C.c_int32)]
        lib.lbm_ensemble_autotune.argtypes = [vp, C.c_int32, P(C.c_int32)]
        lib.lbm_ensemble_launch_count.argtypes = [vp, P(C.c_int64)]
        lib.lbm_ensemble_last_error.argtypes = [vp]
        lib.lbm_ensemble_last_error.restype = C.c_char_p
        lib.lbm_ensemble_destroy.argtypes = [vp]
        for name in EXPORTS:
            if name not in ("lbm_last_error", "lbm_destroy"):
                getattr(lib, name).restype = C.c_int
        lib.lbm_destroy.restype = None
        lib.lbm_ensemble_last_error.restype = C.c_char_p
        lib.lbm_ensemble_destroy.restype = None
        _lib = lib
    return _lib


def make_params(cfg: dict, lib=None) -> LbmParams:
    """lbm_params from a configuration dictionary (same keys as the workload definitions)."""
    lib = lib or load()
    p = LbmParams()
    lib.lbm_params_default(C.byref(p))
    d = dict(cfg)
    p.precision = PRECISION[d.get("precision", "fp32")]
    p.n_comp = int(d.get("n_comp", 1))
    tau = list(d.get("tau", [1.0]))
    p.tau[0] = float(tau[0])
    p.tau[1] = float(tau[1] if len(tau) > 1 else tau[0])
    G = d.get("G", [[0.0, 0.0], [0.0, 0.0]])
    for a in range(2):
        for b in range(2):
            p.G[a][b] = float(G[a][b])
    ga = d.get("G_ads", [0.0, 0.0])
    p.G_ads[0], p.G_ads[1] = float(ga[0]), float(ga[1])
    p.rho_solid = float(d.get("rho_solid", 0.0))
    p.psi_kind = PSI[d.get("psi_kind", "exp")]
    p.rho0 = float(d.get("rho0", 1.0))
    p.forcing = FORCING[d.get("forcing", "guo")]
    g = d.get("g", [0.0, 0.0, 0.0])
    for a in range(3):
        p.g[a] = float(g[a])
    p.collision = COLLISION[d.get("collision", "bgk")]
    rates = d.get("mrt_rates", {})
    p.s_e = float(rates.get("s_e", 1.19))
    p.s_eps = float(rates.get("s_eps", 1.4))
    p.s_q = float(rates.get("s_q", 1.2))
    p.s_pi = float(rates.get("s_pi", 1.0 / p.tau[0]))
    p.s_m = float(rates.get("s_m", 1.98))
    p.n_scal = int(d.get("n_scal", 0))
    tc = list(d.get("tau_c", [1.0]))
    p.tau_c[0] = float(tc[0])
    p.tau_c[1] = float(tc[1] if len(tc) > 1 else tc[0])
    dim = int(d["dim"])
    p.J0 = float(d.get("J0", 0.4 if dim == 2 else 0.25))
    p.k_react = float(d.get("k_react", 0.0))
    p.ade_open_x = int(bool(d.get("ade_open_x", False)))
    ci = list(d.get("C_in", [0.0]))
    p.C_in[0] = float(ci[0])
    p.C_in[1] = float(ci[1] if len(ci) > 1 else 0.0)
    per = d.get("periodic", [1, 1, 1])
    for a in range(3):
        p.periodic[a] = int(per[a])
    p.geo_mode = GEO[d.get("geo_mode", "none")]
    p.V_m = float(d.get("V_m", 1.0))
    p.m_s0 = float(d.get("m_s0", 1.0))
    p.DP = float(d.get("DP", 0.0))
    p.deposit_conservative = int(bool(d.get("deposit_conservative", True)))
    p.N_geo = int(d.get("N_geo", 1))
    p.N_mon = int(d.get("N_mon", 0))
    rr = d.get("rho_ref", [1.0, 1.0])
    p.rho_ref[0], p.rho_ref[1] = float(rr[0]), float(rr[1] if len(rr) > 1 else rr[0])
    cr = d.get("C_ref", [0.0, 0.0])
    p.C_ref[0], p.C_ref[1] = float(cr[0]), float(cr[1] if len(cr) > 1 else cr[0])
    p.block_x = int(d.get("block_x", 0))
    p.device = int(d.get("device", 0))
    p.l2_fetch_bytes = int(d.get("l2_fetch_bytes", 0))
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
    p.product = int(bool(d.get("product", False)))
    p.tau_p = float(d.get("tau_p", 1.0))
    p.C_in_p = float(d.get("C_in_p", 0.0))
    p.conjugate = int(bool(d.get("conjugate", False)))
    p.tau_s = float(d.get("tau_s", 1.0))
    p.c_fs = float(d.get("c_fs", 1.0))
    return p


class DeviceArray:
    """A device array owned by a Solver, exposed through the CUDA array interface (version 3).
    Keeps its solver alive; the data stream is synchronised before it is handed out."""

    def __init__(self, ptr, shape, typestr, owner):
        self.ptr, self.shape, self.typestr, self._owner = int(ptr), tuple(shape), typestr, owner

    @property
    def __cuda_array_interface__(self):
        return {"shape": self.shape, "typestr": self.typestr, "data": (self.ptr, False), "version": 3,
                "strides": None, "stream": None}


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double)) if a is not None else None


MON_KEYS = ["step", "mass0", "mass1", "momx", "momy", "momz", "species0", "species1", "reacted",
            "inflow0", "inflow1", "outflow0", "outflow1", "inj_mass0", "inj_mass1", "inj_spec0",
            "inj_spec1", "rem_mass0", "rem_mass1", "rem_spec0", "rem_spec1", "deposited", "nsolid",
            "nfluid", "nonfinite", "wallx", "residual", "heat", "species_p", "inflow_p", "outflow_p",
            "inj_spec_p", "rem_spec_p", "produced", "tsolid", "heat_s", "heat_src", "solid_rem"]


def save_fields(fields, path):
    """Write a fields dict (as Solver.fields returns it) to `path` (.npz, uncompressed) and
    return the path written."""
    path = str(path)
    if not path.endswith(".npz"):
        path += ".npz"
    np.savez(path, **{k: np.asarray(v) for k, v in fields.items()})
    return path


class Solver:
    """One lattice Boltzmann domain on one GPU (owns an lbm_ctx)."""

    def __init__(self, cfg: dict, stream=None, _handle=None):
        self.lib = load()
        self.cfg = dict(cfg)
        self.dim = int(cfg["dim"])
        nx, ny, nz = int(cfg["nx"]), int(cfg["ny"]), int(cfg.get("nz", 1))
        self.shape = (nz, ny, nx)
        self.N = nx * ny * nz
        self.qf = 19 if self.dim == 3 else 9
        self.qc = 7 if self.dim == 3 else 5
        self.p = make_params(cfg, self.lib)
        if stream is not None:
            self.p.stream = C.c_void_p(int(stream))
        # scalar lattices: the given scalars, then the reaction product (if any)
        self.n_comp, self.n_scal = self.p.n_comp, self.p.n_scal + self.p.product
        self._owner = _handle is None
        if _handle is not None:   # a member context owned by an Ensemble
            self.h = _handle
            return
        h = C.c_void_p()
        lat = LBM_D3Q19_D3Q7 if self.dim == 3 else LBM_D2Q9_D2Q5
        st = self.lib.lbm_create(lat, nx, ny, nz, C.byref(self.p), C.byref(h))
        if st != 0:
            raise LbmError(st, self.lib.lbm_last_error(None).decode())
        self.h = h

    # ------------------------------------------------------------------ helpers
    def _ck(self, st):
        if st != 0:
            raise LbmError(st, self.lib.lbm_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            if self._owner:
                self.lib.lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --------------------------------------------------------------------- API
    def set_geometry(self, flags):
        fl = np.ascontiguousarray(flags, dtype=np.uint8).reshape(-1)
        self._ck(self.lib.lbm_set_geometry(self.h, fl.ctypes.data_as(C.POINTER(C.c_uint8)), fl.size))

    def set_fields(self, rho, u, Cs=None):
        r = np.ascontiguousarray(rho, dtype=np.float64).reshape(self.n_comp, self.N)
        uu = np.ascontiguousarray(u, dtype=np.float64).reshape(3, self.N)
        cc = (np.ascontiguousarray(Cs, dtype=np.float64).reshape(self.n_scal, self.N)
              if self.n_scal else None)
        self._ck(self.lib.lbm_set_fields(self.h, _dp(r), _dp(uu), _dp(cc), self.N))

    def step(self, n=1):
        self._ck(self.lib.lbm_step(self.h, int(n)))

    def sync(self):
        self._ck(self.lib.lbm_sync(self.h))

    def fields(self, out=None):
        """Macroscopic fields as a dict of arrays (rho, u, C, flags, acc; x fastest).  out may be
        such a dict of preallocated C-contiguous arrays (float64; flags uint8) of the same shapes,
        for example in pinned host memory, which are filled in place and returned."""
        nc, ns, N = self.n_comp, self.n_scal, self.N
        sh = self.shape
        if out is None:
            out = {"rho": np.zeros((nc,) + sh), "u": np.zeros((3,) + sh), "C": np.zeros((ns,) + sh),
                   "flags": np.zeros(sh, dtype=np.uint8), "acc": np.zeros(sh)}
        want = {"rho": ((nc,) + sh, np.float64), "u": ((3,) + sh, np.float64), "C": ((ns,) + sh, np.float64),
                "flags": (sh, np.uint8), "acc": (sh, np.float64)}
        for k, (shape, dt) in want.items():
            a = out[k]
            if a.shape != shape or a.dtype != dt or not a.flags["C_CONTIGUOUS"]:
                raise ValueError(f"fields(out): {k} must be a C-contiguous {np.dtype(dt).name} array of shape {shape}")
        self._ck(self.lib.lbm_get_fields(self.h, _dp(out["rho"]), _dp(out["u"]), _dp(out["C"]) if ns else None,
                                         out["flags"].ctypes.data_as(C.POINTER(C.c_uint8)), _dp(out["acc"])))
        return out

    def fields_device(self):
        """The fields left on the device (lbm_get_fields_device): a dict of objects exposing the
        CUDA array interface (no copy; read them with torch.as_tensor(v, device="cuda") or any
        consumer of that interface), in the layouts of fields().  They stay valid until the next
        fields(), fields_device() or set_fields() (flags and acc: until the next step), and never
        after close()."""
        ptr = [C.c_void_p() for _ in range(5)]
        self._ck(self.lib.lbm_get_fields_device(self.h, *[C.byref(p) for p in ptr]))
        nc, ns, sh = self.n_comp, self.n_scal, self.shape
        spec = {"rho": ((nc,) + sh, "<f8"), "u": ((3,) + sh, "<f8"), "C": ((ns,) + sh, "<f8"),
                "flags": (sh, "|u1"), "acc": (sh, "<f8")}
        out = {}
        for (k, (shape, typestr)), p in zip(spec.items(), ptr):
            if p.value is None:
                continue
            out[k] = DeviceArray(p.value, shape, typestr, self)
        return out

    def save_fields(self, path):
        """Write the macroscopic fields (rho, u, C, flags, acc; x fastest) to an .npz file for
        offline plotting."""
        return save_fields(self.fields(), path)

    def pops(self):
        f = np.zeros((self.n_comp, self.qf, self.N))
        h = np.zeros((max(self.n_scal, 1), self.qc, self.N))
        self._ck(self.lib.lbm_get_pops(self.h, _dp(f), _dp(h) if self.n_scal else None))
        return f, h[: self.n_scal]

    def pops_noalloc(self, want_f=True, want_h=True):
        """pops() through lbm_get_pops_noalloc (no device allocation, bounded domain size).
        want_f / want_h = False pass NULL for that output, which then comes back as None."""
        f = np.zeros((self.n_comp, self.qf, self.N)) if want_f else None
        h = np.zeros((max(self.n_scal, 1), self.qc, self.N)) if want_h else None
        self._ck(self.lib.lbm_get_pops_noalloc(self.h, _dp(f) if want_f else None,
                                               _dp(h) if (want_h and self.n_scal) else None))
        return f, (h[: self.n_scal] if want_h else None)

    def set_pops(self, f, h=None):
        f = np.ascontiguousarray(f, dtype=np.float64)
        hh = np.ascontiguousarray(h, dtype=np.float64) if (h is not None and self.n_scal) else None
        self._ck(self.lib.lbm_set_pops(self.h, _dp(f), _dp(hh)))

    def monitors(self):
        m = LbmMonitors()
        self._ck(self.lib.lbm_get_monitors(self.h, C.byref(m)))
        vals = [m.step, m.mass[0], m.mass[1], *m.momentum, m.species[0], m.species[1], m.reacted,
                m.inflow[0], m.inflow[1], m.outflow[0], m.outflow[1], m.injected_mass[0],
                m.injected_mass[1], m.injected_species[0], m.injected_species[1],
                m.removed_mass[0], m.removed_mass[1], m.removed_species[0], m.removed_species[1],
                m.deposited, m.n_solid, m.n_fluid, m.nonfinite, m.wall_exchange, m.residual, m.heat,
                m.species_p, m.inflow_p, m.outflow_p, m.injected_species_p, m.removed_species_p, m.produced,
                m.t_solid, m.heat_solid, m.heat_source, m.solid_removed]
        return dict(zip(MON_KEYS, vals))

    def residual(self):
        r = C.c_double()
        self._ck(self.lib.lbm_residual(self.h, C.byref(r)))
        return r.value

    def get_state(self) -> bytes:
        n = C.c_size_t(0)
        self._ck(self.lib.lbm_get_state(self.h, None, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        self._ck(self.lib.lbm_get_state(self.h, C.cast(buf, C.c_void_p), C.byref(n)))
        return buf.raw

    def set_state(self, blob: bytes):
        buf = C.create_string_buffer(blob, len(blob))
        self._ck(self.lib.lbm_set_state(self.h, C.cast(buf, C.c_void_p), len(blob)))

    def profile(self, on=True):
        self._ck(self.lib.lbm_profile_enable(self.h, 1 if on else 0))

    def profile_read(self):
        ms = C.c_double()
        n = C.c_int64()
        self._ck(self.lib.lbm_profile_read(self.h, C.byref(ms), C.byref(n)))
        return ms.value, n.value

    def launch_count(self):
        n = C.c_int64()
        self._ck(self.lib.lbm_launch_count(self.h, C.byref(n)))
        return n.value


class Ensemble:
    """Independent domains of one lattice advanced together (owns an lbm_ensemble).

    cfgs: one configuration dict per member (same keys as Solver).  members[k] is a Solver view
    of member k for geometry, fields, monitors and read-back."""

    def __init__(self, cfgs, stream=None):
        self.lib = load()
        cfgs = [dict(c) for c in cfgs]
        dims = {int(c["dim"]) for c in cfgs}
        if len(dims) != 1:
            raise ValueError("ensemble members share one lattice")
        dim = dims.pop()
        n = len(cfgs)
        params = (LbmParams * n)()
        sizes = (C.c_int32 * (3 * n))()
        for k, c in enumerate(cfgs):
            params[k] = make_params(c, self.lib)
            if stream is not None:
                params[k].stream = C.c_void_p(int(stream))
            sizes[3 * k:3 * k + 3] = [int(c["nx"]), int(c["ny"]), int(c.get("nz", 1))]
        h = C.c_void_p()
        lat = LBM_D3Q19_D3Q7 if dim == 3 else LBM_D2Q9_D2Q5
        st = self.lib.lbm_ensemble_create(lat, n, sizes, params, C.byref(h))
        if st != 0:
            raise LbmError(st, self.lib.lbm_ensemble_last_error(None).decode())
        self.h = h
        self.members = []
        for k, c in enumerate(cfgs):
            mh = C.c_void_p()
            self._ck(self.lib.lbm_ensemble_member(self.h, k, C.byref(mh)))
            self.members.append(Solver(c, stream=stream, _handle=mh))

    def _ck(self, st):
        if st != 0:
            raise LbmError(st, self.lib.lbm_ensemble_last_error(self.h).decode())

    def step(self, n=1):
        self._ck(self.lib.lbm_ensemble_step(self.h, int(n)))

    def run_to_steady(self, r_tol, max_steps):
        """(steps taken, number of members that reached r_tol and stopped)"""
        s, c = C.c_int64(), C.c_int32()
        self._ck(self.lib.lbm_ensemble_run_to_steady(self.h, float(r_tol), int(max_steps), C.byref(s), C.byref(c)))
        return s.value, c.value

    def autotune(self, steps=8):
        t = C.c_int32()
        self._ck(self.lib.lbm_ensemble_autotune(self.h, int(steps), C.byref(t)))
        return t.value

    def launch_count(self):
        n = C.c_int64()
        self._ck(self.lib.lbm_ensemble_launch_count(self.h, C.byref(n)))
        return n.value

    def close(self):
        if getattr(self, "h", None):
            for m in self.members:
                m.h = None
            self.lib.lbm_ensemble_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
