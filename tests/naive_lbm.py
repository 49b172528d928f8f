"""A second, deliberately naive formulation of one time step, for brute-force checks of the
oracle on tiny lattices.

Written independently of oracle/ (no shared code, tables or helpers) and structured
differently on purpose:
- It streams by pushing post-collision populations to their destinations, where the oracle
  pulls them from their sources.
- MRT is the full moment-space relaxation with the explicit d'Humieres (D3Q19) / Lallemand-Luo
  (D2Q9) polynomial matrix and its numerical inverse, where the oracle builds rows by
  Gram-Schmidt.
- Every node and link is a plain Python loop.
- The coupled interface values (T_b of the temperature-dependent closure and of the solid-link
  exchange) are bracketed roots, where the oracle iterates a fixed point.
- Heat conduction in the solid and its link exchange are pushed after the fluid streaming, and
  the CO2 product is closed from the link rates of the species closure.

The velocity sets come from the paper's printed tables (tests/golden/lattice_tables.json), with
the same readings the project documents: D2Q9 axis weights 1/9, D3Q7 as the first seven D3Q19
directions with rest weight J0, the wet-node closure per link at gather time, inlet
equilibrium ghost and zero-gradient outlet for the scalar, and flow walls on non-periodic
faces.

The state is the populations each fluid node holds at the start of a step (after streaming),
the same quantity the oracle reports.  Fields are indexed [q][z][y][x].
"""
from __future__ import annotations

import json
import os
from fractions import Fraction

import numpy as np

_GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "lattice_tables.json")


def velocity_sets(dim, J0):
    t = json.load(open(_GOLD))
    if dim == 3:
        d = t["D3Q19"]
        cf = np.array([d["cx"], d["cy"], d["cz"]], dtype=int).T
        wf = np.array([float(Fraction(w)) for w in d["w"]])
        cc = cf[:7].copy()
        wc = np.array([J0] + [(1.0 - J0) / 6.0] * 6)
    else:
        d = t["D2Q9"]
        cf = np.array([d["cx"], d["cy"], [0] * 9], dtype=int).T
        wf = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)     # axis weights 1/9 (reading 1)
        e = t["D2Q5"]
        cc = np.array([e["cx"], e["cy"], [0] * 5], dtype=int).T
        wc = np.array([J0] + [(1.0 - J0) / 4.0] * 4)
    return cf, wf, cc, wc


def opposite(c):
    return [next(k for k in range(len(c)) if (c[k] == -c[i]).all()) for i in range(len(c))]


def moment_matrix(dim, cf):
    """Rows of the MRT moment basis as printed polynomials, with each row's relaxation group:
    'c' conserved, 'nu' stress (1/tau), 'e', 'eps', 'q', 'pi', 'm'."""
    rows, grp = [], []
    x, y, z = cf[:, 0].astype(float), cf[:, 1].astype(float), cf[:, 2].astype(float)
    c2 = x * x + y * y + z * z
    one = np.ones_like(x)
    if dim == 3:
        table = [(one, "c"), (19 * c2 - 30, "e"), ((21 * c2 * c2 - 53 * c2 + 24) / 2, "eps"),
                 (x, "c"), ((5 * c2 - 9) * x, "q"), (y, "c"), ((5 * c2 - 9) * y, "q"),
                 (z, "c"), ((5 * c2 - 9) * z, "q"),
                 (3 * x * x - c2, "nu"), ((3 * c2 - 5) * (3 * x * x - c2), "pi"),
                 (y * y - z * z, "nu"), ((3 * c2 - 5) * (y * y - z * z), "pi"),
                 (x * y, "nu"), (y * z, "nu"), (x * z, "nu"),
                 (x * (y * y - z * z), "m"), (y * (z * z - x * x), "m"), (z * (x * x - y * y), "m")]
    else:
        table = [(one, "c"), (3 * c2 - 4, "e"), ((9 * c2 * c2 - 21 * c2 + 8) / 2, "eps"),
                 (x, "c"), ((3 * c2 - 5) * x, "q"), (y, "c"), ((3 * c2 - 5) * y, "q"),
                 (x * x - y * y, "nu"), (x * y, "nu")]
    for r, g in table:
        rows.append(r)
        grp.append(g)
    return np.array(rows), grp


class NaiveLBM:
    def __init__(self, cfg, flags, f, h, T_solid=None):
        self.cfg = cfg
        self.dim = int(cfg["dim"])
        self.nx, self.ny, self.nz = int(cfg["nx"]), int(cfg["ny"]), int(cfg.get("nz", 1))
        self.nc = int(cfg.get("n_comp", 1))
        # scalar lattices: the n_scal given ones, then the reaction product if there is one
        self.n_given = int(cfg.get("n_scal", 0))
        self.prod = bool(cfg.get("product", False))
        self.ns = self.n_given + int(self.prod)
        tc = [float(t) for t in cfg.get("tau_c", [1.0, 1.0])]
        ci = [float(v) for v in cfg.get("C_in", [0.0, 0.0])]
        self.tau_s_list = [tc[s] if s < len(tc) else tc[0] for s in range(self.n_given)]
        self.cin_list = [ci[s] if s < len(ci) else 0.0 for s in range(self.n_given)]
        if self.prod:
            self.tau_s_list.append(float(cfg["tau_p"]))
            self.cin_list.append(float(cfg.get("C_in_p", 0.0)))
        self.J0 = float(cfg.get("J0", 0.25))
        self.cf, self.wf, self.cc, self.wc = velocity_sets(self.dim, self.J0)
        self.of, self.oc = opposite(self.cf), opposite(self.cc)
        self.flags = np.array(flags, dtype=np.uint8).reshape(self.nz, self.ny, self.nx)
        self.f = np.array(f, dtype=np.float64).reshape(self.nc, len(self.cf), self.nz, self.ny, self.nx).copy()
        self.h = np.array(h, dtype=np.float64).reshape(self.ns, len(self.cc), self.nz, self.ny, self.nx).copy() \
            if self.ns else np.zeros((0, len(self.cc), self.nz, self.ny, self.nx))
        self.acc = np.zeros((self.nz, self.ny, self.nx))
        self.t = 0
        # conduction in the solid: its own populations, at rest equilibrium w_j T_s to start, and
        # the rate constant that each reactive link's last exchange found
        self.conj = bool(cfg.get("conjugate", False))
        self.g = np.zeros((len(self.cc), self.nz, self.ny, self.nx))
        if self.conj:
            Ts = np.asarray(T_solid, dtype=np.float64).reshape(self.nz, self.ny, self.nx)
            self.g = self.wc[:, None, None, None] * np.where(self.flags != 0, Ts, 0.0)[None]
        self.kb = {}
        per = cfg.get("periodic", [1, 1, 1])
        self.per_f = [bool(p) for p in per]
        self.per_c = [bool(per[0]) and not cfg.get("ade_open_x", False), bool(per[1]), bool(per[2])]
        if self.dim == 2:
            self.per_f[2] = self.per_c[2] = True
        self.M, self.grp = moment_matrix(self.dim, self.cf)
        self.Minv = np.linalg.inv(self.M)

    # node at (x, y, z) + c, or None outside a non-periodic face
    def _shift(self, x, y, z, c, per):
        p = [x + c[0], y + c[1], z + c[2]]
        for a, n in enumerate((self.nx, self.ny, self.nz)):
            if p[a] < 0 or p[a] >= n:
                if not per[a]:
                    return None
                p[a] %= n
        return p[0], p[1], p[2]

    def _fluid(self, q):
        return q is not None and self.flags[q[2], q[1], q[0]] == 0

    def _feq(self, i, rho, u):
        cu = float(np.dot(self.cf[i], u))
        return self.wf[i] * rho * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * float(np.dot(u, u)))

    def _guo(self, i, u, F):
        c = self.cf[i].astype(float)
        return self.wf[i] * (3 * np.dot(c - u, F) + 9 * np.dot(c, u) * np.dot(c, F))

    def _psi(self, rho):
        if self.cfg.get("psi_kind", "exp") == "identity":
            return rho
        r0 = float(self.cfg.get("rho0", 1.0))
        return r0 * (1 - np.exp(-rho / r0))

    def _close(self, hstate, x, y, z):
        """Closed scalar populations of fluid node (x, y, z) in state hstate, and the reaction
        rate of each reactive link [(solid node, k C_b)]."""
        cfg = self.cfg
        Qc = len(self.cc)
        tauc = [float(t) for t in cfg.get("tau_c", [1.0, 1.0])]
        closed = hstate[:, :, z, y, x].copy()
        reactions = []
        link_rate = {}
        arr = bool(cfg.get("arrhenius", False))
        if arr:
            # temperature-dependent rate k(T) = A exp(-Ta / T) at the interface temperature, heat
            # h_r k C_b entering the temperature lattice (scalar 1) through the link; the
            # interface temperature is the root of its balance, found here by bracketing
            from scipy.optimize import brentq
            A, Ta, hr = float(cfg["arr_A"]), float(cfg["arr_Ta"]), float(cfg["heat_release"])
            fc = tauc[0] / (tauc[0] - 0.5)
            fT = tauc[1] / (tauc[1] - 0.5)
        else:
            k = float(cfg.get("k_react", 0.0))
            Kr = k * tauc[0] / (tauc[0] - 0.5)
        for j in range(1, Qc):
            src = self._shift(x, y, z, -self.cc[j], self.per_c)
            if src is None or self.flags[src[2], src[1], src[0]] != 2:
                continue
            w = self.wc[j]
            hb = hstate[0, self.oc[j], z, y, x]
            if self.conj:
                # the rate constant of the link's last exchange; before its first, k at the heat-
                # capacity-weighted mean of the fluid node's and the solid node's temperatures
                kk = self.kb.get((x, y, z, j))
                if kk is None:
                    cfs = float(cfg["c_fs"])
                    Tm = (cfs * hstate[1, :, z, y, x].sum() + self.g[:, src[2], src[1], src[0]].sum()) / (cfs + 1)
                    kk = A * np.exp(-Ta / Tm)
                cb = 2 * hb / (2 * w + kk * fc)
                closed[0, j] = 2 * w * cb - hb
                reactions.append((src, kk * cb))
                link_rate[j] = kk * cb
                continue
            if not arr:
                Cb = 2 * hb / (2 * w + Kr)
                closed[0, j] = 2 * w * Cb - hb
                reactions.append((src, k * Cb))
                link_rate[j] = k * Cb
                continue
            gb = hstate[1, self.oc[j], z, y, x]

            def interface(T):
                kk = A * np.exp(-Ta / T)
                return kk, 2 * hb / (2 * w + kk * fc)

            def balance(T):
                kk, cb = interface(T)
                return T - (2 * gb + hr * kk * cb * fT) / (2 * w)

            T0 = gb / w
            T1 = T0 + hr * A * (hb / w) * fT / (2 * w) + 1e-9
            Tb = T0 if hr == 0.0 else brentq(balance, T0, T1, xtol=1e-15, rtol=1e-15, maxiter=500)
            kk, cb = interface(Tb)
            closed[0, j] = 2 * w * cb - hb
            closed[1, j] = gb + hr * kk * cb * fT
            reactions.append((src, kk * cb))
            link_rate[j] = kk * cb
        if self.prod:
            # the product enters through each reactive link at the rate the reaction takes scalar 0:
            # (1 - 1/(2 tau_p)) (h_P,j - h_P,opp(j)) = r_j
            P, tp = self.n_given, float(cfg["tau_p"])
            for j, r in link_rate.items():
                closed[P, j] = hstate[P, self.oc[j], z, y, x] + r * tp / (tp - 0.5)
        return closed, reactions

    def _flips(self):
        """Geometry update after the step's streaming (Sec. 2.1.5 solid consumption, Sec. 3.3
        deposition), every N_geo steps; all flips of one update see the state before any."""
        cfg = self.cfg
        mode = cfg.get("geo_mode", "none")
        if mode == "none" or (self.t + 1) % int(cfg.get("N_geo", 1)) != 0:
            return
        nx, ny, nz = self.nx, self.ny, self.nz
        cells = [(x, y, z) for z in range(nz) for y in range(ny) for x in range(nx)]
        if mode == "deposit":
            for (x, y, z) in cells:
                if self.flags[z, y, x] == 0 and self.acc[z, y, x] > 1.0:
                    self.flags[z, y, x] = 1
                    self.f[:, :, z, y, x] = 0.0
                    self.h[:, :, z, y, x] = 0.0
            return
        V_m = float(cfg.get("V_m", 1.0))
        m_s0 = float(cfg.get("m_s0", 1.0))
        new = []
        for (x, y, z) in cells:
            if self.flags[z, y, x] != 2 or not V_m * self.acc[z, y, x] >= m_s0:
                continue
            rs, cs, cnt = np.zeros(self.nc), np.zeros(self.ns), 0
            for i in range(1, len(self.cf)):
                q = self._shift(x, y, z, self.cf[i], self.per_f)
                if not self._fluid(q):
                    continue
                cnt += 1
                rs += self.f[:, :, q[2], q[1], q[0]].sum(axis=1)
                if self.ns:
                    closed, _ = self._close(self.h, *q)
                    cs += closed.sum(axis=1)
            if cnt:
                new.append(((x, y, z), rs / cnt, cs / cnt))
        for (x, y, z), rbar, cbar in new:
            for s in range(self.nc):
                self.f[s, :, z, y, x] = [self._feq(i, rbar[s], np.zeros(3)) for i in range(len(self.cf))]
            for s in range(self.ns):
                self.h[s, :, z, y, x] = self.wc * cbar[s]
            if self.conj:
                # the new fluid node keeps the temperature its solid had
                self.h[1, :, z, y, x] = self.wc * self.g[:, z, y, x].sum()
                self.g[:, z, y, x] = 0.0
            self.flags[z, y, x] = 0

    def _conduct(self, hpost, hnew):
        """Conduction in the solid and its exchange with the fluid temperature (Sec. 2.1.5, Eq.
        therpop_solid, tempCon, fluxCon, reacRate), pushed: a solid link carries ho out of the
        fluid node and go out of the solid node; both sides get back 2 w T_b minus what they
        sent, with T_b the root of
            (h_in - ho) + (g_in - go) / c_fs = h_r k(T_b) C_b(T_b)
        found by bracketing; C_b closes the species population that has just streamed into the
        fluid node against the wall."""
        from scipy.optimize import brentq
        cfg = self.cfg
        Qc = len(self.cc)
        cfs, taus = float(cfg["c_fs"]), float(cfg["tau_s"])
        A, Ta, hr = float(cfg["arr_A"]), float(cfg["arr_Ta"]), float(cfg["heat_release"])
        tauc = [float(t) for t in cfg.get("tau_c", [1.0, 1.0])]
        fc = tauc[0] / (tauc[0] - 0.5)
        cells = [(x, y, z) for z in range(self.nz) for y in range(self.ny) for x in range(self.nx)]
        solid = [q for q in cells if self.flags[q[2], q[1], q[0]] != 0]
        gpost = np.zeros_like(self.g)
        for (x, y, z) in solid:
            Ts = float(self.g[:, z, y, x].sum())
            gpost[:, z, y, x] = self.g[:, z, y, x] - (self.g[:, z, y, x] - self.wc * Ts) / taus
        gnew = np.zeros_like(self.g)
        for (x, y, z) in solid:
            for j in range(Qc):
                t = self._shift(x, y, z, self.cc[j], self.per_c)
                if t is None:
                    gnew[self.oc[j], z, y, x] = gpost[j, z, y, x]       # closed face: reflected
                elif self.flags[t[2], t[1], t[0]] != 0:
                    gnew[j, t[2], t[1], t[0]] = gpost[j, z, y, x]
        for (x, y, z) in cells:
            if self.flags[z, y, x] != 0:
                continue
            for j in range(1, Qc):
                t = self._shift(x, y, z, self.cc[j], self.per_c)
                if t is None or self.flags[t[2], t[1], t[0]] == 0:
                    continue
                w = self.wc[j]
                ho = hpost[1, j, z, y, x]
                go = gpost[self.oc[j], t[2], t[1], t[0]]
                T0 = (cfs * ho + go) / (w * (cfs + 1))
                Tb = T0
                if self.flags[t[2], t[1], t[0]] == 2:
                    hb = hnew[0, j, z, y, x]

                    def source(T):
                        kk = A * np.exp(-Ta / T)
                        return kk, hr * kk * (2 * hb / (2 * w + kk * fc))

                    def balance(T):
                        return T - (cfs * ho + go + 0.5 * cfs * source(T)[1]) / (w * (cfs + 1))

                    if hr != 0.0:
                        T1 = T0 + 0.5 * cfs * hr * A * (hb / w) / (w * (cfs + 1)) + 1e-9
                        Tb = brentq(balance, T0, T1, xtol=1e-15, rtol=1e-15, maxiter=500)
                    self.kb[(x, y, z, self.oc[j])] = source(Tb)[0]
                hnew[1, self.oc[j], z, y, x] = 2 * w * Tb - ho
                gnew[j, t[2], t[1], t[0]] = 2 * w * Tb - go
        self.g = gnew

    def step(self):
        cfg = self.cfg
        nx, ny, nz = self.nx, self.ny, self.nz
        Qf, Qc = len(self.cf), len(self.cc)
        tau = [float(t) for t in cfg.get("tau", [1.0, 1.0])]
        tauc = [float(t) for t in cfg.get("tau_c", [1.0, 1.0])]
        g = np.array(cfg.get("g", [0, 0, 0]), dtype=float)
        if self.dim == 2:
            g[2] = 0.0
        G = cfg.get("G", [[0, 0], [0, 0]])
        Gads = cfg.get("G_ads", [0, 0])
        k = float(cfg.get("k_react", 0.0))
        nodes = [(x, y, z) for z in range(nz) for y in range(ny) for x in range(nx) if self.flags[z, y, x] == 0]

        # wet-node closure at reactive links, from the stored populations
        hc = self.h.copy()
        if self.ns:
            for (x, y, z) in nodes:
                closed, reactions = self._close(self.h, x, y, z)
                hc[:, :, z, y, x] = closed
                for (src, r) in reactions:
                    self.acc[src[2], src[1], src[0]] += r

        # deposition at near-substrate fluid nodes (Sec. 3.3): C_p,s += DP sum_j h_p,j
        if self.ns and cfg.get("geo_mode", "none") == "deposit":
            DP = float(cfg.get("DP", 0.0))
            for (x, y, z) in nodes:
                near = False
                for j in range(1, Qc):
                    t = self._shift(x, y, z, self.cc[j], self.per_c)
                    if t is None:
                        xt = x + self.cc[j][0]
                        near |= not (cfg.get("ade_open_x", False) and (xt < 0 or xt >= nx))
                    else:
                        near |= self.flags[t[2], t[1], t[0]] != 0
                if near:
                    self.acc[z, y, x] += DP * float(hc[0, :, z, y, x].sum())
                    if cfg.get("deposit_conservative", True):
                        hc[0, :, z, y, x] *= (1.0 - DP)

        # densities, momenta and psi of every fluid node before any force
        rho = {n: [float(self.f[s, :, n[2], n[1], n[0]].sum()) for s in range(self.nc)] for n in nodes}
        mom = {n: [self.cf.T.astype(float) @ self.f[s, :, n[2], n[1], n[0]] for s in range(self.nc)] for n in nodes}
        psi = {n: [self._psi(rho[n][s]) for s in range(self.nc)] for n in nodes}
        psi_w = self._psi(float(cfg.get("rho_solid", 0.0)))
        force, vel = {}, {}
        for n in nodes:
            x, y, z = n
            Fs = []
            for s in range(self.nc):
                F = rho[n][s] * g
                for s2 in range(self.nc):
                    if G[s][s2] == 0:
                        continue
                    acc = np.zeros(3)
                    for i in range(1, Qf):
                        q = self._shift(x, y, z, self.cf[i], self.per_f)
                        p = psi[q][s2] if self._fluid(q) else psi_w
                        acc += self.wf[i] * p * self.cf[i]
                    F = F - psi[n][s] * G[s][s2] * acc
                if Gads[s] != 0:
                    acc = np.zeros(3)
                    for i in range(1, Qf):
                        q = self._shift(x, y, z, self.cf[i], self.per_f)
                        acc += self.wf[i] * (0.0 if self._fluid(q) else 1.0) * self.cf[i]
                    F = F - Gads[s] * rho[n][s] * acc
                Fs.append(F)
            force[n] = Fs
            vel[n] = sum(mom[n][s] + 0.5 * Fs[s] for s in range(self.nc)) / sum(rho[n])

        # collision
        fpost = np.zeros_like(self.f)
        hpost = np.zeros_like(self.h)
        # MRT rates of the run (documented defaults: s_e 1.19, s_eps 1.4, s_q 1.2, s_pi = 1/tau, s_m 1.98)
        mr = cfg.get("mrt_rates", {})
        rate = {"e": mr.get("s_e", 1.19), "eps": mr.get("s_eps", 1.4), "q": mr.get("s_q", 1.2),
                "pi": mr.get("s_pi", 1.0 / tau[0]), "m": mr.get("s_m", 1.98)}
        for n in nodes:
            x, y, z = n
            u = vel[n]
            for s in range(self.nc):
                fv = self.f[s, :, z, y, x]
                if cfg.get("forcing", "guo") == "sc_shift":
                    up = sum(mom[n][t] / tau[t] for t in range(self.nc)) / sum(rho[n][t] / tau[t] for t in range(self.nc))
                    ueq = up + tau[s] * force[n][s] / rho[n][s]
                    fpost[s, :, z, y, x] = [fv[i] - (fv[i] - self._feq(i, rho[n][s], ueq)) / tau[s] for i in range(Qf)]
                elif cfg.get("collision", "bgk") == "mrt":
                    fe = np.array([self._feq(i, rho[n][s], u) for i in range(Qf)])
                    Fi = np.array([self._guo(i, u, force[n][s]) for i in range(Qf)])
                    S = np.array([1.0 / tau[s] if gr in ("c", "nu") else rate[gr] for gr in self.grp])
                    m, me, mF = self.M @ fv, self.M @ fe, self.M @ Fi
                    fpost[s, :, z, y, x] = self.Minv @ (m - S * (m - me) + (1 - S / 2) * mF)
                else:
                    fpost[s, :, z, y, x] = [fv[i] - (fv[i] - self._feq(i, rho[n][s], u)) / tau[s]
                                           + (1 - 1 / (2 * tau[s])) * self._guo(i, u, force[n][s]) for i in range(Qf)]
            cs2 = (1.0 - self.J0) / self.dim   # the scalar lattice's own sound speed (reading 3)
            for s in range(self.ns):
                C = float(hc[s, :, z, y, x].sum())
                for j in range(Qc):
                    heq = self.wc[j] * C * (1 + float(np.dot(self.cc[j], u)) / cs2)
                    hpost[s, j, z, y, x] = hc[s, j, z, y, x] - (hc[s, j, z, y, x] - heq) / self.tau_s_list[s]

        # push streaming with halfway bounce-back, inlet ghost and zero-gradient outlet
        cs2 = (1.0 - self.J0) / self.dim
        fnew = np.zeros_like(self.f)
        hnew = np.zeros_like(self.h)
        for n in nodes:
            x, y, z = n
            for s in range(self.nc):
                for i in range(Qf):
                    t = self._shift(x, y, z, self.cf[i], self.per_f)
                    xt = x + self.cf[i][0]
                    if self._fluid(t):
                        fnew[s, i, t[2], t[1], t[0]] = fpost[s, i, z, y, x]
                    elif t is None and cfg.get("flow_open_x", False) and xt < 0:
                        # velocity inlet: a face moving with u_x = 6 U s (1 - s) reflects f_i
                        sy = (y + 0.5) / ny
                        uin = np.array([6.0 * cfg["u_in"] * sy * (1.0 - sy), 0.0, 0.0])
                        fnew[s, self.of[i], z, y, x] = (fpost[s, i, z, y, x]
                                                        - 2 * self.wf[i] * rho[n][s] * float(np.dot(self.cf[i], uin)) * 3.0)
                    elif t is None and cfg.get("flow_open_x", False) and xt >= nx:
                        # zero-gradient outlet: the entering population repeats the node's own
                        fnew[s, self.of[i], z, y, x] = fpost[s, self.of[i], z, y, x]
                    else:
                        v = fpost[s, i, z, y, x]
                        if t is None and y + self.cf[i][1] >= ny:
                            # Ladd's moving wall: the plate beyond y = ny - 1 moves with u_wall
                            uw = np.array(cfg.get("u_wall_ymax", [0, 0, 0]), dtype=float)
                            v -= 2 * self.wf[i] * rho[n][s] * float(np.dot(self.cf[i], uw)) * 3.0
                        fnew[s, self.of[i], z, y, x] = v
            for s in range(self.ns):
                for j in range(Qc):
                    t = self._shift(x, y, z, self.cc[j], self.per_c)
                    xt = x + self.cc[j][0]
                    if self._fluid(t):
                        hnew[s, j, t[2], t[1], t[0]] = hpost[s, j, z, y, x]
                    elif t is None and cfg.get("ade_open_x", False) and (xt < 0 or xt >= nx):
                        pass   # leaves through an open face
                    else:
                        hnew[s, self.oc[j], z, y, x] = hpost[s, j, z, y, x]
                # populations entering through the open faces
                for j in range(Qc):
                    xs = x - self.cc[j][0]
                    if not cfg.get("ade_open_x", False) or self.cc[j][1] or self.cc[j][2]:
                        continue
                    if xs < 0:
                        C_in = self.cin_list[s]
                        hnew[s, j, z, y, x] = self.wc[j] * C_in * (1 + float(np.dot(self.cc[j], vel[n])) / cs2)
                    elif xs >= nx:
                        hnew[s, j, z, y, x] = hpost[s, j, z, y, x]
        if self.conj:
            self._conduct(hpost, hnew)
        self.f, self.h = fnew, hnew
        self._flips()
        self.t += 1
