"""Seeded synthetic inputs: geometries, initial fields and workload configurations.

This module holds no lattice-Boltzmann arithmetic.  It only draws seeded
geometries (numpy.random.default_rng) and lists parameter sets, so the CUDA
path and the CPU oracle can be fed identical inputs.

Flags: 0 fluid, 1 inert solid, 2 reactive solid.  Arrays are indexed
[z, y, x] (x fastest in memory); 2D arrays have a leading z axis of length 1.

The paper's own geometries (the FIB-SEM pore image of Sec. 3.3 and the
four-obstacle combustion channel of Sec. 3.4 with its literature data) are not
available, so seeded stand-ins with the workloads' sizes and porosities are
used instead.
"""
from __future__ import annotations

import numpy as np

FLUID, SOLID, REACTIVE = 0, 1, 2


def circles_2d(nx: int, ny: int, n_circles: int = 12, r_min: int = 4, r_max: int = 8,
               x_margin: int = 8, seed: int = 0, flag: int = REACTIVE) -> np.ndarray:
    """Seeded circular obstacles; radius uniform integer in [r_min, r_max], centres
    uniform with x kept `x_margin` + r away from the inlet/outlet faces, periodic
    wrap in y.  Overlaps are allowed."""
    rng = np.random.default_rng(seed)
    g = np.zeros((1, ny, nx), dtype=np.uint8)
    yy, xx = np.mgrid[0:ny, 0:nx]
    for _ in range(n_circles):
        r = int(rng.integers(r_min, r_max + 1))
        lo, hi = x_margin + r, nx - 1 - x_margin - r
        cx = float(rng.uniform(lo, hi)) if hi > lo else nx / 2.0
        cy = float(rng.uniform(0, ny))
        dy = np.abs(yy - cy)
        dy = np.minimum(dy, ny - dy)
        g[0][(xx - cx) ** 2 + dy ** 2 <= r * r] = flag
    return g


def sphere_packing_3d(n: int, r_min: float = 6.0, r_max: float = 12.0, solid_fraction: float = 0.6,
                      seed: int = 0, flag: int = REACTIVE, shape=None, max_spheres: int = 1_000_000
                      ) -> np.ndarray:
    """Boolean random-sphere packing: radius uniform real in [r_min, r_max],
    centres uniform, periodic wrap; spheres are added until the solid fraction
    reaches `solid_fraction`.  `shape` (nz, ny, nx) overrides the cube n^3."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape if shape is not None else (n, n, n)
    solid = np.zeros((nz, ny, nx), dtype=bool)
    total = solid.size
    n_solid = 0
    count = 0
    while n_solid < solid_fraction * total and count < max_spheres:
        r = float(rng.uniform(r_min, r_max))
        c = rng.uniform(0, 1, size=3) * np.array([nz, ny, nx])
        R = int(np.ceil(r))
        offs = np.arange(-R, R + 1)
        dz, dy, dx = np.meshgrid(offs, offs, offs, indexing="ij")
        iz = np.floor(c[0]).astype(int) + dz
        iy = np.floor(c[1]).astype(int) + dy
        ix = np.floor(c[2]).astype(int) + dx
        d2 = (iz + 0.5 - c[0]) ** 2 + (iy + 0.5 - c[1]) ** 2 + (ix + 0.5 - c[2]) ** 2
        m = d2 <= r * r
        idx = (iz[m] % nz, iy[m] % ny, ix[m] % nx)
        n_solid += int(np.count_nonzero(~solid[idx]))
        solid[idx] = True
        count += 1
    g = np.zeros((nz, ny, nx), dtype=np.uint8)
    g[solid] = flag
    return g


def random_solids(shape, fraction: float, seed: int = 0, reactive_fraction: float = 0.5) -> np.ndarray:
    """Independent random solid nodes (small parity cases), a mix of inert and reactive."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(size=shape)
    g = np.zeros(shape, dtype=np.uint8)
    s = u < fraction
    g[s] = SOLID
    g[s & (rng.uniform(size=shape) < reactive_fraction)] = REACTIVE
    return g


def droplet_fields(shape, radius: float, rho_in: float = 1.0, rho_out: float = 0.05):
    """Sharp spherical (or circular) droplet of component 0 centred in the box;
    component 1 fills the rest; zero velocity."""
    nz, ny, nx = shape
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    cz = nz / 2.0 if nz > 1 else 0.0
    d2 = (xx - nx / 2.0) ** 2 + (yy - ny / 2.0) ** 2 + ((zz - cz) ** 2 if nz > 1 else 0.0)
    inside = d2 < radius * radius
    rho = np.empty((2,) + tuple(shape))
    rho[0] = np.where(inside, rho_in, rho_out)
    rho[1] = np.where(inside, rho_out, rho_in)
    u = np.zeros((3,) + tuple(shape))
    return rho, u


def sessile_droplet_2d(nx=200, ny=80, radius=30.0, G=2.7, g_ads=0.0, precision="fp32", rho_solid=0.0):
    """Two-component Shan-Chen sessile droplet for the contact angle (Sec. 3.2, contact angle):
    a half disc of component 0 (density 1.0, 0.05 of component 1) centred on the bottom wall
    (the halfway face y = -1/2 of a closed y axis), component 1 elsewhere; psi = rho, cross
    cohesion G, adhesion G_ads = (g, -g), periodic x, tau 1.  Solid nodes carry
    psi(rho_solid) in the cohesion sums (0: the wall interacts through G_ads alone)."""
    cfg = dict(dim=2, nx=nx, ny=ny, nz=1, n_comp=2, tau=[1.0, 1.0], G=[[0.0, G], [G, 0.0]],
               psi_kind="identity", G_ads=[g_ads, -g_ads], periodic=[1, 0, 1], precision=precision,
               rho_solid=rho_solid)
    yy, xx = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    inside = (xx - nx / 2.0) ** 2 + (yy + 0.5) ** 2 < radius * radius
    rho = np.empty((2, 1, ny, nx))
    rho[0, 0] = np.where(inside, 1.0, 0.05)
    rho[1, 0] = np.where(inside, 0.05, 1.0)
    return cfg, np.zeros((1, ny, nx), np.uint8), (rho, np.zeros((3, 1, ny, nx)), None)


def uniform_fields(shape, n_comp: int = 1, n_scal: int = 0, rho=1.0, C=0.0, u=(0.0, 0.0, 0.0)):
    rho_a = np.empty((n_comp,) + tuple(shape))
    for s in range(n_comp):
        rho_a[s] = rho[s] if np.ndim(rho) else rho
    u_a = np.empty((3,) + tuple(shape))
    for a in range(3):
        u_a[a] = u[a]
    C_a = np.empty((n_scal,) + tuple(shape))
    for s in range(n_scal):
        C_a[s] = C[s] if np.ndim(C) else C
    return rho_a, u_a, C_a


def perturbed_fields(shape, n_comp: int, n_scal: int, seed: int, amp_rho: float = 1e-3,
                     amp_u: float = 1e-3, amp_C: float = 0.1, rho0=1.0, C0=0.5):
    """Smooth-ish seeded random initial fields for parity tests."""
    rng = np.random.default_rng(seed)
    rho = np.empty((n_comp,) + tuple(shape))
    for s in range(n_comp):
        base = rho0[s] if np.ndim(rho0) else rho0
        rho[s] = base * (1.0 + amp_rho * rng.uniform(-1, 1, size=shape))
    u = amp_u * rng.uniform(-1, 1, size=(3,) + tuple(shape))
    if shape[0] == 1:
        u[2] = 0.0
    C = np.empty((n_scal,) + tuple(shape))
    for s in range(n_scal):
        C[s] = C0 * (1.0 + amp_C * rng.uniform(-1, 1, size=shape))
    return rho, u, C


# --------------------------------------------------------------- workloads
# Plain parameter sets; keys are read by both the CUDA binding and the oracle.

def reactive_channel_2d(nx=128, ny=64, seed=0, precision="fp64"):
    """2D reactive channel: D2Q9 BGK (tau 0.8) driven by body force 1e-6, 12 seeded
    reactive circles (radius 4-8), D2Q5 solute (tau_c 0.7, J0 0.4), inlet C = 1,
    zero-gradient outlet, initial C = 0, k = 1e-3, periodic flow."""
    cfg = dict(dim=2, nx=nx, ny=ny, nz=1, n_comp=1, tau=[0.8], g=[1e-6, 0.0, 0.0],
               collision="bgk", forcing="guo", n_scal=1, tau_c=[0.7], J0=0.4, k_react=1e-3,
               ade_open_x=True, C_in=[1.0], periodic=[1, 1, 1], geo_mode="none",
               precision=precision)
    geom = circles_2d(nx, ny, 12, 4, 8, 8, seed)
    rho, u, C = uniform_fields((1, ny, nx), 1, 1, rho=1.0, C=0.0)
    return cfg, geom, (rho, u, C)


def combustion_channel_2d(nx=420, ny=80, n_obstacles=4, radius=None, precision="fp64"):
    """Stand-in for the reactive porous channel of Sec. 3.4 (Xu et al.'s set-up, whose exact
    geometry is not in the text): a channel of nx x ny nodes with no-slip walls at y = -1/2 and
    ny - 1/2, the parabolic velocity inlet at x = 0 and zero-gradient outlets for every field;
    n_obstacles reactive carbon discs of radius ny/8 (default) on the centre line, evenly spaced
    in the middle three fifths.  O2 (scalar 0) enters at 0.22, CO2 (the product) at 0, and the
    fluid at the temperature 1; the solid starts at 1 too.  Lattice parameters: D2Q9 BGK
    tau 0.8, D2Q5 J0 0.4; tau_O2 0.8, tau_T 0.9, tau_CO2 0.75, tau_s 0.7, c_fs 0.5; with L the
    disc diameter, U the mean inlet velocity and D the O2 diffusivity, Pe = U L / D = 1e-2 and
    Da = k(1) L / D = 3.525e-2 at the inlet temperature (Sec. 3.4), k(T) = A exp(-Ta / T) with
    Ta = 8, and the heat release h_r = 2."""
    r = int(radius if radius is not None else max(2, ny // 8))
    g = np.zeros((1, ny, nx), dtype=np.uint8)
    yy, xx = np.mgrid[0:ny, 0:nx]
    cy = (ny - 1) / 2.0
    for k in range(n_obstacles):
        cx = nx * (0.2 + 0.6 * (k + 0.5) / n_obstacles)
        g[0][(xx - cx) ** 2 + (yy - cy) ** 2 <= r * r] = REACTIVE
    L = 2.0 * r
    D = 0.3 * (0.8 - 0.5)
    U = 1e-2 * D / L
    k_in = 3.525e-2 * D / L
    Ta = 8.0
    cfg = dict(dim=2, nx=nx, ny=ny, nz=1, n_comp=1, tau=[0.8], g=[0.0, 0.0, 0.0], collision="bgk",
               forcing="guo", flow_open_x=True, u_in=U, periodic=[0, 0, 1], n_scal=2,
               tau_c=[0.8, 0.9], J0=0.4, ade_open_x=True, C_in=[0.22, 1.0], arrhenius=True,
               arr_A=k_in * float(np.exp(Ta)), arr_Ta=Ta, heat_release=2.0, n_it=24,
               conjugate=True, tau_s=0.7, c_fs=0.5, product=True, tau_p=0.75, C_in_p=0.0,
               geo_mode="none", precision=precision)
    rho, u, _ = uniform_fields((1, ny, nx), 1, 0)
    C = np.zeros((3, 1, ny, nx))
    C[1] = 1.0
    return cfg, g, (rho, u, C)


def droplet_3d(n=128, radius=16.0, precision="fp32", G=2.7):
    """3D two-component Shan-Chen static droplet: D3Q19 per component, psi = rho,
    cross-cohesion G (0.9 in the w_i/c_s^2 convention = 2.7 in Eq. 1.14's w_i
    convention), densities 1.0 / 0.05, tau 1, periodic."""
    cfg = dict(dim=3, nx=n, ny=n, nz=n, n_comp=2, tau=[1.0, 1.0], G=[[0.0, G], [G, 0.0]],
               psi_kind="identity", collision="bgk", forcing="guo", n_scal=0,
               periodic=[1, 1, 1], geo_mode="none", precision=precision)
    geom = np.zeros((n, n, n), dtype=np.uint8)
    rho, u = droplet_fields((n, n, n), radius)
    return cfg, geom, (rho, u, np.zeros((0, n, n, n)))


# Config-3 transport parameters: tau = 1 (nu = 1/6), J0 = 1/4 (c_s^2 = 1/4 on D3Q7),
# characteristic length L = 9 (mean sphere radius), target Re ~ 1, Pe ~ 10, Da ~ 0.1:
# U ~ Re nu / L = 0.0185, D = U L / Pe = 0.0167, tau_c = D / c_s^2 + 1/2 = 0.5667,
# k = Da D / L = 1.85e-4.  The body force below gives U ~ 0.0185 (mean fluid speed) on
# the seed-0 256^3 packing (calibrated once on the GPU and frozen).
DISSOLUTION_G = 2.2e-4


def dissolution_3d(n=256, seed=0, precision="fp32", shape=None, g=None, radius=(6.0, 12.0)):
    """3D reactive dissolution in a random-sphere packing: D3Q19 MRT (tau 1) flow by
    body force + D3Q7 solute, first-order reaction at reactive links consuming solid mass,
    inlet C = 1 at x = 0, zero-gradient outlet, periodic flow.  Small test domains pass a
    proportionally smaller sphere radius range."""
    shp = shape if shape is not None else (n, n, n)
    cfg = dict(dim=3, nx=shp[2], ny=shp[1], nz=shp[0], n_comp=1, tau=[1.0],
               g=[DISSOLUTION_G if g is None else g, 0.0, 0.0], collision="mrt", forcing="guo",
               n_scal=1, tau_c=[0.5667], J0=0.25, k_react=1.85e-4, ade_open_x=True,
               C_in=[1.0], periodic=[1, 1, 1], geo_mode="dissolve", V_m=1.0, m_s0=1.0,
               C_ref=[1.0], precision=precision)
    geom = sphere_packing_3d(n, radius[0], radius[1], 0.6, seed, REACTIVE, shape=shp)
    rho, u, C = uniform_fields(shp, 1, 1, rho=1.0, C=1.0)
    return cfg, geom, (rho, u, C)


def circle_packing_2d(nx: int, ny: int, r_min: int = 4, r_max: int = 8, solid_fraction: float = 0.5,
                      seed: int = 0, flag: int = REACTIVE, max_circles: int = 1_000_000) -> np.ndarray:
    """Boolean random-circle packing: radius uniform integer in [r_min, r_max], centres
    uniform, periodic wrap; circles are added until the solid fraction is reached."""
    rng = np.random.default_rng(seed)
    solid = np.zeros((ny, nx), dtype=bool)
    n_solid, count = 0, 0
    while n_solid < solid_fraction * solid.size and count < max_circles:
        r = int(rng.integers(r_min, r_max + 1))
        cy, cx = rng.uniform(0, 1, size=2) * np.array([ny, nx])
        offs = np.arange(-r, r + 1)
        dy, dx = np.meshgrid(offs, offs, indexing="ij")
        iy = np.floor(cy).astype(int) + dy
        ix = np.floor(cx).astype(int) + dx
        m = (iy + 0.5 - cy) ** 2 + (ix + 0.5 - cx) ** 2 <= r * r
        idx = (iy[m] % ny, ix[m] % nx)
        n_solid += int(np.count_nonzero(~solid[idx]))
        solid[idx] = True
        count += 1
    g = np.zeros((1, ny, nx), dtype=np.uint8)
    g[0][solid] = flag
    return g


def ensemble_members(n2d: int, n3d: int, seed0: int = 0, side_2d=(64, 512), side_3d=(64, 160),
                     porosity=(0.35, 0.7), precision="fp16"):
    """Uneven ensemble of steady-state flow + solute runs: n2d square 2D domains (side uniform
    integer in side_2d, circles of radius 4-8) and n3d cubic 3D domains (side uniform in
    side_3d, spheres of radius 6-12), porosity uniform in `porosity`, member k seeded with
    seed0 + k.  Transport parameters of the reactive channel (2D) and the dissolution case (3D);
    the geometry stays fixed.  Returns (list_2d, list_3d) of (cfg, geom, fields)."""
    out2, out3 = [], []
    for k in range(n2d + n3d):
        rng = np.random.default_rng(seed0 + k)
        phi = float(rng.uniform(*porosity))
        if k < n2d:
            s = int(rng.integers(side_2d[0], side_2d[1] + 1))
            geom = circle_packing_2d(s, s, 4, 8, 1.0 - phi, seed0 + k)
            cfg = dict(dim=2, nx=s, ny=s, nz=1, n_comp=1, tau=[0.8], g=[1e-5, 0.0, 0.0], collision="bgk",
                       forcing="guo", n_scal=1, tau_c=[0.7], J0=0.4, k_react=1e-3, ade_open_x=True,
                       C_in=[1.0], periodic=[1, 1, 1], geo_mode="none", C_ref=[1.0], precision=precision)
            out2.append((cfg, geom, uniform_fields(geom.shape, 1, 1, rho=1.0, C=1.0)))
        else:
            s = int(rng.integers(side_3d[0], side_3d[1] + 1))
            geom = sphere_packing_3d(s, 6.0, 12.0, 1.0 - phi, seed0 + k, REACTIVE)
            cfg = dict(dim=3, nx=s, ny=s, nz=s, n_comp=1, tau=[1.0], g=[DISSOLUTION_G, 0.0, 0.0],
                       collision="mrt", forcing="guo", n_scal=1, tau_c=[0.5667], J0=0.25, k_react=1.85e-4,
                       ade_open_x=True, C_in=[1.0], periodic=[1, 1, 1], geo_mode="none", C_ref=[1.0],
                       precision=precision)
            out3.append((cfg, geom, uniform_fields(geom.shape, 1, 1, rho=1.0, C=1.0)))
    return out2, out3
