"""Seeded synthetic inputs shaped like the paper's cases.

This module generates inputs only (geometry masks, inlet profiles, rate
fields and the lattice parameters a case is run with).  It holds none of the
time step's arithmetic, so the CUDA path and the CPU oracle can both be fed
from it.  All randomness is numpy's PCG64 seeded explicitly.

Mask convention (uint8, indexed [z, y, x], x fastest):
  0 fluid, 1 reactive solid, 2 Dirichlet solid (fixed concentration).

Cases (sizes are the arguments' defaults):
* ``reactive_wall_1d`` -- 2D strip with a reactive wall row and a Dirichlet
  row (steady reaction-diffusion toward a flat wall).
* ``tilted_channel`` -- 3D slab channel whose walls are tilted about x by
  theta against the grid, with a plane-Poiseuille inlet profile.
* ``sphere_pack`` -- Boolean model of overlapping spheres with radii uniform
  in [r_min, r_max], added until the porosity reaches the target.
* ``annulus`` -- 2D reactive disk inside a Dirichlet circle.
* ``lognormal_k`` -- per-voxel rate k_bar exp(sigma Z - sigma^2 / 2).
* ``case_molins`` -- 2D reactive disc in a channel flow (Sec. 3.3, Table 2).
* ``case_grain_2d`` -- 2D grain growth by precipitation from a star-shaped
  seed inside a circle of fixed concentration (Sec. 3.2).
"""
from __future__ import annotations

import math

import numpy as np

FLUID, REACTIVE, DIRICHLET = 0, 1, 2


def lattice_cs2(q: int, dim: int, rest_fraction: float = -1.0) -> float:
    """Speed of sound squared the case recipes assume for a lattice: 1/3 for
    D2Q9 / D3Q19 / D2Q5, (1 - J0) / dim with a rest fraction J0, and 1/4 for
    D3Q7 without one."""
    if rest_fraction >= 0.0:
        return (1.0 - rest_fraction) / dim
    if dim == 3 and q == 7:
        return 0.25
    return 1.0 / 3.0


def params_from_dimensionless(*, Re=None, Pe=None, Da=None, PeDa=None, L, U, tau_flow=None, tau_solute=None,
                              rest_fraction=None, solute_q=7, dim=3):
    """Lattice parameters for target Re, Pe, Da (Eq. PeDa: Re = U L / nu,
    Pe = U L / D, Da = k_r / U, PeDa = k_r L / D).

    Given tau_flow, Re fixes U (returned as ``U``) unless U is given.  Given
    tau_solute and Pe, the rest fraction J0 is chosen so that
    D = cs^2(J0) (tau_solute - 1/2); given rest_fraction instead, tau_solute
    follows.  k_r comes from Da (k_r = Da U) or PeDa (k_r = PeDa D / L)."""
    out = {}
    if Re is not None and tau_flow is not None:
        nu = (tau_flow - 0.5) / 3.0
        if U is None:
            U = Re * nu / L
        out["tau_flow"] = tau_flow
    out["U"] = U
    D = None
    if Pe is not None:
        D = U * L / Pe
        if rest_fraction is not None and rest_fraction >= 0.0:
            cs2 = lattice_cs2(solute_q, dim, rest_fraction)
            out["tau_solute"] = 0.5 + D / cs2
            out["rest_fraction"] = rest_fraction
        elif tau_solute is not None:
            cs2 = D / (tau_solute - 0.5)
            out["rest_fraction"] = 1.0 - dim * cs2
            out["tau_solute"] = tau_solute
    elif tau_solute is not None:
        cs2 = lattice_cs2(solute_q, dim, -1.0 if rest_fraction is None else rest_fraction)
        D = cs2 * (tau_solute - 0.5)
        out["tau_solute"] = tau_solute
        out["rest_fraction"] = -1.0 if rest_fraction is None else rest_fraction
    out["D"] = D
    if Da is not None:
        out["k_r"] = Da * U
    elif PeDa is not None and D is not None:
        out["k_r"] = PeDa * D / L
    return out


# ---------------------------------------------------------------------------
# Geometries
# ---------------------------------------------------------------------------
def reactive_wall_1d(nx: int = 128, ny: int = 64):
    """Row y = 0 reactive solid, row y = ny-1 Dirichlet solid, fluid between
    (periodic in x).  Distance wall-to-Dirichlet node centres: ny - 1."""
    m = np.zeros((1, ny, nx), np.uint8)
    m[0, 0, :] = REACTIVE
    m[0, ny - 1, :] = DIRICHLET
    return m


def reactive_wall_3d(nx: int = 2, ny: int = 32, nz: int = 2):
    m = np.zeros((nz, ny, nx), np.uint8)
    m[:, 0, :] = REACTIVE
    m[:, ny - 1, :] = DIRICHLET
    return m


def tilted_channel(nx: int = 256, ny: int = 128, nz: int = 128, h: float = 32.0, theta_deg: float = 0.0,
                   u_max: float = 0.0):
    """Slab channel of half-width h whose mid-plane passes through the box
    centre and is tilted about x by theta.  A node is solid when its distance
    to the mid-plane exceeds h; the four box faces normal to y and z are
    solid.  Returns (mask, inlet_ux[nz, ny]) with the plane-Poiseuille
    profile u_max (1 - (d/h)^2) on fluid inlet nodes."""
    th = math.radians(theta_deg)
    z, y = np.meshgrid(np.arange(nz, dtype=np.float64), np.arange(ny, dtype=np.float64), indexing="ij")
    d = (y - (ny - 1) / 2.0) * math.cos(th) + (z - (nz - 1) / 2.0) * math.sin(th)
    solid2d = np.abs(d) > h
    solid2d[:, 0] = solid2d[:, -1] = True
    solid2d[0, :] = solid2d[-1, :] = True
    mask = np.broadcast_to(solid2d[:, :, None], (nz, ny, nx)).astype(np.uint8) * REACTIVE
    inlet = np.where(solid2d, 0.0, u_max * (1.0 - (d / h) ** 2))
    return np.ascontiguousarray(mask), np.ascontiguousarray(inlet)


def sphere_pack(shape, porosity: float = 0.4, r_min: float = 8.0, r_max: float = 16.0, seed: int = 0,
                periodic=(False, True, True), buffer_x: int = 0, batch: int = 64):
    """Boolean model: spheres with radii ~ U[r_min, r_max] and uniform
    centres are added in small batches until the pore fraction (outside the
    x buffers) is <= porosity.  ``periodic`` (x, y, z) wraps spheres across
    those faces; ``buffer_x`` layers at both x ends stay fluid.  Returns a
    uint8 mask with REACTIVE for solid."""
    nz, ny, nx = shape
    rng = np.random.default_rng(seed)
    solid = np.zeros(shape, dtype=bool)
    core = (slice(None), slice(None), slice(buffer_x, nx - buffer_x if buffer_x else nx))
    ncore = solid[core].size
    n = np.array([nx, ny, nz])
    while True:
        for _ in range(batch):
            r = rng.uniform(r_min, r_max)
            c = rng.uniform(0, 1, 3) * n
            lo = np.floor(c - r).astype(int)
            hi = np.floor(c + r).astype(int) + 1
            ax = []
            for a in range(3):
                idx = np.arange(lo[a], hi[a])
                if periodic[a]:
                    ax.append((idx, idx % n[a]))
                else:
                    keep = (idx >= 0) & (idx < n[a])
                    ax.append((idx[keep], idx[keep]))
            dx = (ax[0][0] + 0.5 - c[0]) ** 2
            dy = (ax[1][0] + 0.5 - c[1]) ** 2
            dz = (ax[2][0] + 0.5 - c[2]) ** 2
            inside = dz[:, None, None] + dy[None, :, None] + dx[None, None, :] <= r * r
            zz, yy, xx = np.ix_(ax[2][1], ax[1][1], ax[0][1])
            solid[zz, yy, xx] |= inside
        if buffer_x:
            solid[:, :, :buffer_x] = False
            solid[:, :, nx - buffer_x:] = False
        if 1.0 - solid[core].sum() / ncore <= porosity:
            break
    return solid.astype(np.uint8) * REACTIVE


def annulus(n: int = 72, R: float = 12.0, R2: float = 32.0, offset: float = 0.3):
    """2D reactive disk of radius R inside a Dirichlet circle of radius R2,
    centred at ((n-1)/2 + offset) in x and y."""
    yy, xx = np.mgrid[0:n, 0:n].astype(np.float64)
    c = (n - 1) / 2.0 + offset
    r = np.hypot(xx - c, yy - c)
    m = np.zeros((1, n, n), np.uint8)
    m[0][r <= R] = REACTIVE
    m[0][r >= R2] = DIRICHLET
    return m, c


def lognormal_k(shape, k_bar: float, sigma: float = 0.5, seed: int = 0):
    """Per-voxel rate field k_bar * exp(sigma Z - sigma^2/2), Z ~ N(0, 1)."""
    rng = np.random.default_rng(seed)
    return k_bar * np.exp(sigma * rng.standard_normal(shape) - 0.5 * sigma * sigma)


# ---------------------------------------------------------------------------
# Named cases (geometry + lattice parameters), recipes stated in the docs.
# ---------------------------------------------------------------------------
def case_wall_2d(nx: int = 128, ny: int = 64, tau: float = 0.8, scheme: str = "new", solute_q: int = 9):
    """2D pure diffusion toward a flat reactive wall: D2Q9 (or D2Q5) solute
    lattice, no flow, c = 1 on the Dirichlet row y = ny-1, c_eq = 0, and
    PeDa = k_r (ny-1) / D = 1."""
    mask = reactive_wall_1d(nx, ny)
    D = (tau - 0.5) / 3.0
    p = dict(dim=2, nx=nx, ny=ny, nz=1, flow_q=0, solute_q=solute_q, bc=("periodic", "wall", "periodic"),
             tau_solute=tau, magic_solute=-1.0, rest_fraction=-1.0, k_r=D / (ny - 1), c_eq=0.0,
             c_dirichlet=1.0, c_init=0.0, scheme=scheme, molar_volume=1.0)
    return p, mask, {}


def case_channel(nx: int = 256, ny: int = 128, nz: int = 128, theta_deg: float = 30.0, Pe: float = 10.0,
                 Da: float = 1.0, h: float = 32.0, tau_flow: float = 0.8, tau_solute: float = 1.0,
                 scheme: str = "new"):
    """3D tilted channel with flow: D3Q19 TRT (Lambda = 3/16) flow at
    Re = u_mean * 2h / nu = 1, D3Q7 BGK solute with the rest fraction chosen
    for Pe = u_mean 2h / D at tau_solute (lowered to keep u_max <= cs^2),
    Da = k_r / u_mean, inlet c = 1, c_eq = 0.5."""
    L = 2.0 * h
    nu = (tau_flow - 0.5) / 3.0
    u_mean = 1.0 * nu / L
    u_max = 1.5 * u_mean
    D = u_mean * L / Pe
    # positivity of the linear solute equilibrium needs u_max <= cs^2
    cs2 = D / (tau_solute - 0.5)
    while cs2 < 1.05 * u_max and tau_solute > 0.52:
        tau_solute -= 0.01
        cs2 = D / (tau_solute - 0.5)
    J0 = 1.0 - 3.0 * cs2
    mask, inlet = tilted_channel(nx, ny, nz, h, theta_deg, u_max)
    p = dict(dim=3, nx=nx, ny=ny, nz=nz, flow_q=19, solute_q=7, bc=("open", "wall", "wall"),
             tau_flow=tau_flow, magic_flow=3.0 / 16.0, tau_solute=tau_solute, magic_solute=-1.0,
             rest_fraction=J0, k_r=Da * u_mean, c_eq=0.5, c_init=1.0, c_inlet=1.0, rho_outlet=1.0,
             u_inlet=0.0, molar_volume=1.0, scheme=scheme)
    return p, mask, dict(inlet_ux=inlet)


def case_sphere_pack(n: int = 512, porosity: float = 0.4, seed: int = 2306, tau_flow: float = 0.8,
                     Re: float = 0.1, Pe: float = 100.0, tau_solute: float = 1.0, buffer_x: int = 8,
                     molar_volume: float = 0.1, phase_change: int = 1, c_eq: float = 1.0):
    """3D precipitation in a seeded sphere pack: porosity 0.4, radii U[8,16],
    periodic in y and z, 8 fluid layers at both x ends, plug inlet giving
    Re = U d_mean / nu (d_mean = 24), supersaturated inlet c = 2 c_eq."""
    mask = sphere_pack((n, n, n), porosity, 8.0, 16.0, seed, (False, True, True), buffer_x)
    L = 24.0
    nu = (tau_flow - 0.5) / 3.0
    U = Re * nu / L
    D = U * L / Pe
    cs2 = D / (tau_solute - 0.5)
    while cs2 < 1.05 * 3.0 * U and tau_solute > 0.52:
        tau_solute -= 0.01
        cs2 = D / (tau_solute - 0.5)
    J0 = 1.0 - 3.0 * cs2
    p = dict(dim=3, nx=n, ny=n, nz=n, flow_q=19, solute_q=7, bc=("open", "periodic", "periodic"),
             tau_flow=tau_flow, magic_flow=3.0 / 16.0, tau_solute=tau_solute, magic_solute=-1.0,
             rest_fraction=J0, k_r=1.0 * U, c_eq=c_eq, c_init=c_eq, c_inlet=2.0 * c_eq, u_inlet=U,
             rho_outlet=1.0, molar_volume=molar_volume, phase_change=phase_change, scheme="new")
    return p, mask, {}


def case_batch(n: int = 256, L_min: int = 32, L_max: int = 96, seed: int = 2310, precision: str = "fp32"):
    """Independent 3D dissolution domains of uneven size: cubic edge L ~
    U{L_min..L_max}, seeded Boolean sphere pack with porosity ~ U[0.3, 0.6]
    and radii ~ U[L/12, L/6], periodic in y and z with 3 fluid layers at the
    open x ends, D3Q19 TRT flow (plug inlet, Re = 1 on the mean grain
    diameter), D3Q7 TRT solute with Pe ~ log-U[1, 1000] (capped where the
    lattice cannot reach it with tau >= 0.51 and u_max <= cs^2) via the rest
    fraction, Da ~ log-U[0.01, 10], undersaturated inlet c = 0 against
    c_eq = 1.  Returns a list of (params, mask, init) and the per-domain
    (L, porosity, Pe, Da) actually used."""
    rng = np.random.default_rng(seed)
    out, meta = [], []
    for i in range(n):
        L = int(rng.integers(L_min, L_max + 1))
        por = rng.uniform(0.3, 0.6)
        r_lo, r_hi = L / 12.0, L / 6.0
        mask = sphere_pack((L, L, L), por, r_lo, r_hi, seed=seed * 1000 + i, periodic=(False, True, True),
                           buffer_x=3)
        d = (r_lo + r_hi)  # mean grain diameter
        tau_f = 0.8
        nu = (tau_f - 0.5) / 3.0
        U = 1.0 * nu / d
        Pe = float(np.exp(rng.uniform(np.log(1.0), np.log(1000.0))))
        Da = float(np.exp(rng.uniform(np.log(0.01), np.log(10.0))))
        # reachable Pe: cs^2 >= 3 U (u_max) and tau_solute >= 0.51 -> D >= 0.03 U
        Pe = min(Pe, U * d / (0.03 * U))
        D = U * d / Pe
        tau_s = 1.0
        cs2 = D / (tau_s - 0.5)
        while cs2 < 3.0 * U and tau_s > 0.51:
            tau_s = max(0.51, tau_s - 0.01)
            cs2 = D / (tau_s - 0.5)
        cs2 = min(cs2, 1.0 / 3.0)
        J0 = max(0.0, 1.0 - 3.0 * cs2)
        p = dict(dim=3, nx=L, ny=L, nz=L, flow_q=19, solute_q=7, bc=("open", "periodic", "periodic"),
                 tau_flow=tau_f, magic_flow=3.0 / 16.0, tau_solute=tau_s, magic_solute=0.25, rest_fraction=J0,
                 k_r=Da * U, c_eq=1.0, c_init=0.0, c_inlet=0.0, u_inlet=U, rho_outlet=1.0, molar_volume=0.1,
                 phase_change=0, precision=precision, scheme="new")
        out.append((p, mask, {}))
        meta.append(dict(L=L, porosity=float((mask == 0).mean()), Pe=Pe, Da=Da))
    return out, meta


def case_rect_2d(config: str = "A", peda: float = 1.0, scheme: str = "new", a: float = 100.0, b: float = 80.0,
                 D: float = 0.08, rest_fraction: float = -1.0, magic: float = -1.0, c0: float = 1.0,
                 precision: str = "fp64"):
    """2D reaction-diffusion verification rectangle (D2Q5, no flow): constant
    c0 on the left edge, zero gradient on the right and bottom edges, the
    reactive wall (c_eq = 0, k_r from PeDa = k_r b_e / D) on top.  Config A
    is aligned with the grid, config B rotated by 45 degrees.

    Lattice placement (wet-node boundaries): the Dirichlet cells lie on
    xi = 0 and the reactive cells on eta = b_e, the inert bounce-back walls
    half a cell beyond the last fluid cells, so the effective rectangle is
    a_e = a + 1/2 by b_e = b + 1/2.  Returns (params, mask, init, geom) where
    geom = dict(xi, eta, a_e, b_e, fluid) maps every cell to the rectangle's
    frame for evaluating the analytical solution."""
    ae, be = a + 0.5, b + 0.5
    if config == "A":
        nx, ny = int(a) + 2, int(b) + 1
        yy, xx = np.mgrid[0:ny, 0:nx].astype(np.float64)
        xi, eta = xx, yy + 0.5
        mask = np.full((ny, nx), REACTIVE, np.uint8)
        fluid = (xx >= 1) & (xx <= a) & (yy <= b - 1)
        mask[fluid] = FLUID
        mask[:, 0] = DIRICHLET
        inert = (mask == REACTIVE) & ~(yy == b)
    else:
        n = int(math.ceil((ae + be) / math.sqrt(2.0))) + 6
        nx = ny = n
        yy, xx = np.mgrid[0:ny, 0:nx].astype(np.float64)
        c = (n - 1) / 2.0
        # rectangle centre at the grid centre; xi along (1,1)/sqrt2, eta along (-1,1)/sqrt2
        xi = ((xx - c) + (yy - c)) / math.sqrt(2.0) + ae / 2.0
        eta = (-(xx - c) + (yy - c)) / math.sqrt(2.0) + be / 2.0
        fluid = (xi > 0) & (xi < ae) & (eta > 0) & (eta < be)
        mask = np.full((ny, nx), REACTIVE, np.uint8)
        mask[fluid] = FLUID
        mask[(~fluid) & (xi <= 0)] = DIRICHLET
        inert = (mask == REACTIVE) & ~(eta >= be)
    k_r = peda * D / be
    kf = np.where(inert, 0.0, k_r)[None]
    tau = 0.5 + D / lattice_cs2(5, 2, rest_fraction)
    p = dict(dim=2, nx=nx, ny=ny, nz=1, flow_q=0, solute_q=5, bc=("wall", "wall", "periodic"), tau_solute=tau,
             magic_solute=magic, rest_fraction=rest_fraction, k_r=k_r, c_eq=0.0, c_dirichlet=c0, c_init=c0,
             molar_volume=1.0, scheme=scheme, precision=precision)
    geom = dict(xi=xi[None], eta=eta[None], a_e=ae, b_e=be, fluid=fluid[None])
    return p, mask[None], dict(k_field=kf), geom


# Sec. 3.3 / Table 2: (Pe, Da) of the four cases and the rest fraction the
# paper uses for each Pe.
MOLINS_CASES = {1: (600.0, 178.0), 2: (600.0, 17800.0), 3: (6.0, 178.0), 4: (6.0, 0.178)}
MOLINS_J0 = {600.0: 0.99, 6.0: 1.0 / 3.0}


def case_molins(case: int = 4, scheme: str = "new", scale: float = 1.0, magic_flow: float = 3.0 / 16.0,
                magic_solute: float = 0.25, precision: str = "fp32"):
    """2D reactive disc in a channel flow (Sec. 3.3): channel H x W = 600 x
    1200 cells at scale 1 (0.05 cm x 0.1 cm), disc of diameter 240 cells
    (0.02 cm) at the centre, plug inlet U = 0.001 / scale, rho = 1 outlet,
    bounce-back channel walls; D2Q9 TRT flow at Re = U H / nu = 0.6
    (tau = 3.5 at every scale), D2Q5 TRT solute with the paper's rest
    fraction, Pe = U H / D, Da = k_r / U (Eq. PeDa), c_in = c_init = 1,
    c_eq = 0 on the disc.  Returns (params, mask, init, geom); geom holds
    what the average reaction rate of Eq. avgReactionRateMolins needs and
    the factor from lattice to the paper's unit (1e-8 mol / (cm^2 s)) for
    c_in = 10 mol/m^3 and u_in = 0.12 cm/s."""
    Pe, Da = MOLINS_CASES[case]
    H, W = int(round(600 * scale)), int(round(1200 * scale))
    d_obj = 240.0 * scale
    U = 0.001 / scale
    Re = 0.6
    nu = U * H / Re
    tau_f = 3.0 * nu + 0.5
    J0 = MOLINS_J0[Pe]
    D = U * H / Pe
    cs2 = lattice_cs2(5, 2, J0)
    tau_g = 0.5 + D / cs2
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    cx, cy = (W - 1) / 2.0, (H - 1) / 2.0
    disc = (xx - cx) ** 2 + (yy - cy) ** 2 <= (0.5 * d_obj) ** 2
    mask = np.where(disc, REACTIVE, FLUID).astype(np.uint8)[None]
    p = dict(dim=2, nx=W, ny=H, nz=1, flow_q=9, solute_q=5, bc=("open", "wall", "periodic"), tau_flow=tau_f,
             magic_flow=magic_flow, tau_solute=tau_g, magic_solute=magic_solute, rest_fraction=J0, k_r=Da * U,
             c_eq=0.0, c_init=1.0, c_inlet=1.0, u_inlet=U, rho_outlet=1.0, molar_volume=1.0, scheme=scheme,
             precision=precision)
    # lattice concentration 1 = 10 mol/m^3 = 1e-5 mol/cm^3; lattice velocity
    # U = 0.12 cm/s; result in 1e-8 mol/(cm^2 s)
    to_paper = 1e-5 * (0.12 / U) / 1e-8
    geom = dict(H=H, W=W, d_obj=d_obj, U=U, c_in=1.0, Pe=Pe, Da=Da, to_paper=to_paper,
                steps_hint=int(4.0e6 * scale * scale))
    return p, mask, {}, geom


def case_grain_2d(angle_deg: float = 0.0, scheme: str = "new", n: int = 300, k_r: float = 0.0014,
                  tau: float = 1.0, molar_volume: float = 0.2, c_init: float = 1.0, precision: str = "fp32"):
    """Grain growth during precipitation (Sec. 3.2): an n x n square with
    Dirichlet cells (C = 1) outside the inscribed circle of diameter n, a
    seed in the centre bounded by the curve r(s) = [0.1 + 0.02 cos(8 pi s)] n
    at polar angle 2 pi s, turned clockwise by angle_deg, reacting with
    C_eq = 0 and k_r (precipitation: the seed grows), pure diffusion on D2Q5
    with BGK (tau), phase change on.  Returns (params, mask, init, geom);
    geom holds the centre, the seed mask and the cells inside the circle."""
    yy, xx = np.mgrid[0:n, 0:n].astype(np.float64)
    c = (n - 1) / 2.0
    dx, dy = xx - c, yy - c
    r = np.hypot(dx, dy)
    # polar angle in the seed's own frame: a clockwise turn by angle_deg shows
    # the seed's feature at angle t at grid angle t - angle_deg
    t = np.arctan2(dy, dx) + math.radians(angle_deg)
    seed = r <= (0.1 + 0.02 * np.cos(4.0 * t)) * n
    outside = r > 0.5 * n - 0.5
    mask = np.full((n, n), FLUID, np.uint8)
    mask[seed] = REACTIVE
    mask[outside] = DIRICHLET
    p = dict(dim=2, nx=n, ny=n, nz=1, flow_q=0, solute_q=5, bc=("wall", "wall", "periodic"), tau_solute=tau,
             magic_solute=-1.0, rest_fraction=-1.0, k_r=k_r, c_eq=0.0, c_dirichlet=1.0, c_init=c_init,
             molar_volume=molar_volume, phase_change=1, scheme=scheme, precision=precision)
    geom = dict(centre=(c, c), seed=seed[None], inside=(~outside)[None])
    return p, mask[None], {}, geom
