"""Seeded synthetic inputs for the IMB-LBM-DEM workloads.

This module is the only thing the FP64 oracle (``oracle/``) and the CUDA path
(``paper_1809_07008_gb300``) have in common: it draws particle layouts and
parameter sets from a counter-free splitmix64 stream and holds none of the
method's arithmetic (no equilibrium, collision, overlap area or contact law).

Geometry convention shared by both sides (stated here because both receive
these numbers): lattice cell (i, k) is the unit square [i, i+1) x [k, k+1) and
its node sits at (i + 1/2, k + 1/2); the domain is [0, nx) x [0, ny); wall
boundaries lie on the domain edges, half a cell outside the first and last node
rows (halfway bounce-back).  Particle centres are given in the same frame.

Workloads (lattice units, dx = dt = 1, rho0 = 1):
  * ``c1``  200 x 100 channel, one fixed disk d = 20 at the centre, velocity
            inlet u = 0.01, zero-gradient outlet, no-slip walls, tau = 0.6.
  * ``c2``  2048 x 1024 closed box, 1000 disks d ~ U[16, 24] on a jittered grid
            in a 640-wide left column (granular collapse), tau = 0.52,
            Smagorinsky C = 0.1, linear spring-dashpot DEM with gravity.
  * ``c3``  8192 x 4096, periodic in x, walls in y, 20000 disks d = 20 placed by
            random sequential addition with a one-cell gap, random velocities of
            magnitude 0.005, tau = 0.51, Smagorinsky C = 0.1, DEM on, no gravity.
  * ``c3sub`` the 512 x 512 subdomain of ``c3`` at the same number density.
  * ``happel``  3D (D3Q19): plane Poiseuille flow between walls y = 0 and y = 5N past one
            held sphere of diameter N cells a quarter of the way across, periodic in x and z
            with l_x = l_z = 20 N (the paper's Sec. 3.1 case in lattice units).
  * ``spheres3`` small 3D boxes with seeded held spheres (parity cases).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

MASK64 = (1 << 64) - 1

# boundary codes (same integers in include/imblbm.h and oracle/imb_oracle.h)
BC_PERIODIC = 0
BC_WALL = 1
BC_INLET_OUTLET = 2

EPS_EXACT = 0
EPS_SUBCELL = 1

STORE_FP32 = 0
STORE_FP16 = 1
STORE_BF16 = 2


class SplitMix64:
    """splitmix64 (Steele, Lea & Flood 2014): 64-bit state, golden-ratio increment."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def uniform_range(self, lo: float, hi: float) -> float:
        return lo + (hi - lo) * self.uniform()


@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    tau: float
    C_smag: float = 0.0
    bc_x: int = BC_PERIODIC
    bc_y: int = BC_WALL
    u_in: tuple = (0.0, 0.0)
    force: tuple = (0.0, 0.0)          # body force density on the fluid
    u0: tuple = (0.0, 0.0)             # initial uniform fluid velocity
    rho0: float = 1.0
    eps_mode: int = EPS_EXACT
    n_sub: int = 5
    dem_on: int = 0
    N_sub: int = 100
    kn: float = 1.0e5
    kt: float = 0.5e5
    e_rest: float = 0.5
    ct_ratio: float = 0.5
    mu: float = 0.5
    rho_s: float = 2.65
    gravity: tuple = (0.0, 0.0)
    wall_u: tuple = (0.0, 0.0)         # x velocity of the walls y = 0 and y = ny
    contact_model: int = 0             # 0 linear spring-dashpot, 1 simplified Hertz-Mindlin
    E_young: float = 0.0               # Hertz-Mindlin material
    nu_poisson: float = 0.3
    steps: int = 1000
    x: np.ndarray = field(default_factory=lambda: np.zeros((0, 2)))
    v: np.ndarray = field(default_factory=lambda: np.zeros((0, 2)))
    omega: np.ndarray = field(default_factory=lambda: np.zeros(0))
    r: np.ndarray = field(default_factory=lambda: np.zeros(0))

    @property
    def n_particles(self) -> int:
        return int(self.r.shape[0])

    @property
    def cells(self) -> int:
        return self.nx * self.ny

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)

    def solid_fraction(self) -> float:
        return float(np.sum(math.pi * self.r ** 2) / self.cells)


def _particles(x, v, omega, r):
    return (np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(-1, 2)),
            np.ascontiguousarray(np.asarray(v, dtype=np.float64).reshape(-1, 2)),
            np.ascontiguousarray(np.asarray(omega, dtype=np.float64).reshape(-1)),
            np.ascontiguousarray(np.asarray(r, dtype=np.float64).reshape(-1)))


def random_sequential_addition(nx, ny, n, radius_fn, seed, gap=1.0, periodic_x=True,
                               wall_gap=1.0, region=None, max_attempts=None):
    """Place ``n`` non-overlapping disks by random sequential addition.

    Each attempt draws a centre uniformly in ``region`` (default: the domain, kept
    ``r + wall_gap`` away from non-periodic edges) and keeps it when every placed
    disk is at least ``r_a + r_b + gap`` away (minimum image in periodic x).
    Radii are drawn per disk by ``radius_fn(rng)`` before its first attempt.
    """
    rng = SplitMix64(seed)
    x0, y0, x1, y1 = region if region is not None else (0.0, 0.0, float(nx), float(ny))
    cell = 32.0
    ncx = max(1, int(math.ceil(nx / cell)))
    ncy = max(1, int(math.ceil(ny / cell)))
    grid = {}
    xs, ys, rs = [], [], []
    attempts = 0
    limit = max_attempts if max_attempts is not None else 200 * n + 10000
    while len(rs) < n:
        r = radius_fn(rng)
        placed = False
        while not placed:
            attempts += 1
            if attempts > limit:
                raise RuntimeError(f"random sequential addition stalled at {len(rs)}/{n} disks")
            if periodic_x and region is None:
                cx = rng.uniform_range(0.0, float(nx))
            else:
                cx = rng.uniform_range(x0 + r + wall_gap, x1 - r - wall_gap)
            cy = rng.uniform_range(y0 + r + wall_gap, y1 - r - wall_gap)
            gx, gy = int(cx // cell), int(cy // cell)
            ok = True
            for dy in (-1, 0, 1):
                if not ok:
                    break
                for dx in (-1, 0, 1):
                    kx, ky = gx + dx, gy + dy
                    if periodic_x:
                        kx %= ncx
                    if ky < 0 or ky >= ncy or kx < 0 or kx >= ncx:
                        continue
                    for j in grid.get((kx, ky), ()):
                        ddx = xs[j] - cx
                        if periodic_x:
                            if ddx > nx / 2:
                                ddx -= nx
                            elif ddx < -nx / 2:
                                ddx += nx
                        ddy = ys[j] - cy
                        if ddx * ddx + ddy * ddy < (rs[j] + r + gap) ** 2:
                            ok = False
                            break
                    if not ok:
                        break
            if ok:
                grid.setdefault((gx % ncx if periodic_x else gx, gy), []).append(len(rs))
                xs.append(cx)
                ys.append(cy)
                rs.append(r)
                placed = True
    return np.stack([np.array(xs), np.array(ys)], axis=1), np.array(rs)


def random_directions(n, speed, seed):
    rng = SplitMix64(seed)
    v = np.zeros((n, 2))
    for k in range(n):
        a = 2.0 * math.pi * rng.uniform()
        v[k] = (speed * math.cos(a), speed * math.sin(a))
    return v


def c1(steps=2000, d=20.0, nx=200, ny=100, u_in=0.01, tau=0.6) -> Workload:
    """Fixed disk of diameter ``d`` at the centre of an ``nx`` x ``ny`` channel."""
    x, v, om, r = _particles([[nx / 2.0, ny / 2.0]], [[0.0, 0.0]], [0.0], [d / 2.0])
    return Workload(name=f"c1_channel_{nx}x{ny}_disk_d{d:g}", nx=nx, ny=ny, tau=tau,
                    bc_x=BC_INLET_OUTLET, bc_y=BC_WALL, u_in=(u_in, 0.0), dem_on=0,
                    steps=steps, x=x, v=v, omega=om, r=r)


def c2(steps=20000, n=1000, nx=2048, ny=1024, column=640, seed=1809) -> Workload:
    """Granular column collapse: ``n`` disks d ~ U[16, 24] on a jittered grid."""
    rng = SplitMix64(seed)
    ncol = max(1, int(round(math.sqrt(n * column / ny))))
    nrow = int(math.ceil(n / ncol))
    sx, sy = column / ncol, ny / nrow
    xs, rs = [], []
    for k in range(n):
        i, j = k % ncol, k // ncol
        d = rng.uniform_range(16.0, 24.0)
        d = min(d, min(sx, sy) - 1.0)
        ax = max(0.0, (sx - d - 1.0) / 2.0)
        ay = max(0.0, (sy - d - 1.0) / 2.0)
        cx = (i + 0.5) * sx + rng.uniform_range(-ax, ax)
        cy = (j + 0.5) * sy + rng.uniform_range(-ay, ay)
        xs.append((cx, cy))
        rs.append(d / 2.0)
    x, v, om, r = _particles(xs, np.zeros((n, 2)), np.zeros(n), rs)
    return Workload(name=f"c2_collapse_{nx}x{ny}_{n}disks", nx=nx, ny=ny, tau=0.52, C_smag=0.1,
                    bc_x=BC_WALL, bc_y=BC_WALL, dem_on=1, gravity=(0.0, -1.0e-5),
                    steps=steps, x=x, v=v, omega=om, r=r)


def c3(steps=20000, n=20000, nx=8192, ny=4096, seed=7008, d=20.0, speed=0.005) -> Workload:
    """Periodic-x suspension of ``n`` disks of diameter ``d`` with random velocities."""
    x, r = random_sequential_addition(nx, ny, n, lambda g: d / 2.0, seed, gap=1.0,
                                      periodic_x=True, wall_gap=1.0)
    v = random_directions(n, speed, seed ^ 0x5DEECE66D)
    x, v, om, r = _particles(x, v, np.zeros(n), r)
    return Workload(name=f"c3_suspension_{nx}x{ny}_{n}disks", nx=nx, ny=ny, tau=0.51, C_smag=0.1,
                    bc_x=BC_PERIODIC, bc_y=BC_WALL, dem_on=1, gravity=(0.0, 0.0),
                    steps=steps, x=x, v=v, omega=om, r=r)


def c3sub(steps=1000, nx=512, ny=512, seed=7008) -> Workload:
    """``c3`` at the same disk number density on a smaller lattice."""
    n = int(round(20000 * nx * ny / (8192 * 4096)))
    w = c3(steps=steps, n=n, nx=nx, ny=ny, seed=seed)
    return w.with_(name=f"c3sub_suspension_{nx}x{ny}_{n}disks")


def c2_stack(steps=1000, n=30, nx=256, ny=192, ncols=4, gap=0.2, seed=1809) -> Workload:
    """The collapse case's physics (closed box, d ~ U[16, 24], tau = 0.52, C = 0.1, buoyant
    gravity, DEM on) on a small box: ``n`` disks stacked in ``ncols`` columns, each disk
    ``gap`` cells above the one below it (the lowest ``gap`` above the wall), so that wall and
    pair contacts form within the first coupling cycles."""
    rng = SplitMix64(seed)
    d = [rng.uniform_range(16.0, 24.0) for _ in range(n)]
    pitch = 24.0 + gap
    xs, top = [], [0.0] * ncols
    for k in range(n):
        c = k % ncols
        r = d[k] / 2.0
        y = top[c] + gap + r
        top[c] = y + r
        xs.append(((c + 0.5) * pitch + gap, y))
    if max(top) + gap > ny or ncols * pitch + 2 * gap > nx:
        raise ValueError("the stack does not fit the box")
    x, v, om, r = _particles(xs, np.zeros((n, 2)), np.zeros(n), [di / 2.0 for di in d])
    return Workload(name=f"c2_stack_{nx}x{ny}_{n}disks", nx=nx, ny=ny, tau=0.52, C_smag=0.1,
                    bc_x=BC_WALL, bc_y=BC_WALL, dem_on=1, gravity=(0.0, -1.0e-5),
                    steps=steps, x=x, v=v, omega=om, r=r)


def c4(steps=4000, nx=512, ny=256, n_side=4, d=20.0, seed=1809, u_in=0.02, tau=0.6) -> Workload:
    """Channel with n_side x n_side fixed disks on a jittered grid (velocity inlet, outlet at the
    reference pressure with zero velocity gradient, walls), the case of the drag-gradient
    computation."""
    rng = SplitMix64(seed)
    sx, sy = nx / (n_side + 1), ny / (n_side + 1)
    xs = []
    for j in range(n_side):
        for i in range(n_side):
            xs.append(((i + 1) * sx + rng.uniform_range(-0.15 * sx, 0.15 * sx),
                       (j + 1) * sy + rng.uniform_range(-0.15 * sy, 0.15 * sy)))
    n = len(xs)
    return Workload(name=f"c4_channel_{nx}x{ny}_{n}disks", nx=nx, ny=ny, tau=tau, C_smag=0.0,
                    bc_x=BC_INLET_OUTLET, bc_y=BC_WALL, u_in=(u_in, 0.0), dem_on=0, steps=steps,
                    x=np.array(xs), v=np.zeros((n, 2)), omega=np.zeros(n), r=np.full(n, d / 2.0))


def rsa_periodic(nx, ny, n, r, seed, gap=1.0, attempts_per_disk=40):
    """Up to ``n`` disks of radius ``r`` by random sequential addition in a box periodic in x and
    y, each at least 2 r + gap from every other (minimum image); stops after
    ``attempts_per_disk * n`` attempts (dense arrays jam below the requested count)."""
    rng = SplitMix64(seed)
    pts = np.zeros((0, 2))
    dmin2 = (2.0 * r + gap) ** 2
    for _ in range(attempts_per_disk * n):
        if len(pts) == n:
            break
        c = np.array([rng.uniform_range(0.0, float(nx)), rng.uniform_range(0.0, float(ny))])
        if len(pts):
            d = pts - c
            d[:, 0] -= nx * np.round(d[:, 0] / nx)
            d[:, 1] -= ny * np.round(d[:, 1] / ny)
            if ((d * d).sum(axis=1) < dmin2).any():
                continue
        pts = np.vstack([pts, c])
    return pts


def c5_domain(k, nx, ny, d, phi, tau, Re, seed, C_smag=0.1):
    """One domain of the batched sweep: periodic box with fixed disks of diameter d at solid
    fraction ~phi, driven along x by the body force that a Kozeny-Carman-type permeability
    k = d^2 (1 - phi)^3 / (9 phi^2) turns into the mean speed U = Re nu / d (U capped at 0.02
    for the Mach number; the constant 9 instead of the packed-bed 180 because these random disk
    arrays let the flow through channels -- with 180 the densest domains reached |u| = 0.34);
    Smagorinsky C_smag as in the suspension cases (tau down to 0.51)."""
    r = d / 2.0
    n = max(1, int(round(phi * nx * ny / (np.pi * r * r))))
    x = rsa_periodic(nx, ny, n, r, seed)
    phi_got = len(x) * np.pi * r * r / (nx * ny)
    nu = (tau - 0.5) / 3.0
    U = min(Re * nu / d, 0.02)
    perm = d * d * (1.0 - phi_got) ** 3 / (9.0 * phi_got * phi_got)
    F = nu * U / perm
    m = len(x)
    return Workload(name=f"c5_{k}_{nx}x{ny}", nx=nx, ny=ny, tau=tau, C_smag=C_smag, bc_x=BC_PERIODIC,
                    bc_y=BC_PERIODIC, force=(F, 0.0), dem_on=0, x=x, v=np.zeros((m, 2)), omega=np.zeros(m),
                    r=np.full(m, r))


def c5(n_domains=256, seed=1809):
    """Batched sweep: ``n_domains`` independent periodic domains, sizes 128..512 x 128..256 (in
    steps of 32), disk diameter 10..30, solid fraction 0.1..0.5, tau 0.51..1.0, Re 0.1..100
    (log-uniform), Smagorinsky C = 0.1, all drawn from one seeded generator."""
    rng = SplitMix64(seed)
    out = []
    for k in range(n_domains):
        nx = 128 + 32 * int(rng.uniform() * 13)
        ny = 128 + 32 * int(rng.uniform() * 5)
        d = rng.uniform_range(10.0, 30.0)
        phi = rng.uniform_range(0.1, 0.5)
        tau = rng.uniform_range(0.51, 1.0)
        Re = 10.0 ** rng.uniform_range(-1.0, 2.0)
        out.append(c5_domain(k, nx, ny, d, phi, tau, Re, seed * 1000 + k))
    return out


def poiseuille(H=32, nx=4, tau=0.6, g=1.0e-6, steps=20000) -> Workload:
    """Body-force driven channel, periodic in x, walls at y = 0 and y = H, no particles."""
    return Workload(name=f"poiseuille_H{H}", nx=nx, ny=H, tau=tau, bc_x=BC_PERIODIC, bc_y=BC_WALL,
                    force=(g, 0.0), steps=steps)


WORKLOADS = {"c1": c1, "c2": c2, "c3": c3, "c3sub": c3sub, "c4": c4}


# ------------------------------------------------------------------- 3D (D3Q19)
@dataclass
class Workload3:
    """3D lattice with held spheres: x and z periodic, y walls (``wall_y``) or periodic."""
    name: str
    nx: int
    ny: int
    nz: int
    tau: float
    wall_y: bool = True
    force: tuple = (0.0, 0.0, 0.0)
    n_sub: int = 5
    rho0: float = 1.0
    u0: tuple = (0.0, 0.0, 0.0)
    wall_u: tuple = (0.0, 0.0)         # x velocity of the walls y = 0 and y = ny
    C_smag: float = 0.0                # Smagorinsky constant
    steps: int = 1000
    x: np.ndarray = field(default_factory=lambda: np.zeros((0, 3)))
    v: np.ndarray = field(default_factory=lambda: np.zeros((0, 3)))
    omega: np.ndarray = field(default_factory=lambda: np.zeros((0, 3)))
    R: np.ndarray = field(default_factory=lambda: np.zeros(0))

    @property
    def n_spheres(self) -> int:
        return int(self.R.shape[0])

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz

    def with_(self, **kw) -> "Workload3":
        return replace(self, **kw)


def happel(N=5, tau=1.0, n_sub=5, u_c=2.0e-4, steps=None) -> Workload3:
    """Poiseuille flow past a held sphere (the paper's first benchmark) at N cells per
    diameter: walls 5 N apart, sphere centre N 5/4 from the lower wall and half-way in x and z,
    l_x = l_z = 20 N.  The body force g makes the undisturbed velocity at the centre height
    u_c = 3 g H^2 / (32 nu) (plane Poiseuille flow u(y) = g y (H - y) / (2 nu))."""
    H = 5 * N
    L = 20 * N
    nu = (tau - 0.5) / 3.0
    g = u_c * 32.0 * nu / (3.0 * H * H)
    if steps is None:   # about five viscous times of the wall gap
        steps = int(5.0 * H * H / (nu * math.pi ** 2)) + 500
    x = np.array([[L / 2.0, H / 4.0, L / 2.0]])
    return Workload3(name=f"happel_N{N}_tau{tau:g}_nsub{n_sub}", nx=L, ny=H, nz=L, tau=tau, wall_y=True,
                     force=(g, 0.0, 0.0), n_sub=n_sub, steps=steps, x=x, v=np.zeros((1, 3)),
                     omega=np.zeros((1, 3)), R=np.array([N / 2.0]))


# (Delta P [Pa] across the 10 d_p medium, tau) of the paper's ten packed-bed runs (Sec. 3.3)
PACKED_BED_RUNS = ((1.0, 0.58), (5.0, 0.53), (10.0, 0.524), (20.0, 0.516), (50.0, 0.51), (100.0, 0.508),
                   (200.0, 0.505), (400.0, 0.503), (800.0, 0.502), (1600.0, 0.501))


def packed_bed_units(N, tau, d_p=1.0e-3, rho_f=1000.0, mu_f=1.0e-3):
    """Lattice spacing and time step of the packed bed: dx = d_p / N, and dt from the fluid's
    viscosity, nu_f = (tau - 1/2) / 3 dx^2 / dt."""
    dx = d_p / N
    dt = (tau - 0.5) / 3.0 * dx * dx / (mu_f / rho_f)
    return dx, dt


def packed_bed(N=20, run=9, C_smag=0.3, n_sub=5, offset=0.5, d_p=1.0e-3, rho_f=1000.0, mu_f=1.0e-3,
               steps=1000) -> Workload3:
    """The paper's flow through densely packed particles (Sec. 3.3): 10 x 5 x 5 spheres of
    diameter d_p in a simple cubic arrangement with N cells per diameter, one d_p of free fluid
    before and after the packing in x, periodic in every direction.  Run ``run`` of the ten
    takes its pressure difference Delta P across the 10 d_p medium and its tau; the pressure
    gradient Delta P / (10 d_p) drives the fluid as the body force g = (Delta P / L) dt^2 /
    (rho_f dx) in lattice units.  The lattice sits ``offset`` cells off the packing in every
    direction: at 0 (N even) every contact point lies on a cell face and no cell holds two
    spheres; at 1/2 the contacts fall inside cells, which the two touching spheres share."""
    dP, tau = PACKED_BED_RUNS[run]
    dx, dt = packed_bed_units(N, tau, d_p, rho_f, mu_f)
    g = dP / (10.0 * d_p) * dt * dt / (rho_f * dx)
    x = np.array([[(1.5 + i) * N + offset, (0.5 + j) * N + offset, (0.5 + k) * N + offset]
                  for i in range(10) for j in range(5) for k in range(5)])
    n = x.shape[0]
    return Workload3(name=f"packed_bed_N{N}_dP{dP:g}_tau{tau:g}_C{C_smag:g}", nx=12 * N, ny=5 * N, nz=5 * N,
                     tau=tau, wall_y=False, force=(g, 0.0, 0.0), n_sub=n_sub, C_smag=C_smag, steps=steps, x=x,
                     v=np.zeros((n, 3)), omega=np.zeros((n, 3)), R=np.full(n, N / 2.0))


def spheres3(nx=40, ny=24, nz=36, n=3, r_lo=2.5, r_hi=5.0, seed=3, tau=0.7, wall_y=True,
             force=(2.0e-5, 0.0, 1.0e-5), speed=0.004, spin=0.001, n_sub=5, gap=2.0) -> Workload3:
    """Up to ``n`` spheres by random sequential addition (surfaces at least ``gap`` cells
    apart and from the walls), random velocities of magnitude ``speed`` and spins of
    magnitude ``spin`` (they enter u_s only: the spheres are held)."""
    rng = SplitMix64(seed)
    pts, rad = [], []
    for _ in range(200 * n):
        if len(pts) == n:
            break
        r = rng.uniform_range(r_lo, r_hi)
        c = np.array([rng.uniform_range(0.0, nx), rng.uniform_range(0.0, ny), rng.uniform_range(0.0, nz)])
        if wall_y and (c[1] - r < gap or c[1] + r > ny - gap):
            continue
        ok = True
        for p, rp in zip(pts, rad):
            d = c - p
            d[0] -= nx * round(d[0] / nx)
            d[2] -= nz * round(d[2] / nz)
            if not wall_y:
                d[1] -= ny * round(d[1] / ny)
            if float(np.sqrt((d * d).sum())) < r + rp + gap:
                ok = False
                break
        if ok:
            pts.append(c)
            rad.append(r)
    m = len(pts)
    v = np.array([_unit3(rng) * speed for _ in range(m)]).reshape(-1, 3)
    om = np.array([_unit3(rng) * spin for _ in range(m)]).reshape(-1, 3)
    return Workload3(name=f"spheres3_{nx}x{ny}x{nz}_{m}", nx=nx, ny=ny, nz=nz, tau=tau, wall_y=wall_y,
                     force=force, n_sub=n_sub, x=np.array(pts).reshape(-1, 3), v=v, omega=om,
                     R=np.array(rad))


def _unit3(rng):
    while True:
        a = np.array([rng.uniform_range(-1.0, 1.0) for _ in range(3)])
        n2 = float((a * a).sum())
        if 1e-6 < n2 <= 1.0:
            return a / math.sqrt(n2)
