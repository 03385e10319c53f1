"""ctypes wrapper and build step for the FP64 CPU oracle (``imb_oracle.c``, and the 3D
D3Q19 lattice with spheres in ``imb_oracle3.c``).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
module.  It never imports the CUDA package and the CUDA package never imports
it.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liborc.so")
SRC = os.path.join(HERE, "imb_oracle.c")
HDR = os.path.join(HERE, "imb_oracle.h")
SRC3 = os.path.join(HERE, "imb_oracle3.c")
HDR3 = os.path.join(HERE, "imb_oracle3.h")

PERIODIC, WALL, INLET_OUTLET = 0, 1, 2
EPS_EXACT, EPS_SUBCELL = 0, 1
MAX_SLOTS = 4


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library (plain gcc, no GPU code)."""
    os.makedirs(BUILD, exist_ok=True)
    srcs = (SRC, HDR, SRC3, HDR3)
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(x) for x in srcs)):
        return LIB
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-std=gnu11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           SRC, SRC3, "-o", tmp, "-lm"]
    # OpenMP only spreads the collide and stream loops over host threads (orc_set_threads,
    # default one); without it the same code builds single-threaded
    if subprocess.run(cmd[:-1] + ["-fopenmp", "-lm"], capture_output=True).returncode != 0:
        subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


class Params(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int),
                ("tau", C.c_double), ("C_smag", C.c_double),
                ("bc_x", C.c_int), ("bc_y", C.c_int),
                ("u_in_x", C.c_double), ("u_in_y", C.c_double),
                ("Fx", C.c_double), ("Fy", C.c_double),
                ("rho0", C.c_double), ("ux0", C.c_double), ("uy0", C.c_double),
                ("eps_mode", C.c_int), ("n_sub", C.c_int),
                ("dem_on", C.c_int), ("N_sub", C.c_int),
                ("kn", C.c_double), ("kt", C.c_double), ("e_rest", C.c_double),
                ("ct_ratio", C.c_double), ("mu", C.c_double), ("rho_s", C.c_double),
                ("gx", C.c_double), ("gy", C.c_double),
                ("wall_u_bot", C.c_double), ("wall_u_top", C.c_double),
                ("contact_model", C.c_int), ("E_young", C.c_double), ("nu_poisson", C.c_double)]


class Params3(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("tau", C.c_double),
                ("wall_y", C.c_int), ("Fx", C.c_double), ("Fy", C.c_double), ("Fz", C.c_double),
                ("n_sub", C.c_int), ("rho0", C.c_double), ("ux0", C.c_double), ("uy0", C.c_double),
                ("uz0", C.c_double), ("wall_ux_bot", C.c_double), ("wall_ux_top", C.c_double),
                ("C_smag", C.c_double)]


_lib = None
_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        L.orc_feq.argtypes = [C.c_double, C.c_double, C.c_double, _dp]
        L.orc_B.argtypes = [C.c_double, C.c_double]
        L.orc_B.restype = C.c_double
        L.orc_tau_eff.argtypes = [_dp, C.c_double, C.c_double, C.c_double, C.c_double]
        L.orc_tau_eff.restype = C.c_double
        L.orc_cell_area.argtypes = [C.c_double] * 5
        L.orc_cell_area.restype = C.c_double
        L.orc_eps_subcell.argtypes = [C.c_float, C.c_float, C.c_float, C.c_int]
        L.orc_eps_subcell.restype = C.c_double
        L.orc_covers.argtypes = [C.c_float, C.c_float, C.c_float]
        L.orc_covers.restype = C.c_int
        L.orc_omega_s.argtypes = [_dp] + [C.c_double] * 5 + [_dp]
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_new.argtypes = [C.POINTER(Params)]
        L.orc_new.restype = C.c_void_p
        L.orc_free.argtypes = [C.c_void_p]
        L.orc_set_particles.argtypes = [C.c_void_p, C.c_int, _dp, _dp, _dp, _dp]
        L.orc_step.argtypes = [C.c_void_p, C.c_int]
        L.orc_get_f.argtypes = [C.c_void_p, _dp]
        L.orc_set_f.argtypes = [C.c_void_p, _dp]
        L.orc_get_macro.argtypes = [C.c_void_p, _dp, _dp, _dp]
        L.orc_get_forces.argtypes = [C.c_void_p, _dp, _dp]
        L.orc_set_forces.argtypes = [C.c_void_p, _dp, _dp]
        L.orc_get_particles.argtypes = [C.c_void_p, _dp, _dp, _dp]
        L.orc_cell_map.argtypes = [C.c_void_p, _ip, _ip, _dp]
        L.orc_contacts.argtypes = [C.c_void_p, C.c_int, _ip]
        L.orc_bins.argtypes = [C.c_void_p, C.c_int, _ip, _ip]
        L.orc_dem_substeps.argtypes = [C.c_void_p, C.c_int]
        L.orc_wall_contact_xi.argtypes = [C.c_void_p, C.c_int, C.c_int]
        L.orc_wall_contact_xi.restype = C.c_double
        L.orc_drag_adjoint.argtypes = [C.c_void_p, C.c_int, _dp, _dp, _dp, _dp]
        L.orc3_lattice.argtypes = [_ip, _dp]
        L.orc3_feq.argtypes = [C.c_double] * 4 + [_dp]
        L.orc3_omega_s.argtypes = [_dp] + [C.c_double] * 7 + [_dp]
        L.orc3_subcell_count.argtypes = [C.c_int] * 3 + [C.c_double] * 4 + [C.c_int]
        L.orc3_tau_eff.argtypes = [_dp] + [C.c_double] * 5
        L.orc3_tau_eff.restype = C.c_double
        L.orc3_new.argtypes = [C.POINTER(Params3)]
        L.orc3_new.restype = C.c_void_p
        L.orc3_free.argtypes = [C.c_void_p]
        L.orc3_set_spheres.argtypes = [C.c_void_p, C.c_int, _dp, _dp, _dp, _dp]
        L.orc3_step.argtypes = [C.c_void_p, C.c_int]
        L.orc3_get_f.argtypes = [C.c_void_p, _dp]
        L.orc3_set_f.argtypes = [C.c_void_p, _dp]
        L.orc3_get_macro.argtypes = [C.c_void_p, _dp, _dp, _dp, _dp]
        L.orc3_get_forces.argtypes = [C.c_void_p, _dp, _dp]
        L.orc3_cell_map.argtypes = [C.c_void_p, _ip, _ip]
        _lib = L
    return _lib


_threads = 1


def set_threads(n: int) -> int:
    """Host threads of the oracle's collide and stream loops (default 1); returns the previous
    count.  The results do not depend on it: each cell's arithmetic is the same and the
    particles' forces are summed in the same order."""
    global _threads
    prev, _threads = _threads, max(1, int(n))
    lib().orc_set_threads(_threads)
    return prev


def _d(a):
    return a.ctypes.data_as(_dp)


def _i(a):
    return a.ctypes.data_as(_ip)


def feq(rho, ux, uy):
    out = np.zeros(9)
    lib().orc_feq(rho, ux, uy, _d(out))
    return out


def B(eps, tau):
    return lib().orc_B(eps, tau)


def tau_eff(f9, tau, C_smag, force=(0.0, 0.0)):
    f9 = np.ascontiguousarray(f9, dtype=np.float64)
    return lib().orc_tau_eff(_d(f9), force[0], force[1], tau, C_smag)


def cell_area(a0, a1, b0, b1, r):
    return lib().orc_cell_area(a0, a1, b0, b1, r)


def eps_subcell(lox, loy, r, n):
    return lib().orc_eps_subcell(lox, loy, r, n)


def covers(lox, loy, r):
    return bool(lib().orc_covers(lox, loy, r))


def omega_s(f9, rho, ux, uy, usx, usy):
    f9 = np.ascontiguousarray(f9, dtype=np.float64)
    out = np.zeros(9)
    lib().orc_omega_s(_d(f9), rho, ux, uy, usx, usy, _d(out))
    return out


def params_from_workload(w) -> Params:
    p = Params()
    p.nx, p.ny = w.nx, w.ny
    p.tau, p.C_smag = w.tau, w.C_smag
    p.bc_x, p.bc_y = w.bc_x, w.bc_y
    p.u_in_x, p.u_in_y = w.u_in
    p.Fx, p.Fy = w.force
    p.rho0 = w.rho0
    p.ux0, p.uy0 = w.u0
    p.eps_mode, p.n_sub = w.eps_mode, w.n_sub
    p.dem_on, p.N_sub = w.dem_on, w.N_sub
    p.kn, p.kt, p.e_rest, p.ct_ratio = w.kn, w.kt, w.e_rest, w.ct_ratio
    p.mu, p.rho_s = w.mu, w.rho_s
    p.gx, p.gy = w.gravity
    p.wall_u_bot, p.wall_u_top = w.wall_u
    p.contact_model, p.E_young, p.nu_poisson = w.contact_model, w.E_young, w.nu_poisson
    return p


class Sim:
    """One oracle simulation; mirrors the calls of the C-ABI library."""

    def __init__(self, w, particles: bool = True):
        self.w = w
        self.p = params_from_workload(w)
        self.h = lib().orc_new(C.byref(self.p))
        if not self.h:
            raise ValueError("oracle rejected the parameters")
        self.np = 0
        if particles and w.n_particles:
            self.set_particles(w.x, w.v, w.omega, w.r)

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_free(self.h)
            self.h = None

    def set_particles(self, x, v, omega, r):
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
        v = np.ascontiguousarray(v, dtype=np.float64).reshape(-1)
        omega = np.ascontiguousarray(omega, dtype=np.float64).reshape(-1)
        r = np.ascontiguousarray(r, dtype=np.float64).reshape(-1)
        rc = lib().orc_set_particles(self.h, r.shape[0], _d(x), _d(v), _d(omega), _d(r))
        if rc:
            raise ValueError("oracle rejected the particles")
        self.np = r.shape[0]

    def step(self, n=1):
        rc = lib().orc_step(self.h, n)
        if rc:
            raise RuntimeError(f"oracle step failed with code {rc}")

    def dem_substeps(self, n):
        lib().orc_dem_substeps(self.h, n)

    @property
    def shape(self):
        return (self.w.ny, self.w.nx)

    def f(self):
        out = np.zeros((9, self.w.ny, self.w.nx))
        lib().orc_get_f(self.h, _d(out))
        return out

    def set_f(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        lib().orc_set_f(self.h, _d(f))

    def macro(self):
        rho = np.zeros(self.shape)
        ux = np.zeros(self.shape)
        uy = np.zeros(self.shape)
        lib().orc_get_macro(self.h, _d(rho), _d(ux), _d(uy))
        return rho, ux, uy

    def forces(self):
        F = np.zeros((self.np, 2))
        T = np.zeros(self.np)
        if self.np:
            lib().orc_get_forces(self.h, _d(F), _d(T))
        return F, T

    def set_forces(self, F, T):
        F = np.ascontiguousarray(F, dtype=np.float64)
        T = np.ascontiguousarray(T, dtype=np.float64)
        lib().orc_set_forces(self.h, _d(F), _d(T))

    def particles(self):
        x = np.zeros((self.np, 2))
        v = np.zeros((self.np, 2))
        w = np.zeros(self.np)
        if self.np:
            lib().orc_get_particles(self.h, _d(x), _d(v), _d(w))
        return x, v, w

    def cell_map(self):
        count = np.zeros(self.shape, dtype=np.int32)
        ids = np.zeros(self.shape + (MAX_SLOTS,), dtype=np.int32)
        eps = np.zeros(self.shape + (MAX_SLOTS,))
        rc = lib().orc_cell_map(self.h, _i(count), _i(ids), _d(eps))
        if rc:
            raise RuntimeError("more than four particles cover one cell")
        return count, ids, eps

    def contacts(self):
        n = lib().orc_contacts(self.h, 0, None)
        pairs = np.zeros((max(n, 1), 2), dtype=np.int32)
        lib().orc_contacts(self.h, n, _i(pairs))
        return pairs[:n]

    def bins(self, edge=32):
        nbx = (self.w.nx + edge - 1) // edge
        nby = (self.w.ny + edge - 1) // edge
        start = np.zeros(nbx * nby + 1, dtype=np.int32)
        ids = np.zeros(max(self.np, 1), dtype=np.int32)
        lib().orc_bins(self.h, edge, _i(start), _i(ids))
        return start, ids[:self.np]

    def wall_xi(self, p, wall):
        return lib().orc_wall_contact_xi(self.h, p, wall)

    def drag_adjoint(self, T):
        """Time-averaged drag over T steps from the current state and its gradient with
        respect to u_in_x, tau and the particle centres (reverse mode; see the C source)."""
        J, gu, gt = (C.c_double(0.0) for _ in range(3))
        gx = np.zeros((max(self.np, 1), 2))
        rc = lib().orc_drag_adjoint(self.h, int(T), C.byref(J), C.byref(gu), C.byref(gt), _d(gx))
        if rc:
            raise ValueError(f"drag adjoint outside its scope or failed ({rc})")
        return J.value, gu.value, gt.value, gx[:self.np]

    def drag_average(self, T):
        """Time-averaged total drag sum_p F_x,p over T steps from the current state."""
        s = 0.0
        for _ in range(T):
            self.step(1)
            s += self.forces()[0][:, 0].sum()
        return s / T


# ------------------------------------------------------------------- 3D (D3Q19)
def lattice3():
    c = np.zeros((19, 3), dtype=np.int32)
    w = np.zeros(19)
    lib().orc3_lattice(_i(c), _d(w))
    return c, w


def feq3(rho, ux, uy, uz):
    out = np.zeros(19)
    lib().orc3_feq(rho, ux, uy, uz, _d(out))
    return out


def omega_s3(f19, rho, u, us):
    f19 = np.ascontiguousarray(f19, dtype=np.float64)
    out = np.zeros(19)
    lib().orc3_omega_s(_d(f19), rho, u[0], u[1], u[2], us[0], us[1], us[2], _d(out))
    return out


def tau_eff3(f19, tau, C_smag, force=(0.0, 0.0, 0.0)):
    f19 = np.ascontiguousarray(f19, dtype=np.float64)
    return lib().orc3_tau_eff(_d(f19), force[0], force[1], force[2], tau, C_smag)


def subcell_count3(off, frac, R, n):
    return lib().orc3_subcell_count(int(off[0]), int(off[1]), int(off[2]), float(frac[0]), float(frac[1]),
                                    float(frac[2]), float(R), int(n))


class Sim3:
    """One 3D oracle simulation (``workloads.Workload3``): D3Q19 with held spheres."""

    def __init__(self, w):
        self.w = w
        p = Params3()
        p.nx, p.ny, p.nz = w.nx, w.ny, w.nz
        p.tau, p.wall_y = w.tau, int(w.wall_y)
        p.Fx, p.Fy, p.Fz = w.force
        p.n_sub = w.n_sub
        p.rho0 = w.rho0
        p.ux0, p.uy0, p.uz0 = w.u0
        p.wall_ux_bot, p.wall_ux_top = w.wall_u
        p.C_smag = w.C_smag
        self.p = p
        self.h = lib().orc3_new(C.byref(p))
        if not self.h:
            raise ValueError("oracle rejected the parameters")
        self.np = len(w.R)
        x = np.ascontiguousarray(w.x, dtype=np.float64).reshape(-1)
        v = np.ascontiguousarray(w.v, dtype=np.float64).reshape(-1)
        om = np.ascontiguousarray(w.omega, dtype=np.float64).reshape(-1)
        R = np.ascontiguousarray(w.R, dtype=np.float64).reshape(-1)
        rc = lib().orc3_set_spheres(self.h, self.np, _d(x), _d(v), _d(om), _d(R))
        if rc:
            raise ValueError(f"oracle rejected the spheres ({rc})")

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc3_free(self.h)
            self.h = None

    def step(self, n=1):
        lib().orc3_step(self.h, n)

    def f(self):
        out = np.zeros((19, self.w.nz, self.w.ny, self.w.nx))
        lib().orc3_get_f(self.h, _d(out))
        return out

    def set_f(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        lib().orc3_set_f(self.h, _d(f))

    def macro(self):
        shp = (self.w.nz, self.w.ny, self.w.nx)
        rho, ux, uy, uz = (np.zeros(shp) for _ in range(4))
        lib().orc3_get_macro(self.h, _d(rho), _d(ux), _d(uy), _d(uz))
        return rho, ux, uy, uz

    def forces(self):
        F = np.zeros((max(self.np, 1), 3))
        T = np.zeros((max(self.np, 1), 3))
        lib().orc3_get_forces(self.h, _d(F), _d(T))
        return F[:self.np], T[:self.np]

    def cell_map(self):
        shp = (self.w.nz, self.w.ny, self.w.nx, 4)
        sph = np.zeros(shp, dtype=np.int32)
        cnt = np.zeros(shp, dtype=np.int32)
        lib().orc3_cell_map(self.h, _i(sph), _i(cnt))
        return sph, cnt


def happel_brenner(R, l, U, rho, nu):
    """Eqs. 18-19: drag and torque on a held sphere of radius R whose centre is a distance l
    from a plane wall, in a shear flow whose undisturbed velocity at the centre is U (density
    rho, kinematic viscosity nu).  (The paper's printed values for its case follow with l the
    centre's distance from the nearer wall and U the Poiseuille velocity at the centre.)"""
    a = R / l
    F = 6.0 * math.pi * rho * nu * R * U * (1.0 - a ** 2 / 9.0) / (1.0 - 0.6526 * a + 0.316 * a ** 3 - 0.242 * a ** 4)
    T = 8.0 / 3.0 * math.pi * rho * nu * R ** 2 * U * a * (1.0 + 0.0758 * a + 0.049 * a ** 2)
    return F, T


def ergun_gradient(U, d_p, n, rho, mu):
    """Eq. 21 (Ergun): pressure gradient Delta P / L across a packed bed of particle diameter d_p
    and porosity n at superficial velocity U, a viscous loss linear in U plus an inertial one
    quadratic in U."""
    return 150.0 * mu / d_p ** 2 * (1.0 - n) ** 2 / n ** 3 * U + 1.75 * rho / d_p * (1.0 - n) / n ** 3 * U ** 2


def packed_bed_reynolds(U, d_p, n, rho, mu):
    """Eq. 23: the modified particle Reynolds number rho d_p U / (mu (1 - n))."""
    return rho * d_p * U / (mu * (1.0 - n))


def packed_bed_friction(dPdL, U, d_p, n, rho):
    """Eq. 22, left: the packed bed friction factor (Delta P / L) d_p n^3 / (rho U^2 (1 - n))."""
    return dPdL * d_p * n ** 3 / (rho * U ** 2 * (1.0 - n))


def ergun_friction(Re):
    """Eq. 22, right: the Ergun friction factor 150 / Re*_p + 1.75."""
    return 150.0 / Re + 1.75


def happel_table2():
    """The paper's Table 2 rows (tests/golden/happel_table2.txt): (N, n_sub, tau, err_F %, err_T %)."""
    path = os.path.join(os.path.dirname(HERE), "tests", "golden", "happel_table2.txt")
    rows = []
    for ln in open(path):
        ln = ln.strip()
        if ln and not ln.startswith("#"):
            a = ln.split()
            rows.append((int(a[0]), int(a[1]), float(a[2]), float(a[3]), float(a[4])))
    return rows
