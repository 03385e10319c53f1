"""Thin ctypes binding of ``libimblbm.so`` (the C ABI of ``include/imblbm.h``).

Argument marshalling only: every step of the IMB-LBM-DEM path runs in the CUDA
library.  There is no fallback -- if the library cannot be loaded, or no CUDA
device is present, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

IMB_OK = 0
ERRORS = {
    -1: "IMB_E_INVALID_ARG", -2: "IMB_E_CUDA", -3: "IMB_E_NOMEM", -4: "IMB_E_UNSTABLE",
    -5: "IMB_E_OVERFLOW", -6: "IMB_E_TIMEOUT", -7: "IMB_E_SKIN", -8: "IMB_E_STATE",
}
BC_PERIODIC, BC_WALL, BC_INLET_OUTLET = 0, 1, 2
STORE_FP32, STORE_FP16, STORE_BF16 = 0, 1, 2
STORAGE_NAMES = {"fp32": STORE_FP32, "fp16": STORE_FP16, "bf16": STORE_BF16}
EPS_EXACT, EPS_SUBCELL = 0, 1
MAX_SLOTS = 4

# every symbol include/imblbm.h declares
EXPORTS = (
    "imb_default_params", "imb_init_lattice", "imb_set_particles", "imb_set_kinematics",
    "imb_step", "imb_step_async", "imb_dem_step", "imb_sync", "imb_get_populations",
    "imb_get_macro", "imb_get_forces", "imb_set_forces", "imb_get_particles",
    "imb_get_cell_map", "imb_get_contacts", "imb_get_bins", "imb_set_stream", "imb_get_stream",
    "imb_enable_kernel_timing", "imb_kernel_time", "imb_launch_count", "imb_bytes_per_cell",
    "imb_last_error", "imb_destroy", "imb_bin_particles_noalloc", "imb_drag_gradient", "imb_step_io",
    "imb_drag_gradient_binomial", "imb_binomial_schedule",
    "imb3_default_params", "imb3_init", "imb3_set_spheres", "imb3_step", "imb3_get_populations",
    "imb3_get_macro", "imb3_get_forces", "imb3_get_cell_map", "imb3_enable_kernel_timing",
    "imb3_kernel_time", "imb3_launch_count", "imb3_bytes_per_cell", "imb3_last_error", "imb3_destroy",
    "imb_batch_create", "imb_batch_run", "imb_batch_autotune", "imb_batch_set_launch", "imb_batch_mean_drag",
    "imb_batch_get_populations", "imb_batch_cells", "imb_batch_last_error", "imb_batch_destroy",
)


CK_ADVANCE, CK_STORE, CK_RESTORE, CK_ADJOINT = 1, 2, 3, 4


def binomial_schedule(T: int, snapshots: int):
    """imb_binomial_schedule: the operations [(kind, argument), ...] of the binomial
    checkpointing schedule for reversing T steps with ``snapshots`` free snapshot slots, and
    the number of forward steps it takes.  Host only (no GPU)."""
    L = load()
    n, adv = C.c_int(0), C.c_longlong(0)
    rc = L.imb_binomial_schedule(int(T), int(snapshots), None, 0, C.byref(n), C.byref(adv))
    if rc:
        raise ImbError(rc, "imb_binomial_schedule")
    ops = np.zeros(2 * max(n.value, 1), dtype=np.int32)
    rc = L.imb_binomial_schedule(int(T), int(snapshots), ops.ctypes.data_as(_ip), n.value, C.byref(n), None)
    if rc:
        raise ImbError(rc, "imb_binomial_schedule")
    return [(int(ops[2 * k]), int(ops[2 * k + 1])) for k in range(n.value)], adv.value


def bin_particles_noalloc(d_x: int, n: int, nx: int, ny: int, d_bin_start: int, d_bin_ids: int,
                          stream: int = 0) -> int:
    """imb_bin_particles_noalloc on raw device addresses (e.g. tensor.data_ptr()); returns
    the IMB_* code.  For callers that cannot allocate: nothing is allocated."""
    return load().imb_bin_particles_noalloc(_vp(d_x), int(n), int(nx), int(ny), _vp(d_bin_start),
                                           _vp(d_bin_ids), _vp(stream) if stream else None)


class ImbError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Params3(C.Structure):
    """Mirror of imb3_params (include/imblbm.h)."""
    _fields_ = [("wall_y", C.c_int), ("Fx", C.c_double), ("Fy", C.c_double), ("Fz", C.c_double),
                ("n_sub", C.c_int), ("storage", C.c_int), ("rho0", C.c_double), ("ux0", C.c_double),
                ("uy0", C.c_double), ("uz0", C.c_double), ("timeout_ms", C.c_int),
                ("wall_ux_bot", C.c_double), ("wall_ux_top", C.c_double), ("C_smag", C.c_double)]


class Params(C.Structure):
    _fields_ = [("bc_x", C.c_int), ("bc_y", C.c_int),
                ("u_in_x", C.c_double), ("u_in_y", C.c_double),
                ("Fx", C.c_double), ("Fy", C.c_double),
                ("rho0", C.c_double), ("ux0", C.c_double), ("uy0", C.c_double),
                ("storage", C.c_int), ("eps_mode", C.c_int), ("n_sub", C.c_int),
                ("dem_on", C.c_int), ("N_sub", C.c_int),
                ("kn", C.c_double), ("kt", C.c_double), ("e_rest", C.c_double),
                ("ct_ratio", C.c_double), ("mu", C.c_double), ("rho_s", C.c_double),
                ("gx", C.c_double), ("gy", C.c_double), ("skin", C.c_double),
                ("timeout_ms", C.c_int), ("wall_u_bot", C.c_double), ("wall_u_top", C.c_double),
                ("contact_model", C.c_int), ("E_young", C.c_double), ("nu_poisson", C.c_double),
                ("work_units", C.c_int), ("plain_launches", C.c_int)]


_lib = None
_dp = C.POINTER(C.c_double)
_F64 = np.dtype(np.float64)
_fp = C.POINTER(C.c_float)
_ip = C.POINTER(C.c_int)
_vp = C.c_void_p


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load (building first if needed) the CUDA library and declare its signatures."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build_if_missing else _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"libimblbm.so not found at {path}; run paper_1809_07008_gb300/build.py")
    L = C.CDLL(path)
    L.imb_default_params.argtypes = [C.POINTER(Params)]
    L.imb_default_params.restype = None
    L.imb_init_lattice.argtypes = [C.POINTER(_vp), C.c_int, C.c_int, C.c_double, C.c_double,
                                   C.POINTER(Params)]
    L.imb_set_particles.argtypes = [_vp, C.c_int, _dp, _dp, _dp, _dp]
    L.imb_set_kinematics.argtypes = [_vp, _dp, _dp, _dp]
    for name in ("imb_step", "imb_step_async", "imb_dem_step"):
        getattr(L, name).argtypes = [_vp, C.c_int]
    L.imb_sync.argtypes = [_vp]
    # plain addresses: the per-cycle call takes them from Lattice._io_addr
    L.imb_step_io.argtypes = [_vp, C.c_int, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
    L.imb_get_populations.argtypes = [_vp, _dp]
    L.imb_get_macro.argtypes = [_vp, _dp, _dp, _dp]
    L.imb_get_forces.argtypes = [_vp, _dp, _dp]
    L.imb_set_forces.argtypes = [_vp, _dp, _dp]
    L.imb_get_particles.argtypes = [_vp, _dp, _dp, _dp]
    L.imb_get_cell_map.argtypes = [_vp, _ip, _ip, _fp]
    L.imb_get_contacts.argtypes = [_vp, C.c_int, _ip, _ip]
    L.imb_get_bins.argtypes = [_vp, _ip, _ip]
    L.imb_set_stream.argtypes = [_vp, _vp]
    L.imb_get_stream.argtypes = [_vp]
    L.imb_get_stream.restype = _vp
    L.imb_enable_kernel_timing.argtypes = [_vp, C.c_int]
    L.imb_kernel_time.argtypes = [_vp, _dp, C.POINTER(C.c_longlong)]
    L.imb_launch_count.argtypes = [_vp]
    L.imb_launch_count.restype = C.c_longlong
    L.imb_bytes_per_cell.argtypes = [_vp]
    L.imb_bytes_per_cell.restype = C.c_double
    L.imb_last_error.argtypes = [_vp]
    L.imb_last_error.restype = C.c_char_p
    L.imb_destroy.argtypes = [_vp]
    L.imb_destroy.restype = None
    L.imb_bin_particles_noalloc.argtypes = [_vp, C.c_int, C.c_int, C.c_int, _vp, _vp, _vp]
    L.imb_drag_gradient.argtypes = [_vp, C.c_int, C.c_int, _dp, _dp, _dp, _dp]
    L.imb_drag_gradient_binomial.argtypes = [_vp, C.c_int, C.c_int, _dp, _dp, _dp, _dp]
    L.imb_binomial_schedule.argtypes = [C.c_int, C.c_int, _ip, C.c_int, _ip, C.POINTER(C.c_longlong)]
    L.imb_batch_create.argtypes = [C.POINTER(_vp), C.c_int, _ip, _ip, _dp, _dp, _dp, _dp, _ip, _dp, _dp, C.c_int]
    L.imb_batch_run.argtypes = [_vp, C.c_int]
    L.imb_batch_autotune.argtypes = [_vp, C.c_int, _ip, _ip, _dp]
    L.imb_batch_set_launch.argtypes = [_vp, C.c_int, C.c_int]
    L.imb_batch_mean_drag.argtypes = [_vp, _dp, _dp]
    L.imb_batch_get_populations.argtypes = [_vp, C.c_int, _dp]
    L.imb_batch_cells.argtypes = [_vp]
    L.imb_batch_cells.restype = C.c_longlong
    L.imb_batch_last_error.argtypes = [_vp]
    L.imb_batch_last_error.restype = C.c_char_p
    L.imb_batch_destroy.argtypes = [_vp]
    L.imb_batch_destroy.restype = None
    L.imb3_default_params.argtypes = [C.POINTER(Params3)]
    L.imb3_default_params.restype = None
    L.imb3_init.argtypes = [C.POINTER(_vp), C.c_int, C.c_int, C.c_int, C.c_double, C.POINTER(Params3)]
    L.imb3_set_spheres.argtypes = [_vp, C.c_int, _dp, _dp, _dp, _dp]
    L.imb3_step.argtypes = [_vp, C.c_int]
    L.imb3_get_populations.argtypes = [_vp, _dp]
    L.imb3_get_macro.argtypes = [_vp, _dp, _dp, _dp, _dp]
    L.imb3_get_forces.argtypes = [_vp, _dp, _dp]
    L.imb3_get_cell_map.argtypes = [_vp, _ip, _ip]
    L.imb3_enable_kernel_timing.argtypes = [_vp, C.c_int]
    L.imb3_kernel_time.argtypes = [_vp, _dp, C.POINTER(C.c_longlong)]
    L.imb3_launch_count.argtypes = [_vp]
    L.imb3_launch_count.restype = C.c_longlong
    L.imb3_bytes_per_cell.argtypes = [_vp]
    L.imb3_bytes_per_cell.restype = C.c_double
    L.imb3_last_error.argtypes = [_vp]
    L.imb3_last_error.restype = C.c_char_p
    L.imb3_destroy.argtypes = [_vp]
    L.imb3_destroy.restype = None
    _lib = L
    return L


def _d(a):
    return a.ctypes.data_as(_dp)


def _f64(a, n):
    a = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
    if a.shape[0] != n:
        raise ValueError(f"expected {n} values, got {a.shape[0]}")
    return a


def default_params() -> Params:
    p = Params()
    load().imb_default_params(C.byref(p))
    return p


class Lattice:
    """One lattice context of the CUDA library (see include/imblbm.h for the semantics)."""

    def __init__(self, nx, ny, tau, C_smag=0.0, params: Params | None = None, **kw):
        L = load()
        p = params if params is not None else default_params()
        for k, v in kw.items():
            if k == "storage" and isinstance(v, str):
                v = STORAGE_NAMES[v]
            setattr(p, k, v)
        self.params = p
        self.nx, self.ny = int(nx), int(ny)
        h = _vp()
        rc = L.imb_init_lattice(C.byref(h), self.nx, self.ny, float(tau), float(C_smag), C.byref(p))
        if rc != IMB_OK:
            raise ImbError(rc, L.imb_last_error(None).decode())
        self.h = h
        self.np = 0
        self._addr_table = {}
        self._L = L

    @classmethod
    def from_workload(cls, w, storage="fp32", particles=True, **kw):
        p = default_params()
        p.bc_x, p.bc_y = w.bc_x, w.bc_y
        p.u_in_x, p.u_in_y = w.u_in
        p.Fx, p.Fy = w.force
        p.rho0 = w.rho0
        p.ux0, p.uy0 = w.u0
        p.storage = STORAGE_NAMES[storage] if isinstance(storage, str) else storage
        p.eps_mode, p.n_sub = w.eps_mode, w.n_sub
        p.dem_on, p.N_sub = w.dem_on, w.N_sub
        p.kn, p.kt, p.e_rest, p.ct_ratio = w.kn, w.kt, w.e_rest, w.ct_ratio
        p.mu, p.rho_s = w.mu, w.rho_s
        p.gx, p.gy = w.gravity
        p.wall_u_bot, p.wall_u_top = w.wall_u
        p.contact_model, p.E_young, p.nu_poisson = w.contact_model, w.E_young, w.nu_poisson
        for k, v in kw.items():
            setattr(p, k, v)
        lat = cls(w.nx, w.ny, w.tau, w.C_smag, params=p)
        if particles and w.n_particles:
            lat.set_particles(w.x, w.v, w.omega, w.r)
        return lat

    def _check(self, rc):
        if rc != IMB_OK:
            raise ImbError(rc, self._L.imb_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self._L.imb_destroy(self.h)
            self.h = None
        self._addr_table = {}

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- state
    def set_particles(self, x, v, omega, r):
        r = _f64(r, np.size(r))
        n = r.shape[0]
        x, v, omega = _f64(x, 2 * n), _f64(v, 2 * n), _f64(omega, n)
        self._check(self._L.imb_set_particles(self.h, n, _d(x), _d(v), _d(omega), _d(r)))
        self.np = n

    def set_kinematics(self, x, v, omega):
        n = self.np
        x, v, omega = _f64(x, 2 * n), _f64(v, 2 * n), _f64(omega, n)
        self._check(self._L.imb_set_kinematics(self.h, _d(x), _d(v), _d(omega)))

    def step(self, n=1):
        self._check(self._L.imb_step(self.h, int(n)))

    def _io_addr(self, a):
        """Address of the data of array ``a``, looked up once per array object: the host waits
        on this call every coupling cycle, and numpy's own lookup costs about a microsecond an
        array.  Holding ``a`` in the table keeps its id and its buffer (which numpy cannot
        reallocate while another reference exists) tied to the stored address."""
        e = self._addr_table.get(id(a))
        if e is not None and e[0] is a:
            return e[1]
        if len(self._addr_table) >= 32:
            self._addr_table.clear()
        p = a.ctypes.data
        self._addr_table[id(a)] = (a, p)
        return p

    def step_io(self, n=1, kin_in=None, F=None, T=None, x=None, v=None, w=None):
        """imb_step_io: optional upload of (x, v, omega), n cycles, read-back into the given
        host arrays (any may be None), one wait."""
        n_p = self.np
        xi = vi = wi = None
        keep = None
        if kin_in is not None:
            if len(kin_in) != 3:
                raise ValueError("kin_in must hold x, v and omega")
            kin = []
            for a, k in zip(kin_in, (2, 2, 1)):
                if isinstance(a, np.ndarray) and a.dtype == _F64 and a.size == k * n_p and a.flags.c_contiguous:
                    kin.append(self._io_addr(a))
                else:   # a converted copy, referenced until the call returns
                    a = _f64(a, k * n_p)
                    keep = (keep or ()) + (a,)
                    kin.append(a.ctypes.data)
            xi, vi, wi = kin
        outs = []
        for a, k in ((F, 2), (T, 1), (x, 2), (v, 2), (w, 1)):
            if a is None:
                outs.append(None)
                continue
            if not isinstance(a, np.ndarray) or a.size != k * n_p or a.dtype != _F64 or not a.flags.c_contiguous:
                raise ValueError(f"outputs must be contiguous float64 arrays of {k} x {n_p} values")
            outs.append(self._io_addr(a))
        rc = self._L.imb_step_io(self.h, int(n), xi, vi, wi, *outs)
        del keep
        self._check(rc)

    def step_async(self, n=1):
        self._check(self._L.imb_step_async(self.h, int(n)))

    def sync(self):
        self._check(self._L.imb_sync(self.h))

    def dem_step(self, n=1):
        self._check(self._L.imb_dem_step(self.h, int(n)))

    # ------------------------------------------------------------- readback
    def populations(self):
        out = np.zeros((9, self.ny, self.nx))
        self._check(self._L.imb_get_populations(self.h, _d(out)))
        return out

    def macro(self):
        rho, ux, uy = (np.zeros((self.ny, self.nx)) for _ in range(3))
        self._check(self._L.imb_get_macro(self.h, _d(rho), _d(ux), _d(uy)))
        return rho, ux, uy

    def forces(self, F=None, T=None):
        F = np.zeros((self.np, 2)) if F is None else F
        T = np.zeros(self.np) if T is None else T
        self._check(self._L.imb_get_forces(self.h, _d(F), _d(T)))
        return F, T

    def set_forces(self, F, T):
        F, T = _f64(F, 2 * self.np), _f64(T, self.np)
        self._check(self._L.imb_set_forces(self.h, _d(F), _d(T)))

    def particles(self, x=None, v=None, w=None):
        x = np.zeros((self.np, 2)) if x is None else x
        v = np.zeros((self.np, 2)) if v is None else v
        w = np.zeros(self.np) if w is None else w
        self._check(self._L.imb_get_particles(self.h, _d(x), _d(v), _d(w)))
        return x, v, w

    def drag_gradient(self, T, checkpoint_every=100, snapshots=None):
        """Time-averaged drag over T steps from the current state and its gradient with respect
        to the inlet velocity, tau and the disk centres: uniform checkpoints every
        ``checkpoint_every`` steps (imb_drag_gradient), or binomial checkpointing with
        ``snapshots`` snapshots when that is given (imb_drag_gradient_binomial)."""
        J, gu, gt = C.c_double(0.0), C.c_double(0.0), C.c_double(0.0)
        gx = np.zeros((max(self.np, 1), 2))
        if snapshots is None:
            rc = self._L.imb_drag_gradient(self.h, int(T), int(checkpoint_every), C.byref(J), C.byref(gu),
                                           C.byref(gt), _d(gx))
        else:
            rc = self._L.imb_drag_gradient_binomial(self.h, int(T), int(snapshots), C.byref(J), C.byref(gu),
                                                    C.byref(gt), _d(gx))
        self._check(rc)
        return J.value, gu.value, gt.value, gx[:self.np]

    def cell_map(self):
        count = np.zeros((self.ny, self.nx), dtype=np.int32)
        ids = np.zeros((self.ny, self.nx, MAX_SLOTS), dtype=np.int32)
        eps = np.zeros((self.ny, self.nx, MAX_SLOTS), dtype=np.float32)
        self._check(self._L.imb_get_cell_map(self.h, count.ctypes.data_as(_ip),
                                             ids.ctypes.data_as(_ip), eps.ctypes.data_as(_fp)))
        return count, ids, eps

    def contacts(self):
        n = C.c_int(0)
        self._check(self._L.imb_get_contacts(self.h, 0, None, C.byref(n)))
        pairs = np.zeros((max(n.value, 1), 2), dtype=np.int32)
        self._check(self._L.imb_get_contacts(self.h, n.value, pairs.ctypes.data_as(_ip), C.byref(n)))
        return pairs[:n.value]

    def bins(self):
        nb = ((self.nx + 31) // 32) * ((self.ny + 31) // 32)
        start = np.zeros(nb + 1, dtype=np.int32)
        ids = np.zeros(max(self.np, 1), dtype=np.int32)
        self._check(self._L.imb_get_bins(self.h, start.ctypes.data_as(_ip), ids.ctypes.data_as(_ip)))
        return start, ids[:self.np]

    # ----------------------------------------------------------------- misc
    def set_stream(self, stream_ptr: int | None):
        self._check(self._L.imb_set_stream(self.h, stream_ptr or None))

    @property
    def stream(self) -> int:
        return self._L.imb_get_stream(self.h) or 0

    def enable_kernel_timing(self, on=True):
        self._check(self._L.imb_enable_kernel_timing(self.h, int(on)))

    def kernel_time(self):
        ms = C.c_double(0.0)
        n = C.c_longlong(0)
        self._check(self._L.imb_kernel_time(self.h, C.byref(ms), C.byref(n)))
        return ms.value, n.value

    def launch_count(self) -> int:
        return int(self._L.imb_launch_count(self.h))

    def bytes_per_cell(self) -> float:
        return float(self._L.imb_bytes_per_cell(self.h))


class Batch:
    """Many independent periodic domains with fixed disks, stepped together (imb_batch_*).

    ``domains`` is a sequence of workloads (``workloads.Workload``, periodic in x and y, DEM
    off, disks at rest); their sizes, tau, Smagorinsky constant, body force and disks define
    the batch."""

    def __init__(self, domains, storage="fp16"):
        self._L = load()
        n = len(domains)
        nx = np.array([w.nx for w in domains], dtype=np.int32)
        ny = np.array([w.ny for w in domains], dtype=np.int32)
        tau = np.array([w.tau for w in domains], dtype=np.float64)
        csm = np.array([w.C_smag for w in domains], dtype=np.float64)
        fx = np.array([w.force[0] for w in domains], dtype=np.float64)
        fy = np.array([w.force[1] for w in domains], dtype=np.float64)
        nd = np.array([w.n_particles for w in domains], dtype=np.int32)
        xy = np.ascontiguousarray(np.concatenate([np.asarray(w.x, dtype=np.float64).reshape(-1, 2)
                                                  for w in domains] + [np.zeros((0, 2))]))
        r = np.ascontiguousarray(np.concatenate([np.asarray(w.r, dtype=np.float64).reshape(-1)
                                                 for w in domains] + [np.zeros(0)]))
        if xy.shape[0] == 0:
            xy, r = np.zeros((1, 2)), np.zeros(1)
        st = STORAGE_NAMES[storage] if isinstance(storage, str) else storage
        h = _vp()
        rc = self._L.imb_batch_create(C.byref(h), n, nx.ctypes.data_as(_ip), ny.ctypes.data_as(_ip), _d(tau),
                                      _d(csm), _d(fx), _d(fy), nd.ctypes.data_as(_ip), _d(xy), _d(r), st)
        self.h = h
        self.n = n
        self.shapes = [(int(a), int(b)) for a, b in zip(ny, nx)]
        self._check(rc)

    def _check(self, rc):
        if rc != IMB_OK:
            msg = self._L.imb_batch_last_error(self.h).decode() if self.h else ""
            raise ImbError(rc, msg)

    def run(self, steps):
        self._check(self._L.imb_batch_run(self.h, int(steps)))

    def autotune(self, steps_per_trial=20):
        blk, cpl, ms = C.c_int(0), C.c_int(0), C.c_double(0.0)
        self._check(self._L.imb_batch_autotune(self.h, int(steps_per_trial), C.byref(blk), C.byref(cpl),
                                               C.byref(ms)))
        return blk.value, cpl.value, ms.value

    def set_launch(self, block, cells_per_lane):
        """Pin the launch shape (imb_batch_set_launch)."""
        self._check(self._L.imb_batch_set_launch(self.h, int(block), int(cells_per_lane)))

    def mean_drag(self):
        fx, fy = np.zeros(self.n), np.zeros(self.n)
        self._check(self._L.imb_batch_mean_drag(self.h, _d(fx), _d(fy)))
        return fx, fy

    def populations(self, domain):
        ny, nx = self.shapes[domain]
        out = np.zeros((9, ny, nx))
        self._check(self._L.imb_batch_get_populations(self.h, int(domain), _d(out)))
        return out

    def cells(self):
        return int(self._L.imb_batch_cells(self.h))

    def close(self):
        if getattr(self, "h", None):
            self._L.imb_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Lattice3:
    """A D3Q19 lattice with held spheres (imb3_*; the paper's own lattice): up to two spheres per
    cell, the Smagorinsky closure when ``C_smag`` > 0, walls in y fixed or moving along x."""

    def __init__(self, nx, ny, nz, tau, wall_y=True, force=(0.0, 0.0, 0.0), n_sub=5, storage="fp32",
                 rho0=1.0, u0=(0.0, 0.0, 0.0), wall_u=(0.0, 0.0), C_smag=0.0):
        L = load()
        p = Params3()
        L.imb3_default_params(C.byref(p))
        p.wall_y = int(bool(wall_y))
        p.Fx, p.Fy, p.Fz = map(float, force)
        p.n_sub = int(n_sub)
        p.storage = STORAGE_NAMES[storage] if isinstance(storage, str) else int(storage)
        p.rho0 = float(rho0)
        p.ux0, p.uy0, p.uz0 = map(float, u0)
        p.wall_ux_bot, p.wall_ux_top = map(float, wall_u)
        p.C_smag = float(C_smag)
        h = _vp()
        rc = L.imb3_init(C.byref(h), int(nx), int(ny), int(nz), float(tau), C.byref(p))
        if rc != IMB_OK:
            msg = L.imb3_last_error(h if h.value else None).decode()
            if h.value:
                L.imb3_destroy(h)
            raise ImbError(rc, msg)
        self._L, self.h, self.params = L, h, p
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.np = 0

    @classmethod
    def from_workload(cls, w, storage="fp32"):
        lat = cls(w.nx, w.ny, w.nz, w.tau, wall_y=w.wall_y, force=w.force, n_sub=w.n_sub, storage=storage,
                  rho0=w.rho0, u0=w.u0, wall_u=w.wall_u, C_smag=w.C_smag)
        if w.n_spheres:
            lat.set_spheres(w.x, w.v, w.omega, w.R)
        return lat

    def _check(self, rc):
        if rc != IMB_OK:
            raise ImbError(rc, self._L.imb3_last_error(self.h).decode())

    def set_spheres(self, x, v, omega, R):
        n = int(np.asarray(R).reshape(-1).shape[0])
        self._check(self._L.imb3_set_spheres(self.h, n, _d(_f64(x, 3 * n)), _d(_f64(v, 3 * n)),
                                             _d(_f64(omega, 3 * n)), _d(_f64(R, n))))
        self.np = n

    def step(self, n=1):
        self._check(self._L.imb3_step(self.h, int(n)))

    def populations(self):
        out = np.zeros((19, self.nz, self.ny, self.nx))
        self._check(self._L.imb3_get_populations(self.h, _d(out)))
        return out

    def macro(self):
        shp = (self.nz, self.ny, self.nx)
        rho, ux, uy, uz = (np.zeros(shp) for _ in range(4))
        self._check(self._L.imb3_get_macro(self.h, _d(rho), _d(ux), _d(uy), _d(uz)))
        return rho, ux, uy, uz

    def forces(self):
        F, T = np.zeros((max(self.np, 1), 3)), np.zeros((max(self.np, 1), 3))
        self._check(self._L.imb3_get_forces(self.h, _d(F), _d(T)))
        return F[:self.np], T[:self.np]

    def cell_map(self):
        """Two slots per cell: covering spheres (lower index first, -1 none) and sub-cell counts,
        each [nz][ny][nx][2]."""
        shp = (self.nz, self.ny, self.nx, 2)
        sph, cnt = np.zeros(shp, dtype=np.int32), np.zeros(shp, dtype=np.int32)
        self._check(self._L.imb3_get_cell_map(self.h, sph.ctypes.data_as(_ip), cnt.ctypes.data_as(_ip)))
        return sph, cnt

    def enable_kernel_timing(self, on=True):
        self._check(self._L.imb3_enable_kernel_timing(self.h, int(bool(on))))

    def kernel_time(self):
        ms, n = C.c_double(0.0), C.c_longlong(0)
        self._check(self._L.imb3_kernel_time(self.h, C.byref(ms), C.byref(n)))
        return ms.value, n.value

    def launch_count(self):
        return self._L.imb3_launch_count(self.h)

    def bytes_per_cell(self):
        return self._L.imb3_bytes_per_cell(self.h)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self._L.imb3_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
