"""GPU (sm_103a) path against the FP64 oracle on the same seeded inputs.

Tolerances (FP32 populations, compared after the stated number of steps):
  * velocity field: relative L2 <= 1e-5 over the fluid cells (denominator ||u_oracle||);
  * populations: max |f_gpu - f_oracle| <= 1e-6 (FP32 storage of f - w: ~1e-8 per step);
  * per-particle force: |F_gpu - F_oracle| <= 1e-4 * max(|F_oracle|, mean_p |F_oracle|),
    torque likewise with the scale r * that force;
  * integer bookkeeping (bins, cells covered per particle, contact pairs) bit-exact;
  * solid ratio per cell within 2e-6 of the FP64 overlap area (FP32 geometry).
"""
import math

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def imb():
    import paper_1809_07008_gb300 as imb
    imb.load()
    return imb


def _fluid_mask(orc_sim):
    count, _, _ = orc_sim.cell_map() if orc_sim.np else (np.zeros(orc_sim.shape, int), None, None)
    return count == 0


def _u_rel_l2(g, o, mask):
    gu = np.stack(g[1:])[:, mask]
    ou = np.stack(o[1:])[:, mask]
    return np.linalg.norm(gu - ou) / np.linalg.norm(ou)


def _force_ok(Fg, Tg, Fo, To, r, tol=1e-4):
    scale = max(np.abs(Fo).max(), np.linalg.norm(Fo, axis=1).mean(), 1e-30)
    errF = np.abs(Fg - Fo).max() / scale
    errT = np.abs(Tg - To).max() / (scale * max(r.max(), 1.0))
    return errF, errT


def _run_pair(orc, imb, w, steps, storage="fp32", **kw):
    o = orc.Sim(w)
    g = imb.Lattice.from_workload(w, storage=storage, **kw)
    o.step(steps)
    g.step(steps)
    return o, g


# work units: 1 = tiles handed out to a persistent grid, 2 = eight-row units, one per block
UNITS = [1, 2]


@pytest.mark.parametrize("units", UNITS)
@pytest.mark.parametrize("bc", ["channel", "periodic_forced_smag", "closed_box", "walls_x_periodic_y"])
def test_fluid_only_parity(orc, imb, bc, units):
    # the boundary rules on lattices that are not multiples of the tile (the corners of the
    # ghost frame: bounce-back, periodic images and their precedence)
    if bc == "walls_x_periodic_y":
        w = W.Workload(name="wp", nx=50, ny=37, tau=0.7, bc_x=W.BC_WALL, bc_y=W.BC_PERIODIC,
                       force=(1e-6, 3e-5), u0=(-0.01, 0.02))
    elif bc == "channel":
        w = W.Workload(name="ch", nx=70, ny=45, tau=0.6, bc_x=W.BC_INLET_OUTLET, bc_y=W.BC_WALL,
                       u_in=(0.02, 0.0))
    elif bc == "periodic_forced_smag":
        w = W.Workload(name="pf", nx=67, ny=40, tau=0.52, C_smag=0.15, bc_x=W.BC_PERIODIC,
                       bc_y=W.BC_WALL, force=(2e-5, 1e-6), u0=(0.01, 0.0))
    else:
        w = W.Workload(name="box", nx=64, ny=33, tau=0.8, bc_x=W.BC_WALL, bc_y=W.BC_WALL,
                       u0=(0.03, -0.02))
    o, g = _run_pair(orc, imb, w, 300, work_units=units)
    fo, fg = o.f(), g.populations()
    assert np.abs(fg - fo).max() < 1e-6
    mask = np.ones(o.shape, bool)
    assert _u_rel_l2(g.macro(), o.macro(), mask) < 1e-5


def test_initial_state_and_readback(orc, imb):
    w = W.Workload(name="init", nx=40, ny=35, tau=0.7, bc_x=W.BC_INLET_OUTLET, bc_y=W.BC_WALL,
                   u_in=(0.02, 0.0), u0=(0.01, 0.005), rho0=1.01)
    o = orc.Sim(w)
    g = imb.Lattice.from_workload(w)
    assert np.abs(g.populations() - o.f()).max() < 2e-7


@pytest.mark.parametrize("units", UNITS)
def test_channel_disk_c1_parity(orc, imb, units):
    # 200 x 100 channel, fixed disk d = 20 at the centre, u_in = 0.01, tau = 0.6 (2000 steps)
    w = W.c1(steps=2000)
    o, g = _run_pair(orc, imb, w, w.steps, work_units=units)
    mask = _fluid_mask(o)
    assert _u_rel_l2(g.macro(), o.macro(), mask) < 1e-5
    Fo, To = o.forces()
    Fg, Tg = g.forces()
    errF, errT = _force_ok(Fg, Tg, Fo, To, w.r)
    assert Fo[0, 0] > 0 and errF < 1e-4 and errT < 1e-4


def test_cell_map_bit_exact_and_eps(orc, imb):
    w = W.c3sub(steps=0, nx=256, ny=192)
    o = orc.Sim(w)
    g = imb.Lattice.from_workload(w)
    co, io, eo = o.cell_map()
    cg, ig, eg = g.cell_map()
    assert np.array_equal(co, cg)
    assert np.array_equal(io, ig)
    assert np.abs(eg - eo).max() < 2e-6
    # sum of the solid ratios of each disk equals its area
    for p in range(w.n_particles):
        tot = eg[ig == p].sum(dtype=np.float64)
        assert abs(tot - math.pi * w.r[p] ** 2) < 1e-5 * math.pi * w.r[p] ** 2


def test_cell_map_subcell_bit_exact(orc, imb):
    w = W.c3sub(steps=0, nx=128, ny=128).with_(eps_mode=W.EPS_SUBCELL, n_sub=5)
    o = orc.Sim(w)
    g = imb.Lattice.from_workload(w)
    co, io, eo = o.cell_map()
    cg, ig, eg = g.cell_map()
    assert np.array_equal(co, cg) and np.array_equal(io, ig)
    assert np.abs(eg - eo).max() < 1e-7


def test_bins_bit_exact(orc, imb):
    w = W.c3sub(steps=0, nx=512, ny=512)
    o = orc.Sim(w)
    g = imb.Lattice.from_workload(w)
    so, ido = o.bins(32)
    sg, idg = g.bins()
    assert np.array_equal(so, sg) and np.array_equal(ido, idg)


def _pile(rows=6, cols=10, R=8.0, overlap=3e-4, seed=5, gy=-2e-3, e=0.5, mu=0.5, N_sub=50,
          speed=1e-3):
    """Disks on a triangular lattice in a box just wide enough to hold them: neighbours
    overlap by ~``overlap`` (radii jittered by +-1e-4), the bottom row rests on the wall
    y = 0, small random velocities, gravity down."""
    rng = W.SplitMix64(seed)
    s = 2 * R - overlap
    xs, rs = [], []
    for j in range(rows):
        for i in range(cols):
            xs.append((R + 0.3 + i * s + (j % 2) * s / 2, R - 1e-4 + j * s * math.sqrt(3) / 2))
            rs.append(R + rng.uniform_range(-1e-4, 1e-4))
    n = len(rs)
    v = W.random_directions(n, speed, seed + 1)
    nx = int(math.ceil(2 * R + 0.6 + (cols - 0.5) * s))
    ny = int(rows * s + 3 * R)
    return W.Workload(name="pile", nx=nx, ny=ny, tau=0.6, bc_x=W.BC_WALL, bc_y=W.BC_WALL, dem_on=1,
                      N_sub=N_sub, gravity=(0.0, gy), e_rest=e, mu=mu, x=np.array(xs), v=v,
                      omega=np.zeros(n), r=np.array(rs))


def test_contacts_bit_exact(orc, imb):
    w = _pile()
    o = orc.Sim(w)
    g = imb.Lattice.from_workload(w)
    po, pg = o.contacts(), g.contacts()
    assert len(po) > 10
    assert np.array_equal(po, pg)


def test_dem_only_trajectories_bit_exact(orc, imb):
    # DEM alone (fluid force held at zero): the GPU sub-cycles reproduce the sequential
    # FP64 evaluation of Eqs. 7-11 bit for bit, contacts and walls included
    w = _pile()
    o = orc.Sim(w)
    g = imb.Lattice.from_workload(w)
    cycles = 40
    o.dem_substeps(cycles * w.N_sub)
    g.dem_step(cycles)
    xo, vo, wo = o.particles()
    xg, vg, wg = g.particles()
    assert np.array_equal(xo, xg) and np.array_equal(vo, vg) and np.array_equal(wo, wg)
    assert np.array_equal(o.contacts(), g.contacts())
    assert len(o.contacts()) > 10


def test_dem_only_hertz_mindlin_bit_exact(orc, imb):
    # the paper's contact law (simplified Hertz-Mindlin, Sec. 2.2) on the same pile: the GPU
    # sub-cycles reproduce the oracle bit for bit
    w = _pile().with_(contact_model=1, E_young=2.0e6, nu_poisson=0.3)
    o = orc.Sim(w)
    g = imb.Lattice.from_workload(w)
    cycles = 40
    o.dem_substeps(cycles * w.N_sub)
    g.dem_step(cycles)
    xo, vo, wo = o.particles()
    xg, vg, wg = g.particles()
    assert np.array_equal(xo, xg) and np.array_equal(vo, vg) and np.array_equal(wo, wg)
    assert np.array_equal(o.contacts(), g.contacts())
    assert len(o.contacts()) > 10
    # the pile settles differently under the two laws
    lin = orc.Sim(_pile())
    lin.dem_substeps(cycles * w.N_sub)
    assert not np.array_equal(lin.particles()[0], xo)
    g.close()
    with pytest.raises(imb.ImbError):       # Hertz-Mindlin needs a material
        imb.Lattice.from_workload(_pile().with_(contact_model=1, E_young=0.0))


def test_dem_only_with_frozen_fluid_force_bit_exact(orc, imb):
    w = _pile(rows=4, cols=10, seed=9)
    rng = np.random.default_rng(9)
    F = 1e-2 * rng.standard_normal((w.n_particles, 2))
    T = 1e-2 * rng.standard_normal(w.n_particles)
    o = orc.Sim(w)
    g = imb.Lattice.from_workload(w)
    o.set_forces(F, T)
    g.set_forces(F, T)
    o.dem_substeps(10 * w.N_sub)
    g.dem_step(10)
    for a, b in zip(o.particles(), g.particles()):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("bc_x", [W.BC_WALL, W.BC_PERIODIC])
def test_dem_gas_quiet_and_touching_islands_bit_exact(orc, imb, bc_x):
    # a dilute gas of disks: candidate pairs far enough apart to move freely through the
    # cycle, pairs that collide, separate again and cross the periodic edge, all bit for bit
    nx, ny, n, R = 160, 120, 100, 5.0
    x, r = W.random_sequential_addition(nx, ny, n, lambda g: R + g.uniform_range(-0.5, 0.5), 11, gap=0.3,
                                        periodic_x=bc_x == W.BC_PERIODIC, wall_gap=0.3)
    v = W.random_directions(n, 0.06, 12)
    w = W.Workload(name="gas", nx=nx, ny=ny, tau=0.6, bc_x=bc_x, bc_y=W.BC_WALL, dem_on=1, N_sub=20,
                   gravity=(0.0, -1e-4), e_rest=0.7, mu=0.3, x=x, v=v, omega=np.zeros(n), r=r)
    o = orc.Sim(w)
    g = imb.Lattice.from_workload(w)
    rng = np.random.default_rng(3)
    F = 1e-1 * rng.standard_normal((n, 2))
    T = 1e-1 * rng.standard_normal(n)
    o.set_forces(F, T)
    g.set_forces(F, T)
    touched = 0
    for cycle in range(240):
        o.dem_substeps(w.N_sub)
        g.dem_step(1)
        touched += len(o.contacts()) > 0
        if cycle % 20 == 19:
            for a, b in zip(o.particles(), g.particles()):
                assert np.array_equal(a, b)
    assert touched >= 10


def _edge_velocities(rng, n):
    """Velocity components on the hard cases of the free particles' repeated velocity sums:
    zero, values a few ulps from powers of two (the sums cross into the next binade within a
    cycle), tiny values that change sign, and magnitudes from 1e-9 to 0.1."""
    out = np.empty(n)
    for k in range(n):
        kind = k % 5
        if kind == 0:
            out[k] = 0.0
        elif kind in (1, 2):
            p = 2.0 ** -int(rng.integers(4, 30))
            ulps = int(rng.integers(1, 6)) * (1 if kind == 1 else -1)
            out[k] = np.nextafter(p, np.inf if ulps > 0 else 0.0)
            for _ in range(abs(ulps) - 1):
                out[k] = np.nextafter(out[k], np.inf if ulps > 0 else 0.0)
            out[k] *= rng.choice([-1.0, 1.0])
        elif kind == 3:
            out[k] = rng.uniform(-1e-9, 1e-9)
        else:
            out[k] = rng.choice([-1.0, 1.0]) * 10.0 ** rng.uniform(-9, -1)
    return rng.permutation(out)


def test_free_particles_bit_exact_across_binades(orc, imb):
    # disks far apart in a periodic box (no contacts, no walls): every sub-cycle is a free
    # update (the register-only path, or the sub-cycle loop near the periodic edges);
    # velocities and accelerations chosen so that the sums cross powers of two, pass through
    # zero and fall below the ulp, compared with the oracle's sequential FP64 updates bit for bit
    n = 120
    rng = np.random.default_rng(21)
    x, r = W.random_sequential_addition(480, 360, n, lambda g: 4.0 + g.uniform_range(-0.5, 0.5), 21, gap=12.0,
                                        periodic_x=True, wall_gap=2.0)
    v = np.stack([_edge_velocities(rng, n), _edge_velocities(rng, n)], axis=1)
    om = _edge_velocities(rng, n)
    w = W.Workload(name="free_gas", nx=480, ny=360, tau=0.6, bc_x=W.BC_PERIODIC, bc_y=W.BC_PERIODIC, dem_on=1,
                   N_sub=100, gravity=(0.0, 0.0), x=x, v=v, omega=om, r=r)
    m = w.rho_s * np.pi * r ** 2
    F = (rng.choice([-1.0, 1.0], (n, 2)) * 10.0 ** rng.uniform(-9, -3, (n, 2))) * m[:, None] * 10.0
    F[::7] = 0.0
    T = rng.choice([-1.0, 1.0], n) * 10.0 ** rng.uniform(-9, -3, n) * m * r ** 2 * 5.0
    o = orc.Sim(w)
    g = imb.Lattice.from_workload(w)
    o.set_forces(F, T)
    g.set_forces(F, T)
    for cycle in range(12):
        o.dem_substeps(w.N_sub)
        g.dem_step(1)
        assert len(o.contacts()) == 0
        for a, b in zip(o.particles(), g.particles()):
            assert np.array_equal(a, b), cycle
    g.close()


@pytest.mark.parametrize("units", UNITS)
def test_moving_particles_coupled_parity(orc, imb, units):
    # c3 at the same density on 256 x 192: DEM + IMB + Smagorinsky, tau = 0.51, 1000 coupling
    # cycles (the horizon the FP32 bars are stated for)
    w = W.c3sub(steps=0, nx=256, ny=192)
    o, g = _run_pair(orc, imb, w, 1000, work_units=units)
    mask = _fluid_mask(o)
    assert _u_rel_l2(g.macro(), o.macro(), mask) < 1e-5
    Fo, To = o.forces()
    Fg, Tg = g.forces()
    errF, errT = _force_ok(Fg, Tg, Fo, To, w.r)
    assert errF < 1e-4 and errT < 1e-4
    # trajectories: FP64 DEM driven by forces within the FP32 bar; the disks move ~5 cells
    xo, vo, _ = o.particles()
    xg, vg, _ = g.particles()
    assert np.abs(xo - w.x).max() > 2.0
    assert np.abs(xo - xg).max() < 2e-5
    assert np.abs(vo - vg).max() < 1e-5 * np.abs(vo).max()


@pytest.mark.parametrize("units", UNITS)
def test_doubly_periodic_suspension_parity(orc, imb, units):
    # moving disks in a box periodic in x and y whose sides are not multiples of the tile: the
    # flow crosses the periodic images of the ghost frame, corners included, with gradients
    w = W.c3sub(steps=0, nx=200, ny=150).with_(bc_y=W.BC_PERIODIC)
    o, g = _run_pair(orc, imb, w, 300, work_units=units)
    mask = _fluid_mask(o)
    assert _u_rel_l2(g.macro(), o.macro(), mask) < 1e-5
    Fo, To = o.forces()
    Fg, Tg = g.forces()
    errF, errT = _force_ok(Fg, Tg, Fo, To, w.r)
    assert errF < 1e-4 and errT < 1e-4


def test_collapse_stack_coupled_parity(orc, imb):
    # the collapse case's physics on 256 x 192: a closed box, 30 disks d ~ U[16, 24] stacked
    # 0.2 cells apart above the bottom wall, buoyant gravity, tau = 0.52, Smagorinsky C = 0.1;
    # the fluid, the hydrodynamic forces, wall contacts and then pair contacts, 1000 cycles.
    # Element by element at every 100th cycle while no pair touches: velocity 1e-5, forces 1e-4,
    # positions 2e-5.  Once pairs touch, the contact springs (k_n = 1e5) turn the FP32 force
    # difference into a difference of contact onset, and a position difference of 1e-6 cells
    # into 0.1 of contact force (the hydrodynamic forces are ~0.06): the two runs then separate
    # as any perturbed run of a granular pile does.  What they still share is checked at the
    # end: the same pairs in contact and positions within 5e-3 cells.
    w = W.c2_stack()
    o = orc.Sim(w)
    g = imb.Lattice.from_workload(w)
    first_contact = None
    for k in range(1, 11):
        o.step(100)
        g.step(100)
        if first_contact is None and len(o.contacts()):
            first_contact = 100 * k
        if first_contact is None:
            mask = _fluid_mask(o)
            assert _u_rel_l2(g.macro(), o.macro(), mask) < 1e-5, k
            Fo, To = o.forces()
            Fg, Tg = g.forces()
            errF, errT = _force_ok(Fg, Tg, Fo, To, w.r)
            assert errF < 1e-4 and errT < 1e-4, k
            assert np.abs(g.particles()[0] - o.particles()[0]).max() < 2e-5, k
    assert first_contact is not None and first_contact >= 300
    xo, _, _ = o.particles()
    xg, _, _ = g.particles()
    assert (xo[:, 1] - w.r).min() < 0.05             # disks resting on the bottom wall
    assert len(o.contacts()) >= 3
    assert np.array_equal(g.contacts(), o.contacts())
    assert np.abs(xo - xg).max() < 5e-3


@pytest.mark.parametrize("storage,tol", [("fp16", 1e-2), ("bf16", 5e-2)])
def test_shifted_low_precision_forces_suspension(orc, imb, storage, tol):
    # populations stored as f_i - w_i in 16 bits, FP32 arithmetic: per-particle hydrodynamic
    # forces after 1000 steps of the suspension at the 8192 x 4096 case's disk density, against
    # the FP64 oracle.  Each particle's error is taken relative to its own force, or to the mean
    # force where its own is smaller: FP16 within 1 %, BF16 (8 significant bits) within 5 %.
    w = W.c3sub(steps=0, nx=256, ny=192)
    o, g = _run_pair(orc, imb, w, 1000, storage=storage)
    Fo, _ = o.forces()
    Fg, _ = g.forces()
    mag = np.linalg.norm(Fo, axis=1)
    err = np.linalg.norm(Fg - Fo, axis=1) / np.maximum(mag, mag.mean())
    assert err.max() < tol, (err.max(), err.argmax())


@pytest.mark.parametrize("storage,tol", [("fp16", 1e-2), ("bf16", 2e-2)])
def test_shifted_low_precision_drag_channel(orc, imb, storage, tol):
    # channel with one fixed disk at u_in = 0.01 for 2000 steps: the drag comes from the
    # small residual velocity inside the disk, where 16-bit storage is weakest (measured on a
    # GB300: FP16 0.7 %, BF16 0.8 %; FP16 must stay below 1 %)
    w = W.c1(steps=2000)
    o, g = _run_pair(orc, imb, w, w.steps, storage=storage)
    Fo, _ = o.forces()
    Fg, _ = g.forces()
    assert abs(Fg[0, 0] - Fo[0, 0]) / abs(Fo[0, 0]) < tol


def test_mass_conserved_on_gpu(imb):
    w = W.c3sub(steps=0, nx=128, ny=96).with_(bc_y=W.BC_PERIODIC, tau=0.53)
    g = imb.Lattice.from_workload(w)
    m0 = g.macro()[0].sum()
    g.step(1000)
    assert abs(g.macro()[0].sum() - m0) / m0 < 1e-6   # FP32 storage of f - w


# ----------------------------------------------------------------- error paths
def test_invalid_arguments(imb):
    with pytest.raises(imb.ImbError) as e:
        imb.Lattice(2, 10, 0.6)
    assert e.value.code == -1
    with pytest.raises(imb.ImbError):
        imb.Lattice(64, 64, 0.6, work_units=3)
    with pytest.raises(imb.ImbError):
        imb.Lattice(64, 64, 0.6, plain_launches=2)
    with pytest.raises(imb.ImbError):
        imb.Lattice(10, 10, 0.5)
    lat = imb.Lattice(64, 64, 0.6)
    with pytest.raises(imb.ImbError):
        lat.set_particles([[10.0, 10.0]], [[0, 0]], [0.0], [-1.0])
    with pytest.raises(imb.ImbError):
        lat.set_particles([[70.0, 10.0]], [[0, 0]], [0.0], [5.0])


def test_mach_guard_reports_unstable(imb):
    lat = imb.Lattice(64, 32, 0.6, bc_x=imb.BC_INLET_OUTLET, u_in_x=0.45)
    with pytest.raises(imb.ImbError) as e:
        lat.step(5)
    assert e.value.code == -4


def test_skin_violation_reported(imb):
    # a lone particle crossing two cells in one coupling cycle breaks the neighbour-list skin
    w = _pile(rows=1, cols=3, seed=3)
    w = w.with_(nx=200, ny=100, x=np.array([[30.0, 60.0], [120.0, 8.0], [150.0, 8.0]]),
                v=np.array([[2.0, 0.0], [0.0, 0.0], [0.0, 0.0]]), gravity=(0.0, 0.0))
    lat = imb.Lattice.from_workload(w)
    with pytest.raises(imb.ImbError) as e:
        lat.dem_step(1)
    assert e.value.code == -7


def test_host_wait_is_bounded(imb):
    # a 1 ms bound on a queued 4096^2 step returns IMB_E_TIMEOUT; the context stays usable
    lat = imb.Lattice(4096, 4096, 0.6, timeout_ms=1)
    lat.step_async(50)
    with pytest.raises(imb.ImbError) as e:
        lat.sync()
    assert e.value.code == -6
    import time
    for _ in range(600):
        try:
            lat.sync()
            break
        except imb.ImbError:
            time.sleep(0.05)
    lat.sync()


def test_couette_moving_walls(orc, imb):
    # walls y = 0 and y = H moving along x at -u_w and +u_w (Sec. 3.4): the fluid-only
    # steady profile is the exact line in FP32, and a suspension between the moving walls
    # (DEM on, the 8192 x 4096 case's density) matches the oracle after 200 steps
    H, tau, uw = 16, 0.8, 0.01
    w = W.Workload(name="couette", nx=64, ny=H, tau=tau, bc_x=W.BC_PERIODIC, bc_y=W.BC_WALL, wall_u=(-uw, uw))
    g = imb.Lattice.from_workload(w)
    nu = (tau - 0.5) / 3.0
    g.step(int(30 * H * H / (nu * math.pi ** 2)))
    _, ux, uy = g.macro()
    y = np.arange(H) + 0.5
    assert np.abs(ux - (-uw + 2 * uw * y / H)[:, None]).max() < 2e-6 * uw / 0.01
    assert np.abs(uy).max() < 1e-7
    g.close()
    ws = W.c3sub(steps=0, nx=128, ny=96).with_(wall_u=(-uw, uw))
    o, g = _run_pair(orc, imb, ws, 200)
    assert _u_rel_l2(g.macro(), o.macro(), _fluid_mask(o)) < 1e-5
    Fo, To = o.forces()
    Fg, Tg = g.forces()
    errF, errT = _force_ok(Fg, Tg, Fo, To, ws.r)
    assert errF < 1e-4 and errT < 1e-4
    g.close()


def test_drag_gradient_refuses_moving_walls(imb):
    w = W.c4(steps=0, nx=96, ny=48, n_side=1).with_(wall_u=(0.0, 0.01))
    g = imb.Lattice.from_workload(w)
    with pytest.raises(imb.ImbError):
        g.drag_gradient(10)
    g.close()


@pytest.mark.parametrize("pinned", [False, True])
def test_step_io_equals_separate_calls(imb, pinned):
    # imb_step_io (upload, cycles, read-back, one wait) gives what the separate calls give, to the
    # bit (the forces are summed in a fixed order); pinned host arrays take the one-launch upload
    # and read-back through host memory, pageable ones the copies
    w = W.c3sub(steps=0, nx=128, ny=96)
    a = imb.Lattice.from_workload(w)
    b = imb.Lattice.from_workload(w)
    a.step(3)
    b.step(3)
    x, v, om = a.particles()
    x = x + 0.01
    n = w.n_particles

    def buf(arr):
        if not pinned:
            return np.ascontiguousarray(arr)
        import torch
        return torch.from_numpy(np.ascontiguousarray(arr)).pin_memory().numpy()

    xi, vi, wi = buf(x), buf(v), buf(om)
    F, T = buf(np.zeros((n, 2))), buf(np.zeros(n))
    xo, vo, wo = buf(np.zeros((n, 2))), buf(np.zeros((n, 2))), buf(np.zeros(n))
    a.step_io(2, (xi, vi, wi), F, T, xo, vo, wo)
    b.set_kinematics(x, v, om)
    b.step(2)
    Fb, Tb = b.forces()
    xb, vb, wb = b.particles()
    assert np.array_equal(xo, xb) and np.array_equal(vo, vb) and np.array_equal(wo, wb)
    assert np.array_equal(F, Fb) and np.array_equal(T, Tb)
    assert np.array_equal(a.populations(), b.populations())
    # again with the same arrays (the binding looks each array object's address up once), then
    # with fresh arrays, one input Fortran-ordered (converted to a contiguous copy for the call)
    for fresh in (False, True):
        kin = (xo.copy(), vo.copy(), wo.copy())
        if fresh:
            F, T, xo, vo, wo = (buf(np.zeros_like(o)) for o in (F, T, xo, vo, wo))
            ins = (buf(kin[0]), np.asfortranarray(kin[1]), buf(kin[2]))
        else:
            ins = (xo, vo, wo)
        a.step_io(1, ins, F, T, xo, vo, wo)
        b.set_kinematics(*kin)
        b.step(1)
        Fb, Tb = b.forces()
        xb, vb, wb = b.particles()
        assert np.array_equal(xo, xb) and np.array_equal(vo, vb) and np.array_equal(wo, wb)
        assert np.array_equal(F, Fb) and np.array_equal(T, Tb)
    a.step_io(1)                       # no arrays: just the cycles and the wait
    b.step(1)
    with pytest.raises(ValueError):
        a.step_io(1, None, np.zeros(3))
    # centres outside the lattice, or NaN, are refused before anything is uploaded
    xs, _, _ = a.particles()
    for bad in ((0, 0, w.nx + 0.5), (1, 1, -1e-9), (2, 0, float("nan"))):
        xb = xs.copy()
        xb[bad[0], bad[1]] = bad[2]
        with pytest.raises(imb.ImbError):
            a.set_kinematics(xb, v, om)
        with pytest.raises(imb.ImbError):
            a.step_io(1, (xb, v, om), F, T)
    assert np.array_equal(a.particles()[0], xs)
    a.close()
    b.close()


@pytest.mark.parametrize("units", UNITS)
def test_cycle_graph_equals_launches(imb, units):
    # a coupling cycle with the DEM replays a captured CUDA graph (timed, with its event nodes
    # re-pointed every replay, or untimed) unless plain_launches asks for kernel launches: all
    # three give the same state to the bit and count the same launches and timed cycles, and a
    # new particle set between cycles (another count, another table shape) is taken up
    w = W.c3sub(steps=0, nx=160, ny=96)
    g = imb.Lattice.from_workload(w, work_units=units)
    gt = imb.Lattice.from_workload(w, work_units=units)
    p = imb.Lattice.from_workload(w, work_units=units, plain_launches=1)
    lats = (g, gt, p)
    gt.enable_kernel_timing(True)
    p.enable_kernel_timing(True)
    n0 = [lat.launch_count() for lat in lats]
    for lat in lats:
        lat.step(5)
    assert len({lat.launch_count() - n for lat, n in zip(lats, n0)}) == 1
    (mt, kt), (mp, kp) = gt.kernel_time(), p.kernel_time()
    assert kt == kp == 5 and mt > 0 and mp > 0
    x, v, om = g.particles()
    keep = slice(0, max(1, w.n_particles // 2))
    r = np.asarray(w.r)[keep] * 0.9
    for lat in lats:
        lat.set_particles(x[keep], v[keep], om[keep], r)
        lat.step(4)
    for o in (gt, p):
        for a, b in zip(g.particles() + g.forces(), o.particles() + o.forces()):
            assert np.array_equal(a, b)
        assert np.array_equal(g.populations(), o.populations())
        assert np.array_equal(g.contacts(), o.contacts())
    assert gt.kernel_time()[1] == p.kernel_time()[1] == 4
    for lat in lats:
        lat.close()


@pytest.mark.parametrize("units", UNITS)
def test_lattice_step_graphs_equal_launches(imb, units):
    # without the DEM, untimed runs of eight lattice steps replay a captured graph and the rest
    # are launched: the channel with its fixed disk, 21 steps in calls of 3, 13 and 5 (a call
    # shorter than eight, one with a replay and a remainder), equals plain launches, timed or
    # not, to the bit
    w = W.c1(steps=0)
    g = imb.Lattice.from_workload(w, work_units=units)
    gt = imb.Lattice.from_workload(w, work_units=units)
    p = imb.Lattice.from_workload(w, work_units=units, plain_launches=1)
    lats = (g, gt, p)
    gt.enable_kernel_timing(True)
    p.enable_kernel_timing(True)
    n0 = [lat.launch_count() for lat in lats]
    for k in (3, 13, 5):
        for lat in lats:
            lat.step(k)
    assert len({lat.launch_count() - n for lat, n in zip(lats, n0)}) == 1
    assert gt.kernel_time()[1] == p.kernel_time()[1] == 21
    for o in (gt, p):
        assert np.array_equal(g.populations(), o.populations())
        for a, b in zip(g.forces(), o.forces()):
            assert np.array_equal(a, b)
    for lat in lats:
        lat.close()


def test_lid_driven_cavity_parity(orc, imb):
    # moving top wall meeting the fixed side walls at the corners: GPU against the oracle
    w = W.Workload(name="cavity", nx=96, ny=64, tau=0.7, bc_x=W.BC_WALL, bc_y=W.BC_WALL, wall_u=(0.0, 0.05))
    o, g = _run_pair(orc, imb, w, 500)
    assert np.abs(g.populations() - o.f()).max() < 1e-6
    assert _u_rel_l2(g.macro(), o.macro(), np.ones((w.ny, w.nx), bool)) < 1e-5
    g.close()
