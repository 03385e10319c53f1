"""Pins of the oracle's DEM (Eqs. 7-11, Sec. 2.4 sub-cycling) and particle mapping.

* two-disk head-on collision against the damped linear oscillator: contact time
  pi / omega_d and restitution e (the damping is set from e);
* the simplified Hertz-Mindlin law (the paper's, Sec. 2.2): an undamped head-on impact against
  the closed-form Hertz peak overlap, contact time and rebound speed; with damping the
  restitution falls as e falls and lies near e;
* free flight under buoyancy-reduced gravity against the closed-form sum of the
  leapfrog recurrence;
* a disk sliding on a wall decelerates at mu g until it rolls at 2/3 of its
  initial speed (Coulomb cap of Eq. 9 with the torque of Eq. 11);
* contact lists on hand-built layouts (strict overlap, periodic image);
* bins of the particle-to-lattice map against a stable sort;
* a disk moving with a uniform flow feels no force and leaves the flow uniform
  (Eq. 12 with u_s = u_f).
"""
import math

import numpy as np
import pytest

import workloads as W


def _dem_only(nx=400, ny=200, bc_x=W.BC_PERIODIC, bc_y=W.BC_WALL, N_sub=1000, g=(0.0, 0.0),
              e=0.5, mu=0.5, x=(), v=(), r=()):
    n = len(r)
    return W.Workload(name="dem", nx=nx, ny=ny, tau=0.6, bc_x=bc_x, bc_y=bc_y, dem_on=1,
                      N_sub=N_sub, gravity=g, e_rest=e, mu=mu,
                      x=np.array(x, dtype=float).reshape(n, 2),
                      v=np.array(v, dtype=float).reshape(n, 2), omega=np.zeros(n),
                      r=np.array(r, dtype=float))


@pytest.mark.parametrize("N_sub,tol", [(1000, 1e-2), (4000, 2e-3)])
def test_head_on_collision_matches_damped_oscillator(orc, N_sub, tol):
    # the contact opens at a fraction of a sub-step, so e converges at first order in dt
    R, v0, e = 10.0, 0.01, 0.5
    w = _dem_only(x=[(100.0, 100.0), (120.002, 100.0)], v=[(v0, 0.0), (-v0, 0.0)], r=[R, R], e=e,
                  N_sub=N_sub)
    sim = orc.Sim(w)
    dt = 1.0 / w.N_sub
    m = w.rho_s * math.pi * R * R
    mstar = m / 2
    zeta = -math.log(e) / math.sqrt(math.pi ** 2 + math.log(e) ** 2)
    cn = 2 * zeta * math.sqrt(mstar * w.kn)
    wd = math.sqrt(w.kn / mstar - (cn / (2 * mstar)) ** 2)
    tc = math.pi / wd
    in_contact = 0
    for _ in range(int(0.8 * N_sub)):
        sim.dem_substeps(1)
        x, v, om = sim.particles()
        if len(sim.contacts()):
            in_contact += 1
        assert abs(v[0, 0] + v[1, 0]) < 1e-17          # equal and opposite contact forces
        assert np.all(om == 0.0) and np.all(v[:, 1] == 0.0)
    x, v, _ = sim.particles()
    assert abs(in_contact * dt - tc) <= 2 * dt
    e_meas = (v[1, 0] - v[0, 0]) / (2 * v0)
    assert abs(e_meas - e) < tol
    assert v[0, 0] < 0 < v[1, 0]


def test_free_flight_leapfrog_closed_form(orc):
    g = (0.0, -1.0e-3)
    x0, v0 = (50.3, 120.7), (0.004, 0.002)
    w = _dem_only(N_sub=100, g=g, x=[x0], v=[v0], r=[8.0])
    sim = orc.Sim(w)
    n = 700
    sim.dem_substeps(n)
    x, v, _ = sim.particles()
    dt = 1.0 / w.N_sub
    a = (1.0 - 1.0 / w.rho_s) * g[1]                       # buoyancy-reduced gravity
    # leapfrog: v_k = v0 + k a dt, x_n = x0 + sum_k v_k dt = x0 + n v0 dt + a dt^2 n (n+1) / 2
    assert v[0, 1] == pytest.approx(v0[1] + n * a * dt, rel=1e-12)
    assert x[0, 1] == pytest.approx(x0[1] + n * v0[1] * dt + a * dt * dt * n * (n + 1) / 2, rel=1e-12)
    assert x[0, 0] == pytest.approx(x0[0] + n * v0[0] * dt, rel=1e-12)
    assert v[0, 0] == v0[0]


def test_sliding_disk_decelerates_at_mu_g_then_rolls(orc):
    R, g, mu, v0 = 10.0, 1.0e-2, 0.3, 0.05
    rho_s = 2.65
    m = rho_s * math.pi * R * R
    geff = (1.0 - 1.0 / rho_s) * g
    kn = 1.0e5
    y0 = R - m * geff / kn                                  # resting on the wall y = 0
    w = _dem_only(N_sub=100, g=(0.0, -g), mu=mu, x=[(50.0, y0)], v=[(v0, 0.0)], r=[R])
    sim = orc.Sim(w)
    t, vs, ws = [], [], []
    for k in range(1200):
        sim.dem_substeps(1)
        _, v, om = sim.particles()
        t.append((k + 1) / w.N_sub)
        vs.append(v[0, 0])
        ws.append(om[0])
    t, vs, ws = map(np.array, (t, vs, ws))
    tstar = v0 / (3 * mu * geff)                           # v0 - mu g t = 2 mu g t
    sl = (t > 0.2 * tstar) & (t < 0.8 * tstar)
    slope = np.polyfit(t[sl], vs[sl], 1)[0]
    assert slope == pytest.approx(-mu * geff, rel=2e-2)
    assert vs[-1] == pytest.approx(2 * v0 / 3, rel=1e-2)
    assert -ws[-1] * R == pytest.approx(vs[-1], rel=1e-2)   # rolling: v = -w r for z-up rotation


def test_contact_list_hand_layout(orc):
    # periodic in x (nx = 100): 0-1 overlap by 0.01; 1-2 apart by 0.01; 0-3 touch through the
    # periodic image (distance 8 < 10); 0-4 exactly at contact distance (no overlap: strict)
    x = [(3.0, 30.0), (12.99, 30.0), (23.0, 30.0), (95.0, 30.0), (3.0, 40.0)]
    w = _dem_only(nx=100, ny=60, x=x, v=[(0, 0)] * 5, r=[5.0] * 5)
    sim = orc.Sim(w)
    assert sim.contacts().tolist() == [[0, 1], [0, 3]]


def test_bins_are_a_stable_sort_by_bin(orc):
    rng = np.random.default_rng(21)
    n = 300
    x = np.stack([rng.uniform(0, 200, n), rng.uniform(0, 100, n)], axis=1)
    w = _dem_only(nx=200, ny=100, x=x, v=np.zeros((n, 2)), r=np.full(n, 1.0))
    sim = orc.Sim(w)
    start, ids = sim.bins(32)
    nbx, nby = 7, 4
    b = np.floor(x[:, 1] / 32).astype(int) * nbx + np.floor(x[:, 0] / 32).astype(int)
    assert np.array_equal(np.diff(start), np.bincount(b, minlength=nbx * nby))
    assert np.array_equal(ids, np.argsort(b, kind="stable"))


def test_comoving_disk_feels_no_force(orc):
    u = (0.03, -0.01)
    w = W.Workload(name="comoving", nx=64, ny=48, tau=0.7, bc_x=W.BC_PERIODIC, bc_y=W.BC_PERIODIC,
                   u0=u, x=np.array([[30.2, 20.7]]), v=np.array([u]), omega=np.zeros(1),
                   r=np.array([9.0]))
    sim = orc.Sim(w)
    sim.step(50)
    F, T = sim.forces()
    assert np.max(np.abs(F)) < 1e-14 and abs(T[0]) < 1e-13
    assert np.max(np.abs(sim.f() - orc.feq(1.0, *u)[:, None, None])) < 1e-14


def test_spinning_disk_torque_opposes_rotation(orc):
    w = W.Workload(name="spin", nx=64, ny=64, tau=0.8, bc_x=W.BC_PERIODIC, bc_y=W.BC_PERIODIC,
                   x=np.array([[32.0, 32.0]]), v=np.zeros((1, 2)), omega=np.array([1e-3]),
                   r=np.array([10.0]))
    sim = orc.Sim(w)
    sim.step(200)
    F, T = sim.forces()
    assert T[0] < 0
    assert np.max(np.abs(F)) < 1e-12 * abs(T[0])


def _hertz_collision(orc, E, nu, e, v0=0.01, R=10.0, N_sub=4000, steps=None):
    w = _dem_only(x=[(100.0, 100.0), (120.002, 100.0)], v=[(v0, 0.0), (-v0, 0.0)], r=[R, R], e=e,
                  N_sub=N_sub).with_(contact_model=1, E_young=E, nu_poisson=nu)
    sim = orc.Sim(w)
    in_contact, dmax = 0, 0.0
    for _ in range(steps or N_sub):
        sim.dem_substeps(1)
        x, v, om = sim.particles()
        if len(sim.contacts()):
            in_contact += 1
            dmax = max(dmax, 2 * R - (x[1, 0] - x[0, 0]))
        assert abs(v[0, 0] + v[1, 0]) < 1e-17
    x, v, _ = sim.particles()
    return w, in_contact / N_sub, dmax, (v[1, 0] - v[0, 0]) / (2 * v0)


def test_hertz_mindlin_head_on_collision_matches_closed_form(orc):
    # undamped (e = 1) Hertz impact of two disks: m* delta'' = -K delta^(3/2) with
    # K = 4/3 E* sqrt(R*), E* = E / (2 (1 - nu^2)): peak overlap (5 m* v^2 / (4 K))^(2/5) for the
    # approach speed v, duration 2 (delta_max / v) (2/5) B(2/5, 1/2), rebound at the approach speed
    R, v0, E, nu = 10.0, 0.01, 2.0e5, 0.3
    w, tc_meas, dmax, e_meas = _hertz_collision(orc, E, nu, 1.0, v0=v0, R=R)
    m = w.rho_s * math.pi * R * R
    mstar, Rstar = m / 2, R / 2
    K = 4.0 / 3.0 * E / (2 * (1 - nu * nu)) * math.sqrt(Rstar)
    v = 2 * v0
    delta_max = (5 * mstar * v * v / (4 * K)) ** 0.4
    beta = math.gamma(0.4) * math.gamma(0.5) / math.gamma(0.9)
    tc = 2 * delta_max / v * 0.4 * beta
    assert abs(tc_meas - tc) <= 2.0 / w.N_sub + 1e-3 * tc
    assert abs(dmax - delta_max) < 1e-3 * delta_max
    assert abs(e_meas - 1.0) < 1e-4


def test_hertz_mindlin_damping_gives_the_restitution(orc):
    # the dashpot 2 sqrt(5/6) |beta| sqrt(S_n m*) with beta from e returns the rebound speed
    # e times the approach speed (to the sub-step's first-order error)
    for e in (0.9, 0.5, 0.2):
        assert abs(_hertz_collision(orc, 2.0e5, 0.3, e)[3] - e) < 2e-3
