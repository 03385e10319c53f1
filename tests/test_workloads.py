"""The seeded inputs shared by the oracle and the GPU path.

* splitmix64 reproduces its published outputs (Steele, Lea and Flood; the reference
  implementation's first values for seeds 0 and 1234567), and the doubles drawn from it use
  the top 53 bits;
* random sequential addition keeps every pair of disks (minimum image) and every disk and wall
  at least the stated gap apart, in the suspension, the periodic sweep domains and the sphere
  boxes;
* the batched sweep's 256 domains have the stated sizes, fractions, relaxation times and a
  mean speed capped at 0.02; the Poiseuille-flow-past-a-sphere box has the paper's proportions
  (walls 5 N apart, l_x = l_z = 20 N, radius N / 2, centre N 5/4 above the lower wall) and the body
  force that gives the stated centre-height velocity.
"""
import math

import numpy as np

import workloads as W


def test_splitmix64_published_outputs():
    r = W.SplitMix64(0)
    assert [r.next_u64() for _ in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    assert W.SplitMix64(1234567).next_u64() == 6457827717110365317
    r1, r2 = W.SplitMix64(99), W.SplitMix64(99)
    u = r1.uniform()
    assert u == (r2.next_u64() >> 11) / 2.0 ** 53 and 0.0 <= u < 1.0


def _min_pair_gap(x, r, Lx, Ly, per_x, per_y):
    d = x[:, None, :] - x[None, :, :]
    if per_x:
        d[..., 0] -= Lx * np.round(d[..., 0] / Lx)
    if per_y:
        d[..., 1] -= Ly * np.round(d[..., 1] / Ly)
    dist = np.sqrt((d ** 2).sum(-1))
    gap = dist - (r[:, None] + r[None, :])
    np.fill_diagonal(gap, np.inf)
    return gap.min()


def test_suspension_disks_keep_their_gap():
    w = W.c3sub(steps=0, nx=512, ny=512)
    assert w.n_particles == round(20000 * 512 * 512 / (8192 * 4096))
    assert _min_pair_gap(w.x, w.r, w.nx, w.ny, True, False) >= 1.0 - 1e-12
    assert (w.x[:, 1] - w.r >= 1.0 - 1e-12).all() and (w.x[:, 1] + w.r <= w.ny - 1.0 + 1e-12).all()
    assert np.allclose(np.linalg.norm(w.v, axis=1), 0.005)


def test_sweep_domains():
    ds = W.c5(256)
    assert len(ds) == 256
    for w in ds:
        assert 128 <= w.nx <= 512 and w.nx % 32 == 0 and 128 <= w.ny <= 256 and w.ny % 32 == 0
        assert 0.51 <= w.tau < 1.0 and w.C_smag == 0.1 and w.force[0] > 0.0 and w.force[1] == 0.0
        d = 2 * w.r[0]
        assert 10.0 <= d < 30.0 and np.all(w.r == w.r[0])
        if w.n_particles > 1:
            assert _min_pair_gap(w.x, w.r, w.nx, w.ny, True, True) >= 1.0 - 1e-12
        phi = w.n_particles * math.pi * w.r[0] ** 2 / (w.nx * w.ny)
        assert 0.0 < phi < 0.5 + 1e-9
        nu = (w.tau - 0.5) / 3.0
        k = d * d * (1 - phi) ** 3 / (9 * phi * phi)
        U = w.force[0] * k / nu
        assert U <= 0.02 + 1e-12
    # reproducible from the seed
    again = W.c5(3)
    assert all(np.array_equal(a.x, b.x) and a.tau == b.tau for a, b in zip(again, ds[:3]))


def test_sphere_boxes_and_happel_geometry():
    w = W.spheres3(nx=40, ny=24, nz=36, n=3, seed=3)
    assert w.n_spheres == 3
    for i in range(3):
        for j in range(i + 1, 3):
            d = w.x[i] - w.x[j]
            d[0] -= w.nx * round(d[0] / w.nx)
            d[2] -= w.nz * round(d[2] / w.nz)
            assert np.linalg.norm(d) >= w.R[i] + w.R[j] + 2.0
        assert w.x[i, 1] - w.R[i] >= 2.0 and w.x[i, 1] + w.R[i] <= w.ny - 2.0
    for N in (5, 10, 20):
        h = W.happel(N)
        assert (h.nx, h.ny, h.nz) == (20 * N, 5 * N, 20 * N) and h.R[0] == N / 2
        assert tuple(h.x[0]) == (10 * N, 1.25 * N, 10 * N) and h.wall_y
        nu = (h.tau - 0.5) / 3.0
        yc, H = h.x[0, 1], h.ny
        assert abs(h.force[0] / (2 * nu) * yc * (H - yc) - 2.0e-4) < 1e-15


def test_packed_bed_geometry_and_units(orc):
    # the paper's packing (Sec. 3.3): 10 x 5 x 5 touching spheres in a simple cubic arrangement,
    # one d_p of free fluid at each end, N cells per diameter; its porosity 1 - pi / 6 is the
    # printed n = 0.4764
    N = 20
    w = W.packed_bed(N, run=9)
    assert (w.nx, w.ny, w.nz) == (12 * N, 5 * N, 5 * N) and w.n_spheres == 250 and (w.R == N / 2).all()
    assert not w.wall_y and w.C_smag == 0.3 and w.tau == 0.501
    assert (w.x >= 0).all() and (w.x < np.array([w.nx, w.ny, w.nz])).all()
    d = w.x[:, None, :] - w.x[None, :, :]
    for a, L in enumerate((w.nx, w.ny, w.nz)):
        d[..., a] -= L * np.round(d[..., a] / L)
    dist = np.sqrt((d ** 2).sum(-1))
    np.fill_diagonal(dist, np.inf)
    assert abs(dist.min() - N) < 1e-12                       # neighbours touch
    assert ((np.abs(dist - N) < 1e-12).sum(1) >= 5).all()    # x neighbours at the ends: 5, else 6
    assert w.x[:, 0].min() - w.R[0] == N + 0.5 and w.nx - (w.x[:, 0].max() + w.R[0]) == N - 0.5
    assert round(1.0 - math.pi / 6.0, 4) == 0.4764
    # units: nu_lattice dx^2 / dt is the fluid's viscosity, and Ergun (Eq. 21) solved in lattice
    # units with the body force as the gradient gives the physical velocity times dt / dx
    n, rho, mu, d_p = 1.0 - math.pi / 6.0, 1000.0, 1.0e-3, 1.0e-3
    for run, (dP, tau) in enumerate(W.PACKED_BED_RUNS):
        wr = W.packed_bed(N, run=run)
        dx, dt = W.packed_bed_units(N, tau)
        nu = (tau - 0.5) / 3.0
        assert abs(nu * dx * dx / dt - mu / rho) < 1e-18
        U = _bisect(lambda u: orc.ergun_gradient(u, d_p, n, rho, mu) - dP / (10 * d_p), 0.0, 10.0)
        Ul = _bisect(lambda u: orc.ergun_gradient(u, N, n, 1.0, nu) - wr.force[0], 0.0, 1.0)
        assert abs(Ul - U * dt / dx) < 1e-9 * Ul
        assert abs(orc.packed_bed_reynolds(Ul, N, n, 1.0, nu) - orc.packed_bed_reynolds(U, d_p, n, rho, mu)) < 1e-8


def _bisect(f, lo, hi):
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if f(mid) > 0.0:
            hi = mid
        else:
            lo = mid
    return 0.5 * (lo + hi)



def test_bench_packed_bed_friction_follows_eqs_22_23(orc):
    # the bench's report of the packed bed: with D = (Delta P / L) x area x length (the drag a
    # pressure-driven medium takes) its Re*_p and f* are Eqs. 23 and 22 in lattice units, and at
    # the Ergun gradient of a velocity the two friction factors coincide
    import sys, os
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    n = 1.0 - math.pi / 6.0
    N, tau, area, length = 20, 0.58, 100 * 100, 200
    nu = (tau - 0.5) / 3.0
    for U in (1e-5, 3.5e-4, 0.01):
        G = orc.ergun_gradient(U, N, n, 1.0, nu)
        Re, f, fe = bench.packed_bed_friction(G * area * length, U, N, tau, area, length)
        assert abs(Re - orc.packed_bed_reynolds(U, N, n, 1.0, nu)) < 1e-12 * Re
        assert abs(f - orc.packed_bed_friction(G, U, N, n, 1.0)) < 1e-12 * f
        assert abs(fe - orc.ergun_friction(Re)) < 1e-12 * fe and abs(f - fe) < 1e-10 * fe
