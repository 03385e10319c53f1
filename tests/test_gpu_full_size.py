"""The GPU path at the full 8192 x 4096 suspension size (20 000 disks of diameter 20), in the
launch configuration the benchmark times, with FP32 and FP16 population storage.  The FP64
oracle cannot step the whole lattice in a test, so it checks sampled outputs on small windows:

* the particle-to-cell map (cells covered, covering particle ids, solid ratios) on the interior
  of periodic oracle windows holding the disks whose centres fall inside them;
* one coupling step started from the GPU's own populations: the window oracle takes the GPU's
  f(x, t), steps once, and its populations and per-particle forces are compared with the GPU's.
  The DEM is held for this step (dem_on = 0: disks keep their place and velocity, as in the window).

A window is cut around a sampled disk; disks whose centres lie outside it are left out and the
oracle wraps the window periodically, so only cells at least r_max + 2 from the window's edge
(and particles whose disk stays inside that interior) are compared.

Tolerances: solid ratios 2e-6 (FP32 geometry against the FP64 area), cell counts and ids exact;
populations 2e-6 (FP32) or 4e-5 (FP16: half an ulp of the stored deviation f - w); forces 1e-4
of the force scale (FP32 sums over the covered cells, from the same inputs).
"""
import math

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

S = 96          # window edge (cells)
NWIN = 12       # sampled windows per test


@pytest.fixture(scope="module")
def imb():
    import paper_1809_07008_gb300 as imb
    imb.load()
    return imb


def _windows(w, seed):
    """Window origins around randomly chosen disks, away from the walls and the periodic edge."""
    rng = np.random.default_rng(seed)
    out = []
    for p in rng.permutation(w.n_particles):
        cx, cy = w.x[p]
        x0, y0 = int(math.floor(cx)) - S // 2, int(math.floor(cy)) - S // 2
        if x0 < 4 or y0 < 4 or x0 + S > w.nx - 4 or y0 + S > w.ny - 4:
            continue
        out.append((x0, y0))
        if len(out) == NWIN:
            break
    return out


def _window_workload(w, x, v, om, r, x0, y0, dem_on):
    inside = (x[:, 0] >= x0) & (x[:, 0] < x0 + S) & (x[:, 1] >= y0) & (x[:, 1] < y0 + S)
    idx = np.nonzero(inside)[0]
    shift = np.array([x0, y0], dtype=np.float64)   # integer shift: fractional offsets unchanged
    ww = W.Workload(name="window", nx=S, ny=S, tau=w.tau, C_smag=w.C_smag, bc_x=W.BC_PERIODIC,
                    bc_y=W.BC_PERIODIC, dem_on=dem_on, N_sub=w.N_sub, eps_mode=w.eps_mode,
                    n_sub=w.n_sub, x=x[idx] - shift, v=v[idx], omega=om[idx], r=r[idx])
    return ww, idx


def _interior(r_max):
    m = int(math.ceil(r_max)) + 2
    return slice(m, S - m), m


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_full_size_cell_map_on_windows(orc, imb, storage):
    w = W.c3()
    g = imb.Lattice.from_workload(w, storage=storage)
    count, ids, eps = g.cell_map()
    sl, _ = _interior(w.r.max())
    checked = 0
    for x0, y0 in _windows(w, 1):
        ww, idx = _window_workload(w, w.x, w.v, w.omega, w.r, x0, y0, dem_on=1)
        o = orc.Sim(ww)
        oc, oi, oe = o.cell_map()
        gc = count[y0:y0 + S, x0:x0 + S][sl, sl]
        assert np.array_equal(gc, oc[sl, sl])
        gi = ids[y0:y0 + S, x0:x0 + S][sl, sl]
        ge = eps[y0:y0 + S, x0:x0 + S][sl, sl]
        oi, oe = oi[sl, sl], oe[sl, sl]
        for k in range(4):
            used = gc > k
            assert np.array_equal(gi[..., k][used], idx[oi[..., k][used]])
            assert np.abs(ge[..., k][used] - oe[..., k][used]).max(initial=0.0) < 2e-6
        checked += int((gc > 0).sum())
    assert checked > 5000
    g.close()


@pytest.mark.parametrize("storage,tol_f", [("fp32", 2e-6), ("fp16", 4e-5)])
def test_full_size_step_on_windows(orc, imb, storage, tol_f):
    w = W.c3().with_(dem_on=0)
    g = imb.Lattice.from_workload(w, storage=storage)
    g.step(5)                        # a flow around the moving disks, then one step compared
    f_t = g.populations()
    g.step(1)
    F, T = g.forces()
    f_t1 = g.populations()
    x, v, om = g.particles()
    assert np.array_equal(x, w.x)    # held in place
    sl, m = _interior(w.r.max())
    inner = slice(m + 1, S - m - 1)  # streaming pulls from one cell around
    scale = np.linalg.norm(F, axis=1).mean()
    nf = 0
    for x0, y0 in _windows(w, 2):
        ww, idx = _window_workload(w, x, v, om, w.r, x0, y0, dem_on=0)
        o = orc.Sim(ww)
        o.set_f(f_t[:, y0:y0 + S, x0:x0 + S])
        o.step(1)
        diff = np.abs(o.f()[:, inner, inner] - f_t1[:, y0:y0 + S, x0:x0 + S][:, inner, inner])
        assert diff.max() < tol_f, (x0, y0, diff.max())
        oF, oT = o.forces()
        xs = ww.x
        keep = ((xs - ww.r[:, None] - 1 >= m) & (xs + ww.r[:, None] + 1 < S - m)).all(axis=1)
        for j in np.nonzero(keep)[0]:
            p = idx[j]
            assert np.abs(F[p] - oF[j]).max() < 1e-4 * scale, (p, F[p], oF[j])
            assert abs(T[p] - oT[j]) < 1e-4 * scale * w.r[p], (p, T[p], oT[j])
            nf += 1
    assert nf >= 5
    g.close()
