"""Pins of the oracle's reverse-mode drag gradient: the gradient of the time-averaged drag
with respect to the inlet velocity, the relaxation time and the disk centres must equal central
finite differences of the oracle's own forward steps (FP64, h = 1e-6).

Cases: a channel (velocity inlet, zero-gradient outlet, walls) with two disks, and a box periodic
in x with walls in y holding a decaying uniform flow past two disks.  Radii and centres are chosen
so that no disk edge is tangent to a cell edge (there the cell coverage switches and the drag has
a kink, so no derivative exists)."""
import numpy as np
import pytest

import workloads as W

T = 60
H = 1e-6


def _case(kind, u=0.02, tau=0.6, x=None):
    x = np.array([[20.3, 15.7], [33.6, 17.2]]) if x is None else x
    n = len(x)
    common = dict(x=x, v=np.zeros((n, 2)), omega=np.zeros(n), r=np.array([5.23, 4.37]))
    if kind == "channel":
        return W.Workload(name="adj_channel", nx=52, ny=32, tau=tau, bc_x=W.BC_INLET_OUTLET,
                          bc_y=W.BC_WALL, u_in=(u, 0.0), **common)
    return W.Workload(name="adj_periodic", nx=52, ny=32, tau=tau, bc_x=W.BC_PERIODIC, bc_y=W.BC_WALL,
                      u0=(0.02, 0.0), u_in=(u, 0.0), **common)


def _state(orc, kind):
    s = orc.Sim(_case(kind))
    s.step(20)   # a developed flow around the disks
    return s.f()


def _J(orc, kind, f0, **kw):
    s = orc.Sim(_case(kind, **kw))
    s.set_f(f0)
    return s.drag_average(T)


@pytest.mark.parametrize("kind", ["channel", "periodic"])
def test_drag_gradient_matches_central_differences(orc, kind):
    f0 = _state(orc, kind)
    s = orc.Sim(_case(kind))
    s.set_f(f0)
    J, g_u, g_tau, g_x = s.drag_adjoint(T)
    assert J == pytest.approx(_J(orc, kind, f0), rel=1e-13)
    assert abs(J) > 1e-3
    fd_tau = (_J(orc, kind, f0, tau=0.6 + H) - _J(orc, kind, f0, tau=0.6 - H)) / (2 * H)
    assert g_tau == pytest.approx(fd_tau, rel=1e-6)
    if kind == "channel":   # the inlet velocity only enters through the inlet
        fd_u = (_J(orc, kind, f0, u=0.02 + H) - _J(orc, kind, f0, u=0.02 - H)) / (2 * H)
        assert g_u == pytest.approx(fd_u, rel=1e-6)
    else:
        assert g_u == 0.0
    xb = np.array([[20.3, 15.7], [33.6, 17.2]])
    scale = np.abs(g_x).max()
    for p in range(2):
        for d in range(2):
            xp, xm = xb.copy(), xb.copy()
            xp[p, d] += H
            xm[p, d] -= H
            fd = (_J(orc, kind, f0, x=xp) - _J(orc, kind, f0, x=xm)) / (2 * H)
            assert abs(g_x[p, d] - fd) < 1e-6 * scale, (p, d, g_x[p, d], fd)


def test_drag_adjoint_rejects_moving_particles(orc):
    w = _case("channel").with_(v=np.full((2, 2), 0.01))
    s = orc.Sim(w)
    with pytest.raises(ValueError):
        s.drag_adjoint(5)
