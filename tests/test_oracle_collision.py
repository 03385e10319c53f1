"""Pins of the oracle's per-node building blocks against closed forms.

Equilibrium (Eq. 2), weights (Tab. 1 analogue for D2Q9), the weighting
function B (Eq. 14), the solid operator (Eq. 12) and the Smagorinsky closure
(Sec. 3.3).  Every expected value here comes from a moment identity, a limit
or an algebraic property worked out by hand, never from the oracle itself.
"""
import math

import numpy as np
import pytest

CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
OPP = np.array([0, 3, 4, 1, 2, 7, 8, 5, 6])


def test_d2q9_rest_equilibrium_is_the_weight_table(orc):
    # Qian et al. 1992 D2Q9 weights: 4/9 rest, 1/9 axis, 1/36 diagonal; they sum to 1 (Tab. 1 note)
    fe = orc.feq(1.0, 0.0, 0.0)
    expect = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    assert np.array_equal(fe, expect)
    assert abs(fe.sum() - 1.0) < 1e-15


@pytest.mark.parametrize("rho,ux,uy", [(1.0, 0.0, 0.0), (1.02, 0.05, -0.03), (0.97, -0.08, 0.01),
                                       (1.3, 0.0, 0.09)])
def test_equilibrium_moments_closed_form(orc, rho, ux, uy):
    # Eq. 2 moments: sum f = rho, sum c f = rho u, sum c c f = rho (cs^2 I + u u), cs^2 = 1/3
    fe = orc.feq(rho, ux, uy)
    assert abs(fe.sum() - rho) < 1e-15 * 4
    assert abs((CX * fe).sum() - rho * ux) < 1e-15 * 4
    assert abs((CY * fe).sum() - rho * uy) < 1e-15 * 4
    assert abs((CX * CX * fe).sum() - rho * (1 / 3 + ux * ux)) < 1e-15 * 4
    assert abs((CY * CY * fe).sum() - rho * (1 / 3 + uy * uy)) < 1e-15 * 4
    assert abs((CX * CY * fe).sum() - rho * ux * uy) < 1e-15 * 4


def test_weighting_function_limits_and_order(orc):
    # Eq. 14 / Fig. 3c: B(0) = 0, B(1) = 1, increasing in eps, and the curve rises with tau
    for tau in (0.53, 0.62, 0.8, 1.0):
        assert orc.B(0.0, tau) == 0.0
        assert orc.B(1.0, tau) == 1.0
        e = np.linspace(0, 1, 101)
        b = np.array([orc.B(x, tau) for x in e])
        assert np.all(np.diff(b) > 0)
        assert np.all(b <= e + 1e-15)   # (1 - eps) >= 0 makes B <= eps for every tau
    for eps in (0.1, 0.5, 0.9):
        bs = [orc.B(eps, t) for t in (0.53, 0.62, 0.8, 1.0)]
        assert all(b1 < b2 for b1, b2 in zip(bs, bs[1:]))
    # hand value: eps = 1/2, tau = 0.6 -> 0.5*0.1 / (0.5 + 0.1) = 1/12
    assert abs(orc.B(0.5, 0.6) - 1 / 12) < 1e-16


def _random_f(rng, rho=1.0, u=(0.03, -0.02), amp=1e-3):
    fe = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4) * rho
    cu = CX * u[0] + CY * u[1]
    fe = fe * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * (u[0] ** 2 + u[1] ** 2))
    return fe + amp * rng.standard_normal(9)


def test_solid_operator_conserves_mass_and_exchanges_momentum(orc):
    # Eq. 12: sum_i Omega^s_i = 0 (both equilibria carry rho) and
    # sum_i c_i Omega^s_i = rho (u_s - u) + 2 (rho u - j) for any f
    rng = np.random.default_rng(3)
    for _ in range(20):
        f = _random_f(rng)
        rho = f.sum()
        jx, jy = (CX * f).sum(), (CY * f).sum()
        ux, uy = jx / rho + 1e-3 * rng.standard_normal(), jy / rho
        usx, usy = 0.01 * rng.standard_normal(2)
        om = orc.omega_s(f, rho, ux, uy, usx, usy)
        assert abs(om.sum()) < 1e-15
        assert abs((CX * om).sum() - (rho * (usx - ux) + 2 * (rho * ux - jx))) < 1e-15
        assert abs((CY * om).sum() - (rho * (usy - uy) + 2 * (rho * uy - jy))) < 1e-15


def test_solid_operator_at_rest_is_bounce_back(orc):
    # Eq. 12 with u_f = u_s = 0: the equilibria cancel in pairs and Omega^s_i = f_{-i} - f_i,
    # so f + Omega^s is f reflected (the non-equilibrium bounce-back of Sec. 2.3)
    rng = np.random.default_rng(4)
    f = _random_f(rng, u=(0.0, 0.0))
    om = orc.omega_s(f, f.sum(), 0.0, 0.0, 0.0, 0.0)
    assert np.allclose(f + om, f[OPP], atol=1e-16, rtol=0)


def test_solid_operator_sets_solid_velocity(orc):
    # Sec. 2.3 below Eq. 12: at equilibrium f = f^eq(rho, u_f) the post-collision state of a
    # fully solid cell is f^eq(rho, u_s), i.e. the node moves with the solid
    f = orc.feq(1.01, 0.04, -0.02)
    om = orc.omega_s(f, 1.01, 0.04, -0.02, -0.01, 0.03)
    assert np.allclose(f + om, orc.feq(1.01, -0.01, 0.03), atol=1e-16, rtol=0)


def test_smagorinsky_limits(orc):
    rng = np.random.default_rng(5)
    f = _random_f(rng, amp=1e-3)
    assert orc.tau_eff(f, 0.51, 0.0) == 0.51                       # C = 0 is plain BGK
    fe = orc.feq(1.0, 0.02, 0.01)
    assert abs(orc.tau_eff(fe, 0.51, 0.1) - 0.51) < 1e-15           # no strain, no eddy viscosity


def test_smagorinsky_closure_satisfies_eddy_viscosity_definition(orc):
    # nu_t = (C Delta)^2 |S| with |S| = sqrt(2 S:S) and the LBM strain
    # S = -Pi_neq / (2 rho cs^2 tau_eff), and tau_eff = tau + nu_t / cs^2 (Delta = 1).
    rng = np.random.default_rng(6)
    for C in (0.1, 0.3):
        for _ in range(10):
            f = _random_f(rng, amp=5e-3)
            rho = f.sum()
            ux, uy = (CX * f).sum() / rho, (CY * f).sum() / rho
            fe = orc.feq(rho, ux, uy)
            ne = f - fe
            Pi = np.array([[(CX * CX * ne).sum(), (CX * CY * ne).sum()],
                           [(CX * CY * ne).sum(), (CY * CY * ne).sum()]])
            te = orc.tau_eff(f, 0.51, C)
            S = -Pi / (2 * rho * (1 / 3) * te)
            nu_t = C * C * math.sqrt(2 * (S * S).sum())
            assert abs(te - (0.51 + 3 * nu_t)) < 1e-13
            assert te > 0.51
