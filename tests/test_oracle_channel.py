"""Pins of the oracle's inlet/outlet rule (the channel of the one-disk case; the paper has no
channel inlet, so the rule is a reading: velocity inlet f(0) = f^eq(rho of column 1, u_in),
outlet f(nx-1) = f^eq(1, u of column nx-2), i.e. a prescribed velocity with zero normal density
gradient at the inlet and the reference pressure with zero normal velocity gradient at the
outlet).

What the mathematics fixes for an empty walled channel run from rest to its steady state:
  * a steady state exists (the outlet holds the pressure level);
  * steady mass conservation: with the collision conserving mass and momentum, each column's
    x-momentum sum J(i) = sum_y sum_q c_qx f_q(i, y) equals the mean of the mass fluxes through
    its two faces, and steady column masses make every face flux the same, so J(i) is one
    constant for 1 <= i <= nx-2;
  * the boundary conditions' own meaning, read through the macroscopic fields: u = u_in and
    d rho / dx = 0 at the inlet column, rho = 1 and d u / dx = 0 at the outlet column;
  * far downstream the flow is plane Poiseuille flow driven by the pressure gradient the
    boundaries set up: u(y) = G / (2 nu) (y + 1/2)(H - 1/2 - y) with p = rho / 3 and
    nu = (tau - 1/2) / 3 (Eq. 5), exact for halfway bounce-back at tau = 1/2 + sqrt(3)/4;
  * the inflow tends to u_in sum_y rho(0, y) as the channel widens; the shortfall comes from
    the two wall corners of the inlet column, so it times H is independent of H.
Each plausible mistake in the rule, planted in a patched copy of the oracle source, fails at
least one of these.
"""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

import workloads as W

CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
TAU = 0.5 + np.sqrt(3.0) / 4.0
U_IN = 0.01


class _Lib:
    """The oracle built from a given source (the shipped one, or a patched copy)."""

    def __init__(self, path):
        from oracle import oracle as O
        self.O = O
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        L.orc_new.argtypes = [C.POINTER(O.Params)]
        L.orc_new.restype = C.c_void_p
        L.orc_free.argtypes = [C.c_void_p]
        L.orc_step.argtypes = [C.c_void_p, C.c_int]
        L.orc_get_f.argtypes = [C.c_void_p, dp]
        L.orc_get_macro.argtypes = [C.c_void_p, dp, dp, dp]
        self.L = L

    def channel(self, H, nx, steps):
        """Empty walled channel from rest: returns f, rho, ux, uy at `steps` and the largest
        change of f over the last 1000 steps."""
        O, L = self.O, self.L
        w = W.Workload(name="chan", nx=nx, ny=H, tau=TAU, bc_x=W.BC_INLET_OUTLET, bc_y=W.BC_WALL,
                       u_in=(U_IN, 0.0))
        p = O.params_from_workload(w)
        h = L.orc_new(C.byref(p))
        assert h
        try:
            L.orc_step(h, steps - 1000)
            f0 = np.zeros((9, H, nx))
            L.orc_get_f(h, O._d(f0))
            L.orc_step(h, 1000)
            f = np.zeros((9, H, nx))
            L.orc_get_f(h, O._d(f))
            rho, ux, uy = (np.zeros((H, nx)) for _ in range(3))
            L.orc_get_macro(h, O._d(rho), O._d(ux), O._d(uy))
        finally:
            L.orc_free(h)
        return f, rho, ux, uy, float(np.abs(f - f0).max())


def _pins(f, rho, ux, uy, change, H):
    nx = f.shape[2]
    J = (CX[:, None, None] * f).sum(axis=(0, 1))
    nu = (TAU - 0.5) / 3.0
    xm = (2 * nx) // 3
    G = -(rho[:, xm + 1].mean() - rho[:, xm - 1].mean()) / 6.0 / rho[:, xm].mean()
    y = np.arange(H) + 0.5
    pois = G / (2.0 * nu) * y * (H - y)
    return {
        "steady": change < 1e-13,
        "flux": np.ptp(J[1:-1]) < 1e-10 * abs(J[1:-1]).mean(),
        "inlet_velocity": np.abs(ux[:, 0] - U_IN).max() < 1e-14 and np.abs(uy[:, 0]).max() < 1e-14,
        "inlet_density": np.abs(rho[:, 0] - rho[:, 1]).max() < 1e-14,
        "outlet_density": np.abs(rho[:, -1] - 1.0).max() < 1e-14,
        "outlet_velocity": np.abs(ux[:, -1] - ux[:, -2]).max() < 1e-14 and np.abs(uy[:, -1] - uy[:, -2]).max() < 1e-14,
        "poiseuille": np.abs(ux[:, xm] - pois).max() < 1e-3 * ux[:, xm].max(),
        "_deficit_times_H": H * (1.0 - J[nx // 2] / (U_IN * rho[:, 0].sum())),
    }


STEPS = {8: 40000, 16: 50000}


@pytest.fixture(scope="module")
def shipped(orc):
    return _Lib(orc.build())


def test_channel_reaches_the_steady_state_the_boundaries_fix(shipped):
    d = {}
    for H in (8, 16):
        p = _pins(*shipped.channel(H, 6 * H, STEPS[H]), H)
        for k, v in p.items():
            if not k.startswith("_"):
                assert v, f"H = {H}: pin '{k}' fails"
        d[H] = p["_deficit_times_H"]
    # the inflow shortfall is a corner effect: (1 - flux / (u_in sum rho(0))) H does not depend on H
    assert 0.0 < d[8] < 1.0
    assert abs(d[16] - d[8]) < 0.01 * d[8]


# (name, text in the inlet/outlet block of stream(), mistaken replacement)
MUTANTS = [
    ("inlet density from column 0", "rho1 += s->f[IDX(s, q, k, 1)];", "rho1 += s->f[IDX(s, q, k, 0)];"),
    ("u_in applied as momentum", "orc_feq(rho1, s->p.u_in_x, s->p.u_in_y, fe);",
     "orc_feq(rho1, s->p.u_in_x / rho1, s->p.u_in_y / rho1, fe);"),
    ("outlet velocity from column nx-3", "const double g = s->f[IDX(s, q, k, nx - 2)];",
     "const double g = s->f[IDX(s, q, k, nx - 3)];"),
    ("outlet copies column nx-2 (no pressure level)", "s->f[IDX(s, q, k, nx - 1)] = fo[q];",
     "s->f[IDX(s, q, k, nx - 1)] = s->f[IDX(s, q, k, nx - 2)];"),
]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_inlet_outlet_mistake_fails_a_pin(orc, tmp_path, name, old, new):
    src = open(os.path.join(os.path.dirname(orc.SRC), "imb_oracle.c")).read()
    assert src.count(old) == 1, "the planted mistake must replace exactly one statement"
    (tmp_path / "imb_oracle.c").write_text(src.replace(old, new))
    for h in ("imb_oracle.h", "imb_oracle3.h"):
        (tmp_path / h).write_text(open(os.path.join(os.path.dirname(orc.SRC), h)).read())
    (tmp_path / "imb_oracle3.c").write_text(open(orc.SRC3).read())
    lib = str(tmp_path / "libmut.so")
    subprocess.run(["gcc", "-std=gnu11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                    str(tmp_path / "imb_oracle.c"), str(tmp_path / "imb_oracle3.c"), "-o", lib, "-lm"], check=True)
    H = 8
    with np.errstate(all="ignore"):
        p = _pins(*_Lib(lib).channel(H, 6 * H, STEPS[H]), H)
    failed = [k for k, v in p.items() if not k.startswith("_") and not v]
    assert failed, f"planted mistake '{name}' passes every pin"
