"""Pins of the oracle's no-slip walls and body force (parallel-plate flow, Sec. 5.3 and
Appendix F).  The paper fixes the walls by reference (Zou and He's velocity condition) and
the flow by Eqs. (88)-(89); the oracle's readings are that the node momentum at a wall is
J = -F/2 (u = 0 with the half-force shift of Eq. 6b) and that stencils see beyond a wall the
row mirrored through it."""
import numpy as np
import pytest

import oracle as O
from oracle import thermo

A, TAU = 0.25, 1.0


def _run(model, ny, steps, Tr, fx, rho_col):
    T = thermo.temperature(A, 4.0, 1.0, Tr)
    kw = dict(a=A, b=4.0, R=1.0, T=T, fx=fx, walls=1.0, tau_nu=TAU, tau_e=1.0)
    if model == O.PP:
        sig, _, _ = thermo.sigma_li(A, 4.0, 1.0, Tr)
        kw.update(sigma_Li=sig, tau_q=1 / 1.99)
    else:
        kw.update(kappa=0.5)
    p = O.make_params(**kw)
    f = O.init(model, np.repeat(np.asarray(rho_col)[:, None], 4, axis=1))
    m0 = f.sum()
    f = O.run(model, p, f, steps)
    rho, ux, uy, *_ = O.macro(model, p, f)
    return rho[:, 0], ux, uy, f.sum() / m0 - 1


def _s89(rho_col, fx):
    """Eq. (89) with mu(y) = rho(y) c_s^2 (tau - 1/2), no slip at y = 0 and y = H (trapezoid
    rule on the lattice nodes)."""
    y = np.arange(len(rho_col), dtype=float)
    mu = rho_col / 3.0 * (TAU - 0.5)
    i1 = np.concatenate([[0.0], np.cumsum(0.5 * (y[1:] / mu[1:] + y[:-1] / mu[:-1]))])
    i0 = np.concatenate([[0.0], np.cumsum(0.5 * (1 / mu[1:] + 1 / mu[:-1]))])
    return -fx * i1 + fx * i1[-1] / i0[-1] * i0


@pytest.mark.parametrize("model", [O.PP, O.FE])
def test_single_phase_poiseuille_is_exact(model):
    """Uniform liquid between the plates (H = 20): the steady velocity is the parabola
    F y (H - y) / (2 mu) to rounding, zero at the wall nodes, with mass conserved."""
    ny, fx = 21, 1e-6
    rv, rl, _ = thermo.maxwell(A, 4.0, 1.0, 0.8)
    rho, ux, uy, dm = _run(model, ny, 40000, 0.8, fx, np.full(ny, rl))
    y = np.arange(ny)
    ua = fx / (2 * rl / 3.0 * (TAU - 0.5)) * y * (ny - 1 - y)
    assert np.abs(ux[:, 0] - ua).max() < 1e-9 * ua.max()
    assert np.abs(ux[[0, -1]]).max() < 1e-15 and np.abs(uy).max() < 1e-13
    assert abs(dm) < 1e-10


@pytest.mark.parametrize("model,tol", [(O.PP, 0.015), (O.FE, 0.05)])
def test_two_phase_plate_flow_against_eq89(model, tol):
    """Vapour below, liquid above (101 x 50 geometry of Sec. 5.3, periodic x; the flow is
    uniform in x, so 4 columns suffice), Tr = 0.8, F_x = 1e-6: the converged velocity profile
    against Eq. (89) integrated with the run's own rho(y).  Measured: P 0.7%, FE 3.5% (its
    deviation sits in the vapour next to the interface; the paper also finds FE less accurate
    in this flow than at rest, Sec. 6)."""
    ny, fx = 50, 1e-6
    rv, rl, _ = thermo.maxwell(A, 4.0, 1.0, 0.8)
    y = np.arange(ny, dtype=float)
    rho0 = rv + 0.5 * (rl - rv) * (1 + np.tanh(2 * (y - (ny - 1) / 2) / 5.0))
    rho, ux, uy, dm = _run(model, ny, 150000, 0.8, fx, rho0)
    assert rho[0] < rho[-1]                                   # vapour at the bottom wall
    ua = _s89(rho, fx)
    assert np.abs(ux[:, 0] - ua).max() < tol * ua.max()
    assert np.abs(ux - ux[:, :1]).max() < 1e-14 * ua.max()    # uniform in x
    assert np.abs(uy).max() < 1e-6 * ua.max()
