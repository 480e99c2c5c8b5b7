"""Pins of the oracle's no-slip walls and body force (parallel-plate flow, Sec. 5.3 and
Appendix F).  The paper fixes the walls by reference (Zou and He's velocity condition) and
the flow by Eqs. (88)-(89); the oracle's readings are that the node momentum at a wall is
J = -F/2 (u = 0 with the half-force shift of Eq. 6b) and that stencils see beyond a wall the
row mirrored through it."""
import numpy as np
import pytest

import oracle as O
from oracle import plate, thermo

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
    """Eq. (89) on the lattice nodes: plates on the wall rows, H = ny - 1."""
    return plate.s89(np.arange(len(rho_col), dtype=float), plate.viscosity(rho_col, TAU), fx)


def test_s88_reduces_to_poiseuille_and_matches_at_the_interface():
    """Eq. (88): equal viscosities give F y (H - y)/(2 mu); otherwise no slip at both plates
    and continuity of u and of mu du/dy at y = H/2 (one-sided differences)."""
    H, fx = 49.0, 1e-6
    y = np.linspace(0, H, 99)
    assert np.abs(plate.s88(y, H, 0.1, 0.1, fx) - fx * y * (H - y) / 0.2).max() < 1e-15
    mu1, mu2 = 0.01, 0.13
    assert abs(plate.s88(0.0, H, mu1, mu2, fx)) < 1e-16 and abs(plate.s88(H, H, mu1, mu2, fx)) < 1e-16
    e = 1e-6
    lo, mid, hi = plate.s88([H / 2 - e, H / 2, H / 2 + e], H, mu1, mu2, fx)
    assert abs(lo - mid) < 1e-6 * abs(mid) and abs(hi - mid) < 1e-6 * abs(mid)
    d1 = mu1 * (mid - plate.s88(H / 2 - 1e-4, H, mu1, mu2, fx)) / 1e-4
    d2 = mu2 * (plate.s88(H / 2 + 1e-4, H, mu1, mu2, fx) - mid) / 1e-4
    assert abs(d1 - d2) < 1e-4 * abs(d1)  # one-sided differences: O(F_x h) = 1e-10
    # each branch solves mu u'' = -F_x (second differences away from the interface)
    for yy, mu in ((10.0, mu1), (40.0, mu2)):
        u = plate.s88([yy - 0.5, yy, yy + 0.5], H, mu1, mu2, fx)
        assert abs(mu * (u[0] - 2 * u[1] + u[2]) / 0.25 + fx) < 1e-9 * fx


def test_s89_reduces_to_poiseuille_and_converges_to_s88():
    """Eq. (89): exact (trapezoid rule on linear integrands) for uniform viscosity; for a
    viscosity step at H/2 it tends to Eq. (88) as the nodes refine."""
    H, fx = 49.0, 1e-6
    y = np.linspace(0, H, 50)
    assert np.abs(plate.s89(y, np.full(50, 0.1), fx) - fx * y * (H - y) / 0.2).max() < 1e-15
    mu1, mu2 = 0.01, 0.13
    errs = []
    for n in (1001, 4001):
        yy = np.linspace(0, H, n)
        mu = np.where(yy <= H / 2, mu1, mu2)
        ref = plate.s88(yy, H, mu1, mu2, fx)
        errs.append(np.abs(plate.s89(yy, mu, fx) - ref).max() / ref.max())
    assert errs[1] < 0.3 * errs[0] and errs[1] < 2e-3


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


@pytest.mark.parametrize("model,band", [(O.PP, 2), (O.FE, 3)])
def test_wall_band_widths(model, band):
    """The walled step differs from the periodic one only near the walls: after one step of
    the same random state, the periodic and walled oracles agree bitwise on every row at least
    band + 1 rows from a wall (band = 2 for P: psi one row away; 3 for FE: mu one row away and
    rho one more; the + 1 is streaming), and differ on the row band rows from a wall -- the
    rows a GPU strip step must recompute with the wall kernel."""
    nx, ny = 8, 20
    a = 0.5
    T = thermo.temperature(a, 4.0, 1.0, 0.8)
    rv, rl, _ = thermo.maxwell(a, 4.0, 1.0, 0.8)
    rng = np.random.Generator(np.random.PCG64(21))
    rho0 = rng.uniform(rv * 1.5, rl * 0.8, (ny, nx))
    kw = dict(a=a, b=4.0, R=1.0, T=T, tau_nu=0.9, tau_e=0.85, kappa=0.5, fx=1e-5, fy=-2e-5)
    if model == O.PP:
        kw.update(sigma_Li=0.1, kappa_P=0.7, tau_q=1 / 1.99)
    f0 = O.init(model, rho0)
    fp = O.run(model, O.make_params(**kw), f0, 1)
    fw = O.run(model, O.make_params(walls=1.0, **kw), f0, 1)
    same = np.all(fp == fw, axis=(0, 2))
    assert same[band + 1:ny - band - 1].all()
    assert not same[band] and not same[ny - 1 - band]
