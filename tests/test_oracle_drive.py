"""Pins of the oracle's droplet-collision force (Sec. 5.4): F_x = a_x |rho - rho_ave|, a_x by
side of x = x_split, rho_ave the domain mean every step, switched on after t_on."""
import numpy as np
import pytest

import oracle as O
from oracle import thermo

A = 0.25


def _params(model, **kw):
    T = thermo.temperature(A, 4.0, 1.0, 0.8)
    d = dict(a=A, b=4.0, R=1.0, T=T, tau_nu=0.9, tau_e=0.8, drive_ax_lo=3e-4, drive_ax_hi=-1e-4, drive_x_split=5.0)
    if model == O.PP:
        d.update(sigma_Li=thermo.sigma_li(A, 4.0, 1.0, 0.8)[0], kappa_P=0.7, tau_q=1 / 1.99)
    d.update(kw)
    return O.make_params(**d)


def _momentum_x(f):
    cx = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], dtype=float)
    return float(np.einsum("i,iyx->", cx, f))


@pytest.mark.parametrize("model", [O.PP, O.FE])
def test_drive_momentum_budget_on_a_stratified_state(model):
    """A state at rest whose density varies in y only has no x interaction force (the x
    stencils cancel pairwise), so one step changes the total x momentum by exactly the
    summed drive: sum_x a_x(x) * sum_y |rho(y) - rho_ave| (columns x <= 5 get +3e-4, the
    others -1e-4)."""
    nx, ny = 12, 9
    rng = np.random.Generator(np.random.PCG64(3))
    col = rng.uniform(0.03, 0.28, ny)
    rho0 = np.repeat(col[:, None], nx, axis=1)
    f0 = O.init(model, rho0)
    assert abs(_momentum_x(f0)) < 1e-16
    f1 = O.run(model, _params(model, drive=1.0), f0, 1)
    ax = np.where(np.arange(nx) <= 5, 3e-4, -1e-4)
    expect = ax.sum() * np.abs(col - col.mean()).sum()
    assert abs(_momentum_x(f1) - expect) < 1e-14  # rounding of ~10^3 populations of O(0.1); expect ~6e-4
    # drive off: no x momentum
    assert abs(_momentum_x(O.run(model, _params(model, drive=0.0), f0, 1))) < 1e-16


@pytest.mark.parametrize("model", [O.PP, O.FE])
def test_drive_switches_on_after_t_on_and_conserves_mass(model):
    """run_driven leaves the collisions of states t <= t_on undriven: from t0 = 0 with
    t_on = 2, the first three steps equal the undriven run and the fourth does not; mass is
    conserved throughout."""
    nx, ny = 10, 7
    rng = np.random.Generator(np.random.PCG64(5))
    col = rng.uniform(0.03, 0.28, ny)
    f0 = O.init(model, np.repeat(col[:, None], nx, axis=1))
    p = _params(model)
    f3 = O.run_driven(model, p, f0, 3, t0=0, t_on=2)
    assert np.array_equal(f3, O.run(model, _params(model, drive=0.0), f0, 3))
    f4 = O.run_driven(model, p, f0, 4, t0=0, t_on=2)
    assert abs(_momentum_x(f4)) > 1e-6
    assert abs(f4.sum() / f0.sum() - 1) < 1e-14
    # continuing from t = 3 is the same as one run
    assert np.array_equal(O.run_driven(model, p, f3, 1, t0=3, t_on=2), f4)
