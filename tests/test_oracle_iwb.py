"""Pins of the oracle's full improved well-balanced free-energy model: the viscosity-tuning
term A of Eqs. (20)/(23) and gravity (p_g in Eq. 20, -grad p_g in Eq. 21, buoyancy F_g)."""
import numpy as np
import pytest

import oracle as O
from oracle import thermo

A_EOS = 0.25


def _T(Tr=0.8):
    return thermo.temperature(A_EOS, 4.0, 1.0, Tr)


def _shear_wave(A, tau, L=64, steps=(200, 1200), U=1e-4):
    """Uniform density, u_x = U sin(2 pi y / L): amplitude ratio between two times."""
    rv, rl, _ = thermo.maxwell(A_EOS, 4.0, 1.0, 0.8)
    rho = rl
    nx = 4
    p = O.make_params(a=A_EOS, b=4.0, R=1.0, T=_T(), tau_nu=tau, tau_e=1.0, kappa=0.5, A=A)
    f = O.init(O.FE, np.full((L, nx), rho))
    y = np.arange(L)
    ux = U * np.sin(2 * np.pi * y / L)
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    cx = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
    f = f + (w * cx)[:, None, None] * 3.0 * rho * ux[None, :, None]  # first-order momentum
    amps = []
    t = 0
    for s in steps:
        f = O.run(O.FE, p, f, s - t)
        t = s
        _, u, _, *_ = O.macro(O.FE, p, f)
        amps.append(2.0 / L * np.sum(u[:, 0] * np.sin(2 * np.pi * y / L)))
    k2 = (2 * np.pi / L) ** 2
    return -np.log(amps[1] / amps[0]) / (k2 * (steps[1] - steps[0]))


@pytest.mark.parametrize("A,tau", [(0.0, 1.0), (0.2, 1.0), (-0.2, 0.9)])
def test_shear_wave_viscosity_eq23(A, tau):
    """A shear wave decays at nu k^2 with nu = c_s^2 (tau_nu - 1/2 - A) (Eq. 23) to the
    scheme's O(k^2) accuracy (L = 64): within 0.5%."""
    nu = _shear_wave(A, tau)
    assert abs(nu / ((tau - 0.5 - A) / 3.0) - 1) < 5e-3, nu


def test_equilibrium_moments_eq20():
    """Eq. (20) is built so that its moments are rho, rho u and the momentum flux
    p_g delta + rho (u u + c_s^2 A S); and its third moment is that of the plain equilibrium
    (rho c_s^2 (u_a d_bc + u_b d_ac + u_c d_ab)): p_g and the A term are even."""
    cx = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], dtype=float)
    cy = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1], dtype=float)
    rho, ux, uy, pg, A = 0.31, 0.013, -0.021, 0.0042, 0.17
    Sxx, Sxy, Syy = 2.3e-3, -1.1e-3, -0.7e-3
    f = O.feq_iwb(rho, ux, uy, pg, A, Sxx, Sxy, Syy)
    assert abs(f.sum() - rho) < 1e-16
    assert abs(f @ cx - rho * ux) < 1e-17 and abs(f @ cy - rho * uy) < 1e-17
    cs2 = 1.0 / 3.0
    assert abs(f @ (cx * cx) - (pg + rho * (ux * ux + cs2 * A * Sxx))) < 1e-16
    assert abs(f @ (cy * cy) - (pg + rho * (uy * uy + cs2 * A * Syy))) < 1e-16
    assert abs(f @ (cx * cy) - rho * (ux * uy + cs2 * A * Sxy)) < 1e-17
    assert abs(f @ (cx * cx * cy) - rho * cs2 * uy) < 1e-17
    assert abs(f @ (cx * cy * cy) - rho * cs2 * ux) < 1e-17


def test_buoyancy_momentum_budget():
    """With rho_0 = 0 (p_g = 0, so a periodic lattice is allowed) gravity is the body force
    -rho g: from rest, one step of a uniform state changes the y momentum by exactly -g sum rho
    (no interaction force at uniform density)."""
    rv, rl, _ = thermo.maxwell(A_EOS, 4.0, 1.0, 0.8)
    g = 2e-5
    p = O.make_params(a=A_EOS, b=4.0, R=1.0, T=_T(), tau_nu=0.9, tau_e=0.8, kappa=0.5, g=g, rho_g=0.0)
    rho0 = np.full((7, 6), rl)
    f = O.run(O.FE, p, O.init_iwb(p, rho0), 1)
    cy = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1], dtype=float)
    assert abs(np.einsum("i,iyx->", cy, f) + g * rho0.sum()) < 1e-15


def test_gravity_and_A_off_reproduce_the_plain_model():
    """A = 0, g = 0 (and p_g = 0) run the plain Eq. (20)/(21) model: identical states."""
    rv, rl, _ = thermo.maxwell(A_EOS, 4.0, 1.0, 0.8)
    rng = np.random.Generator(np.random.PCG64(9))
    rho0 = rng.uniform(rv * 2, rl * 0.8, (11, 13))
    p = O.make_params(a=A_EOS, b=4.0, R=1.0, T=_T(), tau_nu=0.9, tau_e=0.8, kappa=0.5)
    f1 = O.run(O.FE, p, O.init(O.FE, rho0), 30)
    f2 = O.run(O.FE, p, O.init_iwb(p, rho0), 30)
    assert np.array_equal(f1, f2)


@pytest.mark.parametrize("force", ["fy", "gravity"])
def test_wall_normal_force_period2_mode(force):
    """A liquid column between walls under a wall-normal force (body force fy = -1e-5, or
    gravity g = 1e-5 with rho_0 = rho_l): with mirrored wall rows (walls = 1) the free-energy
    model's neutral period-2 density mode grows from the walls without bound (the second
    differences of rho keep growing: x3 between 8e3 and 2e4 steps); with the one-sided normal mu
    gradient and a self-consistent wall density (walls = 2) the column is steady (second
    differences below 1e-5 and unchanged, velocity ~ 0)."""
    rv, rl, _ = thermo.maxwell(A_EOS, 4.0, 1.0, 0.8)
    ny, nx = 40, 4
    kw = dict(fy=-1e-5) if force == "fy" else dict(g=1e-5, rho_g=rl)
    amp = {}
    for walls in (1.0, 2.0):
        p = O.make_params(a=A_EOS, b=4.0, R=1.0, T=_T(), tau_nu=1.0, tau_e=1.0, kappa=0.5, walls=walls, **kw)
        f = O.init_iwb(p, np.full((ny, nx), rl))
        f8 = O.run(O.FE, p, f, 8000)
        f20 = O.run(O.FE, p, f8, 12000)
        a8 = np.abs(np.diff(O.macro(O.FE, p, f8)[0][4:-4, 0], 2)).max()
        rho, ux, uy, *_ = O.macro(O.FE, p, f20)
        amp[walls] = (a8, np.abs(np.diff(rho[4:-4, 0], 2)).max(), np.abs(uy).max())
    grow1, grow2 = amp[1.0][1] / amp[1.0][0], amp[2.0][1] / amp[2.0][0]
    assert grow1 > 2.0 and amp[1.0][1] > 1e-3
    assert amp[2.0][1] < 1e-5 and abs(grow2 - 1) < 0.05 and amp[2.0][2] < 1e-7
