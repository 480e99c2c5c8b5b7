"""Pins of the FP64 oracle's cell-level pieces against closed forms of the paper.

Each check uses a relation the paper (or plain lattice algebra) fixes, not a
retyping of the oracle's own formula.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from oracle import brute, thermo
from paper_2403_11167_gb300 import inputs
from conftest import golden

CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def test_minv_matches_printed_s49():
    """T1: the oracle inverts M numerically; the result must equal Eq. (S49) as printed."""
    printed = np.array([[float(Fraction(v)) for v in row] for row in golden("minv_s49.txt")])
    Minv = O.moment_matrix_inverse()
    assert np.abs(Minv - printed).max() < 1e-15
    assert np.abs(O.moment_matrix() @ printed - np.eye(9)).max() < 1e-15
    assert np.abs(brute.MINV - printed).max() < 1e-14


def test_moment_matrix_rows_are_velocity_polynomials():
    """Rows of Eq. (S48) are the Lallemand-Luo polynomials of c_i."""
    M = O.moment_matrix()
    c2 = CX**2 + CY**2
    assert np.array_equal(M[0], np.ones(9))
    assert np.array_equal(M[1], 3 * c2 - 4)
    assert np.array_equal(M[2], (9 * c2**2 - 21 * c2 + 8) / 2)
    assert np.array_equal(M[3], CX) and np.array_equal(M[5], CY)
    assert np.array_equal(M[4], (3 * c2 - 5) * CX) and np.array_equal(M[6], (3 * c2 - 5) * CY)
    assert np.array_equal(M[7], CX**2 - CY**2) and np.array_equal(M[8], CX * CY)


@pytest.mark.parametrize("rho,ux,uy", [(0.3, 0.01, -0.02), (0.02, -0.05, 0.03), (1.0, 0.0, 0.0)])
def test_equilibrium_moments(rho, ux, uy):
    """T2: moments of Eq. (4) per (S21); of Eq. (20) per its well-balanced design (no c_s^2 rho)."""
    uu = ux * ux + uy * uy
    f = O.feq(O.PP, rho, ux, uy)
    assert np.isclose(f.sum(), rho, rtol=1e-14)
    assert np.allclose([f @ CX, f @ CY], [rho * ux, rho * uy], rtol=1e-13, atol=1e-16)
    P = np.array([[f @ (CX * CX), f @ (CX * CY)], [f @ (CY * CX), f @ (CY * CY)]])
    assert np.allclose(P, rho * np.outer([ux, uy], [ux, uy]) + rho / 3 * np.eye(2), rtol=1e-13, atol=1e-16)
    # (S66): m^eq of the standard equilibrium
    m = O.moment_matrix() @ f
    expect = [rho, rho * (-2 + 3 * uu), rho * (1 - 3 * uu), rho * ux, -rho * ux, rho * uy, -rho * uy,
              rho * (ux * ux - uy * uy), rho * ux * uy]
    assert np.allclose(m, expect, rtol=1e-12, atol=1e-16)
    g = O.feq(O.FE, rho, ux, uy)
    assert np.isclose(g.sum(), rho, rtol=1e-14)
    assert np.allclose([g @ CX, g @ CY], [rho * ux, rho * uy], rtol=1e-13, atol=1e-16)
    P = np.array([[g @ (CX * CX), g @ (CX * CY)], [g @ (CY * CX), g @ (CY * CY)]])
    assert np.allclose(P, rho * np.outer([ux, uy], [ux, uy]), rtol=1e-13, atol=1e-16)
    # (S50): e and zeta moments of the well-balanced equilibrium
    mg = O.moment_matrix() @ g
    assert np.allclose(mg[1:3], [rho * (-4 + 3 * uu), rho * (4 - 3 * uu)], rtol=1e-12)


def test_pp_forcing_and_source_moments():
    """T3: (S22) and (S23) for the populations that Eqs. (32) and (13) produce."""
    taus = dict(tau_rho=1.0, tau_e=0.83, tau_zeta=1.13, tau_j=0.91, tau_q=1 / 1.99, tau_nu=0.71)
    p = O.make_params(kappa_P=0.6, kappa_Li=-0.4, sigma_Li=0.118, **taus)
    ux, uy, Fx, Fy, Fix, Fiy, psi = 0.013, -0.021, 3e-3, -1e-3, 2.5e-3, -1.5e-3, 0.17
    Qxx, Qyy, Qxy = 1.1e-3, -0.6e-3, 0.4e-3
    S, C = O.pp_sources(p, ux, uy, Fx, Fy, Fix, Fiy, psi, Qxx, Qyy, Qxy)
    wj, we, wv = 1 / taus["tau_j"], 1 / taus["tau_e"], 1 / taus["tau_nu"]
    u, F = np.array([ux, uy]), np.array([Fx, Fy])
    assert abs(S.sum()) < 1e-17
    assert np.allclose([S @ CX, S @ CY], (1 - wj / 2) * F, rtol=1e-13)
    SS = np.array([[S @ (CX * CX), S @ (CX * CY)], [S @ (CY * CX), S @ (CY * CY)]])
    li = 2 * we * p.kappa_P * p.sigma_Li * (Fix**2 + Fiy**2) / psi**2
    expect = (1 - wv / 2) * (np.outer(u, F) + np.outer(F, u)) + (wv - we) / 2 * np.eye(2) * (u @ F) + li * np.eye(2)
    assert np.allclose(SS, expect, rtol=1e-12, atol=1e-18)
    assert abs(C.sum()) < 1e-17 and abs(C @ CX) < 1e-17 and abs(C @ CY) < 1e-17
    CC = np.array([[C @ (CX * CX), C @ (CX * CY)], [C @ (CY * CX), C @ (CY * CY)]])
    Q = np.array([[Qxx, Qxy], [Qxy, Qyy]])
    expectC = -wv * Q + (wv + 0.5 * we) / 2 * np.eye(2) * (Qxx + Qyy)
    assert np.allclose(CC, expectC, rtol=1e-12, atol=1e-18)


def test_fe_forcing_moments():
    """T3: moments of Eq. (21): sum 0, first moment F, second uF' + F'u + c_s^2 (u.grad rho) I,
    with F' = F + c_s^2 grad rho (the design of the improved well-balanced forcing)."""
    u, F, g = np.array([0.011, -0.007]), np.array([2e-3, 3e-3]), np.array([0.05, -0.02])
    Fi = O.fe_forcing(*u, *F, *g)
    assert abs(Fi.sum()) < 1e-17
    assert np.allclose([Fi @ CX, Fi @ CY], F, rtol=1e-13)
    SS = np.array([[Fi @ (CX * CX), Fi @ (CX * CY)], [Fi @ (CY * CX), Fi @ (CY * CY)]])
    Fp = F + g / 3
    assert np.allclose(SS, np.outer(u, Fp) + np.outer(Fp, u) + np.eye(2) * (u @ g) / 3, rtol=1e-12)


def _quadratic_field(nx, ny, c0, ax, bxy, cy, dx=0.0, dy=0.0):
    yy, xx = np.mgrid[0:ny, 0:nx].astype(float)
    xx -= nx // 2
    yy -= ny // 2
    return c0 + dx * xx + dy * yy + ax * xx**2 + bxy * xx * yy + cy * yy**2


def test_stencils_exact_on_quadratics():
    """T13: the Eq. (24) stencils are exact for quadratic fields."""
    ax, bxy, cy, dx, dy = 0.013, -0.007, 0.004, 0.3, -0.2
    phi = _quadratic_field(16, 16, 1.0, ax, bxy, cy, dx, dy)
    x, y = 9, 6
    X, Y = x - 8, y - 8
    gx, gy, lap = O.stencils(phi, x, y)
    assert np.isclose(gx, dx + 2 * ax * X + bxy * Y, rtol=1e-13)
    assert np.isclose(gy, dy + bxy * X + 2 * cy * Y, rtol=1e-13)
    assert np.isclose(lap, 2 * ax + 2 * cy, rtol=1e-12)


@pytest.mark.parametrize("kP,kLi", [(1.0, 0.0), (0.4, 0.0), (0.7, -1.3), (1.3, 0.5)])
def test_q_tensor_continuum_form(kP, kLi):
    """Eq. (30) against its continuum form Eq. (S41b), exact on a quadratic psi:
    Q = (1 - kP + kLi) G/6 psi d_a d_b psi + (5 kP + kLi - 5) G/12 psi lap psi delta.
    This fixes the reading that the C2 term of Eq. (30b) carries G."""
    ax, bxy, cy = 0.011, -0.006, 0.003
    psi = _quadratic_field(16, 16, 0.5, ax, bxy, cy, 0.02, -0.01)
    p = O.make_params(kappa_P=kP, kappa_Li=kLi)
    x, y = 7, 9
    pc = psi[y, x]
    Qxx, Qyy, Qxy = O.q_tensor(p, psi, x, y)
    G = -1.0
    H = np.array([[2 * ax, bxy], [bxy, 2 * cy]])
    lap = 2 * ax + 2 * cy
    expect = (1 - kP + kLi) * G / 6 * pc * H + (5 * kP + kLi - 5) * G / 12 * pc * lap * np.eye(2)
    assert np.allclose([Qxx, Qyy, Qxy], [expect[0, 0], expect[1, 1], expect[0, 1]], rtol=1e-12, atol=1e-17)


def test_shan_chen_force_continuum_form():
    """Eq. (10) against Eq. (S41a): F = -G psi grad psi, exact on a quadratic psi."""
    ax, bxy, cy, dx, dy = 0.011, -0.006, 0.003, 0.02, -0.01
    rho = np.full((16, 16), 0.1)
    # Build populations at rest whose rho gives a chosen psi is awkward; test the force
    # through oracle.macro on a field with known psi instead: invert psi -> rho per cell.
    a, b, R = 0.5, 4.0, 1.0
    T = thermo.temperature(a, b, R, 0.8)
    eos = thermo.EOS(a, b, R)
    target = _quadratic_field(16, 16, 0.0, ax, bxy, cy, dx, dy) * 0.02 + 0.2
    from scipy import optimize
    rho = np.vectorize(lambda t: optimize.brentq(lambda r: thermo.psi(eos, r, T) - t, 0.005, 0.3))(target)
    p = O.make_params(a=a, b=b, R=R, T=T)
    f = O.init(O.PP, rho)
    _, _, _, Fx, Fy, psi = O.macro(O.PP, p, f)
    assert np.allclose(psi, target, rtol=1e-12)
    x, y = 8, 7
    X, Y = x - 8, y - 8
    gx = 0.02 * (dx + 2 * ax * X + bxy * Y)
    gy = 0.02 * (dy + bxy * X + 2 * cy * Y)
    assert np.isclose(Fx[y, x], psi[y, x] * gx, rtol=1e-11)
    assert np.isclose(Fy[y, x], psi[y, x] * gy, rtol=1e-11)


@pytest.mark.parametrize("model", [O.PP, O.FE])
@pytest.mark.parametrize("shape", [(8, 8), (7, 5)])
def test_brute_force_agreement(model, shape):
    """T14: C oracle and the independent NumPy implementation agree on tiny lattices."""
    nx, ny = shape
    a, b, R, Tr = 0.5, 4.0, 1.0, 0.8
    T = thermo.temperature(a, b, R, Tr)
    rv, rl, _ = thermo.maxwell(a, b, R, Tr)
    rho0 = inputs.random_field(nx, ny, rv * 1.2, rl * 0.9, seed=7)
    pr = dict(a=a, b=b, R=R, T=T, G=-1.0, tau_rho=1.0, tau_e=0.9, tau_zeta=1.1, tau_j=1.0, tau_q=1 / 1.99,
              tau_nu=0.8, kappa_P=0.7, kappa_Li=-0.3, sigma_Li=0.117, kappa=0.5, fx=1e-4, fy=-2e-4)
    f0 = O.init(model, rho0)
    fo = O.run(model, O.make_params(**pr), f0, 30)
    fb = brute.run(model, f0.copy(), pr, 30)
    assert np.abs(fo - fb).max() < 1e-13


@pytest.mark.parametrize("model", [O.PP, O.FE])
def test_mass_conservation(model):
    """T4: Eq. (1) conserves mass exactly on a periodic lattice; in FP64 the drift is bounded
    by rounding, far below 1e-15 relative per step."""
    a, b, R, Tr = 0.25, 4.0, 1.0, 0.8
    T = thermo.temperature(a, b, R, Tr)
    rv, rl, _ = thermo.maxwell(a, b, R, Tr)
    m = thermo.match_pp_to_fe(a, b, R, Tr, 0.5)
    p = O.make_params(a=a, b=b, R=R, T=T, kappa=0.5, tau_e=0.75 if model == O.FE else 1.0,
                      tau_q=1 / 1.99 if model == O.PP else 1.0, kappa_P=m["kappa_P"],
                      kappa_Li=m["kappa_Li"], sigma_Li=m["sigma_Li"])
    rho0 = inputs.droplet(40, 40, 10, rv, rl)
    f = O.run(model, p, O.init(model, rho0), 2000)
    assert abs(f.sum() - rho0.sum()) / rho0.sum() < 2000 * 1e-15


def test_pp_momentum_conservation():
    """Without a body force the Shan-Chen force of Eq. (10) sums to zero over a periodic
    lattice (pairwise antisymmetry), so total momentum sum(f c) is conserved."""
    a, b, R, Tr = 0.5, 4.0, 1.0, 0.8
    T = thermo.temperature(a, b, R, Tr)
    rv, rl, _ = thermo.maxwell(a, b, R, Tr)
    p = O.make_params(a=a, b=b, R=R, T=T, sigma_Li=0.12, kappa_P=0.8, kappa_Li=-0.5)
    f0 = O.init(O.PP, inputs.random_field(24, 20, rv * 1.5, rl * 0.8, seed=3))
    f = O.run(O.PP, p, f0, 200)
    j = [np.tensordot(CX, f, 1).sum(), np.tensordot(CY, f, 1).sum()]
    assert np.abs(j).max() < 1e-14


def _wall_unknown_mask(ny, nx):
    """Populations a wall node receives from beyond the wall (completed by the fill; the C
    oracle returns them completed, the NumPy step leaves what streaming wrapped in)."""
    m = np.ones((9, ny, nx), bool)
    m[[2, 5, 6], 0] = False
    m[[4, 7, 8], ny - 1] = False
    return m


@pytest.mark.parametrize("model,extra", [
    (O.PP, dict(walls=1.0)),
    (O.PP, dict(drive=1.0, drive_ax_lo=3e-4, drive_ax_hi=-2e-4, drive_x_split=3.0)),
    (O.FE, dict(walls=1.0)),
    (O.FE, dict(drive=1.0, drive_ax_lo=3e-4, drive_ax_hi=-2e-4, drive_x_split=3.0)),
    (O.FE, dict(A=0.15)),
    (O.FE, dict(A=-0.1, walls=1.0)),
    (O.FE, dict(g=3e-4, rho_g=0.0)),
    (O.FE, dict(A=0.1, walls=1.0, g=2e-5, rho_g=0.1, y_ref=3.0)),
    (O.FE, dict(walls=2.0)),
    (O.FE, dict(A=0.1, walls=2.0, g=2e-5, rho_g=0.1, y_ref=3.0)),
])
def test_brute_force_agreement_extensions(model, extra):
    """The walls (Zou-He fill, mirrored stencils, odd velocities), the Sec. 5.4 drive, the
    A term and gravity of the C oracle against the independent NumPy step on a 9 x 7 random
    field, 8 steps (the walls' incoming populations are completed only in the C oracle's
    returned state and are left out of the comparison)."""
    nx, ny = 9, 7
    a, b, R, Tr = 0.5, 4.0, 1.0, 0.8
    T = thermo.temperature(a, b, R, Tr)
    rv, rl, _ = thermo.maxwell(a, b, R, Tr)
    rho0 = inputs.random_field(nx, ny, rv * 1.2, rl * 0.9, seed=11)
    pr = dict(a=a, b=b, R=R, T=T, G=-1.0, tau_rho=1.0, tau_e=0.9, tau_zeta=1.1, tau_j=1.0, tau_q=1 / 1.99,
              tau_nu=0.8, kappa_P=0.7, kappa_Li=-0.3, sigma_Li=0.117, kappa=0.5, fx=1e-4, fy=-2e-4)
    pr.update(extra)
    p = O.make_params(**pr)
    f0 = O.init_iwb(p, rho0) if model == O.FE else O.init(model, rho0)
    fo = O.run(model, p, f0, 8)
    fb = brute.run(model, f0.copy(), pr, 8)
    mask = _wall_unknown_mask(ny, nx) if extra.get("walls") else np.ones(fo.shape, bool)
    assert np.abs(fo - fb)[mask].max() < 1e-13
