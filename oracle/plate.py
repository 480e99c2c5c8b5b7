"""Analytic velocity profiles of the two-phase flow between parallel plates (Appendix F).

TEST INFRASTRUCTURE (see the package docstring): only tests and the CPU legs of the
benchmark use it.

Geometry: plates at y = 0 and y = H, body force F_x, no slip at both plates, gravity
neglected; dynamic viscosity mu = rho c_s^2 (tau - 1/2) in lattice units (c_s^2 = 1/3).

* ``s88`` -- discrete interface at y = H/2 (fluid 1 below, fluid 2 above), Eq. (88):
  piecewise parabolas matched in velocity and shear stress at the interface.  The paper
  prints C_2 = -F_x H / (8 mu_1) - C_1 H / 2; no slip at y = 0 (u_1(0) = 0) requires
  C_2 = F_x H^2 / (8 mu_1) - C_1 H / 2, which is what is used (C_1 as printed satisfies the
  other three conditions only with this C_2).
* ``s89`` -- diffuse interface, Eq. (89): u(y) = -F_x int_0^y y'/mu + mu(0) u'(0) int_0^y 1/mu,
  with mu(0) u'(0) fixed by u(H) = 0; integrals by the trapezoid rule on the given nodes.
"""
import numpy as np

CS2 = 1.0 / 3.0


def viscosity(rho, tau):
    """Dynamic viscosity of a lattice fluid, mu = rho c_s^2 (tau - 1/2)."""
    return np.asarray(rho, dtype=np.float64) * CS2 * (tau - 0.5)


def s88(y, H, mu1, mu2, fx):
    """Eq. (88) at positions y (0 <= y <= H)."""
    y = np.asarray(y, dtype=np.float64)
    c1 = fx * H / 4.0 * (mu2 - mu1) / (mu1 * (mu1 + mu2))
    c2 = fx * H * H / (8.0 * mu1) - c1 * H / 2.0
    s = H / 2.0 - y
    u1 = -fx / (2.0 * mu1) * s * s + c1 * s + c2
    t = y - H / 2.0
    u2 = -fx / (2.0 * mu2) * t * t - mu1 * c1 / mu2 * t + c2
    return np.where(y <= H / 2.0, u1, u2)


def _cumtrapz(g, y):
    return np.concatenate([[0.0], np.cumsum(0.5 * (g[1:] + g[:-1]) * np.diff(y))])


def s89(y, mu, fx):
    """Eq. (89) on the nodes y[0] = 0 < ... < y[-1] = H with viscosities mu at the nodes."""
    y = np.asarray(y, dtype=np.float64)
    mu = np.asarray(mu, dtype=np.float64)
    i1 = _cumtrapz(y / mu, y)
    i0 = _cumtrapz(1.0 / mu, y)
    shear0 = fx * i1[-1] / i0[-1]  # mu(0) u'(0)
    return -fx * i1 + shear0 * i0


def theory_rho(y, y_c, r, slope):
    """The planar density profile of Appendix A placed with its mid-density (rho_v + rho_l)/2
    at y = y_c: y(rho) = y_c + int_{rho_mid}^{rho} d rho' / (d rho/dx)(rho'), inverted by linear
    interpolation.  (r, slope) is the model's d rho/dx on a density grid from rho_v to rho_l
    (thermo.fe_profile_slope, thermo.pp_profile_slope); beyond the grid's reach the bulk
    densities are returned."""
    r = np.asarray(r, dtype=np.float64)
    s = np.asarray(slope, dtype=np.float64)
    keep = s > 0.0
    rk, sk = r[keep], s[keep]
    yk = _cumtrapz(1.0 / sk, rk)
    yk -= np.interp(0.5 * (r[0] + r[-1]), rk, yk)
    return np.interp(np.asarray(y, dtype=np.float64) - y_c, yk, rk, left=r[0], right=r[-1])


def mid_crossing(rho_col):
    """Position (linear interpolation) where a monotonic column profile crosses the mean of
    its end values."""
    rho_col = np.asarray(rho_col, dtype=np.float64)
    m = 0.5 * (rho_col[0] + rho_col[-1])
    k = int(np.argmax(rho_col >= m)) if rho_col[-1] > rho_col[0] else int(np.argmax(rho_col <= m))
    return (k - 1) + (m - rho_col[k - 1]) / (rho_col[k] - rho_col[k - 1])
