"""Carnahan-Starling thermodynamics and the theoretical parameter procedure of the paper.

TEST INFRASTRUCTURE (see ``oracle/__init__.py``).  Symbolic derivatives come from
SymPy, root finding and quadrature from SciPy; each function states the passage
of arXiv:2403.11167 it follows.  Lattice units, c_s^2 = 1/3, G = -1.
"""
from __future__ import annotations

import functools
import math
from dataclasses import dataclass

import numpy as np
import sympy as sp
from scipy import integrate, optimize

CS2 = 1.0 / 3.0
G = -1.0

_rho, _T, _a, _b, _R = sp.symbols("rho T a b R", positive=True)
_eta = _b * _rho / 4
# Eq. (28): Carnahan-Starling equation of state.
_P = _rho * _R * _T * (1 + _eta + _eta**2 - _eta**3) / (1 - _eta) ** 3 - _a * _rho**2
# Eq. (29): bulk chemical potential.
_MU = _R * _T * (3 - _eta) / (1 - _eta) ** 3 + _R * _T * sp.log(_rho) + _R * _T - 2 * _a * _rho

_args = (_rho, _T, _a, _b, _R)
p_eos = sp.lambdify(_args, _P, "numpy")
dp_drho = sp.lambdify(_args, sp.diff(_P, _rho), "numpy")
d2p_drho2 = sp.lambdify(_args, sp.diff(_P, _rho, 2), "numpy")
mu_b = sp.lambdify(_args, _MU, "numpy")
dmu_drho = sp.lambdify(_args, sp.diff(_MU, _rho), "numpy")


@dataclass(frozen=True)
class EOS:
    a: float = 0.5
    b: float = 4.0
    R: float = 1.0

    def p(self, rho, T):
        return p_eos(rho, T, self.a, self.b, self.R)

    def dp(self, rho, T):
        return dp_drho(rho, T, self.a, self.b, self.R)

    def mu(self, rho, T):
        return mu_b(rho, T, self.a, self.b, self.R)

    def dmu(self, rho, T):
        return dmu_drho(rho, T, self.a, self.b, self.R)


@functools.lru_cache(maxsize=None)
def critical_point(a: float = 0.5, b: float = 4.0, R: float = 1.0):
    """Critical point (rho_c, T_c, p_c): dp/drho = d^2p/drho^2 = 0 (Sec. 3, Eq. 28).

    Solved with SymPy's multiprecision Newton from the estimates printed below
    Eq. (28) (b ~ 0.5218/rho_c, a ~ 3.8533 p_c/rho_c^2, R = 2.7864 p_c/(rho_c T_c)).
    """
    P = _P.subs({_a: a, _b: b, _R: R})
    eqs = [sp.diff(P, _rho), sp.diff(P, _rho, 2)]
    rho0 = 0.5218 / b
    T0 = 2.7864 * (a * rho0**2 / 3.8533) / (rho0 * R)
    sol = sp.nsolve(eqs, [_rho, _T], [rho0, T0], prec=40)
    rc, Tc = float(sol[0]), float(sol[1])
    pc = float(P.subs({_rho: sol[0], _T: sol[1]}))
    return rc, Tc, pc


def spinodal(eos: EOS, T: float):
    """Densities where dp/drho = 0 (the two extrema of the subcritical isotherm)."""
    rc, Tc, _ = critical_point(eos.a, eos.b, eos.R)
    assert T < Tc
    f = lambda r: eos.dp(r, T)
    # The maximum lies below rho_c, the minimum above it; dp/drho < 0 between.
    lo = optimize.brentq(f, 1e-12, rc, xtol=1e-15, rtol=1e-15)
    hi = optimize.brentq(f, rc, 4.0 / eos.b * (1 - 1e-9), xtol=1e-15, rtol=1e-15)
    return lo, hi


@functools.lru_cache(maxsize=None)
def maxwell(a: float, b: float, R: float, Tr: float):
    """Coexistence (rho_v, rho_l, p0) by equal pressure and equal chemical potential.

    Equal mu and p is the Maxwell rule; Eq. (S12) restates it as an integral
    (checked separately by the tests).  For a trial p0 between the spinodal
    pressures the vapour and liquid roots of p(rho) = p0 are bracketed, and p0 is
    found by Brent's method on mu_l(p0) - mu_v(p0).
    """
    eos = EOS(a, b, R)
    _, Tc, _ = critical_point(a, b, R)
    T = Tr * Tc
    s1, s2 = spinodal(eos, T)
    p_max = eos.p(s1, T)
    p_min = max(eos.p(s2, T), 1e-300)
    rho_top = 4.0 / b * (1 - 1e-12)

    def roots(p0):
        rv = optimize.brentq(lambda r: eos.p(r, T) - p0, 1e-300, s1, xtol=1e-300, rtol=1e-15, maxiter=500)
        rl = optimize.brentq(lambda r: eos.p(r, T) - p0, s2, rho_top, xtol=1e-300, rtol=1e-15, maxiter=500)
        return rv, rl

    def g(p0):
        rv, rl = roots(p0)
        return eos.mu(rl, T) - eos.mu(rv, T)

    eps = 1e-14 * p_max
    p0 = optimize.brentq(g, p_min + eps, p_max - eps, xtol=1e-300, rtol=1e-15, maxiter=500)
    rv, rl = roots(p0)
    return rv, rl, p0


def temperature(a: float, b: float, R: float, Tr: float) -> float:
    return Tr * critical_point(a, b, R)[1]


def psi(eos: EOS, rho, T):
    """Eq. (11): psi = sqrt(2 (p_EOS - rho c_s^2) / G)."""
    return np.sqrt(2.0 * (eos.p(rho, T) - rho * CS2) / G)


def dpsi(eos: EOS, rho, T):
    """d psi / d rho, from psi^2 = 2 (p - rho c_s^2)/G."""
    return (eos.dp(rho, T) - CS2) / (G * psi(eos, rho, T))


def _simpson(fun, lo, hi, n):
    x = np.linspace(lo, hi, n + 1)
    return integrate.simpson(fun(x), x=x)


def sigma_li(a: float, b: float, R: float, Tr: float, tol: float = 1e-13, n0: int = 2000):
    """Appendix B: epsilon such that Eq. (S13) F(eps) = 0, then sigma^Li = -eps/(16 G).

    Newton's method from eps = 2 with Simpson quadrature of Eqs. (S13)/(S14).  The
    derivative used is d/d eps of the integrand of (S13),
    -(p - p0) psi' ln(psi) / psi^(1+eps); (S14) as printed lacks that minus sign,
    which would not change the root but would send Newton the wrong way.  The
    panel count is doubled until eps changes by less than ``tol``.
    Returns (sigma_Li, eps, residual F(eps)).
    """
    eos = EOS(a, b, R)
    T = temperature(a, b, R, Tr)
    rv, rl, p0 = maxwell(a, b, R, Tr)

    def F(eps, n):
        return _simpson(lambda r: (eos.p(r, T) - p0) * dpsi(eos, r, T) / psi(eos, r, T) ** (1 + eps), rv, rl, n)

    def dF(eps, n):
        return _simpson(lambda r: -(eos.p(r, T) - p0) * dpsi(eos, r, T) * np.log(psi(eos, r, T))
                        / psi(eos, r, T) ** (1 + eps), rv, rl, n)

    def solve(n):
        eps = 2.0
        for _ in range(100):
            step = -F(eps, n) / dF(eps, n)
            eps += step
            if abs(step) < 1e-15 * max(1.0, abs(eps)):
                break
        return eps

    n = n0
    eps = solve(n)
    while True:
        n *= 2
        e2 = solve(n)
        if abs(e2 - eps) < tol or n > 2**22:
            eps = e2
            break
        eps = e2
    return -eps / (16.0 * G), eps, F(eps, n)


def _profile_grid(rv, rl, n=200001):
    return np.linspace(rv, rl, n)


def fe_profile_slope(a, b, R, Tr, kappa, n=200001):
    """Eq. (26): (d rho/dx)^2 = (2 rho/kappa) int_{rho_v}^{rho} (p - p0)/rho'^2 d rho'.

    Returns (rho grid, d rho/dx) on a uniform density grid from rho_v to rho_l.
    """
    eos = EOS(a, b, R)
    T = temperature(a, b, R, Tr)
    rv, rl, p0 = maxwell(a, b, R, Tr)
    r = _profile_grid(rv, rl, n)
    inner = integrate.cumulative_simpson((eos.p(r, T) - p0) / r**2, x=r, initial=0.0)
    z2 = 2.0 * r / kappa * inner
    return r, np.sqrt(np.clip(z2, 0.0, None))


def pp_profile_slope(a, b, R, Tr, kappa_P, eps, n=200001):
    """Eq. (S44): (psi' d rho/dx)^2 = 8 psi^eps/(G) int_{rho_v}^{rho} (p0 - p)/kappa^P psi'/psi^(1+eps) d rho'."""
    eos = EOS(a, b, R)
    T = temperature(a, b, R, Tr)
    rv, rl, p0 = maxwell(a, b, R, Tr)
    r = _profile_grid(rv, rl, n)
    ps, dps = psi(eos, r, T), dpsi(eos, r, T)
    inner = integrate.cumulative_simpson((p0 - eos.p(r, T)) / kappa_P * dps / ps ** (1 + eps), x=r, initial=0.0)
    z2 = 8.0 * ps**eps / G * inner / dps**2
    return r, np.sqrt(np.clip(z2, 0.0, None))


def tangent_width(r, slope):
    """Interface width (rho_l - rho_v) / max |d rho/dx| of a planar profile."""
    return (r[-1] - r[0]) / np.max(slope)


def fe_width(a, b, R, Tr, kappa):
    r, s = fe_profile_slope(a, b, R, Tr, kappa)
    return tangent_width(r, s)


def fe_surface_tension(a, b, R, Tr, kappa):
    """gamma = int (p_xx - p_yy) dx = kappa int (d rho/dx)^2 dx = kappa int (d rho/dx) d rho (Eq. 25)."""
    r, s = fe_profile_slope(a, b, R, Tr, kappa)
    return kappa * integrate.simpson(s, x=r)


def pp_width(a, b, R, Tr, kappa_P, eps):
    r, s = pp_profile_slope(a, b, R, Tr, kappa_P, eps)
    return tangent_width(r, s)


def pp_surface_tension(a, b, R, Tr, kappa_P, kappa_Li, eps):
    """Eq. (S46): gamma = -(G/6)(kappa^P - kappa^Li) int psi' (d psi/dx) d rho."""
    eos = EOS(a, b, R)
    T = temperature(a, b, R, Tr)
    r, s = pp_profile_slope(a, b, R, Tr, kappa_P, eps)
    dps = dpsi(eos, r, T)
    return -(G / 6.0) * (kappa_P - kappa_Li) * integrate.simpson(dps * dps * s, x=r)


def match_pp_to_fe(a, b, R, Tr, kappa):
    """Sec. 3 / App. B: P-model parameters reproducing the FE width and surface tension.

    sigma^Li from Eq. (S13); kappa^P from W_P(kappa^P) = W_FE, using that the
    profile of Eq. (S44) scales as 1/sqrt(kappa^P) in slope; kappa^Li from
    gamma_P (Eq. S46) = gamma_FE.  Returns dict(sigma_Li, eps, kappa_P, kappa_Li,
    W, gamma).
    """
    sig, eps, _ = sigma_li(a, b, R, Tr)
    W_fe = fe_width(a, b, R, Tr, kappa)
    g_fe = fe_surface_tension(a, b, R, Tr, kappa)
    W_p1 = pp_width(a, b, R, Tr, 1.0, eps)
    kP = (W_fe / W_p1) ** 2
    g_unit = pp_surface_tension(a, b, R, Tr, kP, 0.0, eps) / kP  # gamma per unit (kappa^P - kappa^Li)
    kLi = kP - g_fe / g_unit
    return dict(sigma_Li=sig, eps=eps, kappa_P=kP, kappa_Li=kLi, W=W_fe, gamma=g_fe)


def maxwell_integral(a, b, R, Tr, rv, rl, p0):
    """Eq. (S12): int_{rho_v}^{rho_l} (p - p0) / rho^2 d rho (zero at coexistence)."""
    eos = EOS(a, b, R)
    T = temperature(a, b, R, Tr)
    val, _ = integrate.quad(lambda r: (eos.p(r, T) - p0) / r**2, rv, rl, epsabs=1e-15, epsrel=1e-13, limit=500)
    return val


def reduced(x, a=0.5, b=4.0, R=1.0):
    return x / critical_point(a, b, R)[0]


__all__ = [
    "EOS", "critical_point", "maxwell", "temperature", "psi", "dpsi", "sigma_li",
    "fe_width", "fe_surface_tension", "pp_width", "pp_surface_tension", "match_pp_to_fe",
    "maxwell_integral", "spinodal", "fe_profile_slope", "pp_profile_slope", "reduced", "CS2", "G",
    "math",
]
