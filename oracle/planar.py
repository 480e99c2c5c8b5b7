"""Discrete planar-interface relations of Appendices D and E, solved directly.

TEST INFRASTRUCTURE (see ``oracle/__init__.py``).

* ``fe_discrete_profile`` solves Eq. (S60),
  mu_b(rho_n) - kappa (rho_{n+1} - 2 rho_n + rho_{n-1}) = mu_0 for every n of a
  periodic row, together with a prescribed total mass, by SciPy's hybrid Newton
  method.  Appendix D shows the FE-LBM steady state obeys it (Eq. S59).
* ``pp_invariant`` evaluates the left-hand side of Eq. (S76),
  c_s^2 rho_n + G/2 psi_n^2 + G/4 kappa^P psi_n (psi_{n+1} - 2 psi_n + psi_{n-1})
  + 2 G^2 kappa^P sigma^Li ((psi_{n+1} - psi_{n-1})/2)^2,
  which Appendix E shows is the same constant at every n of a P-LBM steady
  state with tau_e = tau_nu.
"""
import numpy as np
from scipy import optimize

from . import thermo

CS2 = 1.0 / 3.0


def fe_discrete_profile(a, b, R, Tr, kappa, rho_init: np.ndarray):
    """Solution of Eq. (S60) with the mass of ``rho_init`` (a periodic 1-D row)."""
    eos = thermo.EOS(a, b, R)
    T = thermo.temperature(a, b, R, Tr)
    mass = float(rho_init.sum())

    def residual(z):
        r, mu0 = z[:-1], z[-1]
        lap = np.roll(r, -1) - 2.0 * r + np.roll(r, 1)
        return np.concatenate([eos.mu(r, T) - kappa * lap - mu0, [r.sum() - mass]])

    z0 = np.concatenate([rho_init, [float(eos.mu(rho_init.min(), T))]])
    sol = optimize.root(residual, z0, method="hybr", tol=1e-15)
    if np.abs(residual(sol.x)).max() > 1e-12:
        raise RuntimeError("Eq. (S60) Newton solve did not converge: " + sol.message)
    return sol.x[:-1], sol.x[-1]


def pp_invariant(rho_row, psi_row, kappa_P, sigma_Li, G=-1.0):
    """Left-hand side of Eq. (S76) along a periodic row."""
    pn = psi_row
    pp, pm = np.roll(pn, -1), np.roll(pn, 1)
    return (CS2 * rho_row + G / 2.0 * pn**2 + G / 4.0 * kappa_P * pn * (pp - 2.0 * pn + pm)
            + 2.0 * G * G * kappa_P * sigma_Li * ((pp - pm) / 2.0) ** 2)
