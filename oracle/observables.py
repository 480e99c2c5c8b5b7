"""Observables of a flat interface or a droplet computed from oracle fields.

TEST INFRASTRUCTURE (see ``oracle/__init__.py``).  The paper names these
quantities (Secs. 5.1-5.2) without fixing how they are probed; the readings:

* rho_l, rho_v -- flat (geometry 0): mean over the two columns x = nx/2 - 1,
  nx/2 (liquid, middle of the slab) and over x = 0, nx - 1 (vapour).  Droplet
  (geometry 1): mean over the 4x4 block starting at (nx/2 - 2, ny/2 - 2)
  (liquid) and over the four 4x4 corner blocks (vapour).  Every probe covers
  pairs of neighbouring cells in each direction, so the period-2 (odd-even)
  density modes that the central-difference force stencils cannot see cancel.
* width W -- (rho_l - rho_v) / max_x |(rho[x+1] - rho[x-1]) / 2| along row 0
  (flat) or row ny/2 (droplet): the tangent width (a tanh(2x/W) profile has
  exactly width W; the central difference is blind to period-2 modes too).
* dp -- p_EOS(rho_l) - p_EOS(rho_v), the pressure jump of Sec. 5.2.
* radius -- equimolar radius sqrt(sum(rho - rho_v) / (pi (rho_l - rho_v))).
* u_max -- max |u| over the lattice; mass -- sum of rho.
"""
import math

import numpy as np

from . import thermo


def probes(rho: np.ndarray, geometry: int):
    ny, nx = rho.shape
    if geometry == 0:
        liq = rho[:, [nx // 2 - 1, nx // 2]]
        vap = rho[:, [0, nx - 1]]
        return float(liq.mean()), float(vap.mean())
    cx0, cy0 = nx // 2 - 2, ny // 2 - 2
    liq = rho[cy0:cy0 + 4, cx0:cx0 + 4]
    vap = np.concatenate([rho[:4, :4].ravel(), rho[:4, -4:].ravel(), rho[-4:, :4].ravel(), rho[-4:, -4:].ravel()])
    return float(liq.mean()), float(vap.mean())


def width(rho: np.ndarray, geometry: int, rho_l: float, rho_v: float) -> float:
    ny, nx = rho.shape
    row = rho[0] if geometry == 0 else rho[ny // 2]
    d = np.abs(np.roll(row, -1) - np.roll(row, 1)) / 2.0
    return float((rho_l - rho_v) / d.max())


def equimolar_radius(rho: np.ndarray, rho_l: float, rho_v: float) -> float:
    return math.sqrt(max(float((rho - rho_v).sum()), 0.0) / (math.pi * (rho_l - rho_v)))


def observables(rho, ux, uy, geometry: int, a: float, b: float, R: float, T: float):
    rl, rv = probes(rho, geometry)
    eos = thermo.EOS(a, b, R)
    return dict(
        rho_l=rl, rho_v=rv, width=width(rho, geometry, rl, rv),
        dp=float(eos.p(rl, T) - eos.p(rv, T)),
        u_max=float(np.sqrt(ux**2 + uy**2).max()), mass=float(rho.sum()),
        radius=equimolar_radius(rho, rl, rv) if geometry == 1 else float("nan"),
    )
