"""Observables of a flat interface or a droplet computed from oracle fields.

TEST INFRASTRUCTURE (see ``oracle/__init__.py``).  Definitions (the paper names
these quantities without fixing how they are probed):

* rho_l, rho_v -- flat: mean over the column x = nx/2 (liquid, middle of the
  slab) and over the column x = 0 (vapour); droplet: mean over cells with
  r <= 2 from the centre ((nx-1)/2, (ny-1)/2) and over the four 5x5 corner blocks.
* width W -- (rho_l - rho_v) / max_x |(rho[x+1] - rho[x-1]) / 2| along row 0 of
  a flat interface (tangent width; a tanh(2x/W) profile has exactly width W);
  for a droplet the same along the row through the centre.
* dp -- p_EOS(rho_l) - p_EOS(rho_v), the pressure jump of Sec. 5.2.
* R_e -- equimolar radius sqrt(sum(rho - rho_v) / (pi (rho_l - rho_v))).
* u_max -- max |u| over the lattice, mass -- sum rho.
"""
import math

import numpy as np

from . import thermo


def probes(rho: np.ndarray, geometry: int):
    ny, nx = rho.shape
    if geometry == 0:
        return float(rho[:, nx // 2].mean()), float(rho[:, 0].mean())
    cy, cx = (ny - 1) / 2.0, (nx - 1) / 2.0
    yy, xx = np.mgrid[0:ny, 0:nx]
    core = (yy - cy) ** 2 + (xx - cx) ** 2 <= 4.0
    corners = np.concatenate([rho[:5, :5].ravel(), rho[:5, -5:].ravel(), rho[-5:, :5].ravel(), rho[-5:, -5:].ravel()])
    return float(rho[core].mean()), float(corners.mean())


def width(rho: np.ndarray, geometry: int, rho_l: float, rho_v: float) -> float:
    ny, nx = rho.shape
    row = rho[0] if geometry == 0 else rho[ny // 2]
    d = np.abs(np.roll(row, -1) - np.roll(row, 1)) / 2.0
    return float((rho_l - rho_v) / d.max())


def equimolar_radius(rho: np.ndarray, rho_l: float, rho_v: float) -> float:
    return math.sqrt(float((rho - rho_v).sum()) / (math.pi * (rho_l - rho_v)))


def observables(rho, ux, uy, geometry: int, a: float, b: float, R: float, T: float):
    rl, rv = probes(rho, geometry)
    eos = thermo.EOS(a, b, R)
    return dict(
        rho_l=rl, rho_v=rv, width=width(rho, geometry, rl, rv),
        dp=float(eos.p(rl, T) - eos.p(rv, T)),
        u_max=float(np.sqrt(ux**2 + uy**2).max()), mass=float(rho.sum()),
        radius=equimolar_radius(rho, rl, rv) if geometry == 1 else float("nan"),
    )
