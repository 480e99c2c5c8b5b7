"""Pins of the oracle's observables (oracle/observables.py) against closed forms.

The paper names the observables of Secs. 5.1-5.2 (coexistence densities, interface width,
pressure jump, droplet radius) without fixing how a lattice state is probed; the oracle's
readings are pinned here by what the mathematics fixes, so that a slip in a stencil, a
factor or an index fails:

* tangent width of a tanh(2x/W) slab: the central difference of the profile at its centre is
  (rho_l - rho_v) tanh(2/W) / 2, so the width reads W (2/W) / tanh(2/W) = W (1 + 4/(3 W^2) +
  O(W^-4)) -- exactly, for a centre on a lattice node;
* equimolar radius of a tanh(2(r - R)/W) droplet: the area integral of the Fermi-type
  profile has the Sommerfeld expansion pi R^2 + pi^3 W^2 / 48, so the radius reads
  sqrt(R^2 + pi^2 W^2 / 48) up to the lattice-sum error of a smooth profile; a sharp disk
  reads sqrt(N(R) / pi), N(R) the lattice points inside the circle (Gauss circle problem);
* probes average pairs of neighbouring cells, so planted period-2 modes (-1)^x, (-1)^y and
  (-1)^(x+y) cancel exactly;
* the pressure jump is the Carnahan-Starling pressure (Eq. 28) at the two probe densities.
"""
import math

import numpy as np
import pytest

from oracle import observables as OO
from oracle import thermo

RV, RL = 0.0217232, 0.307196  # Maxwell densities at Tr 0.8 (any two densities would do)


def _slab(nx, ny, W, x1, x2):
    x = np.arange(nx, dtype=np.float64)
    row = RV + 0.5 * (RL - RV) * (np.tanh(2 * (x - x1) / W) - np.tanh(2 * (x - x2) / W))
    return np.tile(row, (ny, 1))


@pytest.mark.parametrize("W", [4.0, 5.0, 10.0, 20.0, 40.0])
def test_width_of_a_tanh_slab(W):
    nx = int(16 * W) * 4
    rho = _slab(nx, 4, W, nx // 4, 3 * nx // 4)  # centres on lattice nodes
    got = OO.width(rho, 0, RL, RV)
    # exact for this profile up to the exponentially small overlap of the two interfaces
    assert abs(got / (W * (2 / W) / math.tanh(2 / W)) - 1) < 1e-12, got
    # O(W^-2) convergence to W: (width/W - 1) W^2 -> 4/3
    assert abs((got / W - 1) * W * W - 4.0 / 3.0) < 2.0 / W**2 + 1e-9


def test_width_is_the_tangent_width_for_off_node_centres():
    """Centres half-way between nodes: the largest central difference straddles the centre at
    distance 1/2, (tanh(3/W) + tanh(1/W)) / 2 of the amplitude."""
    W, nx = 6.0, 256
    rho = _slab(nx, 2, W, nx / 4 + 0.5, 3 * nx / 4 + 0.5)
    d = 0.5 * (math.tanh(3 / W) + math.tanh(1 / W))
    assert abs(OO.width(rho, 0, RL, RV) / (2 / d) - 1) < 1e-12


@pytest.mark.parametrize("R,W", [(20.0, 5.0), (30.0, 5.0), (40.0, 8.0), (60.0, 5.0)])
def test_equimolar_radius_of_a_tanh_droplet(R, W):
    n = int(2 * R + 16 * W) // 2 * 2
    y, x = np.mgrid[0:n, 0:n].astype(np.float64)
    r = np.hypot(x - (n - 1) / 2, y - (n - 1) / 2)
    rho = 0.5 * (RL + RV) - 0.5 * (RL - RV) * np.tanh(2 * (r - R) / W)
    got = OO.equimolar_radius(rho, RL, RV)
    want = math.sqrt(R * R + math.pi**2 * W * W / 48.0)
    assert abs(got - want) < 2e-3, (got, want)
    assert abs(got - R) > 0.5 * (want - R)  # the W^2 correction is really there


@pytest.mark.parametrize("R", [10.3, 25.0, 47.7])
def test_equimolar_radius_of_a_sharp_disk(R):
    n = int(2 * R) + 12
    y, x = np.mgrid[0:n, 0:n].astype(np.float64)
    inside = np.hypot(x - (n - 1) / 2, y - (n - 1) / 2) < R
    rho = np.where(inside, RL, RV)
    got = OO.equimolar_radius(rho, RL, RV)
    assert got == pytest.approx(math.sqrt(inside.sum() / math.pi), rel=1e-14)
    # Gauss circle problem: |N(R) - pi R^2| stays well below 2 pi R (perimeter) here
    assert abs(inside.sum() - math.pi * R * R) < 2 * math.pi * R
    assert abs(got - R) < 1.0


def test_probes_cancel_period_two_modes():
    nx, ny = 64, 48
    rng = np.random.default_rng(3)
    y, x = np.mgrid[0:ny, 0:nx]
    base_flat = _slab(nx, ny, 5.0, nx // 4, 3 * nx // 4)
    ref_flat = OO.probes(base_flat, 0)
    r = np.hypot(x - (nx - 1) / 2, y - (ny - 1) / 2)
    base_drop = 0.5 * (RL + RV) - 0.5 * (RL - RV) * np.tanh(2 * (r - 15.0) / 5.0)
    ref_drop = OO.probes(base_drop, 1)
    for mode in ((-1.0) ** x, (-1.0) ** y, (-1.0) ** (x + y)):
        amp = rng.uniform(1e-4, 1e-3)
        got_flat = OO.probes(base_flat + amp * mode, 0)
        got_drop = OO.probes(base_drop + amp * mode, 1)
        for g, want in zip(got_flat + got_drop, ref_flat + ref_drop):
            assert abs(g - want) < 1e-15
    # the probes are where the readings say: liquid columns nx/2-1, nx/2 of a slab, 4x4 blocks
    planted = np.full((ny, nx), RV)
    planted[:, nx // 2 - 1:nx // 2 + 1] = RL
    assert OO.probes(planted, 0) == (pytest.approx(RL), pytest.approx(RV))
    planted = np.full((ny, nx), RL)
    for sl in (np.s_[:4, :4], np.s_[:4, -4:], np.s_[-4:, :4], np.s_[-4:, -4:]):
        planted[sl] = RV
    assert OO.probes(planted, 1) == (pytest.approx(RL), pytest.approx(RV))


def test_pressure_jump_is_the_eos_at_the_probes():
    a, b, R, Tr = 0.25, 4.0, 1.0, 0.8
    T = thermo.temperature(a, b, R, Tr)
    rho = _slab(128, 2, 5.0, 32, 96) * 1.01
    rl, rv = OO.probes(rho, 0)
    obs = OO.observables(rho, np.zeros_like(rho), np.zeros_like(rho), 0, a, b, R, T)
    eta_l, eta_v = b * rl / 4, b * rv / 4
    cs = lambda r, e: r * R * T * (1 + e + e * e - e**3) / (1 - e) ** 3 - a * r * r  # Eq. (28)
    assert obs["dp"] == pytest.approx(cs(rl, eta_l) - cs(rv, eta_v), rel=1e-13)
    assert obs["mass"] == pytest.approx(rho.sum(), rel=1e-15)
