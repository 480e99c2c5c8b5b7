"""Laplace law on the C2 droplet configuration (256^2, R = 20, 30, 40, 60, 2e4 steps, tau = 1,
a = 0.25, Tr = 0.8) in FP64 on the GPU, whose step equals the FP64 oracle to 1e-11 (the
parity tests): the pressure jump is linear in the inverse equimolar radius through about
zero (Eq. S18 in 2-D) with the surface tension of the planar profile of Eq. (26) (Eq. 25),
for the free-energy model and for the pseudopotential model with kappa_P, kappa_Li matched
to that width and surface tension (Sec. 3, Eqs. S44, S46); the R = 20 droplets' vapour
densities against the Kelvin value printed in Sec. 5.3 (reduced 0.1824)."""
import numpy as np
import pytest

from oracle import thermo
from paper_2403_11167_gb300 import inputs

pytestmark = pytest.mark.gpu

A, TR, KAPPA, L, STEPS = 0.25, 0.8, 0.5, 256, 20000
RADII = (20.0, 30.0, 40.0, 60.0)


@pytest.fixture(scope="module")
def lbm():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2403_11167_gb300 import lbm as L_

    return L_


def _droplets(lbm, model, **kw):
    out = []
    for R in RADII:
        p = lbm.lbm_params_default(model, precision=lbm.LBM_F64, a=A, Tr=TR, tau_nu=1.0, **kw)
        ctx = lbm.Context(p, L, L)
        _, th = ctx.derived()
        ctx.set_density(inputs.droplet(L, L, R, th.rho_v, th.rho_l))
        ctx.step(STEPS)
        out.append(ctx.observables(lbm.DROPLET))
        ctx.close()
    return out, th


def _fit(obs):
    inv = np.array([1.0 / o["radius"] for o in obs])
    dp = np.array([o["dp"] for o in obs])
    A_ = np.column_stack([inv, np.ones_like(inv)])
    (slope, icpt), *_ = np.linalg.lstsq(A_, dp, rcond=None)
    resid = dp - A_ @ np.array([slope, icpt])
    return slope, icpt, dp, resid


def test_fe_laplace_law_per_droplet(lbm):
    """Delta p * R_equimolar / gamma_planar = 1 within 1% for R >= 30 and within 3% at R = 20
    (a curvature correction of order W / R, W ~ 4.5; measured 0.974); the jump falls
    monotonically with R; the straight-line fit through all four points, which that correction
    pulls down, stays within 5%."""
    obs, th = _droplets(lbm, lbm.LBM_FREE_ENERGY, kappa=KAPPA)
    assert all(o["status"] == lbm.LBM_OK for o in obs)
    gamma = thermo.fe_surface_tension(A, 4.0, 1.0, TR, KAPPA)
    law = [o["dp"] * o["radius"] / gamma for o in obs]
    assert abs(law[0] - 1) < 0.03, law
    assert all(abs(x - 1) < 0.01 for x in law[1:]), law
    slope, icpt, dp, resid = _fit(obs)
    assert np.all(np.diff(dp) < 0)
    assert abs(slope / gamma - 1) < 0.05, slope / gamma
    # T16 (Sec. 5.3): vapour density of the R = 20 droplet against the printed Kelvin value
    rho_c = thermo.critical_point(A, 4.0, 1.0)[0]
    assert abs(obs[0]["rho_v"] / rho_c / 0.1824 - 1) < 0.01, obs[0]["rho_v"] / rho_c


def test_pp_matched_laplace_law_and_vapour_density(lbm):
    """Pseudopotential model with kappa_P, kappa_Li matched to the free-energy width and
    surface tension: Delta p * R / gamma_FE = 1 within 3% for every droplet; the R = 20 vapour
    density within 2.5% of the printed Kelvin value 0.1824 (measured 0.1858; the paper's own
    run, whose parameters are not all printed, gave 0.1786)."""
    obs, th = _droplets(lbm, lbm.LBM_PSEUDOPOTENTIAL, match_kappa=KAPPA)
    assert all(o["status"] == lbm.LBM_OK for o in obs)
    gamma = thermo.fe_surface_tension(A, 4.0, 1.0, TR, KAPPA)
    law = [o["dp"] * o["radius"] / gamma for o in obs]
    assert all(abs(x - 1) < 0.03 for x in law), law
    rho_c = thermo.critical_point(A, 4.0, 1.0)[0]
    assert abs(obs[0]["rho_v"] / rho_c / 0.1824 - 1) < 0.025, obs[0]["rho_v"] / rho_c
