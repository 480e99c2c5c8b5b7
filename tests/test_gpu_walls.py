"""GPU parity of the walled channel (no-slip walls on rows 0 and ny-1, Zou-He, body force):
the sm_103a wall kernels through the C ABI against the FP64 oracle, and the two-phase flow
between parallel plates of Sec. 5.3 against the analytic profile of Eq. (89)."""
import numpy as np
import pytest

import oracle as O
from oracle import plate
from paper_2403_11167_gb300 import inputs
from helpers import gpu_context, oracle_params, pop_err, rho_err

pytestmark = pytest.mark.gpu

PP, FE = 0, 1
F32, F64 = 0, 1


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    assert torch.cuda.is_available()


def _oracle(model, rp, th, rho0, steps):
    p = oracle_params(rp, th, walls=True)
    f = O.run(model, p, O.init(model, rho0), steps)
    return f, O.macro(model, p, f)


@pytest.mark.parametrize("model", [PP, FE])
@pytest.mark.parametrize("shape,kind", [((8, 4), "random"), ((37, 9), "random"), ((70, 42), "channel"),
                                        ((130, 23), "channel")])
def test_fp64_walls_against_oracle(model, shape, kind):
    """Every population (wall nodes completed) and the fields after 40 steps: random densities
    on tiny lattices (the minimum 4 rows: two walls, two fluid rows) and a channel whose
    interface is a sine wave (x-gradients at the walls), ragged in x and y, with a body force
    in both directions and non-default relaxation times."""
    nx, ny = shape
    ctx, rp, th = gpu_context(model, F64, nx, ny, walls=True, a=0.25, Tr=0.8, tau_nu=0.9, tau_e=0.95,
                              kappa_P=0.7, body_fx=1e-5, body_fy=-2e-6)
    if kind == "random":
        rho0 = inputs.random_field(nx, ny, th.rho_v * 3.0, th.rho_l * 0.6, seed=nx + 7 * ny)
    else:
        rho0 = inputs.plate_channel(nx, ny, th.rho_v, th.rho_l, amp=3.0)
    ctx.set_density(rho0)
    ctx.step(40)
    f_ref, (rho_ref, ux_ref, uy_ref, *_) = _oracle(model, rp, th, rho0, 40)
    assert pop_err(ctx.populations(), f_ref) < 1e-11
    rho, ux, uy = ctx.fields()
    assert rho_err(rho, rho_ref) < 1e-12
    umax = max(np.abs(ux_ref).max(), np.abs(uy_ref).max())
    assert np.abs(ux - ux_ref).max() < 1e-9 * umax and np.abs(uy - uy_ref).max() < 1e-9 * umax
    # no slip: u = 0 at the wall nodes (J = -F/2)
    assert np.abs(ux[[0, -1]]).max() < 1e-14 and np.abs(uy[[0, -1]]).max() < 1e-14


@pytest.mark.parametrize("model", [PP, FE])
def test_fp32_walls_against_oracle(model):
    """FP32 channel (203 x 61, sine interface, body force), 200 steps: densities within 1e-5
    relative, velocities within 5e-5 of the largest speed (measured 2.3e-6 and 5.5e-6)."""
    nx, ny, steps = 203, 61, 200
    ctx, rp, th = gpu_context(model, F32, nx, ny, walls=True, a=0.25, Tr=0.8, tau_nu=1.0, body_fx=1e-5)
    rho0 = inputs.plate_channel(nx, ny, th.rho_v, th.rho_l, amp=2.0)
    ctx.set_density(rho0)
    ctx.step(steps)
    _, (rho_ref, ux_ref, uy_ref, *_) = _oracle(model, rp, th, rho0, steps)
    rho, ux, uy = ctx.fields()
    umax = max(np.abs(ux_ref).max(), np.abs(uy_ref).max())
    print("fp32 walls", model, rho_err(rho, rho_ref), np.abs(ux - ux_ref).max() / umax,
          np.abs(uy - uy_ref).max() / umax)
    assert rho_err(rho, rho_ref) < 1e-5
    assert np.abs(ux - ux_ref).max() < 5e-5 * umax and np.abs(uy - uy_ref).max() < 5e-5 * umax


@pytest.mark.parametrize("model", [PP, FE])
@pytest.mark.parametrize("shape", [(8, 6), (204, 61), (484, 33), (1024, 77)])
def test_fp32_wall_routes_agree(model, shape, monkeypatch):
    """FP32 lattices with nx % 4 == 0 and ny >= 6 run the periodic strip kernel over the whole
    lattice and then recompute the rows next to each wall with the wall kernel; the direct wall
    kernel alone (LBM_NO_TMA) runs the same per-cell arithmetic.  After 50 steps of a sine-
    perturbed channel with a body force both agree (minimum height, ragged strips), and the
    densities match the oracle."""
    nx, ny = shape
    kw = dict(a=0.25, Tr=0.8, tau_nu=0.9, body_fx=1e-5, body_fy=-2e-6)
    a, rp, th = gpu_context(model, F32, nx, ny, walls=True, **kw)
    monkeypatch.setenv("LBM_NO_TMA", "1")
    b, _, _ = gpu_context(model, F32, nx, ny, walls=True, **kw)
    rho0 = inputs.plate_channel(nx, ny, th.rho_v, th.rho_l, amp=min(3.0, ny / 8))
    a.set_density(rho0)
    b.set_density(rho0)
    a.step(50)
    b.step(50)
    fa, fb = a.populations(), b.populations()
    assert np.abs(fa - fb).max() <= 1e-7 * np.abs(fb).max()
    _, (rho_ref, *_rest) = _oracle(model, rp, th, rho0, 50)
    assert rho_err(fa.sum(0), rho_ref) < 1e-5


@pytest.mark.parametrize("precision,tol", [(F64, 1e-9), (F32, 2e-3)])
@pytest.mark.parametrize("model", [PP, FE])
def test_single_phase_poiseuille(model, precision, tol):
    """Uniform liquid between the plates (H = 20, F_x = 1e-6): the steady profile is the parabola
    F y (H - y)/(2 mu), mu = rho c_s^2 (tau - 1/2); zero velocity at the wall nodes."""
    nx, ny, fx = 16, 21, 1e-6
    ctx, rp, th = gpu_context(model, precision, nx, ny, walls=True, a=0.25, Tr=0.8, tau_nu=1.0, tau_e=1.0,
                              body_fx=fx)
    ctx.set_density(np.full((ny, nx), th.rho_l))
    ctx.step(40000)
    rho, ux, uy = ctx.fields()
    y = np.arange(ny)
    ua = fx * y * (ny - 1 - y) / (2 * plate.viscosity(th.rho_l, 1.0))
    err = np.abs(ux - ua[:, None]).max() / ua.max()
    print("poiseuille", model, precision, err)
    assert err < tol
    assert np.abs(uy).max() < tol * ua.max()


# Sec. 5.3: the body force of each reduced temperature
PLATE_FX = {0.8: 1e-6, 0.7: 5e-7, 0.6: 2e-7}


def _plate_flow(model, Tr, steps):
    nx, ny = 101, 50
    kw = dict(a=0.25, Tr=Tr, tau_nu=1.0, tau_e=1.0, body_fx=PLATE_FX[Tr])
    if model == PP:
        kw["match_kappa"] = 0.5  # P matched to the FE interface width and tension (Sec. 5.3)
    else:
        kw["kappa"] = 0.5
    ctx, rp, th = gpu_context(model, F64, nx, ny, walls=True, **kw)
    ctx.set_density(inputs.plate_channel(nx, ny, th.rho_v, th.rho_l))
    ctx.step(steps)
    rho, ux, uy = ctx.fields()
    return rho, ux, uy, th


@pytest.mark.parametrize("model", [PP, FE])
@pytest.mark.parametrize("Tr", [0.8, 0.7, 0.6])
def test_plate_flow_sec53_against_eq89(model, Tr):
    """101 x 50 channel of Sec. 5.3 (a = 0.25, vapour below, liquid above, F_x by temperature,
    tau_nu = tau_e = 1; FE kappa = 0.5, P matched to it), 2e5 steps in FP64: the velocity
    profile against Eq. (89) integrated with the run's own density profile (plates on the wall
    rows, H = 49).  Prints the deviation from the discrete-interface solution, Eq. (88), too."""
    rho, ux, uy, th = _plate_flow(model, Tr, 200000)
    fx = PLATE_FX[Tr]
    col = rho[:, 0]
    y = np.arange(len(col), dtype=float)
    ua = plate.s89(y, plate.viscosity(col, 1.0), fx)
    err = np.abs(ux[:, 0] - ua).max() / ua.max()
    mu_v, mu_l = plate.viscosity(th.rho_v, 1.0), plate.viscosity(th.rho_l, 1.0)
    ud = plate.s88(y, y[-1], mu_v, mu_l, fx)
    err88 = np.abs(ux[:, 0] - ud).max() / ud.max()
    from oracle import thermo

    if model == FE:
        r, s = thermo.fe_profile_slope(0.25, 4.0, 1.0, Tr, 0.5)
    else:
        m = thermo.match_pp_to_fe(0.25, 4.0, 1.0, Tr, 0.5)
        r, s = thermo.pp_profile_slope(0.25, 4.0, 1.0, Tr, m["kappa_P"], m["eps"])
    rho_th = plate.theory_rho(y, plate.mid_crossing(col), r, s)
    ut = plate.s89(y, plate.viscosity(rho_th, 1.0), fx)
    err_th = np.abs(ux[:, 0] - ut).max() / ut.max()
    print(f"plate flow model={model} Tr={Tr}: Eq.89 (own rho) {err:.4f}  Eq.89 (Appendix A rho) {err_th:.4f}  "
          f"Eq.88 {err88:.4f}  rho_v {col[0] / th.rho_v - 1:+.4f}  u_max {ux.max():.4e}")
    assert np.abs(ux - ux[:, :1]).max() < 1e-9 * ua.max()  # uniform in x
    assert err < PLATE_TOL[(model, Tr)]


# measured deviation from Eq. (89) with the run's own density profile, with a margin:
# P 0.72%, 1.54%, 1.74%; FE 3.49%, 10.1%, 15.1% at Tr 0.8, 0.7, 0.6.  FE's deviation sits in the
# vapour next to the interface and grows as the density ratio grows; the paper also reports
# FE's flow errors growing at low temperature (Sec. 5.3)
PLATE_TOL = {(PP, 0.8): 0.012, (PP, 0.7): 0.025, (PP, 0.6): 0.03, (FE, 0.8): 0.05, (FE, 0.7): 0.13, (FE, 0.6): 0.2}


ONESIDED = 2  # LBM_BC_WALL_ZOUHE_ONESIDED


@pytest.mark.parametrize("shape,kind", [((8, 4), "random"), ((70, 42), "channel")])
def test_fp64_onesided_walls_against_oracle(shape, kind):
    """Free-energy walls with the one-sided wall-normal chemical-potential gradient and the
    self-consistent wall density (GPU: a per-step fixed-point sweep over each wall row), with a
    body force along both axes: every population and the fields after 40 steps."""
    nx, ny = shape
    ctx, rp, th = gpu_context(FE, F64, nx, ny, walls=ONESIDED, a=0.25, Tr=0.8, tau_nu=0.9, tau_e=0.95,
                              body_fx=1e-5, body_fy=-2e-6)
    if kind == "random":
        rho0 = inputs.random_field(nx, ny, th.rho_v * 3.0, th.rho_l * 0.6, seed=nx + 7 * ny)
    else:
        rho0 = inputs.plate_channel(nx, ny, th.rho_v, th.rho_l, amp=3.0)
    ctx.set_density(rho0)
    ctx.step(40)
    p = oracle_params(rp, th, walls=ONESIDED)
    f_ref = O.run(FE, p, O.init(FE, rho0), 40)
    assert pop_err(ctx.populations(), f_ref) < 1e-11
    rho_ref, ux_ref, uy_ref, *_ = O.macro(FE, p, f_ref)
    rho, ux, uy = ctx.fields()
    assert rho_err(rho, rho_ref) < 1e-12
    umax = max(np.abs(ux_ref).max(), np.abs(uy_ref).max())
    assert np.abs(ux - ux_ref).max() < 1e-9 * umax and np.abs(uy - uy_ref).max() < 1e-9 * umax


@pytest.mark.parametrize("precision", [F64, F32])
def test_onesided_walls_hold_a_hydrostatic_column(precision):
    """A liquid column between walls under a wall-normal body force (fy = -1e-5, 40 rows),
    2e4 steps: with the one-sided reading the column is steady (density second differences
    below 1e-5 in the interior, velocity ~ 0), as in the oracle; the mirrored reading's
    free-energy period-2 mode grows instead (oracle test)."""
    nx, ny = 8, 40
    ctx, rp, th = gpu_context(FE, precision, nx, ny, walls=ONESIDED, a=0.25, Tr=0.8, tau_nu=1.0, tau_e=1.0,
                              body_fy=-1e-5)
    ctx.set_density(np.full((ny, nx), th.rho_l))
    ctx.step(8000)
    a8 = np.abs(np.diff(ctx.fields()[0][4:-4, 0], 2)).max()
    ctx.step(12000)
    rho, ux, uy = ctx.fields()
    a20 = np.abs(np.diff(rho[4:-4, 0], 2)).max()
    print("onesided column", precision, a8, a20, np.abs(uy).max())
    assert a20 < 1e-5 and abs(a20 - a8) < 0.05 * a8 + 1e-7
    assert np.abs(uy).max() < (1e-7 if precision == F64 else 1e-5)


@pytest.mark.parametrize("shape", [(8, 6), (204, 61)])
def test_fp32_onesided_wall_routes_agree(shape, monkeypatch):
    """FP32 one-sided free-energy walls: the strip kernel plus the wall bands (nx % 4 == 0,
    ny >= 6) against the direct wall kernel (LBM_NO_TMA) after 50 steps, and the oracle."""
    nx, ny = shape
    kw = dict(a=0.25, Tr=0.8, tau_nu=0.9, body_fx=1e-5, body_fy=-2e-6)
    a, rp, th = gpu_context(FE, F32, nx, ny, walls=ONESIDED, **kw)
    monkeypatch.setenv("LBM_NO_TMA", "1")
    b, _, _ = gpu_context(FE, F32, nx, ny, walls=ONESIDED, **kw)
    rho0 = inputs.plate_channel(nx, ny, th.rho_v, th.rho_l, amp=min(3.0, ny / 8))
    a.set_density(rho0)
    b.set_density(rho0)
    a.step(50)
    b.step(50)
    fa, fb = a.populations(), b.populations()
    assert np.abs(fa - fb).max() <= 1e-7 * np.abs(fb).max()
    p = oracle_params(rp, th, walls=ONESIDED)
    f_ref = O.run(FE, p, O.init(FE, rho0), 50)
    assert rho_err(fa.sum(0), f_ref.sum(0)) < 1e-5
