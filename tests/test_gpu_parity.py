"""GPU parity: the sm_103a kernels (through the C ABI) against the FP64 oracle.

Metric: densities cell by cell, max |rho_gpu - rho_oracle| / rho_oracle (helpers.rho_err);
populations relative to their own cell's density (helpers.pop_err).  Tolerances: FP64 runs
agree to rounding (1e-11 on populations after tens of steps) and meet the stated static bar
(1e-5 after 1e4 steps) by orders of magnitude.  FP32 runs meet both stated bars as written:
1e-5 on static droplets and slabs after 1e4 steps, and 1e-4 over the first 200 steps of a
spinodal run (also at the benchmark's 4096^2 size).  What makes FP32 reach the static bar is
the arithmetic of lbm_kernels.cuh: mirror-equivariant sums (no rigid drift of a symmetric
state), scale-exact c_s^2 and stencil weights (no spurious EOS term in the pseudopotential
model) and the compensated rest population of the free-energy model (no mass random walk).
"""
import os
import tempfile

import numpy as np
import pytest

import oracle as O
from oracle import observables as OO
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


def _oracle_run(model, rp, th, rho0, steps):
    return O.run(model, oracle_params(rp, th), O.init(model, rho0), steps)


@pytest.mark.parametrize("model", [PP, FE])
@pytest.mark.parametrize("shape", [(8, 8), (37, 29), (130, 7), (257, 3), (1, 17), (150, 1), (300, 130)])
def test_fp64_random_fields(model, shape):
    """Random densities on ragged lattices (partial tiles, 1-wide, many tiles): every population
    after 25 steps, with a body force and non-default width/tension parameters."""
    nx, ny = shape
    ctx, rp, th = gpu_context(model, F64, nx, ny, a=0.5, Tr=0.8, tau_nu=0.9, tau_e=0.85, tau_zeta=1.1,
                              kappa_P=0.7, kappa_Li=-0.4, body_fx=1e-5, body_fy=-2e-5)
    rho0 = inputs.random_field(nx, ny, th.rho_v * 3.0, th.rho_l * 0.6, seed=nx * 1000 + ny)
    ctx.set_density(rho0)
    ctx.step(25)
    f_ref = _oracle_run(model, rp, th, rho0, 25)
    assert pop_err(ctx.populations(), f_ref) < 1e-11


@pytest.mark.parametrize("model", [PP, FE])
def test_fp32_random_fields(model):
    nx, ny = 203, 77
    ctx, rp, th = gpu_context(model, F32, nx, ny, a=0.5, Tr=0.85, tau_nu=0.8)
    rho0 = inputs.random_field(nx, ny, th.rho_v * 3.0, th.rho_l * 0.6, seed=5)
    ctx.set_density(rho0)
    ctx.step(20)
    f_ref = _oracle_run(model, rp, th, rho0, 20)
    rho_gpu = ctx.populations().sum(0)
    assert rho_err(rho_gpu, f_ref.sum(0)) < 1e-5


def test_flat_interface_fp64_config():
    """256 x 4 flat interface, Carnahan-Starling a = 0.5, Tr = 0.8, tau = 1, 1e4 steps, FP64:
    rho_l, rho_v and width against the oracle."""
    nx, ny, steps = 256, 4, 10000
    ctx, rp, th = gpu_context(PP, F64, nx, ny, a=0.5, Tr=0.8, tau_nu=1.0)
    rho0 = inputs.flat_slab(nx, ny, th.rho_v, th.rho_l)
    ctx.set_density(rho0)
    ctx.step(steps)
    obs = ctx.observables(0)
    f_ref = _oracle_run(PP, rp, th, rho0, steps)
    rho_ref, ux_ref, uy_ref, *_ = O.macro(PP, oracle_params(rp, th), f_ref)
    rho_gpu, ux_gpu, uy_gpu = ctx.fields()
    assert rho_err(rho_gpu, rho_ref) < 1e-10  # FP64 rounding order only (measured 1.5e-11)
    ref = OO.observables(rho_ref, ux_ref, uy_ref, 0, rp.a, rp.b, rp.R, th.T)
    for k in ("rho_l", "rho_v", "width", "dp", "mass"):
        assert abs(obs[k] / ref[k] - 1) < 1e-9, k
    assert abs(obs["u_max"] - ref["u_max"]) < 1e-12
    assert obs["status"] == 0 and obs["step"] == steps


@pytest.mark.parametrize("precision", [F64, F32])
@pytest.mark.parametrize("model", [PP, FE])
def test_static_droplet_1e4_steps(model, precision):
    """Static droplet (ragged 130 x 126 lattice, R = 25, Tr 0.8, a = 0.25, P parameters matched
    to FE kappa = 0.5), 1e4 steps: density cell by cell within 1e-5 of the oracle (the stated
    static bar; FP64 meets it by orders of magnitude), the pair-averaged probe densities and
    the equimolar radius within 1e-5, and the pressure jump of the Laplace test relative to
    itself."""
    nx, ny, steps = 130, 126, 10000
    kw = dict(a=0.25, Tr=0.8, tau_nu=1.0)
    if model == PP:
        kw["match_kappa"] = 0.5
    ctx, rp, th = gpu_context(model, precision, nx, ny, **kw)
    rho0 = inputs.droplet(nx, ny, 25.0, th.rho_v, th.rho_l)
    ctx.set_density(rho0)
    ctx.step(steps)
    rho_gpu, ux_gpu, uy_gpu = ctx.fields()
    f_ref = _oracle_run(model, rp, th, rho0, steps)
    rho_ref, ux_ref, uy_ref, *_ = O.macro(model, oracle_params(rp, th), f_ref)
    err = rho_err(rho_gpu, rho_ref)
    assert err < (1e-9 if precision == F64 else 1e-5), err
    obs = ctx.observables(1)
    ref = OO.observables(rho_ref, ux_ref, uy_ref, 1, rp.a, rp.b, rp.R, th.T)
    for k in ("rho_l", "rho_v", "radius"):
        assert abs(obs[k] / ref[k] - 1) < (1e-9 if precision == F64 else 1e-5), k
    # dp = p(rho_l) - p(rho_v) (Sec. 5.2) relative to itself: 1e-9 in FP64; in FP32 the probe
    # densities carry the FP32 rounding of the stored state (~6e-8) and the EOS slope
    # p'(rho_l) rho_l / dp ~ 200 at R = 25 amplifies it, so the bar is 1e-3 of dp -- the
    # accuracy to which the Laplace slope is read
    assert abs(obs["dp"] / ref["dp"] - 1) < (1e-9 if precision == F64 else 1e-3), (obs["dp"], ref["dp"])


@pytest.mark.parametrize("model", [PP, FE])
def test_spinodal_fp32_first_200_steps(model):
    """Spinodal decomposition (Tr 0.85, a 0.25, tau 0.8, rho = (rho_l+rho_v)/2 (1 + U(-0.01, 0.01))),
    ragged 300 x 200 lattice, FP32: max relative density error over the first 200 steps <= 1e-4."""
    nx, ny = 300, 200
    ctx, rp, th = gpu_context(model, F32, nx, ny, a=0.25, Tr=0.85, tau_nu=0.8)
    rho0 = inputs.spinodal_noise(nx, ny, 0.5 * (th.rho_l + th.rho_v), 0.01, seed=2403)
    ctx.set_density(rho0)
    op = oracle_params(rp, th)
    f = O.init(model, rho0)
    worst = 0.0
    for chunk in range(4):
        ctx.step(50)
        f = O.run(model, op, f, 50)
        worst = max(worst, rho_err(ctx.fields()[0], O.macro(model, op, f)[0]))
    assert worst < 1e-4


@pytest.mark.parametrize("model", [PP, FE])
def test_full_size_4096_sampled(model):
    """The benchmark's 4096^2 spinodal lattice and launch configuration: 16 FP32 steps, populations
    at 6 sampled cells against the oracle run on the periodic crop that holds each cell's domain
    of dependence (radius 2 cells per step for P, 3 for FE; a margin makes the crop exact)."""
    nx = ny = 4096
    steps = 16
    ctx, rp, th = gpu_context(model, F32, nx, ny, a=0.25, Tr=0.85, tau_nu=0.8)
    rho0 = inputs.spinodal_noise(nx, ny, 0.5 * (th.rho_l + th.rho_v), 0.01, seed=2403)
    ctx.set_density(rho0)
    ctx.step(steps)
    pts = [(0, 0), (4095, 4095), (127, 128), (2048, 1), (3000, 4000), (129, 2047)]
    got = ctx.populations_at([p[0] for p in pts], [p[1] for p in pts])
    h = (2 if model == PP else 3) * steps + 2
    op = oracle_params(rp, th)
    for k, (x, y) in enumerate(pts):
        ys = np.arange(y - h, y + h + 1) % ny
        xs = np.arange(x - h, x + h + 1) % nx
        crop = rho0[np.ix_(ys, xs)]
        fc = O.run(model, op, O.init(model, crop), steps)
        ref = fc[:, h, h]
        assert abs(got[k].sum() / ref.sum() - 1) < 1e-5, (x, y)
        assert np.abs(got[k] - ref).max() / ref.sum() < 1e-5, (x, y)
    ctx.close()


@pytest.mark.parametrize("model", [PP, FE])
def test_full_size_4096_sampled_200_steps(model):
    """The chaotic-run bar at the benchmark's size: the 4096^2 spinodal lattice in the
    benchmark's launch configuration, 200 FP32 steps, populations at 3 sampled cells against
    the oracle on each cell's periodic domain-of-dependence crop (805^2 for P, 1205^2 for FE);
    relative density error of each sampled cell <= 1e-4 (and each population relative to it)."""
    nx = ny = 4096
    steps = 200
    ctx, rp, th = gpu_context(model, F32, nx, ny, a=0.25, Tr=0.85, tau_nu=0.8)
    rho0 = inputs.spinodal_noise(nx, ny, 0.5 * (th.rho_l + th.rho_v), 0.01, seed=2403)
    ctx.set_density(rho0)
    ctx.step(steps)
    pts = [(0, 0), (2047, 3001), (4095, 1234)]
    got = ctx.populations_at([p[0] for p in pts], [p[1] for p in pts])
    h = (2 if model == PP else 3) * steps + 2
    op = oracle_params(rp, th)
    for k, (x, y) in enumerate(pts):
        ys = np.arange(y - h, y + h + 1) % ny
        xs = np.arange(x - h, x + h + 1) % nx
        fc = O.run(model, op, O.init(model, rho0[np.ix_(ys, xs)]), steps)
        ref = fc[:, h, h]
        assert abs(got[k].sum() / ref.sum() - 1) < 1e-4, (x, y)  # the cell's density
        assert np.abs(got[k] - ref).max() / ref.sum() < 1e-4, (x, y)  # each population
    ctx.close()


@pytest.mark.parametrize("model", [PP, FE])
def test_mass_conservation_fp64(model):
    nx, ny = 96, 80
    ctx, rp, th = gpu_context(model, F64, nx, ny, a=0.25, Tr=0.7, tau_nu=1.0)
    rho0 = inputs.droplet(nx, ny, 20.0, th.rho_v, th.rho_l)
    ctx.set_density(rho0)
    ctx.step(3000)
    obs = ctx.observables(1)
    assert abs(obs["mass"] / rho0.sum() - 1) < 3000 * 1e-15


@pytest.mark.parametrize("model", [PP, FE])
def test_graph_replay_equals_single_launches(model):
    """lbm_step(n) replays captured 64-step graphs; n single-step calls launch one kernel each.
    Same kernels, same order: bitwise equal."""
    nx, ny = 64, 48
    a, rp, th = gpu_context(model, F32, nx, ny, Tr=0.8)
    b, _, _ = gpu_context(model, F32, nx, ny, Tr=0.8)
    rho0 = inputs.droplet(nx, ny, 12.0, th.rho_v, th.rho_l)
    a.set_density(rho0)
    b.set_density(rho0)
    a.step(131)
    for _ in range(131):
        b.step(1)
    assert np.array_equal(a.populations(), b.populations())


@pytest.mark.parametrize("model,nx", [(PP, 70), (FE, 70), (FE, 72)])
def test_checkpoint_roundtrip(model, nx):
    """n + m steps equal n steps, save, load into a fresh context, m steps (bitwise; for the
    FP32 free-energy model this includes the rest population's extension, on the direct kernel
    (nx = 70) and on the strip kernel (nx = 72))."""
    ny = 50
    a, rp, th = gpu_context(model, F32, nx, ny, Tr=0.8)
    rho0 = inputs.droplet(nx, ny, 15.0, th.rho_v, th.rho_l)
    a.set_density(rho0)
    a.step(150)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "ck.bin")
        a.save(path)
        a.step(77)
        b, _, _ = gpu_context(model, F32, nx, ny, Tr=0.8)
        b.load(path)
        assert b.observables(1)["step"] == 150
        b.step(77)
    assert np.array_equal(a.populations(), b.populations())


def test_checkpoint_rejects_other_parameters():
    """A checkpoint continues the run it came from: loading it into a context of another
    temperature (or any other resolved parameter) is an argument error, and the context keeps
    its own state."""
    from paper_2403_11167_gb300 import lbm

    nx, ny = 40, 24
    a, rp, th = gpu_context(FE, F32, nx, ny, Tr=0.8)
    a.set_density(inputs.droplet(nx, ny, 8.0, th.rho_v, th.rho_l))
    a.step(10)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "ck.bin")
        a.save(path)
        for kw in (dict(Tr=0.75), dict(Tr=0.8, kappa=0.6), dict(Tr=0.8, tau_nu=0.9)):
            b, _, th_b = gpu_context(FE, F32, nx, ny, **kw)
            b.set_density(inputs.droplet(nx, ny, 8.0, th_b.rho_v, th_b.rho_l))
            before = b.populations()
            with pytest.raises(lbm.LBMError) as e:
                b.load(path)
            assert e.value.code == lbm.LBM_ERR_ARG, kw
            assert np.array_equal(b.populations(), before)
            b.close()
        c, _, _ = gpu_context(FE, F32, nx, ny, Tr=0.8)
        c.load(path)
        assert np.array_equal(c.populations(), a.populations())


def test_set_get_populations_roundtrip():
    nx, ny = 33, 21
    ctx, rp, th = gpu_context(FE, F64, nx, ny)
    rng = np.random.default_rng(1)
    f = rng.uniform(0.001, 0.1, size=(9, ny, nx))
    ctx.set_populations(f)
    assert np.array_equal(ctx.populations(), f)


def test_divergence_is_reported_not_crashed():
    """A NaN injected on the host is caught by the observables check and reported as
    LBM_ERR_DIVERGED; later steps refuse to run.  No device fault involved."""
    from paper_2403_11167_gb300 import lbm

    nx, ny = 40, 30
    ctx, rp, th = gpu_context(PP, F32, nx, ny)
    f = O.init(PP, inputs.droplet(nx, ny, 8.0, th.rho_v, th.rho_l))
    f[3, 10, 10] = np.nan
    ctx.set_populations(f)
    ctx.step(5)
    obs = ctx.observables(1)
    assert obs["status"] == lbm.LBM_ERR_DIVERGED
    with pytest.raises(lbm.LBMError) as e:
        ctx.step(1)
    assert e.value.code == lbm.LBM_ERR_DIVERGED


@pytest.mark.parametrize("model", [PP, FE])
@pytest.mark.parametrize("shape", [(8, 4), (300, 200), (132, 7), (1024, 70), (244, 9), (484, 33), (4100, 6)])
def test_tma_pipeline_matches_direct_kernel(model, shape, monkeypatch):
    """The TMA-fed FP32 kernels (row pipeline through shared memory; for the pseudopotential
    model the warp-window kernel) and the direct-load kernels run the same per-cell
    arithmetic: on lattices with nx % 4 == 0 (single tile, ragged and uneven strips, thin
    strips, a 4-column last strip) their populations agree after 50 steps."""
    nx, ny = shape
    a, rp, th = gpu_context(model, F32, nx, ny, Tr=0.85, tau_nu=0.8)
    monkeypatch.setenv("LBM_NO_TMA", "1")
    b, _, _ = gpu_context(model, F32, nx, ny, Tr=0.85, tau_nu=0.8)
    rho0 = inputs.spinodal_noise(nx, ny, 0.5 * (th.rho_l + th.rho_v), 0.01, seed=7)
    a.set_density(rho0)
    b.set_density(rho0)
    a.step(50)
    b.step(50)
    fa, fb = a.populations(), b.populations()
    assert np.abs(fa - fb).max() <= 1e-7 * np.abs(fb).max()
    f_ref = _oracle_run(model, rp, th, rho0, 50)
    assert rho_err(fa.sum(0), f_ref.sum(0)) < 1e-5
