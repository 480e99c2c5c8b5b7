"""GPU parity of the droplet-collision drive (Sec. 5.4: F_x = a_x |rho - rho_ave| by side,
rho_ave reduced every step, switched on after t_on) against the FP64 oracle, and the
collision of Sec. 5.4 itself (merge times of both models)."""
import numpy as np
import pytest

import oracle as O
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


def _drive_params(rp, th, lo, hi, split):
    p = oracle_params(rp, th)
    p.drive_ax_lo, p.drive_ax_hi, p.drive_x_split = lo, hi, split
    return p


@pytest.mark.parametrize("model", [PP, FE])
@pytest.mark.parametrize("shape", [(80, 40), (70, 29)])
def test_fp64_drive_against_oracle(model, shape):
    """Two droplets driven together (a_x = +5e-4 left of the middle column, -3e-4 beyond),
    t_on = 10: 150 steps cross the switch-on (single launches, then graph replays of driven
    steps); every population and the velocity (which carries the drive) against the oracle."""
    nx, ny = shape
    ctx, rp, th = gpu_context(model, F64, nx, ny, a=0.25, Tr=0.8, tau_nu=1.0, **({"match_kappa": 0.5} if model == PP else {}))
    rho0 = inputs.two_droplets(nx, ny, [(nx / 4, ny / 2), (3 * nx / 4, ny / 2)], ny / 4, th.rho_v, th.rho_l)
    split = nx // 2
    ctx.set_density(rho0)
    ctx.set_drive(5e-4, -3e-4, split, 10)
    ctx.step(150)
    p = _drive_params(rp, th, 5e-4, -3e-4, split)
    f_ref = O.run_driven(model, p, O.init(model, rho0), 150, t0=0, t_on=10)
    assert pop_err(ctx.populations(), f_ref) < 1e-11
    p.drive = 1.0
    rho_ref, ux_ref, uy_ref, *_ = O.macro(model, p, f_ref)
    rho, ux, uy = ctx.fields()
    assert rho_err(rho, rho_ref) < 1e-12
    assert np.abs(ux - ux_ref).max() < 1e-9 * np.abs(ux_ref).max()
    assert np.abs(ux_ref).max() > 1e-4  # the drive moved the droplets


@pytest.mark.parametrize("model", [PP, FE])
def test_fp32_drive_against_oracle(model):
    """FP32, 200 x 100 pair of Sec. 5.4 with a 10x stronger drive switched on at t = 50,
    300 steps: densities within 1e-5 relative."""
    nx, ny = 200, 100
    ctx, rp, th = gpu_context(model, F32, nx, ny, a=0.25, Tr=0.8, tau_nu=1.0, **({"match_kappa": 0.5} if model == PP else {}))
    rho0 = inputs.two_droplets(nx, ny, [(50, 50), (150, 50)], 25.0, th.rho_v, th.rho_l)
    ctx.set_density(rho0)
    ctx.set_drive(5e-5, -5e-5, 100, 50)
    ctx.step(300)
    f_ref = O.run_driven(model, _drive_params(rp, th, 5e-5, -5e-5, 100), O.init(model, rho0), 300, t0=0, t_on=50)
    err = rho_err(ctx.populations().sum(0), f_ref.sum(0))
    print("fp32 drive", model, err)
    assert err < 1e-5


@pytest.mark.parametrize("model", [PP, FE])
def test_fp32_driven_strip_kernels_match_direct_kernels(model, monkeypatch):
    """The driven FP32 strip kernels against the driven direct kernels, both with the drive on
    from t = 0 on a 256 x 128 droplet pair for 200 steps.
    - Strip kernels: rho_ave from the masses the previous step stored. The block-sum reduction
      runs only at the first step of each 64-step graph and at single steps.
    - Direct kernels: the block-sum reduction every step.
    Both sum the same stored populations in different orders, so rho_ave differs by rounding
    and the populations agree to rounding, not bit for bit. Mass is conserved alike."""
    nx, ny = 256, 128
    kw = dict(a=0.25, Tr=0.8, tau_nu=1.0, **({"match_kappa": 0.5} if model == PP else {}))
    a, rp, th = gpu_context(model, F32, nx, ny, **kw)
    monkeypatch.setenv("LBM_NO_TMA", "1")
    b, _, _ = gpu_context(model, F32, nx, ny, **kw)
    rho0 = inputs.two_droplets(nx, ny, [(64, 64), (192, 64)], 30.0, th.rho_v, th.rho_l)
    m0 = None
    for ctx in (a, b):
        ctx.set_density(rho0)
        m0 = ctx.populations().sum()
        ctx.set_drive(5e-5, -5e-5, nx // 2, 0)
        ctx.step(200)
    fa, fb = a.populations(), b.populations()
    print("driven strip vs direct", model, pop_err(fa, fb), rho_err(fa.sum(0), fb.sum(0)))
    assert pop_err(fa, fb) < 1e-6
    assert rho_err(fa.sum(0), fb.sum(0)) < 1e-6
    # the drive moved the droplets: the comparison is not of two static states
    ux = a.fields()[1]
    assert np.abs(ux).max() > 1e-4
    for f in (fa, fb):
        assert abs(f.sum() / m0 - 1) < 1e-6
    a.close()
    b.close()


def _merge_time(model, precision=F64, every=10, t_max=9000):
    """Sec. 5.4: 200 x 100, a = 0.25, Tr = 0.8, droplets of diameter 50 at (50, 50) and
    (150, 50), a_x = +-5e-6 by side of x = 100, on after t = 2000; FE tau_e = 0.75, kappa = 0.5;
    P tau_nu = tau_e = 1, tau_q = 1/1.99, matched to FE.  Returns the first t (checked every
    `every` steps) at which the density along y = 50 stays above rho_m = (rho_v + rho_l)/2
    from one droplet centre to the other (the rho_m contours have joined)."""
    nx, ny = 200, 100
    kw = dict(a=0.25, Tr=0.8, tau_nu=1.0)
    kw.update({"match_kappa": 0.5, "tau_e": 1.0} if model == PP else {"tau_e": 0.75, "kappa": 0.5})
    ctx, rp, th = gpu_context(model, precision, nx, ny, **kw)
    ctx.set_density(inputs.two_droplets(nx, ny, [(50, 50), (150, 50)], 25.0, th.rho_v, th.rho_l))
    ctx.set_drive(5e-6, -5e-6, 100, 2000)
    rho_m = 0.5 * (th.rho_v + th.rho_l)
    ctx.step(4000)
    t = 4000
    while t < t_max:
        ctx.step(every)
        t += every
        rho, _, _ = ctx.fields()
        if rho[50, 50:151].min() > rho_m:
            return t
    return None


# Sec. 5.4: P had merged at t* = 1.935, FE only at t* = 1.961 (snapshots; both "almost" at 1.923)
PAPER_MERGE = {PP: 1.935, FE: 1.961}


def test_droplet_collision_sec54_merge_times():
    """Both models merge the droplets, P first, each within 6% of the paper's merge time
    (t* = t sqrt(a_d / D_d), a_d = 5e-6, D_d = 50).  Measured: P t* = 1.875, FE 2.033 (the
    paper reads its merge times off snapshots and gives neither its merge criterion nor the
    droplets' initial profile beyond "as the static droplet")."""
    scale = np.sqrt(5e-6 / 50.0)
    tp = _merge_time(PP)
    tf = _merge_time(FE)
    print(f"merge: P t={tp} t*={tp * scale if tp else None}  FE t={tf} t*={tf * scale if tf else None}")
    assert tp is not None and tf is not None
    assert tp < tf
    assert abs(tp * scale / PAPER_MERGE[PP] - 1) < 0.06 and abs(tf * scale / PAPER_MERGE[FE] - 1) < 0.06
