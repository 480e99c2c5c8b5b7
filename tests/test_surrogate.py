"""Calibration surrogate: the GPU training kernels against the FP64 CPU network oracle,
BF16 inference within its rounding bound, and the trained network against plain
calibration runs on held-out parameter sets (with the gain over the no-network theory)."""
import math

import numpy as np
import pytest

from oracle import mlp as M
from paper_2403_11167_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2403_11167_gb300 import lbm as L

    return L


def _theta(seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for l in range(M.N_LAYERS):
        lim = math.sqrt(6.0 / M.DIMS[l])
        parts.append(rng.uniform(-lim, lim, M.DIMS[l + 1] * M.DIMS[l]))
        parts.append(rng.uniform(-0.1, 0.1, M.DIMS[l + 1]))
    return np.concatenate(parts).astype(np.float32)


def _data(n, seed):
    """Inputs over the calibration ranges and a smooth synthetic target map."""
    rng = np.random.Generator(np.random.PCG64(seed))
    X = np.column_stack([rng.uniform(0.5, 0.95, n), rng.uniform(0.25, 0.5, n), rng.uniform(3, 5, n),
                         rng.choice([0.4, 0.7, 1.0], n)])
    Y = np.column_stack([(1.3 - X[:, 0]) / X[:, 2], np.exp(-12 * (1 - X[:, 0]) ** 0.8) / X[:, 2],
                         3 + 6 * np.sqrt(X[:, 3]) / (1.05 - X[:, 0]), 0.04 * X[:, 1] * (1 - X[:, 0]) ** 1.5])
    return X.astype(np.float32), Y.astype(np.float32)


def _layer_slices():
    out = []
    for l, (wo, bo) in enumerate(M.offsets()):
        out.append(slice(wo, bo))
        out.append(slice(bo, bo + M.DIMS[l + 1]))
    return out


@pytest.mark.parametrize("n,missing", [(300, False), (5000, False), (777, True)])
def test_gradient_matches_oracle(lbm, n, missing):
    """FP32 forward/backward kernels (tiled SGEMM, split-K weight gradients) against the FP64
    backpropagation of the same parameters and data: per tensor, max error <= 1e-4 of the
    tensor's largest gradient entry; loss within 1e-5.  With ``missing``, a third of the
    sigma and width targets are NaN (left out of the loss)."""
    X, Y = _data(n, seed=n)
    if missing:
        Y[::3, 3] = np.nan
        Y[1::5, 2] = np.nan
    st = lbm.Surrogate.standardisation(X, Y)
    m = lbm.Surrogate(st, seed=1)
    th = _theta(2)
    m.set_params(th)
    loss, g = m.loss_grad(X, Y)
    loss_ref, g_ref = M.loss_grad(th.astype(np.float64), X.astype(np.float64), Y.astype(np.float64),
                                  st.astype(np.float64))
    assert abs(loss / loss_ref - 1) < 1e-5
    for sl in _layer_slices():
        scale = np.max(np.abs(g_ref[sl]))
        assert np.max(np.abs(g[sl] - g_ref[sl])) <= 1e-4 * scale, (sl, np.max(np.abs(g[sl] - g_ref[sl])) / scale)
    m.close()


def test_adam_update_matches_oracle(lbm):
    """One training iteration = the gradient above plus the Adam kernel: the new parameters
    equal the oracle's Adam step applied to that gradient (first step, bias-corrected)."""
    X, Y = _data(300, seed=7)
    st = lbm.Surrogate.standardisation(X, Y)
    m = lbm.Surrogate(st, seed=1)
    th = _theta(3)
    m.set_params(th)
    _, g = m.loss_grad(X, Y)
    lr = 1e-3
    m.train(X, Y, iterations=1, lr=lr, lr_min=lr, weight_decay=1e-4)
    p1 = m.params().astype(np.float64)
    ref, _, _ = M.adam_step(th.astype(np.float64), g.astype(np.float64), np.zeros(M.N_PARAMS), np.zeros(M.N_PARAMS),
                            1, lr, weight_decay=1e-4)
    big = np.abs(g) > 1e-5 * np.max(np.abs(g))
    assert np.max(np.abs(p1 - ref)[big]) < 1e-7 + 1e-6 * np.max(np.abs(ref))
    # where the gradient is at rounding level the step is still bounded by lr (first Adam step)
    assert np.all(np.abs(p1 - th) <= lr * (1 + 1e-4) + lr * 1e-4 * np.abs(th) + 1e-7)
    m.close()


def test_fp32_forward_matches_oracle(lbm):
    X, Y = _data(1000, seed=11)
    st = lbm.Surrogate.standardisation(X, Y)
    m = lbm.Surrogate(st, seed=1)
    th = _theta(4)
    m.set_params(th)
    P = m.predict_fp32(X)
    st64 = st.astype(np.float64)
    ref = M.forward(th.astype(np.float64), M.standardise_x(X.astype(np.float64), st64))[0][-1]
    # standardised space (outputs of a random network cross zero; rho_v is compared in log)
    err = np.abs(M.standardise_y(P.astype(np.float64), st64) - ref)
    assert np.max(err) < 1e-5 * max(1.0, np.max(np.abs(ref)))
    m.close()


@pytest.mark.parametrize("n", [4096, 1000, 1])
@pytest.mark.parametrize("mode", ["split", "single"])
def test_bf16_inference_within_rounding_bound(lbm, n, mode):
    """Fused tensor-core inference (BF16 operands, FP32 accumulation) against the FP64 forward
    pass: every standardised output within the oracle's first-order rounding bound, with unit
    roundoff 2^-8 for single BF16 operands and 2^-14 for split (hi + lo) operands (three
    products per tile, the lo*lo term dropped, FP32 accumulation).  Single-mode rounding is
    visible; split mode is near FP32."""
    X, Y = _data(max(n, 64), seed=13)
    X = X[:n]
    st = lbm.Surrogate.standardisation(*_data(2000, seed=5))
    m = lbm.Surrogate(st, seed=1)
    th = _theta(5)
    m.set_params(th)
    md = lbm.LBM_INFER_SPLIT_BF16 if mode == "split" else lbm.LBM_INFER_BF16
    P = m.predict(X, mode=md)
    st64 = st.astype(np.float64)
    yn = M.standardise_y(P.astype(np.float64), st64)
    ref = M.forward(th.astype(np.float64), M.standardise_x(X.astype(np.float64), st64))[0][-1]
    u = 2.0 ** -14 if mode == "split" else 2.0 ** -8
    bound = M.bf16_error_bound(th.astype(np.float64), X.astype(np.float64), st64, u=u)
    err = np.abs(yn - ref)
    assert np.all(err <= bound + 1e-5), np.max(err - bound)
    if n >= 1000 and mode == "single":
        assert np.max(err) > 1e-5
    if mode == "split":
        assert np.max(err) < 1e-3
    m.close()


def test_device_inference_equals_host_inference(lbm):
    import torch

    X, Y = _data(4096, seed=17)
    st = lbm.Surrogate.standardisation(X, Y)
    m = lbm.Surrogate(st, seed=3)
    P = m.predict(X)
    Xd = torch.from_numpy(X).cuda()
    Yd = torch.empty_like(Xd)
    m.predict_device(Xd, Yd)
    torch.cuda.synchronize()
    assert np.array_equal(Yd.cpu().numpy(), P)
    m.close()


def test_training_fits_smooth_map(lbm):
    X, Y = _data(4000, seed=19)
    Xh, Yh = _data(500, seed=23)
    st = lbm.Surrogate.standardisation(X, Y)
    m = lbm.Surrogate(st, seed=0)
    loss0, _ = m.loss_grad(X, Y)
    loss = m.train(X, Y, iterations=4000, lr=2e-3, lr_min=1e-5)
    assert loss < loss0 / 1000
    err = np.abs(m.predict(Xh) / Yh - 1)
    assert np.mean(err[:, 0]) < 3e-3 and np.mean(err[:, 1]) < 5e-3 and np.max(err[:, 1]) < 0.05
    m.close()


def test_surrogate_argument_errors(lbm):
    st = np.ones(16, np.float32)
    st[4] = 0.0
    with pytest.raises(lbm.LBMError) as e:
        lbm.Surrogate(st)
    assert e.value.code == lbm.LBM_ERR_ARG
    m = lbm.Surrogate(np.ones(16, np.float32))
    with pytest.raises(lbm.LBMError):
        m.train(np.zeros((4, 4), np.float32), np.ones((4, 4), np.float32), iterations=10, lr=-1.0)
    m.close()


N_TRAIN_SETS = 8000
N_HELD_OUT = 256


@pytest.fixture(scope="module")
def calibrated(lbm):
    """Seeded training sets calibrated by the batched solver, a trained surrogate, and the
    held-out sets' own calibrations (never trained on)."""
    from paper_2403_11167_gb300 import calibration as C

    tr = inputs.surrogate_sets(N_TRAIN_SETS, seed=4032)
    ho = inputs.surrogate_sets(N_HELD_OUT, seed=1116)
    r = C.calibrate_batched(tr)
    rh = C.calibrate_batched(ho)
    X = C.features(tr)
    m, loss, _ = C.fit_surrogate(X[r["ok"]], r["Y"][r["ok"]])
    yield dict(C=C, tr=tr, ho=ho, r=r, rh=rh, m=m, loss=loss)
    m.close()


def test_calibration_data_quality(calibrated):
    """Most sets give stationary flat runs; sigma is measured for most kappa_P >= 0.7 sets."""
    C, r, tr = calibrated["C"], calibrated["r"], calibrated["tr"]
    X = C.features(tr)
    assert r["ok"].mean() > 0.85
    wide = r["ok"] & (X[:, 3] >= 0.7)
    assert np.isfinite(r["Y"][wide, 3]).mean() > 0.8


def test_batched_calibration_equals_plain_calibration(calibrated):
    """The plain calibration (one lbm_ctx per lattice) is the surrogate's reference; the batched sweep
    that labels the held-out sets is bitwise the same computation (three sets checked)."""
    C, ho, rh = calibrated["C"], calibrated["ho"], calibrated["rh"]
    rp = C.calibrate_plain(ho[:3])
    assert np.array_equal(rp["Y"], rh["Y"][:3], equal_nan=True)
    assert np.array_equal(rp["raw"], rh["raw"][:len(rp["raw"])], equal_nan=True)


def test_surrogate_error_on_held_out_sets(calibrated):
    """BF16 surrogate against the calibration runs of 256 held-out seeded parameter sets:
    max relative error <= 1% on rho_l and rho_v (valid sets), <= 3% on sigma (sets where the
    droplets give a sigma)."""
    C, ho, rh, m = calibrated["C"], calibrated["ho"], calibrated["rh"], calibrated["m"]
    ok = rh["ok"]
    P = m.predict(C.features(ho)[ok])
    err = C.relative_errors(P, rh["Y"][ok])
    assert ok.sum() > 0.85 * N_HELD_OUT
    assert np.max(err[:, 0]) <= 0.01
    assert np.max(err[:, 1]) <= 0.01
    sig = np.isfinite(err[:, 3])
    assert sig.sum() > 0.5 * ok.sum()
    assert np.max(err[sig, 3]) <= 0.03


def test_surrogate_gain_over_theory(calibrated):
    """Without the network the parameters come from the Appendix-B theory, which predicts
    Maxwell coexistence densities; at Tr <= 0.6 the model's vapour density departs from them.
    The surrogate's rho_v error there is at least 10x smaller, and its sigma and W errors are
    smaller than those of the continuum theory (Eqs. S44, S46) over all valid sets."""
    C, ho, rh, m = calibrated["C"], calibrated["ho"], calibrated["rh"], calibrated["m"]
    X = C.features(ho)
    ok = rh["ok"]
    T = C.theory(ho)
    P = m.predict(X)
    low = ok & (X[:, 0] <= 0.6)
    assert low.sum() >= 20
    e_theory = np.abs(T[low, 1] / rh["Y"][low, 1] - 1)
    e_net = np.abs(P[low, 1] / rh["Y"][low, 1] - 1)
    assert np.mean(e_net) * 10 < np.mean(e_theory)
    sig = ok & np.isfinite(rh["Y"][:, 3])
    for j in (2, 3):
        m_ = sig if j == 3 else ok
        assert np.mean(np.abs(P[m_, j] / rh["Y"][m_, j] - 1)) < np.mean(np.abs(T[m_, j] / rh["Y"][m_, j] - 1))


def test_plain_calibration_is_the_fallback_outside_the_trained_domain(calibrated):
    """Sets inside the trained domain get the network's answer; a set beyond the trained
    temperatures, one with an untrained width parameter and one with kappa_P = 0.4 (whose
    training sets mostly lack a measurable sigma) are calibrated by running their lattices,
    exactly as a plain calibration does."""
    C, r, m, tr = calibrated["C"], calibrated["r"], calibrated["m"], calibrated["tr"]
    sc = C.SurrogateCalibration(m, C.features(tr), r["Y"], r["ok"])
    assert not sc.sigma_ok[0.4] and sc.sigma_ok[0.7] and sc.sigma_ok[1.0]
    inside = [dict(Tr=0.6, a=0.3, b=3.5, kappa_P=0.7), dict(Tr=0.7, a=0.45, b=4.5, kappa_P=1.0),
              dict(Tr=0.8, a=0.26, b=4.0, kappa_P=0.7), dict(Tr=0.9, a=0.4, b=3.2, kappa_P=1.0)]
    outside = [dict(Tr=0.97, a=0.3, b=4.0, kappa_P=1.0), dict(Tr=0.7, a=0.3, b=4.0, kappa_P=0.85),
               dict(Tr=0.7, a=0.3, b=4.0, kappa_P=0.4)]
    Y, src = sc.calibrate(inside + outside)
    assert list(src) == ["surrogate"] * 4 + ["calibration"] * 3
    assert np.array_equal(Y[:4], m.predict(C.features(inside)))
    assert np.array_equal(Y[4:], C.calibrate_batched(outside)["Y"], equal_nan=True)
