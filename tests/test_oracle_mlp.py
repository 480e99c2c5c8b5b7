"""Pins of the surrogate network's CPU oracle (finite differences, closed forms)."""
import math

import numpy as np
import pytest

from oracle import mlp as M


def _theta(seed=0, scale=1.0):
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for l in range(M.N_LAYERS):
        lim = math.sqrt(6.0 / M.DIMS[l]) * scale
        parts.append(rng.uniform(-lim, lim, M.DIMS[l + 1] * M.DIMS[l]))
        parts.append(rng.uniform(-0.1, 0.1, M.DIMS[l + 1]))
    return np.concatenate(parts)


def _data(n, seed=1):
    rng = np.random.Generator(np.random.PCG64(seed))
    X = np.column_stack([rng.uniform(0.5, 0.95, n), rng.uniform(0.25, 0.5, n), rng.uniform(3, 5, n),
                         rng.choice([0.4, 0.7, 1.0], n)])
    Y = np.column_stack([rng.uniform(0.2, 0.4, n), np.exp(rng.uniform(-7, -2, n)), rng.uniform(3, 12, n),
                         rng.uniform(0.001, 0.05, n)])
    return X, Y


def _stats(X, Y):
    Yp = Y.copy()
    Yp[:, 1] = np.log(Yp[:, 1])
    return np.concatenate([X.mean(0), X.std(0), Yp.mean(0), Yp.std(0)])


def test_parameter_count():
    assert M.N_PARAMS == 34180
    th = _theta()
    assert np.array_equal(M.pack(M.unpack(th)), th)


def test_gelu_closed_forms():
    z = np.linspace(-6, 6, 241)
    g = M.gelu(z)
    assert M.gelu(np.array([0.0]))[0] == 0.0
    # GELU(z) - GELU(-z) = z (Phi(z) + Phi(-z) = 1)
    assert np.max(np.abs(g - M.gelu(-z) - z)) < 1e-14
    assert abs(M.gelu(np.array([1.0]))[0] - 0.5 * (1 + math.erf(1 / math.sqrt(2)))) < 1e-15
    # derivative by central differences
    h = 1e-6
    fd = (M.gelu(z + h) - M.gelu(z - h)) / (2 * h)
    assert np.max(np.abs(fd - M.gelu_grad(z))) < 1e-8
    # Lipschitz constant of GELU is attained at sqrt(2)
    zz = np.linspace(-10, 10, 200001)
    assert abs(np.max(np.abs(M.gelu_grad(zz))) - M.GELU_LIPSCHITZ) < 1e-4


def test_zero_weights_give_last_bias():
    th = np.zeros(M.N_PARAMS)
    wo, bo = M.offsets()[-1]
    th[bo:bo + 4] = [0.3, -1.0, 2.0, 0.5]
    X, Y = _data(7)
    st = _stats(X, Y)
    pre, _ = M.forward(th, M.standardise_x(X, st))
    assert np.array_equal(pre[-1], np.tile([0.3, -1.0, 2.0, 0.5], (7, 1)))


def test_selected_path_is_nested_gelu():
    """A network whose weights route input 2 -> hidden 3 -> hidden 5 -> hidden 7 -> output 1
    computes y_1 = GELU(GELU(GELU(x_2 + c1) + c2) + c3) + c4 (an index or transpose error
    breaks the routing)."""
    th = np.zeros(M.N_PARAMS)
    offs = M.offsets()
    route = [(3, 2), (5, 3), (7, 5), (1, 7)]  # (out, in) per layer
    biases = [0.2, -0.1, 0.3, 0.05]
    for l, ((o, i), c) in enumerate(zip(route, biases)):
        wo, bo = offs[l]
        th[wo + o * M.DIMS[l] + i] = 1.0
        th[bo + o] = c
    Xn = np.linspace(-2, 2, 9)[:, None] * np.array([[0.0, 0.0, 1.0, 0.0]]) + np.array([[5.0, -3.0, 0.0, 7.0]])
    pre, _ = M.forward(th, Xn)
    g = lambda v: 0.5 * v * (1 + math.erf(v / math.sqrt(2)))
    for k, x in enumerate(Xn[:, 2]):
        ref = g(g(g(x + 0.2) - 0.1) + 0.3) + 0.05
        assert abs(pre[-1][k, 1] - ref) < 1e-15
        assert pre[-1][k, 0] == 0.0 and pre[-1][k, 2] == 0.0 and pre[-1][k, 3] == 0.0


def test_standardisation_roundtrip_and_log_rho_v():
    X, Y = _data(11)
    st = _stats(X, Y)
    Yn = M.standardise_y(Y, st)
    assert np.max(np.abs(M.destandardise_y(Yn, st) / Y - 1)) < 1e-14
    assert abs(Yn[:, 1].mean()) < 1e-12 and abs(Yn[:, 1].std() - 1) < 1e-12


@pytest.mark.parametrize("n", [5, 37])
def test_gradient_matches_central_differences(n):
    th = _theta(3)
    X, Y = _data(n, seed=4)
    st = _stats(X, Y)
    loss, g = M.loss_grad(th, X, Y, st)
    rng = np.random.Generator(np.random.PCG64(5))
    # every bias of every layer and a sample of each layer's weights
    idx = []
    for l, (wo, bo) in enumerate(M.offsets()):
        idx += list(rng.choice(np.arange(wo, bo), 12, replace=False))
        idx += list(range(bo, bo + M.DIMS[l + 1]))[:16]
    h = 1e-6
    for i in idx:
        tp, tm = th.copy(), th.copy()
        tp[i] += h
        tm[i] -= h
        fd = (M.loss_grad(tp, X, Y, st)[0] - M.loss_grad(tm, X, Y, st)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(g[i])) + 1e-9, (i, fd, g[i])


def test_loss_definition():
    th = _theta(6)
    X, Y = _data(13)
    st = _stats(X, Y)
    loss, _ = M.loss_grad(th, X, Y, st)
    P = M.predict(th, X, st)
    Pn = M.standardise_y(P, st)
    Yn = M.standardise_y(Y, st)
    assert abs(loss - np.mean((Pn - Yn) ** 2)) < 1e-13 * max(1.0, loss)


def test_adam_constant_gradient_steps():
    th = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    m1 = np.zeros(3)
    m2 = np.zeros(3)
    lr = 0.01
    for t in range(1, 4):
        new, m1, m2 = M.adam_step(th, g, m1, m2, t, lr)
        # bias-corrected moments of a constant gradient are g and g^2
        assert np.max(np.abs((th - new) - lr * g / (np.abs(g) + 1e-8))) < 1e-15
        th = new
    # decoupled weight decay adds lr * wd * theta
    new, _, _ = M.adam_step(np.array([2.0]), np.array([0.0]), np.zeros(1), np.zeros(1), 1, 0.1, weight_decay=0.5)
    assert abs(new[0] - (2.0 - 0.1 * 0.5 * 2.0)) < 1e-15


def test_cosine_schedule_end_points():
    assert M.lr_at(0, 100, 1e-3, 1e-5) == 1e-3
    assert abs(M.lr_at(99, 100, 1e-3, 1e-5) - 1e-5) < 1e-18
    assert abs(M.lr_at(49.5, 100, 1e-3, 1e-5) - 0.5 * (1e-3 + 1e-5)) < 1e-15
    assert M.lr_at(0, 1, 1e-3, 1e-5) == 1e-3


def test_training_fits_a_smooth_map():
    """A few hundred full-batch Adam steps cut the loss of a smooth synthetic map by 20x."""
    rng = np.random.Generator(np.random.PCG64(8))
    X, _ = _data(64, seed=9)
    Y = np.column_stack([0.3 - 0.1 * X[:, 0], np.exp(-4 * X[:, 0] * X[:, 1] * 4 / X[:, 2]), 2 + 5 * X[:, 3],
                         0.02 * (1 - X[:, 0]) ** 1.5])
    st = _stats(X, Y)
    th = _theta(10) * 0.5
    _, losses = M.train(th, X, Y, st, 300, 3e-3, 3e-4)
    assert losses[-1] < losses[0] / 20


def test_bf16_bound_is_first_order_and_covers_emulation():
    """The bound covers an FP64 emulation of BF16 rounding of inputs, weights and
    activations (round to nearest even of the top 8 significand bits)."""
    def rbf16(v):
        v = np.asarray(v, dtype=np.float32)
        b = v.view(np.uint32).astype(np.uint64)
        b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
        return b.astype(np.uint32).view(np.float32).astype(np.float64)

    th = _theta(12)
    X, Y = _data(200, seed=13)
    st = _stats(X, Y)
    bound = M.bf16_error_bound(th, X, st)
    a = rbf16(M.standardise_x(X, st))
    for l, (W, b) in enumerate(M.unpack(th)):
        z = a @ rbf16(W).T + b
        a = rbf16(M.gelu(z)) if l < M.N_LAYERS - 1 else z
    exact = M.forward(th, M.standardise_x(X, st))[0][-1]
    err = np.abs(a - exact)
    assert np.all(err <= bound)
    assert np.max(err) > 0


def test_missing_targets_drop_out_of_loss_and_gradient():
    """A NaN target contributes nothing: the loss over a set with missing sigma equals the
    loss over the same set with sigma replaced by the prediction, rescaled by the count."""
    th = _theta(14)
    X, Y = _data(9, seed=15)
    st = _stats(X, Y)
    P = M.predict(th, X, st)
    Ym = Y.copy()
    Ym[[1, 4, 7], 3] = np.nan
    Yf = Y.copy()
    Yf[[1, 4, 7], 3] = P[[1, 4, 7], 3]
    lm, gm = M.loss_grad(th, X, Ym, st)
    lf, gf = M.loss_grad(th, X, Yf, st)
    assert abs(lm * (36 - 3) - lf * 36) < 1e-12 * lf * 36
    assert np.max(np.abs(gm * (36 - 3) - gf * 36)) < 1e-10 * np.max(np.abs(gf * 36))
