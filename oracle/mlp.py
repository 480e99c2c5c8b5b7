"""FP64 CPU oracle of the calibration surrogate's network (test infrastructure only).

Only tests, the smoke check and the benchmark's CPU leg use this module; the product
path never does.  Plain NumPy in float64, one operation per line of the definitions:

* network: x -> z1 = W1 x + b1 -> a1 = GELU(z1) -> ... -> y = W4 a3 + b4, widths
  4, 128, 128, 128, 4; GELU(z) = z Phi(z) with Phi the standard normal CDF (via erf);
* parameters: one flat vector, per layer W_l [out][in] row-major, then b_l;
* inputs and targets standardised with stats16 = (mean X, std X, mean Y', std Y'),
  Y' = (rho_l, ln rho_v, W, sigma); loss = mean over the finite target entries of the
  squared standardised error (NaN marks a missing target);
* gradient by the chain rule (backpropagation), Adam with bias correction and decoupled
  weight decay, cosine learning-rate decay from lr to lr_min over the run;
* a first-order bound of the error of BF16 inputs/weights/activations with exact
  accumulation (the inference kernel accumulates in FP32).

Pins (tests/test_oracle_mlp.py): central finite differences of the loss against the
gradient; networks whose weights select one path reduce to GELU(GELU(GELU(x))) written
with math.erf; zero weights give the last bias; Adam's first steps under a constant
gradient move by lr g / (|g| + eps); the cosine schedule's end points.
"""
import math

import numpy as np
from scipy.special import erf

DIMS = (4, 128, 128, 128, 4)
N_LAYERS = len(DIMS) - 1


def offsets():
    """[(w_offset, b_offset)] per layer in the flat parameter vector."""
    out, o = [], 0
    for l in range(N_LAYERS):
        nw = DIMS[l + 1] * DIMS[l]
        out.append((o, o + nw))
        o += nw + DIMS[l + 1]
    return out


N_PARAMS = offsets()[-1][1] + DIMS[-1]


def unpack(theta):
    theta = np.asarray(theta, dtype=np.float64)
    assert theta.shape == (N_PARAMS,)
    layers = []
    for l, (wo, bo) in enumerate(offsets()):
        W = theta[wo:bo].reshape(DIMS[l + 1], DIMS[l])
        b = theta[bo:bo + DIMS[l + 1]]
        layers.append((W, b))
    return layers


def pack(layers):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in layers])


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    Phi = 0.5 * (1.0 + erf(z / math.sqrt(2.0)))
    phi = np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)
    return Phi + z * phi


def standardise_x(X, stats):
    stats = np.asarray(stats, dtype=np.float64)
    return (np.asarray(X, dtype=np.float64) - stats[0:4]) / stats[4:8]


def standardise_y(Y, stats):
    stats = np.asarray(stats, dtype=np.float64)
    Yp = np.array(Y, dtype=np.float64)
    Yp[:, 1] = np.log(Yp[:, 1])
    return (Yp - stats[8:12]) / stats[12:16]


def destandardise_y(Yn, stats):
    stats = np.asarray(stats, dtype=np.float64)
    Y = np.asarray(Yn, dtype=np.float64) * stats[12:16] + stats[8:12]
    Y[:, 1] = np.exp(Y[:, 1])
    return Y


def forward(theta, Xn):
    """Pre-activations z_l and activations a_l (a_0 = Xn) of standardised inputs (n x 4)."""
    a = np.asarray(Xn, dtype=np.float64)
    acts, pre = [a], []
    layers = unpack(theta)
    for l, (W, b) in enumerate(layers):
        z = a @ W.T + b
        pre.append(z)
        if l < N_LAYERS - 1:
            a = gelu(z)
            acts.append(a)
    return pre, acts


def predict(theta, X, stats):
    pre, _ = forward(theta, standardise_x(X, stats))
    return destandardise_y(pre[-1], stats)


def loss_grad(theta, X, Y, stats):
    """Mean squared standardised error and its gradient (flat vector)."""
    Xn, Yn = standardise_x(X, stats), standardise_y(Y, stats)
    pre, acts = forward(theta, Xn)
    layers = unpack(theta)
    # a NaN target is missing: it adds neither loss nor gradient; the mean runs over the rest
    valid = np.isfinite(Yn)
    count = int(valid.sum())
    r = np.where(valid, pre[-1] - np.where(valid, Yn, 0.0), 0.0)
    loss = float(np.sum(r * r) / count)
    dz = 2.0 * r / count
    grads = [None] * N_LAYERS
    for l in range(N_LAYERS - 1, -1, -1):
        W, _ = layers[l]
        dW = dz.T @ acts[l]
        db = dz.sum(axis=0)
        grads[l] = (dW, db)
        if l > 0:
            da = dz @ W
            dz = da * gelu_grad(pre[l - 1])
    return loss, pack(grads)


def lr_at(it, iterations, lr, lr_min):
    """Cosine decay: lr at the first iteration, lr_min at the last."""
    frac = it / (iterations - 1) if iterations > 1 else 0.0
    return lr_min + 0.5 * (lr - lr_min) * (1.0 + math.cos(math.pi * frac))


def adam_step(theta, g, m1, m2, t, lr, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0):
    """One Adam update (t = 1 for the first) with decoupled weight decay; returns new arrays."""
    m1 = beta1 * m1 + (1.0 - beta1) * g
    m2 = beta2 * m2 + (1.0 - beta2) * g * g
    mhat = m1 / (1.0 - beta1 ** t)
    vhat = m2 / (1.0 - beta2 ** t)
    theta = theta - lr * (mhat / (np.sqrt(vhat) + eps) + weight_decay * theta)
    return theta, m1, m2


def train(theta, X, Y, stats, iterations, lr, lr_min, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0):
    """Full-batch Adam training; returns (theta, list of losses before each update)."""
    theta = np.array(theta, dtype=np.float64)
    m1 = np.zeros_like(theta)
    m2 = np.zeros_like(theta)
    losses = []
    for it in range(iterations):
        loss, g = loss_grad(theta, X, Y, stats)
        losses.append(loss)
        theta, m1, m2 = adam_step(theta, g, m1, m2, it + 1, lr_at(it, iterations, lr, lr_min), beta1, beta2, eps,
                                  weight_decay)
    return theta, losses


GELU_LIPSCHITZ = 1.1289  # max |GELU'(z)|, at z = sqrt(2): Phi(sqrt 2) + sqrt(2) phi(sqrt 2)


def bf16_error_bound(theta, X, stats, u=2.0 ** -8):
    """First-order bound on |y_n(BF16) - y_n(exact)| per output (standardised space) when the
    standardised inputs, the weights and each hidden activation are rounded to BF16 (unit
    roundoff u = 2^-8) and products are accumulated exactly; biases stay FP32."""
    Xn = standardise_x(X, stats)
    pre, acts = forward(theta, Xn)
    layers = unpack(theta)
    e = u * np.abs(Xn)
    for l, (W, _) in enumerate(layers):
        ez = (e + u * np.abs(acts[l])) @ np.abs(W).T
        if l < N_LAYERS - 1:
            e = GELU_LIPSCHITZ * ez + u * np.abs(acts[l + 1])
        else:
            return ez
