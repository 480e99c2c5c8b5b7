"""Second, NumPy-only literal implementation of one time step of each model.

TEST INFRASTRUCTURE (see ``oracle/__init__.py``).  Written independently of
``lbm_oracle.c`` (whole-lattice array form, neighbour access by ``np.roll``,
M typed from Eq. (S48), M^-1 from ``numpy.linalg.inv``) so that a typo in one of
the two oracles shows up as a disagreement on small lattices.  Slow; meant for
lattices of a few hundred cells.
"""
import numpy as np

CS2 = 1.0 / 3.0
# Eq. (2)
C = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1], [1, 1], [-1, 1], [-1, -1], [1, -1]])
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
# Eq. (10): omega(|c|^2)
OMEGA = np.array([0.0] + [1 / 3] * 4 + [1 / 12] * 4)
# Eq. (S48)
M = np.array([
    [1, 1, 1, 1, 1, 1, 1, 1, 1],
    [-4, -1, -1, -1, -1, 2, 2, 2, 2],
    [4, -2, -2, -2, -2, 1, 1, 1, 1],
    [0, 1, 0, -1, 0, 1, -1, -1, 1],
    [0, -2, 0, 2, 0, 1, -1, -1, 1],
    [0, 0, 1, 0, -1, 1, 1, -1, -1],
    [0, 0, -2, 0, 2, 1, 1, -1, -1],
    [0, 1, -1, 1, -1, 0, 0, 0, 0],
    [0, 0, 0, 0, 0, 1, -1, 1, -1],
], dtype=float)
MINV = np.linalg.inv(M)


def shifted(phi, i):
    """phi(x + c_i) on a periodic lattice indexed [y, x]."""
    return np.roll(phi, shift=(-C[i, 1], -C[i, 0]), axis=(0, 1))


def stream(fstar):
    """f_i(x + c_i) = f*_i(x)."""
    return np.stack([np.roll(fstar[i], shift=(C[i, 1], C[i, 0]), axis=(0, 1)) for i in range(9)])


def p_eos(rho, a, b, R, T):
    eta = b * rho / 4
    return rho * R * T * (1 + eta + eta**2 - eta**3) / (1 - eta) ** 3 - a * rho**2


def mu_bulk(rho, a, b, R, T):
    eta = b * rho / 4
    return R * T * (3 - eta) / (1 - eta) ** 3 + R * T * np.log(rho) + R * T - 2 * a * rho


def lam(pr):
    return np.diag(1.0 / np.array([pr["tau_rho"], pr["tau_e"], pr["tau_zeta"], pr["tau_j"], pr["tau_q"],
                                   pr["tau_j"], pr["tau_q"], pr["tau_nu"], pr["tau_nu"]]))


def collide_and_stream(f, feq, MF, MC, pr):
    """Eq. (1) in matrix form on every cell, then streaming."""
    L = lam(pr)
    ny, nx = f.shape[1:]
    fv = f.reshape(9, -1)
    Omega = -MINV @ L @ M @ (fv - feq.reshape(9, -1))
    S = MINV @ (np.eye(9) - L / 2) @ MF.reshape(9, -1)
    Ci = MINV @ MC.reshape(9, -1)
    return stream((fv + Omega + S + Ci).reshape(9, ny, nx))


def pp_step(f, pr):
    """One MP-LBM step; pr holds a, b, R, T, G, taus, kappa_P, kappa_Li, sigma_Li, fx, fy."""
    G = pr["G"]
    rho = f.sum(0)
    psi = np.sqrt(2 * (p_eos(rho, pr["a"], pr["b"], pr["R"], pr["T"]) - rho * CS2) / G)
    Fint = np.zeros((2,) + rho.shape)
    for i in range(1, 9):
        Fint += -G * psi * OMEGA[i] * shifted(psi, i) * C[i][:, None, None]
    F = Fint + np.array([pr["fx"], pr["fy"]])[:, None, None]
    C1 = 5 / 6 * (pr["kappa_P"] - 1)
    C2 = 0.5 * (1 - pr["kappa_P"])
    Q = np.zeros((2, 2) + rho.shape)
    for i in range(1, 9):
        cc = np.outer(C[i], C[i])
        Ci = C1 * G * np.eye(2) + C2 * G * (cc - CS2 * np.eye(2)) + pr["kappa_Li"] * G / 2 * cc
        Q += OMEGA[i] * Ci[:, :, None, None] * (shifted(psi, i) - psi)
    Q *= psi
    j = np.tensordot(C.T.astype(float), f, axes=(1, 0))
    u = (j + F / 2) / rho
    uu = (u**2).sum(0)
    feq = np.empty_like(f)
    for i in range(9):
        cu = C[i, 0] * u[0] + C[i, 1] * u[1]
        feq[i] = W[i] * rho * (1 + cu / CS2 + (cu**2 - CS2 * uu) / (2 * CS2**2))
    uF = (u * F).sum(0)
    F2 = (Fint**2).sum(0)
    kP, sL = pr["kappa_P"], pr["sigma_Li"]
    MF = np.stack([
        0 * rho,
        6 * uF + 12 * kP * sL * F2 / (psi**2 * (pr["tau_e"] - 0.5)),
        -6 * uF - 12 * kP * sL * F2 / (psi**2 * (pr["tau_zeta"] - 0.5)),
        F[0], -F[0], F[1], -F[1],
        2 * (u[0] * F[0] - u[1] * F[1]),
        u[0] * F[1] + u[1] * F[0],
    ])
    trQ = Q[0, 0] + Q[1, 1]
    MC = np.stack([
        0 * rho, 1.5 / pr["tau_e"] * trQ, -1.5 / pr["tau_zeta"] * trQ,
        0 * rho, 0 * rho, 0 * rho, 0 * rho,
        -(Q[0, 0] - Q[1, 1]) / pr["tau_nu"], -Q[0, 1] / pr["tau_nu"],
    ])
    return collide_and_stream(f, feq, MF, MC, pr)


def grad(phi):
    """Eq. (24) gradient, read with the weights w_i."""
    g = np.zeros((2,) + phi.shape)
    for i in range(9):
        g += W[i] * shifted(phi, i) * C[i][:, None, None]
    return g / CS2


def lap(phi):
    """Eq. (24) Laplacian."""
    return 2 / CS2 * sum(W[i] * (shifted(phi, i) - phi) for i in range(9))


def fe_step(f, pr):
    """One IWB-FE-LBM step (A = 0, p_g = 0)."""
    rho = f.sum(0)
    mu = mu_bulk(rho, pr["a"], pr["b"], pr["R"], pr["T"]) - pr["kappa"] * lap(rho)
    F = -rho * grad(mu) + np.array([pr["fx"], pr["fy"]])[:, None, None]
    grho = grad(rho)
    j = np.tensordot(C.T.astype(float), f, axes=(1, 0))
    u = (j + F / 2) / rho
    uu = (u**2).sum(0)
    feq = np.empty_like(f)
    Fi = np.empty_like(f)
    ug = (u * grho).sum(0)
    for i in range(9):
        cu = C[i, 0] * u[0] + C[i, 1] * u[1]
        if i == 0:
            feq[i] = rho - W[0] * rho * uu / (2 * CS2)
        else:
            feq[i] = W[i] * rho * (cu / CS2 + (cu**2 - CS2 * uu) / (2 * CS2**2))
        cF = C[i, 0] * F[0] + C[i, 1] * F[1]
        Fp = F + CS2 * grho
        t2 = sum((C[i, a] * C[i, b] - CS2 * (a == b)) * u[a] * Fp[b] for a in range(2) for b in range(2))
        Fi[i] = W[i] * (cF / CS2 + t2 / CS2**2 + 0.5 * ((C[i] ** 2).sum() / CS2 - 2) * ug)
    MF = np.tensordot(M, Fi, axes=(1, 0))
    return collide_and_stream(f, feq, MF, np.zeros_like(f), pr)


def run(model, f, pr, nsteps):
    step = pp_step if model == 0 else fe_step
    for _ in range(nsteps):
        f = step(f, pr)
    return f
