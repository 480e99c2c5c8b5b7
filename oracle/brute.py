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


def shifted(phi, i, walls=False, odd=False):
    """phi(x + c_i) on a lattice indexed [y, x], periodic in x; in y periodic, or (walls)
    reflected through the wall rows 0 and ny-1, with the sign flipped beyond a wall when odd."""
    if not walls:
        return np.roll(phi, shift=(-C[i, 1], -C[i, 0]), axis=(0, 1))
    ny = phi.shape[0]
    yy = np.arange(ny) + C[i, 1]
    beyond = (yy < 0) | (yy > ny - 1)
    yy = np.where(yy < 0, -yy, np.where(yy > ny - 1, 2 * (ny - 1) - yy, yy))
    out = np.roll(phi[yy], shift=-C[i, 0], axis=1)
    if odd:
        out[beyond] *= -1.0
    return out


def zou_he(f, Jx, Jy):
    """Completes the wall rows' incoming populations so that their momentum is (Jx, Jy)
    (arrays over the row): the bottom row lacks i = 2, 5, 6, the top row i = 4, 7, 8."""
    for y, up in ((0, 1), (f.shape[1] - 1, -1)):
        jx, jy = Jx[y], Jy[y]
        h = (f[1, y] - f[3, y]) / 2
        if up == 1:
            f[2, y] = f[4, y] + 2 / 3 * jy
            f[5, y] = f[7, y] - h + jx / 2 + jy / 6
            f[6, y] = f[8, y] + h - jx / 2 + jy / 6
        else:
            f[4, y] = f[2, y] - 2 / 3 * jy
            f[7, y] = f[5, y] + h - jx / 2 - jy / 6
            f[8, y] = f[6, y] - h + jx / 2 - jy / 6


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
    """One MP-LBM step; pr holds a, b, R, T, G, taus, kappa_P, kappa_Li, sigma_Li, fx, fy and
    optionally walls (Zou-He rows 0 and ny-1, mirrored psi) and the Sec. 5.4 drive (an external
    force: in F, not in the sigma^Li term's F_int)."""
    f = f.copy()
    ny, nx = f.shape[1:]
    walls = bool(pr.get("walls", 0.0))
    G = pr["G"]
    if walls:
        zou_he(f, np.zeros((ny, nx)), np.full((ny, nx), -pr["fy"] / 2))
    rho = f.sum(0)
    psi = np.sqrt(2 * (p_eos(rho, pr["a"], pr["b"], pr["R"], pr["T"]) - rho * CS2) / G)
    Fint = np.zeros((2,) + rho.shape)
    for i in range(1, 9):
        Fint += -G * psi * OMEGA[i] * shifted(psi, i, walls) * C[i][:, None, None]
    if walls:
        Fint[1][[0, -1]] = 0.0  # mirrored neighbours: no wall-normal interaction force
    Fx_ext = pr["fx"] * np.ones((ny, nx))
    if pr.get("drive", 0.0):
        ax = np.where(np.arange(nx)[None, :] <= pr["drive_x_split"], pr["drive_ax_lo"], pr["drive_ax_hi"])
        Fx_ext = Fx_ext + ax * np.abs(rho - rho.mean())
    F = Fint + np.stack([Fx_ext, pr["fy"] * np.ones((ny, nx))])
    C1 = 5 / 6 * (pr["kappa_P"] - 1)
    C2 = 0.5 * (1 - pr["kappa_P"])
    Q = np.zeros((2, 2) + rho.shape)
    for i in range(1, 9):
        cc = np.outer(C[i], C[i])
        Ci = C1 * G * np.eye(2) + C2 * G * (cc - CS2 * np.eye(2)) + pr["kappa_Li"] * G / 2 * cc
        Q += OMEGA[i] * Ci[:, :, None, None] * (shifted(psi, i, walls) - psi)
    Q *= psi
    if walls:
        zou_he(f, -F[0] / 2, -F[1] / 2)
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


def grad(phi, walls=False, odd=False):
    """Eq. (24) gradient, read with the weights w_i."""
    g = np.zeros((2,) + phi.shape)
    for i in range(9):
        g += W[i] * shifted(phi, i, walls, odd) * C[i][:, None, None]
    return g / CS2


def lap(phi, walls=False):
    """Eq. (24) Laplacian."""
    return 2 / CS2 * sum(W[i] * (shifted(phi, i, walls) - phi) for i in range(9))


def fe_step(f, pr):
    """One IWB-FE-LBM step: Eq. (20) with A and p_g = rho_0 g (y - y_ref), Eq. (21) with
    grad p_g, the buoyancy -(rho - rho_0) g, the Sec. 5.4 drive and, with walls, the Zou-He
    rows (u = 0 with the half force: J = -F/2), mirrored stencils and odd velocities beyond
    the walls.  Optional keys: A, g, rho_g, y_ref, walls, drive, drive_ax_lo, drive_ax_hi,
    drive_x_split.  walls = 2: the wall rows' normal grad mu one-sided (ghost 2 mu(0) - mu(1))
    with the wall densities iterated to the fixed point of fill and normal force."""
    f = f.copy()
    ny, nx = f.shape[1:]
    walls = bool(pr.get("walls", 0.0))
    one_sided = pr.get("walls", 0.0) == 2.0
    A, g, rg, yref = pr.get("A", 0.0), pr.get("g", 0.0), pr.get("rho_g", 0.0), pr.get("y_ref", 0.0)
    yv = np.arange(ny, dtype=float)[:, None] * np.ones((1, nx))
    wall_row = np.zeros((ny, nx), bool)
    if walls:
        wall_row[[0, -1]] = True
        zou_he(f, np.zeros((ny, nx)), np.full((ny, nx), -pr["fy"] / 2))
    rho = f.sum(0)
    if walls and not one_sided and g != 0.0:
        # wall rows: the node's own buoyancy enters its normal force; rho = K + Jy (bottom),
        # K - Jy (top), Jy = -(fy - (rho - rho_0) g)/2
        K0 = rho[0] + pr["fy"] / 2
        K1 = rho[-1] - pr["fy"] / 2
        r0 = (K0 - pr["fy"] / 2 - rg * g / 2) / (1 - g / 2)
        r1 = (K1 + pr["fy"] / 2 + rg * g / 2) / (1 + g / 2)
        Fyw = np.zeros((ny, nx))
        Fyw[0] = pr["fy"] - (r0 - rg) * g
        Fyw[-1] = pr["fy"] - (r1 - rg) * g
        zou_he(f, np.zeros((ny, nx)), -Fyw / 2)
        rho = f.sum(0)
    def wall_dmu(mu):
        # one-sided wall-normal gradient at rows 0 and ny-1 (Eq. 24 weights, extrapolated ghost)
        g = np.zeros((ny, nx))
        for y, yi, sgn in ((0, 1, 1.0), (ny - 1, ny - 2, -1.0)):
            d = mu[yi] - mu[y]
            g[y] = sgn * 2 * (W[2] * d + W[5] * (np.roll(d, -1) + np.roll(d, 1))) / CS2
        return g

    if one_sided:
        for _ in range(200):
            mu = mu_bulk(rho, pr["a"], pr["b"], pr["R"], pr["T"]) - pr["kappa"] * lap(rho, True)
            Fyw = -rho * wall_dmu(mu) + pr["fy"] - (rho - rg) * g
            zou_he(f, np.zeros((ny, nx)), -Fyw / 2)
            new = f.sum(0)
            done = np.abs(new - rho).max() <= 1e-16 * rho[0, 0]
            rho = new
            if done:
                break
    mu = mu_bulk(rho, pr["a"], pr["b"], pr["R"], pr["T"]) - pr["kappa"] * lap(rho, walls)
    Fx_ext = pr["fx"] * np.ones((ny, nx))
    if pr.get("drive", 0.0):
        ax = np.where(np.arange(nx)[None, :] <= pr["drive_x_split"], pr["drive_ax_lo"], pr["drive_ax_hi"])
        Fx_ext = Fx_ext + ax * np.abs(rho - rho.mean())
    F = -rho * grad(mu, walls) + np.stack([Fx_ext, pr["fy"] - (rho - rg) * g])
    grho = grad(rho, walls)
    F[1][wall_row] = (pr["fy"] - (rho - rg) * g - (rho * wall_dmu(mu) if one_sided else 0.0))[wall_row]
    grho[1][wall_row] = 0.0
    if walls:
        zou_he(f, -F[0] / 2, -F[1] / 2)
    j = np.tensordot(C.T.astype(float), f, axes=(1, 0))
    u = (j + F / 2) / rho
    S = np.zeros((2, 2, ny, nx))
    if A != 0.0:
        du = [grad(u[a], walls, odd=True) for a in range(2)]  # du[a][b] = d_b u_a
        for a in range(2):
            for b in range(2):
                S[a, b] = du[b][a] + du[a][b]
    X = u[:, None] * u[None, :] + CS2 * A * S
    trX = X[0, 0] + X[1, 1]
    pg = rg * g * (yv - yref)
    dpg = np.array([0.0, rg * g])
    feq = np.empty_like(f)
    Fi = np.empty_like(f)
    ug = (u * grho).sum(0)
    for i in range(9):
        cu = C[i, 0] * u[0] + C[i, 1] * u[1]
        cXc = sum(C[i, a] * C[i, b] * X[a, b] for a in range(2) for b in range(2))
        if i == 0:
            feq[i] = rho - (1 - W[0]) * pg / CS2 - W[0] * rho * trX / (2 * CS2)
        else:
            feq[i] = W[i] * pg / CS2 + W[i] * rho * (cu / CS2 + (cXc - CS2 * trX) / (2 * CS2**2))
        cF = C[i, 0] * F[0] + C[i, 1] * F[1]
        Fp = F - dpg[:, None, None] + CS2 * grho
        t2 = sum((C[i, a] * C[i, b] - CS2 * (a == b)) * u[a] * Fp[b] for a in range(2) for b in range(2))
        Fi[i] = W[i] * (cF / CS2 + t2 / CS2**2 + 0.5 * ((C[i] ** 2).sum() / CS2 - 2) * ug)
    MF = np.tensordot(M, Fi, axes=(1, 0))
    return collide_and_stream(f, feq, MF, np.zeros_like(f), pr)


def run(model, f, pr, nsteps):
    step = pp_step if model == 0 else fe_step
    for _ in range(nsteps):
        f = step(f, pr)
    return f
