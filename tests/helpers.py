"""Shared test helpers: build a GPU context and the matching oracle parameters."""
import numpy as np

import oracle as O


def oracle_params(rp, th, walls=False):
    """Oracle parameters equal to a resolved ``lbm_params`` (rp) and its thermodynamics (th);
    walls: no-slip walls on rows 0 and ny-1 (1 or True: mirrored reading, 2: the free-energy
    one-sided wall-normal chemical-potential gradient)."""
    return O.make_params(a=rp.a, b=rp.b, R=rp.R, T=th.T, tau_rho=1.0, tau_e=rp.tau_e, tau_zeta=rp.tau_zeta,
                         tau_q=rp.tau_q, tau_j=rp.tau_j, tau_nu=rp.tau_nu, kappa_P=rp.kappa_P,
                         kappa_Li=rp.kappa_Li, sigma_Li=rp.sigma_Li, kappa=rp.kappa, fx=rp.body_fx,
                         fy=rp.body_fy, walls=float(walls) if walls else 0.0, A=rp.A)


def gpu_context(model, precision, nx, ny, walls=False, **kw):
    from paper_2403_11167_gb300 import lbm

    p = lbm.lbm_params_default(model, precision=precision, **kw)
    ctx = lbm.Context(p, nx, ny, walls=walls)
    rp, th = ctx.derived()
    return ctx, rp, th


def rho_err(a, b):
    """Largest relative density error, cell by cell: max over cells of |a - b| / |b| (every cell
    against its own density, so a vapour cell counts as much as a liquid one)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b) / np.abs(b)))


def pop_err(f, f_ref):
    """Largest population error relative to its own cell's density: max over i and cells of
    |f_i - f_ref_i| / rho_ref (populations can vanish, the density of their cell cannot)."""
    f = np.asarray(f, dtype=np.float64)
    f_ref = np.asarray(f_ref, dtype=np.float64)
    return float(np.max(np.abs(f - f_ref) / np.abs(f_ref.sum(0))))
