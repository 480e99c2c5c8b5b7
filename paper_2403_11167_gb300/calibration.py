"""Calibration runs of the pseudopotential model and the learned surrogate built on them.

The pseudopotential model fixes its parameters against preliminary simulations (Secs. 3,
5.1, 5.2).  One calibration of a parameter set (Tr, a, b, kappa_P; R = 1, tau = 1,
kappa_Li = 0, sigma_Li from the Appendix-B theory) here is four lattices:

* a flat interface, 256 x 4, 10^4 steps: rho_l, rho_v and the tangent width W;
* three centred droplets of radius 20, 30 and 40 on 128 x 128, 8000 steps: the pressure
  jump dp against the inverse equimolar radius, whose least-squares slope (with an
  intercept) is the surface tension sigma (2-D Laplace law, dp = sigma / R).

``calibrate_batched`` runs many sets as ``lbm_batch`` sweeps; ``calibrate_plain`` runs the
same lattices one ``lbm_ctx`` at a time (the plain calibration that judges the surrogate).
Both are bitwise the same computation.  ``fit_surrogate`` trains the MLP on the GPU.
"""
from __future__ import annotations

import time

import numpy as np

from . import inputs
from . import lbm as L

FLAT_NX, FLAT_NY = 256, 4
DROP_L = 128
RADII = (20.0, 30.0, 40.0)
STEPS_FLAT = 10000
STEPS_DROPLET = 8000
LATTICES_PER_SET = 1 + len(RADII)


def set_params(s) -> "L.lbm_params":
    return L.lbm_params_default(L.LBM_PSEUDOPOTENTIAL, a=s["a"], b=s["b"], Tr=s["Tr"], kappa_P=s["kappa_P"],
                                tau_nu=1.0, kappa_Li=0.0)


def features(sets) -> np.ndarray:
    """Network inputs (Tr, a, b, kappa_P), one row per set."""
    return np.array([[s[k] for k in L.SURROGATE_INPUTS] for s in sets], dtype=np.float64)


def lattices(sets, steps_flat=STEPS_FLAT, steps_droplet=STEPS_DROPLET):
    """Batch specs and initial densities of every set's four lattices (sets whose parameters
    do not resolve get none).  Returns (specs, rho0s, owner set index, per-set resolve status,
    per-set (params, thermo))."""
    resolved = L.lbm_resolve_params_many([set_params(s) for s in sets])
    specs, rhos, owner = [], [], []
    status = np.zeros(len(sets), dtype=int)
    derived = []
    for i, (st, rp, th) in enumerate(resolved):
        status[i] = st
        derived.append((rp, th))
        if st != L.LBM_OK:
            continue
        flat = dict(nx=FLAT_NX, ny=FLAT_NY, geometry=L.FLAT, nsteps=steps_flat, params=rp)
        specs.append(flat)
        rhos.append(inputs.flat_slab(FLAT_NX, FLAT_NY, th.rho_v, th.rho_l))
        owner.append(i)
        for R in RADII:
            specs.append(dict(nx=DROP_L, ny=DROP_L, geometry=L.DROPLET, nsteps=steps_droplet, params=rp))
            rhos.append(inputs.droplet(DROP_L, DROP_L, R, th.rho_v, th.rho_l))
            owner.append(i)
    return specs, rhos, owner, status, derived


def targets_from_observables(obs4):
    """(rho_l, rho_v, W, sigma) of one set from its flat run and three droplet runs, or None
    when a run diverged or the fit is degenerate."""
    if any(o["status"] != L.LBM_OK for o in obs4):
        return None
    flat, drops = obs4[0], obs4[1:]
    inv_r = np.array([1.0 / d["radius"] for d in drops])
    dp = np.array([d["dp"] for d in drops])
    if not (np.all(np.isfinite(inv_r)) and np.all(np.isfinite(dp))):
        return None
    A = np.column_stack([inv_r, np.ones_like(inv_r)])
    sigma, _ = np.linalg.lstsq(A, dp, rcond=None)[0]
    y = (flat["rho_l"], flat["rho_v"], flat["width"], sigma)
    if not (all(np.isfinite(y)) and flat["rho_v"] > 0 and sigma > 0):
        return None
    return y


def _collect(sets, owner, obs):
    per = [[] for _ in sets]
    for i, o in zip(owner, obs):
        per[i].append(o)
    Y = np.full((len(sets), 4), np.nan)
    ok = np.zeros(len(sets), dtype=bool)
    for i, o4 in enumerate(per):
        if len(o4) == LATTICES_PER_SET:
            y = targets_from_observables(o4)
            if y is not None:
                Y[i] = y
                ok[i] = True
    return Y, ok


def calibrate_batched(sets, chunk=1000, steps_flat=STEPS_FLAT, steps_droplet=STEPS_DROPLET):
    """Calibrate every set with batched sweeps of ``chunk`` sets (4 lattices each).
    Returns (Y n x 4 with NaN rows where a run failed, ok mask, seconds, lattice count)."""
    Y = np.full((len(sets), 4), np.nan)
    ok = np.zeros(len(sets), dtype=bool)
    t0 = time.perf_counter()
    count = 0
    for c0 in range(0, len(sets), chunk):
        part = sets[c0:c0 + chunk]
        specs, rhos, owner, _, _ = lattices(part, steps_flat, steps_droplet)
        if not specs:
            continue
        b = L.Batch(specs, rhos)
        b.run()
        obs = b.observables()
        b.close()
        count += len(specs)
        Yc, okc = _collect(part, owner, obs)
        Y[c0:c0 + len(part)] = Yc
        ok[c0:c0 + len(part)] = okc
    return Y, ok, time.perf_counter() - t0, count


def calibrate_plain(sets, steps_flat=STEPS_FLAT, steps_droplet=STEPS_DROPLET):
    """The same calibration, one lattice at a time through ``lbm_create``/``lbm_step``.
    Returns (Y, ok, seconds)."""
    t0 = time.perf_counter()
    specs, rhos, owner, _, _ = lattices(sets, steps_flat, steps_droplet)
    obs = []
    for s, r in zip(specs, rhos):
        ctx = L.Context(s["params"], s["nx"], s["ny"])
        ctx.set_density(r)
        ctx.step(s["nsteps"])
        obs.append(ctx.observables(s["geometry"]))
        ctx.close()
    Y, ok = _collect(sets, owner, obs)
    return Y, ok, time.perf_counter() - t0


def theory(sets) -> np.ndarray:
    """The method without a network (Appendix B, Eqs. S44, S46): Maxwell rho_l and rho_v,
    the continuum width and surface tension of the pseudopotential profile."""
    out = np.full((len(sets), 4), np.nan)
    for i, (st, rp, th) in enumerate(L.lbm_resolve_params_many([set_params(s) for s in sets])):
        if st == L.LBM_OK:
            out[i] = (th.rho_l, th.rho_v, th.width, th.gamma)
    return out


def relative_errors(P, Y):
    return np.abs(P / Y - 1.0)


DEFAULT_TRAIN = dict(iterations=30000, lr=2e-3, lr_min=1e-5)


def fit_surrogate(X, Y, seed=0, **train_cfg):
    """Standardise on (X, Y), create a surrogate and train it; returns (surrogate, final loss,
    seconds)."""
    cfg = dict(DEFAULT_TRAIN)
    cfg.update(train_cfg)
    m = L.Surrogate(L.Surrogate.standardisation(X, Y), seed=seed)
    t0 = time.perf_counter()
    loss = m.train(X, Y, **cfg)
    return m, loss, time.perf_counter() - t0
