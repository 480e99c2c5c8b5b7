"""Calibration runs of the pseudopotential model and the learned surrogate built on them.

The pseudopotential model fixes its parameters against preliminary simulations (Secs. 3,
5.1, 5.2).  One calibration of a parameter set (Tr, a, b, kappa_P; R = 1, tau = 1,
kappa_Li = 0, sigma_Li from the Appendix-B theory) here is four lattices:

* a flat interface, 256 x 4, 40,000 steps: rho_l, rho_v and the tangent width W; the same
  slab run 10,000 steps longer checks that these are stationary;
* three centred droplets measured in units of l = max(W_th, 4), W_th the continuum width of
  Eq. (S44): radii 3l, 4l, 5l on an L x L lattice, L = 16 l rounded up to a multiple of 8,
  for 7000 (L / 64)^2 steps (the slowest transient, viscous relaxation, scales with L^2).
  The pressure jump dp against the inverse equimolar radius gives the surface tension
  sigma as the least-squares slope with an intercept (2-D Laplace law, dp = sigma / R).

A set is valid when its flat runs are finite and stationary (rho_l and rho_v agree to
1e-3 and W to 5e-3 between the two run lengths); otherwise it gives no targets.  Its
sigma is valid when the three droplets are quasi-static (spurious velocity u_max <= 0.005),
each equimolar radius is within 20% of its initial radius and the slope is positive;
otherwise sigma is missing (NaN) and the set still supplies rho_l, rho_v and W.  (Thin
interfaces, kappa_P = 0.4, carry large spurious currents: their droplets mostly diverge
and some of their slabs never settle.  Wide interfaces, Tr > 0.9, need the large lattices
the width scaling gives them.)

``calibrate_batched`` runs many sets as ``lbm_batch`` sweeps; ``calibrate_plain`` runs the
same lattices one ``lbm_ctx`` at a time (the plain calibration, the reference of the surrogate).
Both are bitwise the same computation.  ``fit_surrogate`` trains the MLP on the GPU.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import inputs
from . import lbm as L

FLAT_NX, FLAT_NY = 256, 4
STEPS_FLAT = 40000
STEPS_FLAT_CHECK = 10000       # extra steps of the stationarity run
STATIONARY_RHO = 1e-3
STATIONARY_W = 5e-3
DROP_U_MAX = 0.005
DROP_UNIT_MIN = 4.0
DROP_RADII = (3.0, 4.0, 5.0)   # in units of l
DROP_L = 16.0                  # lattice side in units of l
DROP_STEPS_64 = 7000           # steps of a 64 x 64 droplet lattice
LATTICES_PER_SET = 2 + len(DROP_RADII)
RADIUS_TOLERANCE = 0.2


def droplet_geometry(width_theory, steps_64=DROP_STEPS_64):
    """(L, radii, steps) of the droplet runs of a set whose continuum width is width_theory."""
    l = max(float(width_theory), DROP_UNIT_MIN)
    Lx = int(math.ceil(DROP_L * l / 8.0) * 8)
    steps = int(round(steps_64 * (Lx / 64.0) ** 2))
    return Lx, tuple(r * l for r in DROP_RADII), steps


def set_params(s) -> "L.lbm_params":
    return L.lbm_params_default(L.LBM_PSEUDOPOTENTIAL, a=s["a"], b=s["b"], Tr=s["Tr"], kappa_P=s["kappa_P"],
                                tau_nu=1.0, kappa_Li=0.0)


def features(sets) -> np.ndarray:
    """Network inputs (Tr, a, b, kappa_P), one row per set."""
    return np.array([[s[k] for k in L.SURROGATE_INPUTS] for s in sets], dtype=np.float64)


def lattices(sets, steps_flat=STEPS_FLAT, steps_64=DROP_STEPS_64):
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
        for n in (steps_flat, steps_flat + STEPS_FLAT_CHECK):
            specs.append(dict(nx=FLAT_NX, ny=FLAT_NY, geometry=L.FLAT, nsteps=n, params=rp))
            rhos.append(inputs.flat_slab(FLAT_NX, FLAT_NY, th.rho_v, th.rho_l))
            owner.append(i)
        Lx, radii, steps = droplet_geometry(th.width, steps_64)
        for R in radii:
            specs.append(dict(nx=Lx, ny=Lx, geometry=L.DROPLET, nsteps=steps, params=rp, radius=R))
            rhos.append(inputs.droplet(Lx, Lx, R, th.rho_v, th.rho_l))
            owner.append(i)
    return specs, rhos, owner, status, derived


def targets_from_observables(obs5, radii0):
    """(rho_l, rho_v, W, sigma) of one set from its two flat runs and three droplet runs
    (initial radii radii0); None when the flat runs are invalid or not stationary, sigma NaN
    when the droplets are invalid."""
    flat, later, drops = obs5[0], obs5[1], obs5[2:]
    y = [flat["rho_l"], flat["rho_v"], flat["width"], math.nan]
    for f in (flat, later):
        if f["status"] != L.LBM_OK or not all(np.isfinite([f["rho_l"], f["rho_v"], f["width"]])) or not f["rho_v"] > 0:
            return None
    if (abs(later["rho_l"] / flat["rho_l"] - 1) > STATIONARY_RHO or abs(later["rho_v"] / flat["rho_v"] - 1) >
            STATIONARY_RHO or abs(later["width"] / flat["width"] - 1) > STATIONARY_W):
        return None
    ok = all(d["status"] == L.LBM_OK and np.isfinite(d["dp"]) and np.isfinite(d["radius"]) and
             d["u_max"] <= DROP_U_MAX and abs(d["radius"] / r0 - 1.0) <= RADIUS_TOLERANCE
             for d, r0 in zip(drops, radii0))
    if ok:
        inv_r = np.array([1.0 / d["radius"] for d in drops])
        dp = np.array([d["dp"] for d in drops])
        A = np.column_stack([inv_r, np.ones_like(inv_r)])
        sigma = float(np.linalg.lstsq(A, dp, rcond=None)[0][0])
        if sigma > 0:
            y[3] = sigma
    return tuple(y)


def _collect(sets, specs, owner, obs):
    per = [[] for _ in sets]
    r0 = [[] for _ in sets]
    for sp, i, o in zip(specs, owner, obs):
        per[i].append(o)
        if sp["geometry"] == L.DROPLET:
            r0[i].append(sp["radius"])
    Y = np.full((len(sets), 4), np.nan)
    ok = np.zeros(len(sets), dtype=bool)
    for i, o4 in enumerate(per):
        if len(o4) == LATTICES_PER_SET:
            y = targets_from_observables(o4, r0[i])
            if y is not None:
                Y[i] = y
                ok[i] = True
    return Y, ok


OBS_FIELDS = ("rho_l", "rho_v", "width", "dp", "u_max", "mass", "radius", "status")


def raw_table(specs, owner, obs):
    """Per-lattice record (set index, geometry, initial radius, side, steps, observables)."""
    rows = []
    for sp, i, o in zip(specs, owner, obs):
        rows.append([i, sp["geometry"], sp.get("radius", 0.0), sp["nx"], sp["nsteps"]] + [o[k] for k in OBS_FIELDS])
    return np.array(rows, dtype=np.float64).reshape(-1, 5 + len(OBS_FIELDS))


def calibrate_batched(sets, chunk=2000, steps_flat=STEPS_FLAT, steps_64=DROP_STEPS_64):
    """Calibrate every set with batched sweeps of ``chunk`` sets (4 lattices each).  Returns a
    dict: Y (n x 4; NaN rows where the flat run is invalid, NaN sigma where the droplets are),
    ok (valid flat runs), seconds, lattices, updates (lattice site updates), raw (per-lattice
    table of ``raw_table``)."""
    Y = np.full((len(sets), 4), np.nan)
    ok = np.zeros(len(sets), dtype=bool)
    raws = []
    t0 = time.perf_counter()
    count = updates = 0
    for c0 in range(0, len(sets), chunk):
        part = sets[c0:c0 + chunk]
        specs, rhos, owner, _, _ = lattices(part, steps_flat, steps_64)
        if not specs:
            continue
        b = L.Batch(specs, rhos)
        b.run()
        obs = b.observables()
        b.close()
        count += len(specs)
        updates += sum(sp["nx"] * sp["ny"] * sp["nsteps"] for sp in specs)
        Yc, okc = _collect(part, specs, owner, obs)
        Y[c0:c0 + len(part)] = Yc
        ok[c0:c0 + len(part)] = okc
        raw = raw_table(specs, owner, obs)
        raw[:, 0] += c0
        raws.append(raw)
    raw = np.concatenate(raws) if raws else np.zeros((0, 5 + len(OBS_FIELDS)))
    return dict(Y=Y, ok=ok, seconds=time.perf_counter() - t0, lattices=count, updates=updates, raw=raw)


def calibrate_plain(sets, steps_flat=STEPS_FLAT, steps_64=DROP_STEPS_64):
    """The same calibration, one lattice at a time through ``lbm_create``/``lbm_step``.
    Returns the dict of ``calibrate_batched``."""
    t0 = time.perf_counter()
    specs, rhos, owner, _, _ = lattices(sets, steps_flat, steps_64)
    obs = []
    for s, r in zip(specs, rhos):
        ctx = L.Context(s["params"], s["nx"], s["ny"])
        ctx.set_density(r)
        ctx.step(s["nsteps"])
        obs.append(ctx.observables(s["geometry"]))
        ctx.close()
    Y, ok = _collect(sets, specs, owner, obs)
    return dict(Y=Y, ok=ok, seconds=time.perf_counter() - t0, lattices=len(specs),
                updates=sum(sp["nx"] * sp["ny"] * sp["nsteps"] for sp in specs), raw=raw_table(specs, owner, obs))


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


DEFAULT_TRAIN = dict(iterations=60000, lr=2e-3, lr_min=1e-6, weight_decay=1e-5)
# rho_v carries the tightest error target relative to its spread (ln rho_v spans ~5 units)
LOSS_WEIGHTS = (1.0, 4.0, 1.0, 1.0)


def fit_surrogate(X, Y, seed=0, weights=LOSS_WEIGHTS, **train_cfg):
    """Standardise on (X, Y) with the output weights, create a surrogate and train it on the
    GPU; returns (surrogate, final loss, seconds)."""
    cfg = dict(DEFAULT_TRAIN)
    cfg.update(train_cfg)
    m = L.Surrogate(L.Surrogate.standardisation(X, Y, weights), seed=seed)
    t0 = time.perf_counter()
    loss = m.train(X, Y, **cfg)
    return m, loss, time.perf_counter() - t0


class SurrogateCalibration:
    """Calibration with the trained surrogate and the plain calibration runs as its fallback.

    The surrogate answers a parameter set only inside the domain it was trained on: Tr, a
    and b within the ranges of the valid training sets, kappa_P one of the trained values.
    Its sigma is used only for kappa_P values where at least ``min_sigma_fraction`` of the
    valid training sets had a measurable sigma (thin interfaces, kappa_P = 0.4, mostly have
    none).  Every other set is calibrated by running its lattices (``calibrate_batched``,
    bitwise the plain one-lattice-at-a-time calibration), and its whole row comes from that
    run.
    """

    def __init__(self, surrogate, X_train, Y_train, ok_train, min_sigma_fraction=0.5):
        X = np.asarray(X_train, dtype=np.float64)[ok_train]
        Y = np.asarray(Y_train, dtype=np.float64)[ok_train]
        self.m = surrogate
        self.lo = X[:, :3].min(axis=0)
        self.hi = X[:, :3].max(axis=0)
        self.kappas = np.unique(X[:, 3])
        self.sigma_ok = {float(k): float(np.isfinite(Y[X[:, 3] == k, 3]).mean()) >= min_sigma_fraction
                         for k in self.kappas}

    def inside(self, X):
        X = np.asarray(X, dtype=np.float64)
        in_box = np.all((X[:, :3] >= self.lo) & (X[:, :3] <= self.hi), axis=1)
        known = np.isin(X[:, 3], self.kappas)
        with_sigma = np.array([self.sigma_ok.get(float(k), False) for k in X[:, 3]])
        return in_box & known & with_sigma

    def calibrate(self, sets):
        """(Y n x 4, source: 'surrogate' or 'calibration' per set)."""
        X = features(sets)
        use = self.inside(X)
        Y = np.full((len(sets), 4), np.nan)
        if use.any():
            Y[use] = self.m.predict(X[use])
        rest = [s for s, u in zip(sets, use) if not u]
        if rest:
            Y[~use] = calibrate_batched(rest)["Y"]
        return Y, np.where(use, "surrogate", "calibration")
