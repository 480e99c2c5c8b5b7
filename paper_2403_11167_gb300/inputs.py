"""Seeded synthetic initial density fields (the input recipes of the workloads).

This module holds no arithmetic of the lattice Boltzmann method: it only draws
or shapes initial densities, given the two bulk densities as arguments.  Both
the CUDA path and the FP64 oracle are fed from here.

Recipes (the paper initialises every run from f = f^eq(rho0, u = 0), Secs. 5.3-5.4):

* ``flat_slab`` -- liquid slab in the middle half of x, vapour elsewhere,
  rho(x) = rho_v + (rho_l - rho_v)/2 [tanh(2(x - nx/4)/W0) - tanh(2(x - 3nx/4)/W0)].
* ``droplet`` -- rho = (rho_l + rho_v)/2 - (rho_l - rho_v)/2 tanh(2(r - R)/W0),
  r measured from ((nx - 1)/2, (ny - 1)/2).
* ``spinodal_noise`` -- rho = rho_mean (1 + U(-amp, amp)), i.i.d. per cell from
  NumPy's PCG64 with the given seed (spinodal decomposition from a uniform state).
* ``random_field`` -- i.i.d. uniform densities in [lo, hi] (brute-force checks).
* ``plate_channel`` -- the parallel-plate channel of Sec. 5.3: vapour in the bottom half,
  liquid in the top half, rho(x, y) = rho_v + (rho_l - rho_v)/2 [1 + tanh(2(y - h(x))/W0)]
  with the interface at h(x) = (ny - 1)/2 + amp sin(2 pi x / nx) (amp = 0: the paper's flat
  interface; amp > 0 gives parity runs x-gradients).
* ``two_droplets`` -- the droplet pair of Sec. 5.4: rho = rho_v + (rho_l - rho_v)/2
  sum_k [1 - tanh(2(r_k - R)/W0)], r_k measured from each centre (well-separated droplets).
"""
import numpy as np


def flat_slab(nx: int, ny: int, rho_v: float, rho_l: float, w0: float = 5.0) -> np.ndarray:
    x = np.arange(nx, dtype=np.float64)
    x1, x2 = nx / 4.0, 3.0 * nx / 4.0
    prof = rho_v + 0.5 * (rho_l - rho_v) * (np.tanh(2.0 * (x - x1) / w0) - np.tanh(2.0 * (x - x2) / w0))
    return np.ascontiguousarray(np.broadcast_to(prof, (ny, nx)))


def droplet(nx: int, ny: int, radius: float, rho_v: float, rho_l: float, w0: float = 5.0) -> np.ndarray:
    yy, xx = np.mgrid[0:ny, 0:nx].astype(np.float64)
    r = np.sqrt((xx - (nx - 1) / 2.0) ** 2 + (yy - (ny - 1) / 2.0) ** 2)
    return 0.5 * (rho_l + rho_v) - 0.5 * (rho_l - rho_v) * np.tanh(2.0 * (r - radius) / w0)


def spinodal_noise(nx: int, ny: int, rho_mean: float, amp: float = 0.01, seed: int = 2403) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return rho_mean * (1.0 + rng.uniform(-amp, amp, size=(ny, nx)))


def random_field(nx: int, ny: int, lo: float, hi: float, seed: int = 0) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(lo, hi, size=(ny, nx))


def plate_channel(nx: int, ny: int, rho_v: float, rho_l: float, w0: float = 5.0, amp: float = 0.0) -> np.ndarray:
    yy, xx = np.mgrid[0:ny, 0:nx].astype(np.float64)
    h = (ny - 1) / 2.0 + amp * np.sin(2.0 * np.pi * xx / nx)
    return rho_v + 0.5 * (rho_l - rho_v) * (1.0 + np.tanh(2.0 * (yy - h) / w0))


def two_droplets(nx: int, ny: int, centres, radius: float, rho_v: float, rho_l: float,
                 w0: float = 5.0) -> np.ndarray:
    yy, xx = np.mgrid[0:ny, 0:nx].astype(np.float64)
    rho = np.full((ny, nx), rho_v)
    for cx, cy in centres:
        r = np.sqrt((xx - cx) ** 2 + (yy - cy) ** 2)
        rho += 0.5 * (rho_l - rho_v) * (1.0 - np.tanh(2.0 * (r - radius) / w0))
    return rho


def calibration_sweep(n: int = 512, seed: int = 11167, step_range=(5000, 20000), w0: float = 5.0):
    """Seeded parameter sets of a pseudopotential calibration sweep (uneven lattices).

    Half flat slabs (nx in {64, 128, 256, 512}, ny = 4), half centred droplets on L x L
    lattices (L in {64, 128, 192, 256, 384, 512}, radius R ~ U[10, 80] redrawn until
    L >= 2R + 8 w0).  Tr ~ U[0.5, 0.95], width factor kappa_P in {0.4, 0.7, 1.0},
    tau ~ U[0.6, 1.2], steps ~ U{step_range}, a = 0.25, b = 4, R = 1.  Returns a list of
    dicts; the caller builds each initial density from the lattice's Maxwell densities
    with ``flat_slab`` / ``droplet``.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(n):
        flat = i % 2 == 0
        d = dict(a=0.25, Tr=float(rng.uniform(0.5, 0.95)), kappa_P=float(rng.choice([0.4, 0.7, 1.0])),
                 tau=float(rng.uniform(0.6, 1.2)),
                 nsteps=int(rng.integers(step_range[0], step_range[1] + 1)))
        if flat:
            d.update(geometry=0, nx=int(rng.choice([64, 128, 256, 512])), ny=4, radius=0.0)
        else:
            L = int(rng.choice([64, 128, 192, 256, 384, 512]))
            while True:
                R = float(rng.uniform(10.0, 80.0))
                if L >= 2 * R + 8 * w0:
                    break
            d.update(geometry=1, nx=L, ny=L, radius=R)
        out.append(d)
    return out


def sweep_density(spec: dict, rho_v: float, rho_l: float, w0: float = 5.0) -> np.ndarray:
    """Initial density of one sweep lattice (flat slab or droplet) from its bulk densities."""
    if spec["geometry"] == 0:
        return flat_slab(spec["nx"], spec["ny"], rho_v, rho_l, w0)
    return droplet(spec["nx"], spec["ny"], spec["radius"], rho_v, rho_l, w0)


def surrogate_sets(n: int, seed: int = 4032):
    """Seeded parameter sets (Tr, a, b, kappa_P) of surrogate calibration runs.

    Tr ~ U[0.5, 0.95], a ~ U[0.25, 0.5], b ~ U[3, 5], kappa_P uniform over {0.4, 0.7, 1.0};
    R = 1, tau = 1, kappa_Li = 0, sigma_Li from the Appendix-B theory.  Training sets use
    seed 4032, held-out sets seed 1116 (independent streams).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    Tr = rng.uniform(0.5, 0.95, n)
    a = rng.uniform(0.25, 0.5, n)
    b = rng.uniform(3.0, 5.0, n)
    kP = rng.choice([0.4, 0.7, 1.0], n)
    return [dict(Tr=float(Tr[i]), a=float(a[i]), b=float(b[i]), kappa_P=float(kP[i])) for i in range(n)]
