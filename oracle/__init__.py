"""FP64 CPU oracle for the D2Q9 MP-LBM and IWB-FE-LBM time steps (arXiv:2403.11167).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` may import this package.  The
product library never imports, links or calls anything here, and this package
imports nothing from the product.

Contents
--------
``lbm_oracle.c`` (loaded here through ctypes)
    Plain cell-by-cell FP64 time step of both models with explicit 9x9 moment
    matrices: Eq. (1) with Eqs. (2)-(4), (6), (10), (11), (13), (20), (21),
    (24), (28)-(32) and the matrix of Eq. (S48).
``thermo.py``
    Carnahan-Starling thermodynamics, critical point, Maxwell construction,
    sigma^Li by the Newton/Simpson procedure of Appendix B, theoretical planar
    profiles and surface tensions (Eqs. 17, 26, S44, S46).
``planar.py``
    The discrete planar-interface relations of Appendices D and E
    (Eqs. S59/S60 and S75/S76) solved directly by Newton's method.
``brute.py``
    A second, NumPy-only literal implementation of one time step (whole-lattice
    array form) for brute-force cross-checks of the C oracle on tiny lattices.
``observables.py``
    Probe means, interface width, pressure jump and equimolar radius computed
    from oracle fields.
"""
import ctypes
import os

import numpy as np

from . import build as _build

PP = 0  # modified pseudopotential model (Sec. 4)
FE = 1  # improved well-balanced free-energy model (Sec. 2.2)


class Params(ctypes.Structure):
    """Mirror of ``orc_params`` in lbm_oracle.c."""

    _fields_ = [
        ("a", ctypes.c_double), ("b", ctypes.c_double), ("R", ctypes.c_double),
        ("T", ctypes.c_double), ("G", ctypes.c_double),
        ("tau_rho", ctypes.c_double), ("tau_e", ctypes.c_double),
        ("tau_zeta", ctypes.c_double), ("tau_j", ctypes.c_double),
        ("tau_q", ctypes.c_double), ("tau_nu", ctypes.c_double),
        ("kappa_P", ctypes.c_double), ("kappa_Li", ctypes.c_double),
        ("sigma_Li", ctypes.c_double), ("kappa", ctypes.c_double),
        ("fx", ctypes.c_double), ("fy", ctypes.c_double),
        ("walls", ctypes.c_double),
        ("drive", ctypes.c_double), ("drive_ax_lo", ctypes.c_double),
        ("drive_ax_hi", ctypes.c_double), ("drive_x_split", ctypes.c_double),
        ("A", ctypes.c_double), ("g", ctypes.c_double), ("rho_g", ctypes.c_double),
        ("y_ref", ctypes.c_double),
    ]


def make_params(**kw) -> Params:
    """Build oracle parameters; unspecified relaxation times default to 1, G to -1."""
    d = dict(a=0.5, b=4.0, R=1.0, T=0.0, G=-1.0, tau_rho=1.0, tau_e=1.0, tau_zeta=1.0,
             tau_j=1.0, tau_q=1.0, tau_nu=1.0, kappa_P=1.0, kappa_Li=0.0, sigma_Li=0.0,
             kappa=0.5, fx=0.0, fy=0.0, walls=0.0, drive=0.0, drive_ax_lo=0.0, drive_ax_hi=0.0,
             drive_x_split=0.0, A=0.0, g=0.0, rho_g=0.0, y_ref=0.0)
    unknown = set(kw) - set(d)
    if unknown:
        raise KeyError(f"unknown oracle parameter(s): {sorted(unknown)}")
    d.update(kw)
    return Params(**{k: float(v) for k, v in d.items()})


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        pp = ctypes.POINTER(Params)
        L.orc_run.argtypes = [ctypes.c_int, pp, ctypes.c_int, ctypes.c_int, dp, ctypes.c_long, ctypes.c_int]
        L.orc_run.restype = ctypes.c_long
        L.orc_init.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp]
        L.orc_init_iwb.argtypes = [pp, ctypes.c_int, ctypes.c_int, dp, dp]
        L.orc_feq_iwb.argtypes = [ctypes.c_double] * 8 + [dp]
        L.orc_macro.argtypes = [ctypes.c_int, pp, ctypes.c_int, ctypes.c_int, dp, dp, dp, dp, dp, dp, dp]
        L.orc_macro.restype = ctypes.c_int
        L.orc_feq.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp]
        L.orc_fe_forcing.argtypes = [ctypes.c_double] * 6 + [dp]
        L.orc_pp_sources.argtypes = [pp] + [ctypes.c_double] * 10 + [dp, dp]
        L.orc_q_tensor.argtypes = [pp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp]
        L.orc_stencils.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp]
        L.orc_p_eos.argtypes = [pp, ctypes.c_double]
        L.orc_p_eos.restype = ctypes.c_double
        L.orc_mu_bulk.argtypes = [pp, ctypes.c_double]
        L.orc_mu_bulk.restype = ctypes.c_double
        L.orc_moment_matrix.argtypes = [dp]
        L.orc_moment_matrix_inverse.argtypes = [dp]
        L.orc_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def moment_matrix() -> np.ndarray:
    out = np.zeros(81)
    lib().orc_moment_matrix(_ptr(out))
    return out.reshape(9, 9)


def moment_matrix_inverse() -> np.ndarray:
    out = np.zeros(81)
    lib().orc_moment_matrix_inverse(_ptr(out))
    return out.reshape(9, 9)


def init(model: int, rho0: np.ndarray) -> np.ndarray:
    """Populations f = f^eq(rho0, u = 0) of the model, shape (9, ny, nx)."""
    rho0 = np.ascontiguousarray(rho0, dtype=np.float64)
    ny, nx = rho0.shape
    f = np.zeros((9, ny, nx))
    lib().orc_init(model, nx, ny, _ptr(rho0), _ptr(f))
    return f


def feq_iwb(rho, ux, uy, pg=0.0, A=0.0, Sxx=0.0, Sxy=0.0, Syy=0.0) -> np.ndarray:
    """Eq. (20) in full at one cell (p_g, A and the strain rate S)."""
    out = np.zeros(9)
    lib().orc_feq_iwb(rho, ux, uy, pg, A, Sxx, Sxy, Syy, _ptr(out))
    return out


def init_iwb(p: Params, rho0: np.ndarray) -> np.ndarray:
    """Free-energy populations f = f^eq of Eq. (20) at rest with the gravitational reference
    pressure p_g = rho_0 g (y - y_ref) of p, shape (9, ny, nx)."""
    rho0 = np.ascontiguousarray(rho0, dtype=np.float64)
    ny, nx = rho0.shape
    f = np.zeros((9, ny, nx))
    lib().orc_init_iwb(ctypes.byref(p), nx, ny, _ptr(rho0), _ptr(f))
    return f


def run(model: int, p: Params, f: np.ndarray, nsteps: int, nthreads: int = 0) -> np.ndarray:
    """Advance a copy of f by nsteps; raises if the state becomes invalid."""
    f = np.array(f, dtype=np.float64, order="C", copy=True)
    _, ny, nx = f.shape
    done = lib().orc_run(model, ctypes.byref(p), nx, ny, _ptr(f), int(nsteps), int(nthreads))
    if done != nsteps:
        raise FloatingPointError(f"oracle state became invalid after {done} of {nsteps} steps")
    return f


def run_driven(model: int, p: Params, f: np.ndarray, nsteps: int, t0: int, t_on: int) -> np.ndarray:
    """Advance a state at time t0 by nsteps with the droplet-collision force of Sec. 5.4 (the
    drive_* fields of p) acting on the collisions of states at times t > t_on only."""
    import copy

    off = copy.copy(p)
    off.drive = 0.0
    on = copy.copy(p)
    on.drive = 1.0
    n_off = max(0, min(nsteps, t_on + 1 - t0))
    if n_off:
        f = run(model, off, f, n_off)
    if nsteps - n_off:
        f = run(model, on, f, nsteps - n_off)
    return f


def macro(model: int, p: Params, f: np.ndarray):
    """(rho, ux, uy, Fx, Fy, aux) with aux = psi (PP) or mu (FE)."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    _, ny, nx = f.shape
    outs = [np.zeros((ny, nx)) for _ in range(6)]
    rc = lib().orc_macro(model, ctypes.byref(p), nx, ny, _ptr(f), *[_ptr(o) for o in outs])
    if rc != 0:
        raise FloatingPointError("invalid state (rho <= 0 or negative psi radicand)")
    return tuple(outs)


def feq(model: int, rho: float, ux: float, uy: float) -> np.ndarray:
    out = np.zeros(9)
    lib().orc_feq(model, rho, ux, uy, _ptr(out))
    return out


def fe_forcing(ux, uy, Fx, Fy, gx, gy) -> np.ndarray:
    out = np.zeros(9)
    lib().orc_fe_forcing(ux, uy, Fx, Fy, gx, gy, _ptr(out))
    return out


def pp_sources(p: Params, ux, uy, Fx, Fy, Fix, Fiy, psi, Qxx, Qyy, Qxy):
    S = np.zeros(9)
    C = np.zeros(9)
    lib().orc_pp_sources(ctypes.byref(p), ux, uy, Fx, Fy, Fix, Fiy, psi, Qxx, Qyy, Qxy, _ptr(S), _ptr(C))
    return S, C


def q_tensor(p: Params, psi: np.ndarray, x: int, y: int) -> np.ndarray:
    psi = np.ascontiguousarray(psi, dtype=np.float64)
    ny, nx = psi.shape
    out = np.zeros(3)
    lib().orc_q_tensor(ctypes.byref(p), _ptr(psi), nx, ny, x, y, _ptr(out))
    return out


def stencils(phi: np.ndarray, x: int, y: int) -> np.ndarray:
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    ny, nx = phi.shape
    out = np.zeros(3)
    lib().orc_stencils(_ptr(phi), nx, ny, x, y, _ptr(out))
    return out


def p_eos(p: Params, rho: float) -> float:
    return lib().orc_p_eos(ctypes.byref(p), rho)


def mu_bulk(p: Params, rho: float) -> float:
    return lib().orc_mu_bulk(ctypes.byref(p), rho)


def num_threads() -> int:
    return lib().orc_num_threads()
