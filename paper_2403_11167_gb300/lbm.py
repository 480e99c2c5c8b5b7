"""Thin ctypes binding of ``liblbm.so`` (the C ABI of ``include/lbm.h``).

Argument marshalling only: every step of the method runs in the library's CUDA
kernels.  Functions keep the C names.  ``Context`` is a convenience owner of a
``lbm_ctx*`` whose device workspace is a PyTorch tensor (PyTorch provides device
memory and the stream; nothing else).

The library must have been built (``python -m paper_2403_11167_gb300.build`` or
``__graft_entry__.build()``); importing this module without it raises.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblbm.so")

LBM_OK = 0
LBM_ERR_ARG = -1
LBM_ERR_UNSUPPORTED = -2
LBM_ERR_CUDA = -3
LBM_ERR_DIVERGED = -4
LBM_ERR_TIMEOUT = -5
LBM_ERR_NOCONVERGE = -6
LBM_ERR_STATE = -7
LBM_ERR_IO = -8

LBM_PSEUDOPOTENTIAL = 0
LBM_FREE_ENERGY = 1
LBM_F32 = 0
LBM_F64 = 1
LBM_BC_PERIODIC = 0
LBM_BC_WALL_ZOUHE = 1
LBM_BC_WALL_ZOUHE_ONESIDED = 2
FLAT = 0
DROPLET = 1


class lbm_params(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int), ("precision", ctypes.c_int)] + [
        (n, ctypes.c_double) for n in (
            "a", "b", "R", "Tr", "tau_nu", "tau_e", "tau_zeta", "tau_q", "tau_j",
            "kappa_P", "kappa_Li", "sigma_Li", "match_kappa", "kappa", "A", "body_fx", "body_fy")]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class lbm_thermo(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in
                ("T", "Tc", "rho_c", "p_c", "rho_v", "rho_l", "p0", "eps", "width", "gamma")]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class lbm_batch_lattice(ctypes.Structure):
    pass


class lbm_obs(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("rho_l", "rho_v", "width", "dp", "u_max", "mass", "radius")] + [
        ("step", ctypes.c_longlong), ("status", ctypes.c_int), ("pad_", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad_"}


class lbm_train_cfg(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int)] + [(n, ctypes.c_float) for n in (
        "lr", "lr_min", "beta1", "beta2", "eps", "weight_decay")]


lbm_batch_lattice._fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("geometry", ctypes.c_int),
                              ("pad_", ctypes.c_int), ("nsteps", ctypes.c_longlong), ("params", lbm_params)]


class LBMError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        msg = f"{what}: {lbm_strerror(code)} ({code})"
        if code == LBM_ERR_CUDA:
            msg += " -- " + " ".join(getattr(_lib(), f)().decode() for f in (
                "lbm_last_cuda_error", "lbm_batch_last_error", "lbm_surrogate_last_error"))
        super().__init__(msg)


_L = None


def _lib():
    global _L
    if _L is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2403_11167_gb300.build` "
                               "(the library has no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        P, T, O = ctypes.POINTER(lbm_params), ctypes.POINTER(lbm_thermo), ctypes.POINTER(lbm_obs)
        dp, vp = ctypes.POINTER(ctypes.c_double), ctypes.c_void_p
        fp = ctypes.POINTER(ctypes.c_float)
        sig = {
            "lbm_params_default": ([ctypes.c_int, P], ctypes.c_int),
            "lbm_resolve_params": ([P, P, T], ctypes.c_int),
            "lbm_workspace_bytes": ([ctypes.c_int, ctypes.c_int, ctypes.c_int], ctypes.c_size_t),
            "lbm_create": ([P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp, ctypes.c_size_t,
                            ctypes.POINTER(vp)], ctypes.c_int),
            "lbm_derived": ([vp, P, T], ctypes.c_int),
            "lbm_set_density": ([vp, dp], ctypes.c_int),
            "lbm_set_drive": ([vp, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_longlong],
                              ctypes.c_int),
            "lbm_set_gravity": ([vp, ctypes.c_double, ctypes.c_double, ctypes.c_double], ctypes.c_int),
            "lbm_set_density_device": ([vp, vp], ctypes.c_int),
            "lbm_set_populations": ([vp, dp], ctypes.c_int),
            "lbm_get_populations": ([vp, dp], ctypes.c_int),
            "lbm_step": ([vp, ctypes.c_longlong], ctypes.c_int),
            "lbm_observables": ([vp, ctypes.c_int, O], ctypes.c_int),
            "lbm_get_fields": ([vp, dp, dp, dp], ctypes.c_int),
            "lbm_get_populations_at": ([vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), dp],
                                       ctypes.c_int),
            "lbm_device_populations": ([vp, ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_longlong)], ctypes.c_int),
            "lbm_observables_fields_static": ([ctypes.c_int, vp, vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                               ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                               ctypes.c_int, vp, vp], ctypes.c_int),
            "lbm_save": ([vp, ctypes.c_char_p], ctypes.c_int),
            "lbm_load": ([vp, ctypes.c_char_p], ctypes.c_int),
            "lbm_stream": ([vp], vp),
            "lbm_destroy": ([vp], None),
            "lbm_strerror": ([ctypes.c_int], ctypes.c_char_p),
            "lbm_build_info": ([], ctypes.c_char_p),
            "lbm_last_cuda_error": ([], ctypes.c_char_p),
            "lbm_batch_create": ([ctypes.c_int, ctypes.POINTER(lbm_batch_lattice),
                                  ctypes.POINTER(ctypes.POINTER(ctypes.c_double)), ctypes.POINTER(vp)], ctypes.c_int),
            "lbm_batch_run": ([vp], ctypes.c_int),
            "lbm_batch_observables": ([vp, O], ctypes.c_int),
            "lbm_batch_populations": ([vp, ctypes.c_int, dp], ctypes.c_int),
            "lbm_batch_info": ([vp] + [ctypes.POINTER(ctypes.c_int)] * 4, ctypes.c_int),
            "lbm_batch_stream": ([vp], vp),
            "lbm_batch_destroy": ([vp], None),
            "lbm_batch_last_error": ([], ctypes.c_char_p),
            "lbm_selftest_bounded_wait": ([ctypes.c_int, ctypes.c_int], ctypes.c_int),
            "lbm_resolve_params_many": ([ctypes.c_int, P, P, T, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
            "lbm_kelvin_2d": ([ctypes.c_double] * 6 + [dp, dp], ctypes.c_int),
            "lbm_surrogate_num_params": ([], ctypes.c_int),
            "lbm_surrogate_create": ([fp, ctypes.c_uint, ctypes.POINTER(vp)], ctypes.c_int),
            "lbm_surrogate_stats": ([vp, fp], ctypes.c_int),
            "lbm_surrogate_set_params": ([vp, fp], ctypes.c_int),
            "lbm_surrogate_get_params": ([vp, fp], ctypes.c_int),
            "lbm_surrogate_loss_grad": ([vp, fp, fp, ctypes.c_int, fp, fp], ctypes.c_int),
            "lbm_surrogate_train": ([vp, fp, fp, ctypes.c_int, ctypes.POINTER(lbm_train_cfg), fp], ctypes.c_int),
            "lbm_surrogate_predict": ([vp, fp, ctypes.c_int, fp, ctypes.c_int], ctypes.c_int),
            "lbm_surrogate_predict_device": ([vp, vp, ctypes.c_int, vp, ctypes.c_int, vp], ctypes.c_int),
            "lbm_surrogate_predict_fp32": ([vp, fp, ctypes.c_int, fp], ctypes.c_int),
            "lbm_surrogate_destroy": ([vp], None),
            "lbm_surrogate_last_error": ([], ctypes.c_char_p),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _L = L
    return _L


def lib():
    return _lib()


def _check(rc, what):
    if rc != LBM_OK:
        raise LBMError(rc, what)


def _dptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def lbm_strerror(code: int) -> str:
    return _lib().lbm_strerror(code).decode()


def lbm_build_info() -> str:
    return _lib().lbm_build_info().decode()


def lbm_params_default(model: int, **overrides) -> lbm_params:
    p = lbm_params()
    _check(_lib().lbm_params_default(model, ctypes.byref(p)), "lbm_params_default")
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def lbm_resolve_params(p: lbm_params):
    out, th = lbm_params(), lbm_thermo()
    _check(_lib().lbm_resolve_params(ctypes.byref(p), ctypes.byref(out), ctypes.byref(th)), "lbm_resolve_params")
    return out, th


LBM_STATIC_MAX_BLOCKS = 1024


def lbm_observables_fields_static(precision, rho_ptr, ux_ptr, uy_ptr, nx, ny, geometry, a, b, R, T, nblocks,
                                  out_ptr, stream_ptr):
    """Marshal raw device pointers to the no-allocation observables entry point."""
    return _lib().lbm_observables_fields_static(precision, ctypes.c_void_p(rho_ptr), ctypes.c_void_p(ux_ptr),
                                                ctypes.c_void_p(uy_ptr), nx, ny, geometry, a, b, R, T, nblocks,
                                                ctypes.c_void_p(out_ptr), ctypes.c_void_p(stream_ptr))


def lbm_workspace_bytes(precision: int, nx: int, ny: int) -> int:
    return int(_lib().lbm_workspace_bytes(precision, nx, ny))


class Context:
    """Owner of one ``lbm_ctx``.  The workspace is a torch uint8 CUDA tensor and the
    stream a torch stream (its handle is passed to the library)."""

    def __init__(self, params: lbm_params, nx: int, ny: int, stream=None, device="cuda", walls=False):
        """walls: False (periodic in y), True or LBM_BC_WALL_ZOUHE (no-slip Zou-He walls on rows 0
        and ny-1), or LBM_BC_WALL_ZOUHE_ONESIDED (the same walls with the free-energy model's
        one-sided wall-normal chemical-potential gradient)."""
        import torch

        self.nx, self.ny = nx, ny
        self.torch = torch
        nbytes = lbm_workspace_bytes(params.precision, nx, ny)
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
        base = self.workspace.data_ptr()
        aligned = (base + 255) & ~255
        self.stream = stream if stream is not None else torch.cuda.Stream(device=device)
        handle = ctypes.c_void_p()
        rc = _lib().lbm_create(ctypes.byref(params), nx, ny, LBM_BC_PERIODIC,
                               (LBM_BC_WALL_ZOUHE if walls is True else int(walls)) if walls else LBM_BC_PERIODIC,
                               ctypes.c_void_p(self.stream.cuda_stream), ctypes.c_void_p(aligned),
                               ctypes.c_size_t(nbytes), ctypes.byref(handle))
        _check(rc, "lbm_create")
        self.h = handle

    def close(self):
        if getattr(self, "h", None):
            _lib().lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def derived(self):
        p, th = lbm_params(), lbm_thermo()
        _check(_lib().lbm_derived(self.h, ctypes.byref(p), ctypes.byref(th)), "lbm_derived")
        return p, th

    def set_density(self, rho0: np.ndarray):
        rho0 = np.ascontiguousarray(rho0, dtype=np.float64)
        assert rho0.shape == (self.ny, self.nx)
        _check(_lib().lbm_set_density(self.h, _dptr(rho0)), "lbm_set_density")

    def set_density_device(self, rho0_tensor):
        _check(_lib().lbm_set_density_device(self.h, ctypes.c_void_p(rho0_tensor.data_ptr())),
               "lbm_set_density_device")

    def set_populations(self, f: np.ndarray):
        f = np.ascontiguousarray(f, dtype=np.float64)
        assert f.shape == (9, self.ny, self.nx)
        _check(_lib().lbm_set_populations(self.h, _dptr(f)), "lbm_set_populations")

    def populations(self) -> np.ndarray:
        f = np.zeros((9, self.ny, self.nx))
        _check(_lib().lbm_get_populations(self.h, _dptr(f)), "lbm_get_populations")
        return f

    def populations_at(self, xs, ys) -> np.ndarray:
        xs = np.ascontiguousarray(xs, dtype=np.int32)
        ys = np.ascontiguousarray(ys, dtype=np.int32)
        out = np.zeros((len(xs), 9))
        ip = ctypes.POINTER(ctypes.c_int)
        _check(_lib().lbm_get_populations_at(self.h, len(xs), xs.ctypes.data_as(ip), ys.ctypes.data_as(ip),
                                             _dptr(out)), "lbm_get_populations_at")
        return out

    def set_drive(self, ax_lo: float, ax_hi: float, x_split: float, t_on: int):
        """Droplet-collision drive of Sec. 5.4 (lbm_set_drive)."""
        _check(_lib().lbm_set_drive(self.h, float(ax_lo), float(ax_hi), float(x_split), int(t_on)), "lbm_set_drive")

    def set_gravity(self, g: float, rho_ref: float, y_ref: float = 0.0):
        """Free-energy gravity of Eqs. (20)-(21) (lbm_set_gravity)."""
        _check(_lib().lbm_set_gravity(self.h, float(g), float(rho_ref), float(y_ref)), "lbm_set_gravity")

    def step(self, n: int):
        _check(_lib().lbm_step(self.h, int(n)), "lbm_step")

    def observables(self, geometry: int = FLAT) -> dict:
        o = lbm_obs()
        rc = _lib().lbm_observables(self.h, geometry, ctypes.byref(o))
        if rc not in (LBM_OK, LBM_ERR_DIVERGED):
            _check(rc, "lbm_observables")
        return o.as_dict()

    def fields(self):
        n = self.nx * self.ny
        rho, ux, uy = (np.zeros(n) for _ in range(3))
        _check(_lib().lbm_get_fields(self.h, _dptr(rho), _dptr(ux), _dptr(uy)), "lbm_get_fields")
        s = (self.ny, self.nx)
        return rho.reshape(s), ux.reshape(s), uy.reshape(s)

    def device_populations(self):
        p = ctypes.c_void_p()
        pitch = ctypes.c_longlong()
        _check(_lib().lbm_device_populations(self.h, ctypes.byref(p), ctypes.byref(pitch)), "lbm_device_populations")
        return p.value, pitch.value

    def save(self, path: str):
        _check(_lib().lbm_save(self.h, path.encode()), "lbm_save")

    def load(self, path: str):
        _check(_lib().lbm_load(self.h, path.encode()), "lbm_load")

    def synchronize(self):
        self.stream.synchronize()


class Batch:
    """Owner of one ``lbm_batch`` (batched pseudopotential calibration sweep)."""

    def __init__(self, specs, rho0s):
        n = len(specs)
        arr = (lbm_batch_lattice * n)()
        self._keep = []
        ptrs = (ctypes.POINTER(ctypes.c_double) * n)()
        self.shapes = []
        for i, (s, r) in enumerate(zip(specs, rho0s)):
            arr[i].nx, arr[i].ny, arr[i].geometry = s["nx"], s["ny"], s["geometry"]
            arr[i].nsteps = s["nsteps"]
            arr[i].params = s["params"]
            r = np.ascontiguousarray(r, dtype=np.float64)
            assert r.shape == (s["ny"], s["nx"])
            self._keep.append(r)
            ptrs[i] = _dptr(r)
            self.shapes.append((s["ny"], s["nx"]))
        h = ctypes.c_void_p()
        _check(_lib().lbm_batch_create(n, arr, ptrs, ctypes.byref(h)), "lbm_batch_create")
        self.h = h
        self.n = n

    def run(self):
        _check(_lib().lbm_batch_run(self.h), "lbm_batch_run")

    def observables(self):
        out = (lbm_obs * self.n)()
        _check(_lib().lbm_batch_observables(self.h, out), "lbm_batch_observables")
        return [o.as_dict() for o in out]

    def populations(self, i):
        ny, nx = self.shapes[i]
        f = np.zeros((9, ny, nx))
        _check(_lib().lbm_batch_populations(self.h, i, _dptr(f)), "lbm_batch_populations")
        return f

    def info(self):
        vals = [ctypes.c_int() for _ in range(4)]
        _check(_lib().lbm_batch_info(self.h, *[ctypes.byref(v) for v in vals]), "lbm_batch_info")
        return dict(zip(("n_resident", "n_items", "resident_threads", "strip_rows"), [v.value for v in vals]))

    def synchronize(self):
        import torch

        torch.cuda.synchronize()

    def close(self):
        if getattr(self, "h", None):
            _lib().lbm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sweep_specs(entries, precision=LBM_F32):
    """lbm_batch_lattice-ready dicts (with resolved Maxwell densities) from
    ``inputs.calibration_sweep`` entries; the initial densities come from ``inputs``."""
    from . import inputs

    specs, rhos = [], []
    for e in entries:
        p = lbm_params_default(LBM_PSEUDOPOTENTIAL, precision=precision, a=e["a"], Tr=e["Tr"], tau_nu=e["tau"],
                               kappa_P=e["kappa_P"])
        _, th = lbm_resolve_params(p)
        specs.append(dict(nx=e["nx"], ny=e["ny"], geometry=e["geometry"], nsteps=e["nsteps"], params=p))
        rhos.append(inputs.sweep_density(e, th.rho_v, th.rho_l))
    return specs, rhos


def lbm_kelvin_2d(a, b, R, T, gamma, radius, rho_v0, rho_l0):
    """Consistent (rho_v, rho_l) of a 2-D droplet (equal mu, Laplace jump gamma / radius)."""
    rv, rl = ctypes.c_double(rho_v0), ctypes.c_double(rho_l0)
    _check(_lib().lbm_kelvin_2d(a, b, R, T, gamma, radius, ctypes.byref(rv), ctypes.byref(rl)), "lbm_kelvin_2d")
    return rv.value, rl.value


def lbm_resolve_params_many(params_list):
    """``lbm_resolve_params`` over a list on all host cores; returns [(status, params, thermo)]."""
    n = len(params_list)
    if n == 0:
        return []
    inp, outp, th = (lbm_params * n)(*params_list), (lbm_params * n)(), (lbm_thermo * n)()
    st = (ctypes.c_int * n)()
    _check(_lib().lbm_resolve_params_many(n, inp, outp, th, st), "lbm_resolve_params_many")
    return [(st[i], outp[i], th[i]) for i in range(n)]


def _fptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def _f32(a, cols=4):
    a = np.ascontiguousarray(a, dtype=np.float32)
    if a.ndim != 2 or a.shape[1] != cols:
        raise ValueError(f"expected an n x {cols} array, got {a.shape}")
    return a


SURROGATE_INPUTS = ("Tr", "a", "b", "kappa_P")
LBM_INFER_SPLIT_BF16 = 0
LBM_INFER_BF16 = 1
SURROGATE_OUTPUTS = ("rho_l", "rho_v", "width", "sigma")


class Surrogate:
    """Owner of one ``lbm_surrogate`` (the MLP calibration surrogate).

    X rows are (Tr, a, b, kappa_P); Y rows are (rho_l, rho_v, W, sigma)."""

    def __init__(self, stats16, seed=0):
        st = np.ascontiguousarray(stats16, dtype=np.float32).reshape(16)
        h = ctypes.c_void_p()
        _check(_lib().lbm_surrogate_create(_fptr(st), seed, ctypes.byref(h)), "lbm_surrogate_create")
        self.h = h
        self.n_params = _lib().lbm_surrogate_num_params()

    @staticmethod
    def standardisation(X, Y, weights=(1.0, 1.0, 1.0, 1.0)):
        """stats16 of a training set: mean/std of X and of (rho_l, ln rho_v, W, sigma).  An
        output's scale is its std / sqrt(weight), so the MSE weighs it by ``weight``."""
        X = np.asarray(X, dtype=np.float64)
        Yp = np.array(Y, dtype=np.float64)
        Yp[:, 1] = np.log(Yp[:, 1])
        sx, sy = X.std(0), np.nanstd(Yp, 0)
        sx[sx == 0] = 1.0
        sy[sy == 0] = 1.0
        sy = sy / np.sqrt(np.asarray(weights, dtype=np.float64))
        return np.concatenate([X.mean(0), sx, np.nanmean(Yp, 0), sy]).astype(np.float32)

    def stats(self):
        st = np.zeros(16, np.float32)
        _check(_lib().lbm_surrogate_stats(self.h, _fptr(st)), "lbm_surrogate_stats")
        return st

    def params(self):
        p = np.zeros(self.n_params, np.float32)
        _check(_lib().lbm_surrogate_get_params(self.h, _fptr(p)), "lbm_surrogate_get_params")
        return p

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.shape == (self.n_params,)
        _check(_lib().lbm_surrogate_set_params(self.h, _fptr(p)), "lbm_surrogate_set_params")

    def loss_grad(self, X, Y):
        X, Y = _f32(X), _f32(Y)
        loss = np.zeros(1, np.float32)
        g = np.zeros(self.n_params, np.float32)
        _check(_lib().lbm_surrogate_loss_grad(self.h, _fptr(X), _fptr(Y), len(X), _fptr(loss), _fptr(g)),
               "lbm_surrogate_loss_grad")
        return float(loss[0]), g

    def train(self, X, Y, iterations=20000, lr=2e-3, lr_min=2e-5, beta1=0.9, beta2=0.999, eps=1e-8,
              weight_decay=0.0):
        X, Y = _f32(X), _f32(Y)
        cfg = lbm_train_cfg(iterations, lr, lr_min, beta1, beta2, eps, weight_decay)
        loss = np.zeros(1, np.float32)
        _check(_lib().lbm_surrogate_train(self.h, _fptr(X), _fptr(Y), len(X), ctypes.byref(cfg), _fptr(loss)),
               "lbm_surrogate_train")
        return float(loss[0])

    def predict(self, X, mode=None):
        """Tensor-core inference (default: split-BF16 operands, FP32 accumulation)."""
        X = _f32(X)
        Y = np.zeros_like(X)
        mode = LBM_INFER_SPLIT_BF16 if mode is None else mode
        _check(_lib().lbm_surrogate_predict(self.h, _fptr(X), len(X), _fptr(Y), mode), "lbm_surrogate_predict")
        return Y

    def predict_fp32(self, X):
        X = _f32(X)
        Y = np.zeros_like(X)
        _check(_lib().lbm_surrogate_predict_fp32(self.h, _fptr(X), len(X), _fptr(Y)), "lbm_surrogate_predict_fp32")
        return Y

    def predict_device(self, X_dev, Y_dev, stream=None, mode=None):
        """Inference on device tensors (float32, n x 4, contiguous); asynchronous."""
        mode = LBM_INFER_SPLIT_BF16 if mode is None else mode
        _check(_lib().lbm_surrogate_predict_device(self.h, X_dev.data_ptr(), X_dev.shape[0], Y_dev.data_ptr(),
                                                   mode, stream), "lbm_surrogate_predict_device")

    def close(self):
        if getattr(self, "h", None):
            _lib().lbm_surrogate_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lbm_selftest_bounded_wait(arrive: bool, polls: int) -> int:
    """Status of one bounded device wait (LBM_OK or LBM_ERR_TIMEOUT); see include/lbm.h."""
    return _lib().lbm_selftest_bounded_wait(1 if arrive else 0, polls)
