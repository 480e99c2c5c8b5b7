"""CPU checks of the C ABI library: it loads, exports every declared symbol, and its
host-only parameter derivation agrees with the oracle's thermodynamics."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

from conftest import ROOT
from oracle import thermo


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2403_11167_gb300 import lbm

    return lbm


def _declared_functions():
    names = set()
    for hdr in os.listdir(os.path.join(ROOT, "include")):
        if not hdr.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", hdr)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*[A-Za-z_][\w\s\*]*?\b(lbm_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert len(names) >= 20
    so = ctypes.CDLL(lib.LIB_PATH)
    missing = [n for n in names if not hasattr(so, n)]
    assert not missing, f"declared but not exported: {missing}"


@pytest.mark.parametrize("model", [0, 1])
@pytest.mark.parametrize("a,Tr", [(0.5, 0.8), (0.25, 0.6), (0.25, 0.85), (0.5, 0.95), (0.25, 0.5)])
def test_resolve_params_matches_oracle_thermo(lib, model, a, Tr):
    out, th = lib.lbm_resolve_params(lib.lbm_params_default(model, a=a, Tr=Tr))
    rv, rl, p0 = thermo.maxwell(a, 4.0, 1.0, Tr)
    rc, Tc, pc = thermo.critical_point(a, 4.0, 1.0)
    assert abs(th.Tc / Tc - 1) < 1e-13 and abs(th.rho_c / rc - 1) < 1e-12
    assert abs(th.rho_v / rv - 1) < 1e-11 and abs(th.rho_l / rl - 1) < 1e-12 and abs(th.p0 / p0 - 1) < 1e-11
    if model == 0:
        sig, eps, _ = thermo.sigma_li(a, 4.0, 1.0, Tr)
        assert abs(out.sigma_Li / sig - 1) < 1e-11
        assert out.tau_e == out.tau_nu and abs(out.tau_q - 1 / 1.99) < 1e-15
        _, eps, _ = thermo.sigma_li(a, 4.0, 1.0, Tr)
        assert abs(th.width / thermo.pp_width(a, 4.0, 1.0, Tr, 1.0, eps) - 1) < 1e-4
    else:
        assert abs(out.tau_e - 0.75) < 1e-15 and out.kappa == 0.5
        assert abs(th.width / thermo.fe_width(a, 4.0, 1.0, Tr, 0.5) - 1) < 1e-4
        assert abs(th.gamma / thermo.fe_surface_tension(a, 4.0, 1.0, Tr, 0.5) - 1) < 1e-4


def test_match_to_free_energy(lib):
    """Sec. 3 / App. B: kappa_P and kappa_Li reproducing the FE width and surface tension."""
    out, th = lib.lbm_resolve_params(lib.lbm_params_default(0, a=0.25, Tr=0.6, match_kappa=0.5))
    m = thermo.match_pp_to_fe(0.25, 4.0, 1.0, 0.6, 0.5)
    assert abs(out.kappa_P / m["kappa_P"] - 1) < 1e-5
    assert abs(out.kappa_Li / m["kappa_Li"] - 1) < 1e-5
    assert abs(th.width / m["W"] - 1) < 1e-4 and abs(th.gamma / m["gamma"] - 1) < 1e-4


def test_argument_errors(lib):
    bad = [dict(Tr=1.2), dict(Tr=0.0), dict(tau_nu=0.5), dict(a=-1.0), dict(tau_e=0.4)]
    for kw in bad:
        with pytest.raises(lib.LBMError) as e:
            lib.lbm_resolve_params(lib.lbm_params_default(0, **kw))
        assert e.value.code == lib.LBM_ERR_ARG
    with pytest.raises(lib.LBMError) as e:  # A belongs to the free-energy equilibrium
        lib.lbm_resolve_params(lib.lbm_params_default(0, A=0.1))
    assert e.value.code == lib.LBM_ERR_UNSUPPORTED
    with pytest.raises(lib.LBMError) as e:  # nu = c_s^2 (tau - 1/2 - A) <= 0
        lib.lbm_resolve_params(lib.lbm_params_default(1, A=0.5, tau_nu=1.0))
    assert e.value.code == lib.LBM_ERR_ARG
    out, _ = lib.lbm_resolve_params(lib.lbm_params_default(1, A=0.2, tau_nu=1.0))
    assert out.A == 0.2
    assert lib.lbm_strerror(lib.LBM_ERR_DIVERGED).startswith("simulation diverged")
    assert lib.lbm_workspace_bytes(0, 0, 5) == 0
    assert lib.lbm_workspace_bytes(1, 256, 4) > 2 * 9 * 256 * 4 * 8
    assert "sm_103a" in lib.lbm_build_info()


def test_free_energy_accepts_A_and_gravity_is_documented(lib):
    """The viscosity-tuning term A of Eq. (20) belongs to the free-energy model: lbm_resolve_params
    accepts A != 0 there (with nu = c_s^2 (tau - 1/2 - A) > 0, Eq. 23) and rejects it for the
    pseudopotential model; the header documents exactly that, and names lbm_set_gravity."""
    for A in (-0.2, 0.15, 0.3):
        out, _ = lib.lbm_resolve_params(lib.lbm_params_default(lib.LBM_FREE_ENERGY, A=A, tau_nu=1.0))
        assert out.A == A
        with pytest.raises(lib.LBMError) as e:
            lib.lbm_resolve_params(lib.lbm_params_default(lib.LBM_PSEUDOPOTENTIAL, A=A, tau_nu=1.0))
        assert e.value.code == lib.LBM_ERR_UNSUPPORTED
    text = open(os.path.join(ROOT, "include", "lbm.h")).read()
    assert "A = 0 and no gravity" not in text
    assert "LBM_ERR_UNSUPPORTED for A != 0 with the pseudopotential model" in text
    assert "lbm_set_gravity" in text.split("typedef enum")[0]  # named in the model summary


def test_create_rejects_bad_sizes_and_boundaries_before_any_device_call(lib):
    """lbm_create validates sizes and boundaries before touching the device (so this runs
    without a GPU): empty lattices and more than 2^31 cells are argument errors, walls need
    ny >= 4, walls in x are not built; *out is left NULL."""
    L = lib._lib()
    p = lib.lbm_params_default(lib.LBM_FREE_ENERGY)
    cases = [((0, 5, lib.LBM_BC_PERIODIC, lib.LBM_BC_PERIODIC), lib.LBM_ERR_ARG),
             ((5, 0, lib.LBM_BC_PERIODIC, lib.LBM_BC_PERIODIC), lib.LBM_ERR_ARG),
             ((1 << 16, (1 << 15) + 1, lib.LBM_BC_PERIODIC, lib.LBM_BC_PERIODIC), lib.LBM_ERR_ARG),
             ((16, 3, lib.LBM_BC_PERIODIC, lib.LBM_BC_WALL_ZOUHE), lib.LBM_ERR_ARG),
             ((16, 3, lib.LBM_BC_PERIODIC, lib.LBM_BC_WALL_ZOUHE_ONESIDED), lib.LBM_ERR_ARG),
             ((16, 8, lib.LBM_BC_WALL_ZOUHE, lib.LBM_BC_PERIODIC), lib.LBM_ERR_UNSUPPORTED),
             ((16, 8, lib.LBM_BC_PERIODIC, 7), lib.LBM_ERR_UNSUPPORTED)]
    for (nx, ny, bx, by), code in cases:
        h = ctypes.c_void_p(1)
        rc = L.lbm_create(ctypes.byref(p), nx, ny, bx, by, None, None, ctypes.c_size_t(0), ctypes.byref(h))
        assert rc == code, ((nx, ny, bx, by), rc)
        assert h.value is None
    # the workspace a context needs grows with the lattice and covers the one-sided walls' scratch
    assert lib.lbm_workspace_bytes(0, 64, 64) > 2 * 9 * 64 * 64 * 4 + 14 * 64 * 4
