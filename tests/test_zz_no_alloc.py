"""The no-allocation observables entry point against the regular one.

lbm_observables_fields_static serves callers that cannot call cudaMalloc (their
device memory belongs to another allocator, or their loop must not pay for an
allocation): its reduction scratch is a static device array instead of a context
workspace.  Here it is fed the fields of a context (uploaded as caller-owned
device tensors) and must reproduce what lbm_observables reports for the same
state, on two calls in a row (the static scratch keeps the first call's partial
sums, which the second must not pick up).  This file is collected last.
"""
import ctypes

import numpy as np
import pytest

from paper_2403_11167_gb300 import inputs

pytestmark = pytest.mark.gpu

KEYS = ("rho_l", "rho_v", "width", "dp", "u_max", "mass", "radius")


def _static_obs(lbm, torch, precision, rho, ux, uy, geometry, rp, th, nblocks, stream):
    dt = torch.float32 if precision == lbm.LBM_F32 else torch.float64
    dev = [torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dt) for a in (rho, ux, uy)]
    out = torch.full((8,), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    ny, nx = rho.shape
    rc = lbm.lbm_observables_fields_static(precision, dev[0].data_ptr(), dev[1].data_ptr(), dev[2].data_ptr(), nx, ny,
                                           geometry, rp.a, rp.b, rp.R, th.T, nblocks, out.data_ptr(),
                                           stream.cuda_stream)
    assert rc == lbm.LBM_OK, lbm.lbm_strerror(rc)
    stream.synchronize()
    return dict(zip(KEYS + ("bad",), out.cpu().numpy().tolist()))


@pytest.mark.parametrize("precision", [0, 1])
def test_static_observables_match_context(precision):
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2403_11167_gb300 import lbm

    stream = torch.cuda.Stream()
    tol = 1e-12 if precision == lbm.LBM_F64 else 1e-6
    results = []
    # first call: a droplet on a large lattice with many blocks; second: a flat slab with
    # fewer blocks, so stale partial sums of the first call would corrupt the second
    cases = [(1, 300, 260, 700), (0, 256, 6, 37)]
    for geometry, nx, ny, nblocks in cases:
        p = lbm.lbm_params_default(0, precision=precision, a=0.25, Tr=0.8)
        ctx = lbm.Context(p, nx, ny, stream=stream)
        rp, th = ctx.derived()
        rho0 = (inputs.droplet(nx, ny, 40.0, th.rho_v, th.rho_l) if geometry == 1
                else inputs.flat_slab(nx, ny, th.rho_v, th.rho_l))
        ctx.set_density(rho0)
        ctx.step(300)
        ref = ctx.observables(geometry)
        rho, ux, uy = ctx.fields()
        got = _static_obs(lbm, torch, precision, rho, ux, uy, geometry, rp, th, nblocks, stream)
        results.append((ref, got, geometry))
        ctx.close()
    for ref, got, geometry in results:
        assert got["bad"] == 0
        for k in KEYS:
            if k == "radius" and geometry == 0:
                assert np.isnan(got[k])
                continue
            assert abs(got[k] - ref[k]) <= tol * max(abs(ref[k]), 1e-30), (k, got[k], ref[k])


def test_static_observables_rejects_oversize():
    import torch

    from paper_2403_11167_gb300 import lbm

    x = torch.ones(16, dtype=torch.float32, device="cuda")
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    for nb in (0, lbm.LBM_STATIC_MAX_BLOCKS + 1):
        rc = lbm.lbm_observables_fields_static(0, x.data_ptr(), x.data_ptr(), x.data_ptr(), 4, 4, 0, 0.25, 4.0, 1.0,
                                               0.02, nb, out.data_ptr(), 0)
        assert rc == lbm.LBM_ERR_ARG
