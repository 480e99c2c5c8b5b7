"""The paper's parameter studies as batched GPU jobs (paper_2403_11167_gb300.experiments):
Table 1 against the FP64 oracle and the paper's pattern; Fig. 5's droplet vapour density
against surface tension."""
import numpy as np
import pytest

import oracle as O
from oracle import thermo
from paper_2403_11167_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    assert torch.cuda.is_available()


def _oracle_table1(steps, fe_steps, nx=100):
    a, Tr, kappa = 0.5, 0.65, 0.5
    T = thermo.temperature(a, 4.0, 1.0, Tr)
    rv, rl, _ = thermo.maxwell(a, 4.0, 1.0, Tr)
    m = thermo.match_pp_to_fe(a, 4.0, 1.0, Tr, kappa)
    rho0 = inputs.flat_slab(nx, 1, rv, rl)
    out = {}
    for tq in (1.0, 1 / 1.99):
        for tn in (0.55, 0.75, 1.0, 1.2):
            p = O.make_params(a=a, b=4.0, R=1.0, T=T, kappa_P=m["kappa_P"], sigma_Li=m["sigma_Li"], tau_q=tq,
                              tau_nu=tn, tau_e=1.0, tau_zeta=1.0)
            r = O.macro(O.PP, p, O.run(O.PP, p, O.init(O.PP, rho0), steps))[0][0]
            out[("P", tq, tn)] = 100 * (0.5 * (r[0] + r[-1]) - rv) / rv
    for tn in (0.55, 0.75, 1.0, 1.2):
        p = O.make_params(a=a, b=4.0, R=1.0, T=T, kappa=kappa, tau_nu=tn, tau_e=1.0, tau_zeta=1.0, tau_q=1.0)
        r = O.macro(O.FE, p, O.run(O.FE, p, O.init(O.FE, rho0), fe_steps))[0][0]
        out[("FE", 1.0, tn)] = 100 * (0.5 * (r[0] + r[-1]) - rv) / rv
    return out


def test_table1_batched_against_oracle(paper_numbers):
    """Table 1 on the GPU (P rows one FP32 batch for 6e4 steps, FE rows FP64 contexts for 3e4
    steps) against the oracle and the paper's pattern.  P vapour densities agree with the
    oracle within the FP32 static bar, 1e-5.  FE (FP64) within 1e-5 as well: Tr = 0.65 at
    a = 0.5 is the free-energy model's stability limit (Sec. 5.1); its planar state carries a
    period-2 density mode of 3-4% of rho_v, and after about 3.5e4 steps a nonlinear event whose
    timing depends on rounding flips the sign of the vapour deviation (the oracle's own values
    at 6e4 steps spread by 2e-4 under 1e-15 perturbations of the start), so the rows are read
    at 3e4 steps, where 1e-15 perturbations move them by less than 1e-6.
    Pattern: FE of the order of the printed 0.0605% for every tau_nu; P with tau_q = 1/1.99
    flat in tau_nu; P with tau_q = 1 falling with tau_nu; both P rows equal at tau_nu = 1."""
    from paper_2403_11167_gb300 import experiments

    steps, fe_steps = 60000, 30000
    gpu = experiments.table1(steps=steps, fe_steps=fe_steps)
    ref = _oracle_table1(steps, fe_steps)
    for k in sorted(ref):
        print(f"Table 1 {k}: GPU {gpu[k]:+.5f}%  oracle {ref[k]:+.5f}%  rho_v ratio - 1 = "
              f"{(1 + gpu[k] / 100) / (1 + ref[k] / 100) - 1:+.2e}")
    for k in sorted(ref):
        assert abs((1 + gpu[k] / 100) / (1 + ref[k] / 100) - 1) < 1e-5, k
    fe = [abs(gpu[("FE", 1.0, t)]) for t in (0.55, 0.75, 1.0, 1.2)]
    # same order as the printed 0.0605% for every tau_nu (the discrete planar relation gives 0.054%)
    assert max(fe) < 3 * paper_numbers["table1_fe_vapour_error_percent"]
    q199 = [abs(gpu[("P", 1 / 1.99, t)]) for t in (0.55, 0.75, 1.0, 1.2)]
    q1 = [abs(gpu[("P", 1.0, t)]) for t in (0.55, 0.75, 1.0, 1.2)]
    assert max(q199) / min(q199) < 1.05
    assert q1[0] > q1[1] > q1[2] > q1[3] and q1[0] / q1[3] > 2
    assert abs(q1[2] / q199[2] - 1) < 1e-3


def test_fig5_pp_droplet_vapour_density_vs_surface_tension(paper_numbers):
    """Fig. 5 (P, Tr 0.6, a = 0.25, R = 20, empirical epsilon and kappa^P, kappa^Li varied, one
    FP32 batch of 120^2 droplets, 2e4 steps): every droplet equals the FP64 oracle's run of the
    same droplet within the static bar (density cell by cell, vapour probe and radius 1e-5);
    the vapour density matches the consistent one
    only near the empirical kappa^Li = -1.70 and departs monotonically on either side; at
    kappa^Li = 0 the model's tension is the printed 0.0046 and the densities are the printed
    0.0355 (numerical) and 0.0251 (consistent).  Measured: 1.7% at -1.70; 0.00457, 0.03549,
    0.02470 (43.7%) at 0."""
    from oracle import observables as OO
    from paper_2403_11167_gb300 import experiments
    from helpers import oracle_params, rho_err

    steps = 20000
    rows = experiments.fig5(steps=steps, fields=True)
    for r in rows:
        print(f"Fig. 5 kappa_Li {r['kappa_li']:+.2f} gamma {r['gamma']:.5f} R {r['radius']:.2f}: "
              f"rho_v/rho_c {r['rho_v']:.5f} consistent {r['rho_v_consistent']:.5f} error {100 * r['rel_err']:+.2f}%")
    assert all(r["status"] == 0 for r in rows)
    # the same droplets in the FP64 oracle: density cell by cell (static bar), vapour probe and
    # equimolar radius
    for r in rows:
        rp, th = r["params"]
        op = oracle_params(rp, th)
        rr, ux, uy, *_ = O.macro(O.PP, op, O.run(O.PP, op, O.init(O.PP, r["rho0"]), steps))
        ref = OO.observables(rr, ux, uy, 1, rp.a, rp.b, rp.R, th.T)
        e = rho_err(r["rho"], rr)
        print(f"Fig. 5 kappa_Li {r['kappa_li']:+.2f} against the oracle: rho_err {e:.2e} rho_v {r['rho_v_abs'] / ref['rho_v'] - 1:+.2e} "
              f"radius {r['radius'] / ref['radius'] - 1:+.2e}")
        assert e < 1e-5, (r["kappa_li"], e)
        assert abs(r["rho_v_abs"] / ref["rho_v"] - 1) < 1e-5 and abs(r["radius"] / ref["radius"] - 1) < 1e-5
    by = {r["kappa_li"]: r for r in rows}
    # the empirical kappa^Li of Sec. 5.2 is the one that matches the consistent density
    assert abs(by[-1.7]["rel_err"]) < 0.03
    errs = [abs(r["rel_err"]) for r in rows]
    k = [r["kappa_li"] for r in rows].index(-1.7)
    assert all(errs[i] > errs[i + 1] for i in range(k)) and all(errs[i] < errs[i + 1] for i in range(k, len(rows) - 1))
    # Sec. 5.2's case: gamma = 0.0046, numerical 0.0355 vs consistent 0.0251 (41%)
    r0 = by[0.0]
    assert abs(r0["gamma"] / paper_numbers["fig5_gamma"] - 1) < 0.02
    assert abs(r0["rho_v"] / paper_numbers["fig5_rho_v_numerical"] - 1) < 0.02
    assert abs(r0["rho_v_consistent"] / paper_numbers["fig5_rho_v_consistent"] - 1) < 0.03
    assert 0.35 < r0["rel_err"] < 0.50
