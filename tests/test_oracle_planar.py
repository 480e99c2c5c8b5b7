"""Planar-interface pins of the oracle time step against the paper (Secs. 4, 5.1; Apps. D, E).

All runs are one-row periodic lattices (the planar problem has no y dependence),
Lx = 100 unless stated, initialised from f^eq of a tanh slab.
"""
import numpy as np
import pytest

import oracle as O
from oracle import planar, thermo
from paper_2403_11167_gb300 import inputs


def _run_flat(model, a, Tr, nx=100, steps=40000, w0=5.0, rho0=None, **kw):
    T = thermo.temperature(a, 4.0, 1.0, Tr)
    rv, rl, _ = thermo.maxwell(a, 4.0, 1.0, Tr)
    if rho0 is None:
        rho0 = inputs.flat_slab(nx, 1, rv, rl, w0=w0)
    p = O.make_params(a=a, b=4.0, R=1.0, T=T, **kw)
    f = O.run(model, p, O.init(model, rho0), steps)
    return p, f, rv, rl


def _vapour_error(rho_row, rv):
    """Vapour density (mean of the two cells straddling x = 0) relative to Maxwell."""
    return (0.5 * (rho_row[0] + rho_row[-1]) - rv) / rv


def test_pp_discrete_invariant_s76():
    """T5: at a P-LBM steady state with tau_e = tau_nu the left side of Eq. (S76) is the same
    constant at every node, equal to the bulk pressure.  This exercises the whole MP-LBM step
    (Eqs. 10, 11, 13, 30-32) and fixes the reading of Eq. (30b)."""
    a, Tr, kP, kLi = 0.5, 0.7, 0.6, -0.8
    sig, _, _ = thermo.sigma_li(a, 4.0, 1.0, Tr)
    p, f, rv, rl = _run_flat(O.PP, a, Tr, nx=64, steps=40000, kappa_P=kP, kappa_Li=kLi,
                             sigma_Li=sig, tau_e=0.8, tau_nu=0.8, tau_zeta=1.1, tau_q=1 / 1.99)
    rho, ux, _, _, _, psi = O.macro(O.PP, p, f)
    inv = planar.pp_invariant(rho[0], psi[0], kP, sig)
    assert np.abs(ux).max() < 1e-13
    assert inv.max() - inv.min() < 1e-14
    eos = thermo.EOS(a, 4.0, 1.0)
    # far from the interface the gradient terms fade and the constant is the bulk pressure
    assert abs(inv.mean() / eos.p(rho[0, 0], p.T) - 1) < 1e-3


def test_kappa_p_controls_width_not_densities():
    """T6 / Fig. 1: kappa^P changes the interface width (W ~ sqrt(kappa^P), Eq. S44) while the
    coexistence densities stay put (Sec. 4; eps is unchanged, Appendix C)."""
    a, Tr = 0.5, 0.7
    sig, _, _ = thermo.sigma_li(a, 4.0, 1.0, Tr)
    res = {}
    for kP in (0.4, 1.0):
        p, f, rv, rl = _run_flat(O.PP, a, Tr, kappa_P=kP, sigma_Li=sig, tau_q=1 / 1.99)
        r = O.macro(O.PP, p, f)[0][0]
        rho_l = 0.5 * (r[49] + r[50])
        rho_v = 0.5 * (r[0] + r[-1])
        W = (rho_l - rho_v) / np.max(np.abs(np.roll(r, -1) - np.roll(r, 1)) / 2)
        res[kP] = (rho_v, rho_l, W)
    assert abs(res[0.4][1] / res[1.0][1] - 1) < 1e-4       # liquid
    assert abs(res[0.4][0] / res[1.0][0] - 1) < 1e-2       # vapour, O(dx^2) discretisation
    ratio = res[0.4][2] / res[1.0][2]
    assert abs(ratio - np.sqrt(0.4)) < 0.1 * np.sqrt(0.4)


def test_fe_discrete_relation_s60():
    """T7: the FE-LBM steady state satisfies mu = const (Eq. S59), i.e. Eq. (S60).  Started from
    the Newton solution of (S60) plus a smooth perturbation, the oracle relaxes back onto it."""
    a, Tr, kappa = 0.5, 0.7, 0.5
    rv, rl, _ = thermo.maxwell(a, 4.0, 1.0, Tr)
    r_s60, mu0 = planar.fe_discrete_profile(a, 4.0, 1.0, Tr, kappa, inputs.flat_slab(100, 1, rv, rl, w0=3.0)[0])
    x = np.arange(100)
    r1 = r_s60 * (1 + 1e-3 * np.sin(2 * np.pi * x / 100))
    r1 *= r_s60.sum() / r1.sum()
    p, f, _, _ = _run_flat(O.FE, a, Tr, steps=60000, rho0=r1[None, :].copy(), kappa=kappa, tau_e=1.0)
    rho, ux, _, _, _, mu = O.macro(O.FE, p, f)
    assert np.abs(rho[0] - r_s60).max() < 1e-6
    assert np.abs(mu - mu0).max() < 1e-6
    assert np.abs(ux).max() < 1e-7


def test_table1_fe_vapour_error(paper_numbers):
    """T8 / Table 1: the FE planar vapour density is within 0.0605% of Maxwell (Tr 0.65, a 0.5,
    kappa 0.5, Lx 100).  The discrete relation (S60) gives 0.054%: same magnitude (the printed
    value carries the run's own small residuals)."""
    a, Tr, kappa = 0.5, 0.65, 0.5
    rv, rl, _ = thermo.maxwell(a, 4.0, 1.0, Tr)
    r, _ = planar.fe_discrete_profile(a, 4.0, 1.0, Tr, kappa, inputs.flat_slab(100, 1, rv, rl, w0=3.0)[0])
    err = 100 * abs(_vapour_error(r, rv))
    assert 0.5 * paper_numbers["table1_fe_vapour_error_percent"] < err < 1.5 * paper_numbers["table1_fe_vapour_error_percent"]


def test_discretisation_orders_eq34_eq35():
    """Eq. (34) vs Eq. (35): the FE planar error falls at least as dx^4 as the interface widens
    (kappa x4 = width x2), the P error about as dx^2 (kappa^P x3 = width x sqrt(3))."""
    a, Tr = 0.5, 0.65
    rv, rl, _ = thermo.maxwell(a, 4.0, 1.0, Tr)
    e_fe = []
    for k, L in ((0.5, 100), (2.0, 200)):
        r, _ = planar.fe_discrete_profile(a, 4.0, 1.0, Tr, k, inputs.flat_slab(L, 1, rv, rl, w0=3 * np.sqrt(k / 0.5))[0])
        e_fe.append(abs(_vapour_error(r, rv)))
    assert e_fe[0] / e_fe[1] > 16.0
    sig, _, _ = thermo.sigma_li(a, 4.0, 1.0, Tr)
    e_pp = []
    for kP, L in ((1.0, 140), (3.0, 250)):
        p, f, _, _ = _run_flat(O.PP, a, Tr, nx=L, steps=60000, w0=5 * np.sqrt(kP), kappa_P=kP, sigma_Li=sig,
                               tau_q=1 / 1.99)
        e_pp.append(abs(_vapour_error(O.macro(O.PP, p, f)[0][0], rv)))
    order = 2 * np.log(e_pp[0] / e_pp[1]) / np.log(3.0)
    assert 1.5 < order < 3.0
    # and FE beats P at the same width (the paper's conclusion, Sec. 6)
    assert e_fe[0] < 0.1 * e_pp[0]


def test_pp_tr06_discrepancy(paper_numbers):
    """Sec. 5.2: with theoretical parameters the planar P-LBM misses Maxwell by about 4% at
    Tr 0.6 (a 0.25, parameters matched to FE kappa 0.5)."""
    a, Tr = 0.25, 0.6
    m = thermo.match_pp_to_fe(a, 4.0, 1.0, Tr, 0.5)
    p, f, rv, rl = _run_flat(O.PP, a, Tr, kappa_P=m["kappa_P"], kappa_Li=m["kappa_Li"], sigma_Li=m["sigma_Li"],
                             tau_q=1 / 1.99)
    err = 100 * abs(_vapour_error(O.macro(O.PP, p, f)[0][0], rv))
    assert abs(err - paper_numbers["pp_vapour_error_percent_tr06"]) < 1.0


def test_pp_empirical_parameters_match_maxwell(paper_numbers):
    """Sec. 5.2: the empirical eps = 1.9168, kappa^Li = -1.70, kappa^P = 0.919 make the planar
    P-LBM match the FE/Maxwell densities at Tr 0.6 (a 0.25)."""
    a, Tr = 0.25, 0.6
    p, f, rv, rl = _run_flat(O.PP, a, Tr, kappa_P=paper_numbers["pp_empirical_kappa_p_tr06"],
                             kappa_Li=paper_numbers["pp_empirical_kappa_li_tr06"],
                             sigma_Li=paper_numbers["pp_empirical_eps_tr06"] / 16.0, tau_q=1 / 1.99)
    r = O.macro(O.PP, p, f)[0][0]
    assert 100 * abs(_vapour_error(r, rv)) < 0.1
    assert abs(0.5 * (r[49] + r[50]) / rl - 1) < 1e-3


def test_table1_pp_tau_dependence(paper_numbers):
    """Table 1 (P-LBM rows): with tau_q = 1 the vapour error falls as tau_nu grows; with
    tau_q = 1/1.99 it is flat in tau_nu; both agree at tau_nu = tau_e = 1.  The oracle
    reproduces this pattern (its magnitudes are ~10x below the printed ones, which are at odds
    with the 4%-at-Tr-0.6 statement of Sec. 5.2; recorded as a reading)."""
    a, Tr = 0.5, 0.65
    m = thermo.match_pp_to_fe(a, 4.0, 1.0, Tr, 0.5)
    errs = {}
    for tq in (1.0, 1 / 1.99):
        for tn in (0.55, 1.0, 1.2):
            p, f, rv, _ = _run_flat(O.PP, a, Tr, steps=60000, kappa_P=m["kappa_P"], sigma_Li=m["sigma_Li"],
                                    tau_q=tq, tau_nu=tn, tau_e=1.0, tau_zeta=1.0)
            errs[(tq, tn)] = abs(_vapour_error(O.macro(O.PP, p, f)[0][0], rv))
    flat = errs[(1 / 1.99, 0.55)] / errs[(1 / 1.99, 1.2)]
    assert abs(flat - 1) < 0.02
    printed = paper_numbers["table1_pp_tq1_tau_nu_055"] / paper_numbers["table1_pp_tq1_tau_nu_120"]
    steep = errs[(1.0, 0.55)] / errs[(1.0, 1.2)]
    assert steep > 2.0 and printed > 2.0
    assert abs(errs[(1.0, 1.0)] / errs[(1 / 1.99, 1.0)] - 1) < 1e-6


def test_table1_pp_rows_with_a_fitted_consistency_parameter(paper_numbers):
    """Table 1's P-LBM magnitudes: no reading of the stated parameters reproduces them (width-
    matched kappa^P or kappa^P = 1, tau_e = 1 or tau_e = tau_nu, kappa^Li = 0 or matched; sigma^Li
    = 0 diverges), all giving 2-6% where 18-51% is printed.  One parameter the table does not
    state does: with the consistency parameter eps = -16 G sigma^Li = 2.053 in place of the
    Appendix-B value 1.867 for this condition, the oracle gives the whole tau_q = 1/1.99 row
    (27.7, 27.7, 27.6, 27.6) within 0.15 percentage points, and the 27.6% that both rows share at
    tau_nu = 1.  The tau_q = 1 row then spans 30.9 .. 26.3%, against the printed 50.6 .. 18.4%:
    the direction of the tau_nu dependence (Wu et al. 2018) is reproduced, its size is not."""
    a, Tr = 0.5, 0.65
    m = thermo.match_pp_to_fe(a, 4.0, 1.0, Tr, 0.5)
    eps = 2.053
    got = {}
    for tq, tns in ((1 / 1.99, (0.55, 0.75, 1.0, 1.2)), (1.0, (0.55, 1.2))):
        for tn in tns:
            p, f, rv, _ = _run_flat(O.PP, a, Tr, steps=60000, kappa_P=m["kappa_P"], sigma_Li=eps / 16.0,
                                    tau_q=tq, tau_nu=tn, tau_e=1.0, tau_zeta=1.0)
            got[(tq, tn)] = 100.0 * _vapour_error(O.macro(O.PP, p, f)[0][0], rv)
    for tn, key in ((0.55, "table1_pp_tq199_tau_nu_055"), (0.75, "table1_pp_tq199_tau_nu_075"),
                    (1.0, "table1_pp_tq199_tau_nu_100"), (1.2, "table1_pp_tq199_tau_nu_120")):
        assert abs(got[(1 / 1.99, tn)] - paper_numbers[key]) < 0.15, (tn, got[(1 / 1.99, tn)])
    # tau_q = 1: falls with tau_nu, as printed, but by far less
    assert got[(1.0, 0.55)] > got[(1 / 1.99, 1.0)] > got[(1.0, 1.2)]
    assert got[(1.0, 0.55)] - got[(1.0, 1.2)] < 0.3 * (paper_numbers["table1_pp_tq1_tau_nu_055"]
                                                      - paper_numbers["table1_pp_tq1_tau_nu_120"])
