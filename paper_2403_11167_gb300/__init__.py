"""GB300-native D2Q9 multiphase lattice Boltzmann library (arXiv:2403.11167).

The compute path is the C-ABI library ``liblbm.so`` (sm_103a kernels, ``include/lbm.h``);
``lbm`` binds it with the same names.  Typical use::

    from paper_2403_11167_gb300 import inputs, lbm

    p = lbm.lbm_params_default(lbm.LBM_FREE_ENERGY, a=0.25, Tr=0.8, tau_nu=1.0)  # Eqs. 20-29
    ctx = lbm.Context(p, nx, ny)                   # periodic; walls=True: Zou-He rows 0, ny-1
    _, th = ctx.derived()                          # Maxwell densities, width, surface tension
    ctx.set_density(inputs.droplet(nx, ny, 25.0, th.rho_v, th.rho_l))
    ctx.step(10000)                                # fused collide + stream, CUDA graphs
    obs = ctx.observables(lbm.DROPLET)             # rho_l, rho_v, width, dp, radius, ...

Extensions of the paper's flow tests: ``walls=True`` with ``body_fx`` (Sec. 5.3),
``ctx.set_drive`` (droplet collision, Sec. 5.4), ``A`` and ``ctx.set_gravity`` (free-energy
model, Eqs. 20-23).  ``lbm.Batch`` runs hundreds of pseudopotential lattices in one launch
sequence; ``calibration`` builds the calibration runs and the learned surrogate;
``experiments`` runs Table 1 and Fig. 5 as batched jobs.
"""
