"""Host logic of the batched paper studies: the consistent droplet densities used by the
Fig. 5 study (paper_2403_11167_gb300.experiments.kelvin_2d) against the oracle's
thermodynamics."""
import numpy as np
import pytest

from oracle import thermo


def _exp():
    import importlib

    return importlib.import_module("paper_2403_11167_gb300.experiments")


@pytest.mark.parametrize("Tr,gamma,R", [(0.6, 0.0046, 20.0), (0.8, 0.01, 30.0), (0.7, 0.0, 25.0)])
def test_kelvin_2d_equal_mu_and_laplace(Tr, gamma, R):
    """Solution satisfies mu(rho_v) = mu(rho_l) and p(rho_l) - p(rho_v) = gamma / R with the
    oracle's EOS; gamma = 0 returns the Maxwell pair; the vapour density rises with gamma/R
    (Kelvin)."""
    E = _exp()
    a = 0.25
    T = thermo.temperature(a, 4.0, 1.0, Tr)
    rv0, rl0, _ = thermo.maxwell(a, 4.0, 1.0, Tr)
    rv, rl = E.kelvin_2d(a, 4.0, 1.0, T, gamma, R, rv0, rl0)
    eos = thermo.EOS(a, 4.0, 1.0)
    assert abs(eos.mu(rv, T) - eos.mu(rl, T)) < 1e-12
    assert abs(eos.p(rl, T) - eos.p(rv, T) - gamma / R) < 1e-12
    if gamma == 0.0:
        assert abs(rv / rv0 - 1) < 1e-10 and abs(rl / rl0 - 1) < 1e-10
    else:
        assert rv > rv0 and rl > rl0
