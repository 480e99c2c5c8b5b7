"""Failure detection without a GPU fault: the bounded waits that guard the TMA row
pipelines give up after their poll limit and report LBM_ERR_TIMEOUT, and the device stays
usable afterwards (a lattice steps and matches a fresh run)."""
import numpy as np
import pytest

from paper_2403_11167_gb300 import inputs
from helpers import gpu_context

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2403_11167_gb300 import lbm as L

    return L


def test_wait_that_nothing_completes_times_out(lbm):
    assert lbm.lbm_selftest_bounded_wait(False, 2000) == lbm.LBM_ERR_TIMEOUT


def test_completed_wait_succeeds(lbm):
    assert lbm.lbm_selftest_bounded_wait(True, 2000) == lbm.LBM_OK


def test_selftest_rejects_bad_limits(lbm):
    assert lbm.lbm_selftest_bounded_wait(False, 0) == lbm.LBM_ERR_ARG
    assert lbm.lbm_selftest_bounded_wait(False, (1 << 22) + 1) == lbm.LBM_ERR_ARG


@pytest.mark.parametrize("model", [0, 1])
def test_device_usable_after_timeout(lbm, model):
    """After a timed-out wait, the TMA-fed step still runs and reproduces a run made before."""
    nx, ny = 244, 33
    a, rp, th = gpu_context(model, lbm.LBM_F32, nx, ny, Tr=0.85, tau_nu=0.8)
    rho0 = inputs.spinodal_noise(nx, ny, 0.5 * (th.rho_l + th.rho_v), 0.01, seed=3)
    a.set_density(rho0)
    a.step(20)
    before = a.populations()
    assert lbm.lbm_selftest_bounded_wait(False, 500) == lbm.LBM_ERR_TIMEOUT
    a.set_density(rho0)
    a.step(20)
    assert np.array_equal(a.populations(), before)
    assert a.observables(0)["status"] == lbm.LBM_OK
