"""The failure path of the bounded device-side waits, exercised without a GPU fault: a kernel's
wait on an mbarrier that nothing completes runs out after a fixed number of polls, the library
reports QMC_ERR_TIMEOUT through its sticky error word, and the context stays usable (a small
estimate afterwards still matches the oracle).  Runs after every other kernel test but the
allocation-free entry point's (collected last), so that nothing else shares the word."""
import numpy as np
import pytest
import torch

from tests.gpu_common import integrand, need_gpu
from oracle import qmc_oracle as O
from paper_2305_11645_gb300 import _lib as L
from paper_2305_11645_gb300 import api
from paper_2305_11645_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_context_survives():
    need_gpu()
    lib = L.load()
    assert lib.qmc_device_status(1) == L.QMC_OK
    assert lib.qmc_selftest_wait_timeout(4096, None) == L.QMC_OK
    assert lib.qmc_device_status(0) == L.QMC_ERR_TIMEOUT
    assert "bit 31" in lib.qmc_last_error().decode()
    assert lib.qmc_device_status(1) == L.QMC_ERR_TIMEOUT        # read and clear
    assert lib.qmc_device_status(0) == L.QMC_OK
    p = I.random_problem(3, f_kind=I.F_MEAN_COS)
    est = api.integrate(api.Rule.from_problem(p), torch.from_numpy(p.A).cuda(), integrand(p)).cpu().numpy()
    _, mean = O.estimate(p)
    assert abs(est[-1] - mean) <= 1e-12 * abs(mean)
    assert np.isfinite(est).all()
