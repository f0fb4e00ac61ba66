"""qmc_integrate_noalloc: the allocation-free form of qmc_integrate.

It serves callers that cannot allocate device memory when they call the
library (a framework that forbids cudaMalloc while capturing a stream, a host
that reserves all device memory up front, a foreign-function caller without a
device allocator): its scratch space is a static array inside the library.
Here it is called through the C ABI and compared with qmc_integrate (which
uses a caller workspace) on the same inputs, twice in a row, at the tolerances
of the other parity tests.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2305_11645_gb300 import _lib as L
from paper_2305_11645_gb300 import api
from paper_2305_11645_gb300 import inputs as I
from tests.gpu_common import integrand, need_gpu

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def noalloc(rule, A, f, device_rule=True):
    est = torch.empty(rule.R_eff + 1, dtype=torch.float64, device=A.device)
    r = rule.struct(A.device if device_rule else None)
    prec = L.QMC_FP64 if A.dtype == torch.float64 else L.QMC_FP32
    st = L.load().qmc_integrate_noalloc(ctypes.byref(r), A.data_ptr(), A.shape[1], ctypes.byref(f.struct()), prec,
                                        est.data_ptr(), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    L.check(st)
    return est


CASES = [
    ("c2_full_fp32", lambda: I.c2(dtype=np.float32)),
    ("c1_fp64", I.c1),
    ("net_shifts_fp32", lambda: I.random_problem(21, kind=I.DIGITAL_NET, m=12, s=48, tau=70, R=3, dtype=np.float32,
                                                 f_kind=I.F_GAUSS_NORM2)),
    ("lattice_lse_fp64", lambda: I.random_problem(22, kind=I.LATTICE, m=10, s=33, tau=9, R=2, f_kind=I.F_LOGSUMEXP)),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("device_rule", [True, False])
def test_matches_integrate_two_calls_in_a_row(name, make, device_rule):
    p = make()
    rule = api.Rule.from_problem(p)
    A = torch.from_numpy(p.A).to(DEV)
    f = integrand(p)
    want = api.integrate(rule, A, f).cpu().numpy()
    tol = 1e-12 if p.A.dtype == np.float64 else 2e-5
    for _ in range(2):
        got = noalloc(rule, A, f, device_rule).cpu().numpy()
        assert np.all(np.abs(got - want) <= tol * np.abs(want)), (got, want)


def test_rejects_problems_beyond_the_static_scratch():
    p = I.c3()
    rule = api.Rule.from_problem(p)
    A = torch.from_numpy(p.A).to(DEV)
    with pytest.raises(L.QmcError) as exc:
        noalloc(rule, A, integrand(p))
    assert exc.value.status == L.QMC_ERR_NO_MEMORY
    assert "static array" in str(exc.value)
