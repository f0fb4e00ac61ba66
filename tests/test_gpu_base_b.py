"""Lattices (Sec. 1.3, N = b^m) and reduced Monte Carlo (Sec. 5, N_j = b^(m-w_j)) in a prime base
b > 2 on the GPU, every tier, against the oracle.

The points u / b^q are formed in double by the same formula on both sides (one rounded division,
the shift as the rounded sum less 1 when it reaches 1), so the FP64 tier matches the oracle to
1e-12; the float tiers (the tensor-core tiers compute in FP32 on the CUDA cores in base b) are held
to the FP32 dot-product bound elementwise and 2e-5 on estimates and gradients.  The integer
numerators u are compared bit for bit."""
import numpy as np
import pytest
import torch

from oracle import qmc_oracle as O
from paper_2305_11645_gb300 import _lib as L
from paper_2305_11645_gb300 import api
from paper_2305_11645_gb300 import inputs as I
from tests.gpu_common import fp32_product_bound, integrand, need_gpu, norm_rel, u32

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
CASES = [(3, 7), (5, 5), (7, 4)]          # (b, m): N = 2187, 3125, 2401


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


@pytest.mark.parametrize("b,m", CASES)
def test_numerators_bit_exact(b, m):
    p = I.base_b_problem(1 + b, b, m, 29, 3, R=2)
    rule = api.Rule.from_problem(p)
    got = u32(api.gen_points(rule, "full", device=DEV)).reshape(p.N, p.s)
    num = O.lattice_numerators(b, m, p.w, p.z)              # k b^w z mod b^m (unreduced definition)
    want = np.stack([num[:, j] // b ** min(int(p.w[j]), m) for j in range(p.s)], axis=1)
    assert np.array_equal(got, want.astype(np.uint32))
    dist = u32(api.gen_points(rule, "distinct", device=DEV))
    off = 0
    for j in range(p.s):
        n = b ** (m - min(int(p.w[j]), m))
        assert np.array_equal(dist[off:off + n], want[:n, j])
        off += n


@pytest.mark.parametrize("b,m", CASES)
@pytest.mark.parametrize("precision", ["fp64", "fp32", "split", "bf16"])
def test_reduced_matmul(b, m, precision):
    dtype = np.float64 if precision == "fp64" else np.float32
    p = I.base_b_problem(10 + b, b, m, 37, 45, R=2, transform=I.T_INV_NORMAL, dtype=dtype)
    rule = api.Rule.from_problem(p)
    P = api.reduced_matmul(rule, torch.from_numpy(p.A).to(DEV),
                           precision=None if precision in ("fp64", "fp32") else precision).cpu().numpy()
    for r in range(p.R_eff):
        X = O.points(p, r)
        want = O.product(X, p.A)
        if precision == "fp64":
            assert norm_rel(P[r], want) <= 1e-12
        else:
            assert np.all(np.abs(P[r] - want) <= fp32_product_bound(X, p.A) + 1e-30)


FK = [(I.F_LOGSUMEXP, (0, 0, 0, 0)), (I.F_CALL_MEAN_EXP, (0.3, 0.9, 0, 0)), (I.F_GAUSS_NORM2, (0, 0, 0, 0)),
      (I.F_PDE_INV_SQ, (0.5, 0, 0, 0))]


@pytest.mark.parametrize("b,m", CASES)
@pytest.mark.parametrize("precision", ["fp64", "fp32", "split"])
@pytest.mark.parametrize("fk", range(len(FK)))
@pytest.mark.parametrize("kind", [I.LATTICE, I.REDUCED_MC])
def test_integrate_and_backward(b, m, precision, fk, kind):
    f_kind, f_params = FK[fk]
    dtype = np.float64 if precision == "fp64" else np.float32
    transform = I.T_CENTER if f_kind == I.F_PDE_INV_SQ else I.T_IDENTITY
    p = I.base_b_problem(20 + 3 * fk + b, b, m, 31, 19, R=2, kind=kind, transform=transform, dtype=dtype,
                         f_kind=f_kind, f_params=f_params)
    rule = api.Rule.from_problem(p)
    A = torch.from_numpy(p.A).to(DEV)
    f = integrand(p)
    prec = None if precision in ("fp64", "fp32") else precision
    est, rowf = api.integrate(rule, A, f, rowf=True, precision=prec)
    est = est.cpu().numpy()
    Q, mean = O.estimate(p)
    tol = 1e-12 if precision == "fp64" else 2e-5
    assert np.all(np.abs(est[:-1] - Q) <= tol * np.abs(Q)), (est, Q)
    assert abs(est[-1] - mean) <= tol * abs(mean)
    for r in range(p.R_eff):
        want = O.integrand(p.f_kind, p.f_params, O.reduced_matmul(p, r))
        assert norm_rel(rowf[0][r].cpu().numpy(), want) <= tol
    G = api.integrate_backward(rule, A, f, torch.tensor([0.7], dtype=torch.float64, device=DEV),
                               precision=prec)[0].double().cpu().numpy()
    assert norm_rel(G, 0.7 * O.grad(p)) <= tol
