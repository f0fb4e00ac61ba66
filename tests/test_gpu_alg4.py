"""Non-periodic reduced digital nets (Sec. 4, Algorithm 4's case) on the GPU, every tier.

The reduction zeroes the last w_j rows of each generating matrix; when the matrices have
nonzero columns beyond m - w_j the points do not repeat periodically in the index, so every
column has N distinct rows and the product is formed over all N points.  The oracle forms the
points from the definition (O2) and the product densely (O5); O11 forms the product as Sec. 4
does, from the table of grid multiples of each a_j.  Tolerances as in the other parity tests:
FP64 1e-12, FP32 and the split tier the dot-product bound elementwise (2e-5 on estimates and
gradients), bf16 2^-7 sum_j |x_j a_j| (2e-3 / 2e-2)."""
import numpy as np
import pytest
import torch

from oracle import qmc_oracle as O
from paper_2305_11645_gb300 import _lib as L
from paper_2305_11645_gb300 import api
from paper_2305_11645_gb300 import inputs as I
from tests.gpu_common import U32, fp32_product_bound, integrand, need_gpu, norm_rel, u32

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()
    L.device_status(clear=True)
    yield
    L.device_status(clear=True)


def nonperiodic_net(seed, m, s, tau, R, transform=I.T_IDENTITY, dtype=np.float64, f_kind=I.F_NONE,
                    f_params=(0.0, 0.0, 0.0, 0.0), w=None):
    g = I.rng(200, I.P_MISC, seed)
    w = I.log2_weights(s, m + 1) if w is None else np.asarray(w, dtype=np.uint32)
    C = I.nonsingular_net_masks(g, m, s)
    A = (g.standard_normal((s, tau)) / np.sqrt(s)).astype(dtype)
    D = I.random_shifts(g, R, s, force_odd=transform == I.T_INV_NORMAL) if R else None
    return I.Problem(I.DIGITAL_NET, m, w, A, C=C, shifts=D, transform=transform, f_kind=f_kind,
                     f_params=tuple(f_params), name=f"nonper{seed}")


def is_nonperiodic(p):
    for j in range(p.s):
        wcl = min(int(p.w[j]), p.m)
        Ch = O.reduced_net_matrix(p.C[j], p.m, wcl)
        if np.any(Ch[:, p.m - wcl:]):
            return True
    return False


@pytest.mark.parametrize("seed", range(4))
def test_points_bit_exact_and_not_periodic(seed):
    p = nonperiodic_net(seed, m=9 + seed % 3, s=23, tau=3, R=2)
    assert is_nonperiodic(p)
    rule = api.Rule.from_problem(p)
    for r in range(p.R_eff):
        got = u32(api.gen_points(rule, "full", r, device=DEV))
        assert np.array_equal(got, O.x32_points(p, r))
        dist = u32(api.gen_points(rule, "distinct", r, device=DEV))
        assert np.array_equal(dist, O.x32_points(p, r).T.reshape(-1))     # all N rows of every column
    # each column's unshifted values: every grid value v 2^-q exactly 2^w times (Sec. 4)
    X = O.x32_points(I.Problem(I.DIGITAL_NET, p.m, p.w, p.A, C=p.C), 0)
    for j in range(p.s):
        q = p.m - min(int(p.w[j]), p.m)
        vals, counts = np.unique(X[:, j] >> np.uint32(32 - q) if q else np.zeros(1 << p.m), return_counts=True)
        assert len(vals) == 1 << q and np.all(counts == 1 << (p.m - q))


def test_product_equals_algorithm_4():
    """Unshifted: the library's X A equals the oracle's Algorithm 4 (the table of multiples)."""
    p = nonperiodic_net(11, m=10, s=40, tau=17, R=0)
    rule = api.Rule.from_problem(p)
    P = api.reduced_matmul(rule, torch.from_numpy(p.A).to(DEV)).cpu().numpy()[0]
    assert norm_rel(P, O.alg4_product(p.m, p.w, p.C, p.A)) <= 1e-12
    assert norm_rel(P, O.reduced_matmul(p, 0)) <= 1e-12


def product_bound(X, A, precision):
    XA = np.abs(X) @ np.abs(np.asarray(A, dtype=np.float64))
    s = X.shape[1]
    if precision == "split":
        return (s + 16) * 4 * U32 * XA
    if precision == "bf16":
        return 2.0 ** -7 * XA + (s + 16) * U32 * XA
    return fp32_product_bound(X, A)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "split", "bf16"])
@pytest.mark.parametrize("transform", [I.T_IDENTITY, I.T_INV_NORMAL])
def test_reduced_matmul_every_tier(precision, transform):
    dtype = np.float64 if precision == "fp64" else np.float32
    p = nonperiodic_net(20 + transform, m=11, s=70, tau=140, R=2, transform=transform, dtype=dtype)
    rule = api.Rule.from_problem(p)
    P = api.reduced_matmul(rule, torch.from_numpy(p.A).to(DEV), precision=None if precision in ("fp64", "fp32")
                           else precision).cpu().numpy()
    for r in range(p.R_eff):
        X = O.points(p, r)
        want = O.product(X, p.A)
        if precision == "fp64":
            assert norm_rel(P[r], want) <= 1e-12
        else:
            assert np.all(np.abs(P[r] - want) <= product_bound(X, p.A, precision) + 1e-30)


FK = [(I.F_GAUSS_NORM2, (0, 0, 0, 0)), (I.F_LOGSUMEXP, (0, 0, 0, 0)), (I.F_CALL_MEAN_EXP, (0.3, 0.9, 0, 0))]
TOL = {"fp64": (1e-12, 1e-12), "fp32": (2e-5, 2e-5), "split": (2e-5, 2e-5), "bf16": (2e-3, 2e-2)}


@pytest.mark.parametrize("precision", ["fp64", "fp32", "split", "bf16"])
@pytest.mark.parametrize("fk", range(len(FK)))
def test_integrate_and_backward_every_tier(precision, fk):
    f_kind, f_params = FK[fk]
    dtype = np.float64 if precision == "fp64" else np.float32
    p = nonperiodic_net(30 + fk, m=10, s=48, tau=37, R=3, dtype=dtype, f_kind=f_kind, f_params=f_params)
    rule = api.Rule.from_problem(p)
    A = torch.from_numpy(p.A).to(DEV)
    f = integrand(p)
    prec = None if precision in ("fp64", "fp32") else precision
    est = api.integrate(rule, A, f, precision=prec).cpu().numpy()
    Q, mean = O.estimate(p)
    tol, gtol = TOL[precision]
    if precision == "bf16":
        # first-order bound: N^-1 sum_k sum_t |df/dy_t| |dy_t|, |dy| <= 2^-7 sum_j |x_j a_j|
        for r in range(p.R_eff):
            X = O.points(p, r)
            Y = O.product(X, p.A)
            dy = product_bound(X, p.A, "bf16")
            bound = np.mean(np.sum(np.abs(O.integrand_grad(p.f_kind, p.f_params, Y)) * dy, axis=1))
            assert abs(est[r] - Q[r]) <= 2 * bound + 1e-12
    else:
        assert np.all(np.abs(est[:-1] - Q) <= tol * np.abs(Q)), (est, Q)
        assert abs(est[-1] - mean) <= tol * abs(mean)
    G = api.integrate_backward(rule, A, f, torch.ones(1, dtype=torch.float64, device=DEV),
                               precision=prec)[0].double().cpu().numpy()
    assert norm_rel(G, O.grad(p)) <= gtol


@pytest.mark.parametrize("precision", ["fp64", "fp32", "split", "bf16"])
def test_pde_matrix_assembly(precision):
    """Sec. 1's D_k = sum_j x_{j,k} C_j for the stiffness terms of an affine random coefficient,
    through api.assemble (the reduced product with tau = M^2), against the oracle's sum of
    matrices; elementwise within the tier's product bound."""
    dtype = np.float64 if precision == "fp64" else np.float32
    s, M = 48, 9
    p = I.pde_assembly(m=11, s=s, M=M, R=2)
    C = I.stiffness_terms(s, M)
    rule = api.Rule.from_problem(p)
    Ct = torch.from_numpy(C.astype(dtype)).to(DEV)
    D = api.assemble(rule, Ct, precision=None if precision in ("fp64", "fp32") else precision).cpu().numpy()
    assert D.shape == (p.R_eff, p.N, M, M)
    Cq = C.astype(dtype).astype(np.float64)
    for r in range(p.R_eff):
        want = O.assemble(p, Cq, r)
        X = O.points(p, r)
        if precision == "fp64":
            assert norm_rel(D[r], want) <= 1e-12
        else:
            bound = product_bound(X, Cq.reshape(s, M * M), precision).reshape(want.shape)
            assert np.all(np.abs(D[r] - want) <= bound + 1e-30)
