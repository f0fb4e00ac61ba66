"""Parity of the tensor-core tiers with the FP64 oracle.

QMC_SPLIT computes the coarse block products X_I A_I (Algorithm 2) and the block gradients
X_I^T F_I with three bf16 pieces per FP32 operand and six piece products (bf16x6), QMC_BF16
with one bf16 rounding per operand; everything else runs as in the FP32 tier.  The product
bounds below add to the FP32 tier's dot-product bound the error of the block products:
  split: every piece product is exact in the FP32 accumulator's input, the three dropped
         products are below 2^-23 |x a|, and the tensor core's FP32 accumulation adds at most
         a few units of 2^-24 per term; (s + 16) 2^-22 sum_j |x_j a_j| covers both with margin.
  bf16:  x and a are each rounded once to 8 significant bits, |bf16(x) bf16(a) - x a| <=
         (2^-8 + 2^-16) |x a|; 2^-7 sum_j |x_j a_j| covers it with the accumulation.
"""
import numpy as np
import pytest
import torch

from gpu_common import U32, integrand, need_gpu, norm_rel
from oracle import qmc_oracle as O
from paper_2305_11645_gb300 import _lib as L
from paper_2305_11645_gb300 import api
from paper_2305_11645_gb300 import inputs as I
from test_gpu_parity import FKINDS, SHAPES, rel, shaped_problem

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()
    L.device_status(clear=True)
    yield
    L.device_status(clear=True)        # no bounded wait ran out in any test of this module


def product_bound(X, A, precision):
    XA = np.abs(X) @ np.abs(np.asarray(A, dtype=np.float64))
    s = X.shape[1]
    if precision == "split":
        return (s + 16) * 4 * U32 * XA
    return 2.0 ** -7 * XA + (s + 16) * U32 * XA


# Shapes for the tensor-core tiles on top of the band shapes: a coarse level with fewer
# distinct rows than a 128-row tile and a K of 100 (four K chunks, both stages reused), a
# level whose K is cut into two entries, 128-column tiles with a ragged last tile, levels
# with several 128-row tiles, and a level eight above the band (m = 14, w = 12: its root
# gradients are folded on the fly while the block gradient loads them).
TC_SHAPES = SHAPES + [
    dict(m=10, w=np.array([0] + [4] * 100 + [6] * 70 + [10] * 3), tau=200),
    dict(m=13, w=np.array([0, 1, 1] + [5] * 40 + [7] * 300), tau=136),
    dict(m=14, w=I.log2_weights(600, 14), tau=64),
    dict(m=14, w=np.array([0, 1, 1, 2, 2, 2, 2] + [3] * 8 + [6] * 40 + [12] * 5), tau=72),
]
FOLD_SHAPE = len(TC_SHAPES) - 1


@pytest.mark.parametrize("precision", ["split", "bf16"])
@pytest.mark.parametrize("shape", range(len(TC_SHAPES)))
@pytest.mark.parametrize("kind", [I.LATTICE, I.DIGITAL_NET])
def test_products(precision, shape, kind):
    transform = [I.T_CENTER, I.T_INV_NORMAL, I.T_IDENTITY, I.T_TENT][(shape + kind) % 4]
    p = shaped_problem(TC_SHAPES[shape], kind, 300 + shape, transform=transform, R=2, dtype=np.float32)
    P = api.reduced_matmul(api.Rule.from_problem(p), torch.from_numpy(p.A).to(DEV), precision=precision)
    P = P.cpu().numpy()
    for r in range(p.R_eff):
        X = O.points(p, r)
        want = O.product(X, p.A)
        err = np.abs(P[r] - want)
        bound = product_bound(X, p.A, precision)
        assert np.all(err <= bound), (r, float(np.max(err / np.maximum(bound, 1e-300))))


def test_split_is_at_least_as_accurate_as_bf16_and_close_to_fp32():
    p = shaped_problem(TC_SHAPES[-1], I.LATTICE, 77, transform=I.T_INV_NORMAL, R=1, dtype=np.float32)
    rule, A = api.Rule.from_problem(p), torch.from_numpy(p.A).to(DEV)
    want = O.reduced_matmul(p, 0)
    err = {pr: norm_rel(api.reduced_matmul(rule, A, precision=pr)[0].cpu().numpy(), want)
           for pr in ("fp32", "split", "bf16")}
    assert err["split"] <= 4 * err["fp32"] + 1e-7, err
    assert err["bf16"] > 10 * err["split"], err
    assert err["bf16"] <= 2e-2, err


@pytest.mark.parametrize("precision", ["split", "bf16"])
@pytest.mark.parametrize("fk", range(len(FKINDS)))
@pytest.mark.parametrize("shape", [0, 3, 4, 5, FOLD_SHAPE])
def test_integrate_and_backward(precision, fk, shape):
    f_kind, f_params = FKINDS[fk]
    kind = I.LATTICE if (fk + shape) % 2 == 0 else I.DIGITAL_NET
    transform = I.T_CENTER if f_kind == I.F_PDE_INV_SQ else I.T_IDENTITY
    if f_kind == I.F_CALL_MEAN_EXP:
        f_params = (0.2, 0.9, 0, 0)
    p = shaped_problem(TC_SHAPES[shape], kind, 400 + 7 * fk + shape, transform=transform, R=2, dtype=np.float32,
                       f_kind=f_kind, f_params=f_params)
    rule = api.Rule.from_problem(p)
    A = torch.from_numpy(p.A).to(DEV)
    f = integrand(p)
    est = api.integrate(rule, A, f, precision=precision).cpu().numpy()
    Q, mean = O.estimate(p)
    if precision == "split":
        for r in range(p.R_eff):
            assert rel(est[r], Q[r]) <= 2e-5, (r, est[r], Q[r])
        assert rel(est[-1], mean) <= 2e-5
    else:
        # first-order bound: |dQ| <= N^-1 sum_k sum_t |df/dy_t| |dy_t|, |dy_t| <= 2^-7 sum_j |x_j a_jt|
        # (a relative tolerance would fail on estimates that cancel, e.g. the linear mean)
        bounds = []
        for r in range(p.R_eff):
            X = O.points(p, r)
            Y = O.product(X, p.A)
            dY = product_bound(X, p.A, "bf16")
            bounds.append(np.mean(np.sum(np.abs(O.integrand_grad(p.f_kind, p.f_params, Y)) * dY, axis=1)))
            assert abs(est[r] - Q[r]) <= bounds[-1], (r, est[r], Q[r], bounds[-1])
        assert abs(est[-1] - mean) <= np.mean(bounds)
    gtol = 2e-5 if precision == "split" else 2e-2
    up = torch.tensor([1.3], dtype=torch.float64, device=DEV)
    G = api.integrate_backward(rule, A, f, up, precision=precision)[0].cpu().numpy()
    assert norm_rel(G, 1.3 * O.grad(p)) <= gtol
    G2 = api.integrate_backward(rule, A, f, up, precision=precision)[0].cpu().numpy()
    assert np.array_equal(G, G2)                      # fixed reduction order: deterministic


@pytest.mark.parametrize("precision", ["split", "bf16"])
@pytest.mark.parametrize("shape", [0, 4, 5, 6, FOLD_SHAPE])
@pytest.mark.parametrize("path", [1, 2])
def test_backward_adjoint_paths(precision, shape, path):
    """Both coarse adjoints of the tensor-core tiers, pinned by the schedule: 1 (one fold of the root
    gradients, the cp.async block-gradient kernel; the model's choice for these small shapes) and 2
    (the fused fold-gradient kernel on the lowest coarse levels, then the TMA block-gradient kernel,
    the rest on the first path).  The shapes cover one, two and three fused levels, fused levels
    without columns, entries cut at 128 columns and levels folded on the fly."""
    kind = I.LATTICE if shape % 2 == 0 else I.DIGITAL_NET
    p = shaped_problem(TC_SHAPES[shape], kind, 900 + 11 * shape + path, R=3, dtype=np.float32,
                       f_kind=I.F_LOGSUMEXP)
    rule = api.Rule.from_problem(p)
    A = torch.from_numpy(p.A).to(DEV)
    f = integrand(p)
    api.tune_clear()
    try:
        api.tune_set(rule, A.shape[1], f, precision, bwd_path=path)
        up = torch.tensor([0.7], dtype=torch.float64, device=DEV)
        G = api.integrate_backward(rule, A, f, up, precision=precision)[0].cpu().numpy()
        assert np.all(np.isfinite(G))
        assert norm_rel(G, 0.7 * O.grad(p)) <= (2e-5 if precision == "split" else 2e-2)
        G2 = api.integrate_backward(rule, A, f, up, precision=precision)[0].cpu().numpy()
        assert np.array_equal(G, G2)
    finally:
        api.tune_clear()


@pytest.mark.parametrize("precision", ["split", "bf16"])
@pytest.mark.parametrize("shape", [0, FOLD_SHAPE])
@pytest.mark.parametrize("kind", [I.REDUCED_MC, I.POLY_LATTICE])
def test_mc_and_poly_lattice_tiers(precision, shape, kind):
    """Reduced MC replicas and shifted polynomial lattices in the tensor-core tiers: the
    materialised product within the tier's elementwise bound, the mean estimate and its gradient
    against the oracle."""
    p = shaped_problem(TC_SHAPES[shape], kind, 600 + shape, transform=I.T_INV_NORMAL, R=2,
                       dtype=np.float32, f_kind=I.F_CALL_MEAN_EXP, f_params=(0.2, 0.9, 0, 0))
    rule = api.Rule.from_problem(p)
    A = torch.from_numpy(p.A).to(DEV)
    P = api.reduced_matmul(rule, A, precision=precision).cpu().numpy()
    for r in range(p.R_eff):
        X = O.points(p, r)
        assert np.all(np.abs(P[r] - O.product(X, p.A)) <= product_bound(X, p.A, precision))
    f = integrand(p)
    est = api.integrate(rule, A, f, precision=precision).cpu().numpy()
    Q, mean = O.estimate(p)
    if precision == "split":
        assert rel(est[-1], mean) <= 2e-5
    else:       # the first-order bound of the bf16 products' error (as for the lattices and nets)
        bounds = []
        for r in range(p.R_eff):
            X = O.points(p, r)
            Y = O.product(X, p.A)
            dY = product_bound(X, p.A, "bf16")
            bounds.append(np.mean(np.sum(np.abs(O.integrand_grad(p.f_kind, p.f_params, Y)) * dY, axis=1)))
            assert abs(est[r] - Q[r]) <= bounds[-1]
        assert abs(est[-1] - mean) <= np.mean(bounds)
    up = torch.ones(1, dtype=torch.float64, device=DEV)
    G = api.integrate_backward(rule, A, f, up, precision=precision)[0].cpu().numpy()
    assert norm_rel(G, O.grad(p)) <= (2e-5 if precision == "split" else 2e-2)


@pytest.mark.parametrize("precision", ["split", "bf16"])
def test_graph_integrator_and_autograd(precision):
    p = shaped_problem(TC_SHAPES[4], I.DIGITAL_NET, 9, transform=I.T_INV_NORMAL, R=3, dtype=np.float32,
                       f_kind=I.F_LOGSUMEXP)
    rule, f = api.Rule.from_problem(p), integrand(p)
    A = torch.from_numpy(p.A).to(DEV)
    it = api.Integrator(rule, A, f, backward=True, graph=True, precision=precision)
    est, grad = it.run()
    torch.cuda.synchronize()
    e_eager = api.integrate(rule, A, f, precision=precision)
    g_eager = api.integrate_backward(rule, A, f, torch.ones(1, dtype=torch.float64, device=DEV),
                                     precision=precision)[0]
    assert torch.equal(est, e_eager) and torch.equal(grad, g_eager)
    Aq = A.clone().requires_grad_(True)
    Q = api.qmc_estimate(Aq, rule, f, precision=precision)
    Q.backward()
    assert torch.equal(Aq.grad, g_eager)
    tol = 2e-5 if precision == "split" else 2e-3
    assert rel(Q.item(), O.estimate(p)[1]) <= tol
    L.device_status(clear=False)


def test_precision_argument_checks():
    p = shaped_problem(SHAPES[0], I.LATTICE, 1, dtype=np.float64)
    rule, A = api.Rule.from_problem(p), torch.from_numpy(p.A).to(DEV)
    with pytest.raises(TypeError):
        api.reduced_matmul(rule, A, precision="split")        # the tensor-core tiers take float32 A
    with pytest.raises(ValueError):
        api.reduced_matmul(rule, A.float(), precision="fp16")
