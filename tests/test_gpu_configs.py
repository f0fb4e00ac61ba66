"""Parity on the five named workloads at full size, in the launch configuration
the benchmark uses.  c1 and c2 are compared with the full oracle computed here;
c3-c5 (N = 2^14..2^20, s, tau up to 4096, up to 16 shifts) with the oracle's
full-size values stored by tests/golden/make_full_size.py (estimates of every
shift, the c5 gradient and its central differences), with rows the oracle
computes one by one, and with the closed forms that hold at any size (exact
column sums of the point sets give the linear integrand's estimate; softmax
rows give the log-sum-exp gradient's row sums).

Tolerances (relative; gradients in the max norm): FP64 1e-12; split 1e-6 on
estimates and gradients; FP32 2e-5; plain bf16 2e-3 on estimates and 2e-2 on
gradients (one bf16 product per term, 2^-8 relative, summed with cancellation)."""
import numpy as np
import pytest
import torch

from oracle import qmc_oracle as O
from paper_2305_11645_gb300 import api
from paper_2305_11645_gb300 import inputs as I
from tests.gpu_common import golden, golden_grad, integrand, need_gpu, norm_rel, oracle_rows

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


def column_sums(p, r):
    out = np.zeros(p.s)
    for j, wj in enumerate(p.w):
        wj = min(int(wj), p.m); q = p.m - wj
        D = 0 if p.shifts is None else int(p.shifts[r, j])
        Dlo = D % (1 << (32 - q))
        x = 2.0 ** wj * ((2.0 ** q - 1) / 2 + 2.0 ** q * Dlo * 2.0 ** -32)
        out[j] = x - (0.5 * p.N if p.transform == I.T_CENTER else 0.0)
    return out


def linear_closed_form(p):
    return np.array([column_sums(p, r) @ np.asarray(p.A, dtype=np.float64).sum(axis=1) / (p.N * p.tau)
                     for r in range(p.R_eff)])


def linear_term_scale(p):
    """The scale of the terms the linear integrand's estimate sums, N^-1 tau^-1 sum_k sum_t sum_j
    |x_kj a_jt| (exact from the column sums when the points are nonnegative; centred points give an
    upper bound through |x - 1/2| <= 1/2).  The estimate itself can cancel far below this scale,
    so its error is held to the tier's tolerance relative to it."""
    absA = np.abs(np.asarray(p.A, dtype=np.float64)).sum(axis=1)
    if p.transform == I.T_CENTER:
        return 0.5 * absA.sum() / p.tau
    return max(column_sums(p, r) @ absA / (p.N * p.tau) for r in range(p.R_eff))


def test_c1_full():
    p = I.c1()
    rule = api.Rule.from_problem(p)
    A = torch.from_numpy(p.A).to(DEV)
    P = api.reduced_matmul(rule, A)[0].cpu().numpy()
    assert norm_rel(P, O.reduced_matmul(p, 0)) <= 1e-12
    est = api.integrate(rule, A, integrand(p)).cpu().numpy()
    Q, mean = O.estimate(p)
    assert rel(est[0], Q[0]) <= 1e-12 and rel(est[-1], mean) <= 1e-12
    G = api.integrate_backward(rule, A, integrand(p), torch.ones(1, dtype=torch.float64, device=DEV))[0]
    assert norm_rel(G.cpu().numpy(), O.grad(p)) <= 1e-12


_C2_ORACLE = {}


def c2_oracle(dtype):
    """The full-size oracle estimate and gradient of the c2 workload (cached per dtype of A)."""
    key = np.dtype(dtype).name
    if key not in _C2_ORACLE:
        p = I.c2(dtype=dtype)
        _C2_ORACLE[key] = (O.estimate(p), O.grad(p))
    return _C2_ORACLE[key]


# estimate and gradient tolerances per tier: FP64 1e-12 (both); FP32 2e-5; split 1e-6 on the
# estimate (the split path's stated tolerance); plain bf16 2e-3 on the estimate
# (split: the stated 1e-6 on both the estimate and the gradient)
C2_TIERS = [(np.float64, None, 1e-12, 1e-12), (np.float32, None, 2e-5, 2e-5),
            (np.float32, "split", 1e-6, 1e-6), (np.float32, "bf16", 2e-3, 2e-2)]


@pytest.mark.parametrize("tier", range(len(C2_TIERS)))
def test_c2_full(tier):
    dtype, precision, tol, gtol = C2_TIERS[tier]
    p = I.c2(dtype=dtype)
    rule = api.Rule.from_problem(p)
    A = torch.from_numpy(p.A).to(DEV)
    est = api.integrate(rule, A, integrand(p), precision=precision).cpu().numpy()
    (Q, mean), grad = c2_oracle(dtype)
    assert rel(est[0], Q[0]) <= tol, (est, Q)
    G = api.integrate_backward(rule, A, integrand(p), torch.ones(1, dtype=torch.float64, device=DEV),
                               precision=precision)[0]
    assert norm_rel(G.cpu().numpy(), grad) <= gtol


def sampled_rows_check(p, rowf, nsample=96, tol=2e-5):
    g = np.random.default_rng(12345)
    ks = np.unique(np.concatenate([[0, 1, p.N - 1], g.integers(0, p.N, size=nsample)]))
    for r in range(p.R_eff):
        want = O.integrand(p.f_kind, p.f_params, oracle_rows(p, r, ks))
        got = rowf[0][r].cpu().numpy()[ks]
        assert np.all(np.abs(got - want) <= tol * np.maximum(np.abs(want), np.abs(want).mean())), r


# (precision, estimate tolerance, gradient tolerance) of the float tiers
FLOAT_TIERS = {"split": ("split", 1e-6, 1e-6), "fp32": (None, 2e-5, 2e-5), "bf16": ("bf16", 2e-3, 2e-2)}


@pytest.mark.parametrize("tier", list(FLOAT_TIERS))
def test_c3_full_estimates_against_the_oracle(tier):
    """Every shift's estimate and their mean against the oracle's full-size values (2^20 points,
    s = tau = 1024, 16 digital shifts), in each float tier."""
    prec, tol, _ = FLOAT_TIERS[tier]
    p = I.c3()
    g = golden("c3")
    rule = api.Rule.from_problem(p)
    A = torch.from_numpy(p.A).to(DEV)
    est = api.integrate(rule, A, integrand(p), precision=prec).cpu().numpy()
    Q = np.array(g["Q"])
    assert np.all(np.abs(est[:-1] - Q) <= tol * np.abs(Q)), np.max(np.abs(est[:-1] - Q) / np.abs(Q))
    assert rel(est[-1], g["mean"]) <= tol


def test_c3_full_sampled_rows_and_closed_form():
    p = I.c3()
    rule = api.Rule.from_problem(p)
    A = torch.from_numpy(p.A).to(DEV)
    est, rowf = api.integrate(rule, A, integrand(p), rowf=True, precision="split")
    sampled_rows_check(p, rowf)
    lin = api.integrate(rule, A, api.Integrand(I.F_LINEAR_MEAN), precision="split").cpu().numpy()
    want = linear_closed_form(p)
    assert np.all(np.abs(lin[:-1] - want) <= 1e-6 * linear_term_scale(p))


@pytest.mark.parametrize("tier", ["split", "fp32"])
@pytest.mark.parametrize("inst", range(len(I.C4_INSTANCES)))
def test_c4_instances_against_the_oracle(inst, tier):
    prec, tol, _ = FLOAT_TIERS[tier]
    p = I.c4(inst)
    g = golden("c4")[inst]
    rule = api.Rule.from_problem(p)
    A = torch.from_numpy(p.A).to(DEV)
    est, rowf = api.integrate(rule, A, integrand(p), rowf=True, precision=prec)
    est = est.cpu().numpy()
    Q = np.array(g["Q"])
    assert np.all(np.abs(est[:-1] - Q) <= tol * np.abs(Q)), np.max(np.abs(est[:-1] - Q) / np.abs(Q))
    assert rel(est[-1], g["mean"]) <= tol
    sampled_rows_check(p, rowf, nsample=48)
    lin = api.integrate(rule, A, api.Integrand(I.F_LINEAR_MEAN), precision=prec).cpu().numpy()
    want = linear_closed_form(p)
    assert np.all(np.abs(lin[:-1] - want) <= tol * linear_term_scale(p))


@pytest.mark.parametrize("tier", ["split", "fp32"])
def test_c4_batched_call_against_the_oracle(tier):
    """The 8 uneven instances in one call: every instance's estimates against the oracle, and
    bit-identical to the instance called alone."""
    prec, tol, _ = FLOAT_TIERS[tier]
    ps = [I.c4(i) for i in range(len(I.C4_INSTANCES))]
    rules = [api.Rule.from_problem(p) for p in ps]
    As = [torch.from_numpy(p.A).to(DEV) for p in ps]
    fs = [integrand(p) for p in ps]
    est = api.integrate(rules, As, fs, precision=prec).cpu().numpy()
    off = 0
    for i, (rule, A, f, p) in enumerate(zip(rules, As, fs, ps)):
        g = golden("c4")[i]
        got = est[off:off + p.R_eff + 1]
        assert np.all(np.abs(got[:-1] - np.array(g["Q"])) <= tol * np.abs(np.array(g["Q"])))
        assert rel(got[-1], g["mean"]) <= tol
        single = api.integrate(rule, A, f, precision=prec).cpu().numpy()
        assert np.array_equal(got, single)
        off += p.R_eff + 1


@pytest.mark.parametrize("tier", list(FLOAT_TIERS))
def test_c5_gradient_against_the_oracle_and_finite_differences(tier):
    """The adjoint at full size (2^20 points, s = tau = 1024, 8 shifts, log-sum-exp): the estimate,
    the gradient elementwise against the oracle's X^T G, the 64 seeded entries against the oracle's
    central differences, and the softmax row-sum invariant."""
    prec, tol, gtol = FLOAT_TIERS[tier]
    p = I.c5()
    g = golden("c5")
    rule = api.Rule.from_problem(p)
    A = torch.from_numpy(p.A).to(DEV)
    f = integrand(p)
    est = api.integrate(rule, A, f, precision=prec).cpu().numpy()
    assert np.all(np.abs(est[:-1] - np.array(g["Q"])) <= tol * np.abs(np.array(g["Q"])))
    assert rel(est[-1], g["mean"]) <= tol
    G = api.integrate_backward(rule, A, f, torch.ones(1, dtype=torch.float64, device=DEV), precision=prec)[0]
    G = G.double().cpu().numpy()
    Gref = golden_grad("c5")
    assert norm_rel(G, Gref) <= gtol
    pairs = np.array(g["fd_pairs"])
    fd = np.array(g["fd"])
    scale = np.abs(Gref).max()
    assert np.all(np.abs(G[pairs[:, 0], pairs[:, 1]] - fd) <= gtol * scale)
    # log-sum-exp: softmax rows sum to one, so sum_t dQ/dA_jt = mean over shifts and points of x_kj
    want = np.mean([column_sums(p, r) for r in range(p.R_eff)], axis=0) / p.N
    assert np.all(np.abs(G.sum(axis=1) - want) <= max(gtol, 2e-5) * np.abs(want).max())
