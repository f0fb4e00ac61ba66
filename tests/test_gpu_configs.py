"""Parity on the five named workloads at full size, in the launch configuration
the benchmark uses.  c1 and c2 are compared with the full oracle; for c3-c5
(N = 2^18..2^20, s, tau up to 4096) the oracle computes sampled rows one by one
and the closed forms that hold at any size (exact column sums of the point
sets give the linear integrand's estimate; softmax rows give the LSE gradient's
row sums)."""
import numpy as np
import pytest
import torch

from oracle import qmc_oracle as O
from paper_2305_11645_gb300 import api
from paper_2305_11645_gb300 import inputs as I
from tests.gpu_common import integrand, need_gpu, norm_rel, oracle_rows

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
    assert norm_rel(G.cpu().numpy(), O.grad(p)) <= 1e-11


_C2_ORACLE = {}


def c2_oracle(dtype):
    """The full-size oracle estimate and gradient of the c2 workload (cached per dtype of A)."""
    key = np.dtype(dtype).name
    if key not in _C2_ORACLE:
        p = I.c2(dtype=dtype)
        _C2_ORACLE[key] = (O.estimate(p), O.grad(p))
    return _C2_ORACLE[key]


# estimate and gradient tolerances per tier: FP64 1e-12 / 1e-11; FP32 2e-5; split 1e-6 on the
# estimate (the split path's stated tolerance); plain bf16 2e-3 on the estimate
# (split: the stated 1e-6 on both the estimate and the gradient)
C2_TIERS = [(np.float64, None, 1e-12, 1e-11), (np.float32, None, 2e-5, 2e-5),
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


def test_c3_full_sampled_and_closed_form():
    p = I.c3()
    rule = api.Rule.from_problem(p)
    A = torch.from_numpy(p.A).to(DEV)
    est, rowf = api.integrate(rule, A, integrand(p), rowf=True)
    sampled_rows_check(p, rowf)
    est = est.cpu().numpy()
    rf = rowf[0].double().mean(dim=1).cpu().numpy()
    assert np.all(np.abs(est[:-1] - rf) <= 1e-5 * np.abs(rf))
    lin = api.integrate(rule, A, api.Integrand(I.F_LINEAR_MEAN)).cpu().numpy()
    want = linear_closed_form(p)
    assert np.all(np.abs(lin[:-1] - want) <= 2e-5 * np.abs(want).max())


@pytest.mark.parametrize("inst", range(len(I.C4_INSTANCES)))
def test_c4_instances_sampled_and_closed_form(inst):
    p = I.c4(inst)
    rule = api.Rule.from_problem(p)
    A = torch.from_numpy(p.A).to(DEV)
    est, rowf = api.integrate(rule, A, integrand(p), rowf=True)
    sampled_rows_check(p, rowf, nsample=48)
    lin = api.integrate(rule, A, api.Integrand(I.F_LINEAR_MEAN)).cpu().numpy()
    want = linear_closed_form(p)
    assert np.all(np.abs(lin[:-1] - want) <= 2e-5 * max(np.abs(want).max(), 1e-3))


def test_c4_batched_call_matches_single_calls():
    ps = [I.c4(i) for i in range(len(I.C4_INSTANCES))]
    rules = [api.Rule.from_problem(p) for p in ps]
    As = [torch.from_numpy(p.A).to(DEV) for p in ps]
    fs = [integrand(p) for p in ps]
    est = api.integrate(rules, As, fs).cpu().numpy()
    off = 0
    for rule, A, f, p in zip(rules, As, fs, ps):
        single = api.integrate(rule, A, f).cpu().numpy()
        assert np.array_equal(est[off:off + p.R_eff + 1], single)
        off += p.R_eff + 1


def test_c5_forward_sampled_and_gradient_invariant():
    p = I.c5()
    rule = api.Rule.from_problem(p)
    A = torch.from_numpy(p.A).to(DEV)
    est, rowf = api.integrate(rule, A, integrand(p), rowf=True)
    sampled_rows_check(p, rowf)
    G = api.integrate_backward(rule, A, integrand(p), torch.ones(1, dtype=torch.float64, device=DEV))[0]
    G = G.double().cpu().numpy()
    # log-sum-exp: softmax rows sum to one, so sum_t dQ/dA_jt = mean over shifts and points of x_kj
    want = np.mean([column_sums(p, r) for r in range(p.R_eff)], axis=0) / p.N
    assert np.all(np.abs(G.sum(axis=1) - want) <= 2e-5 * np.abs(want).max())
