"""Parity of the CUDA path (through the C ABI) with the CPU oracle on small,
seeded cases that span several tiles and ragged tails.

Tolerances: points bit-exact; FP64 tier 1e-12 (norm-wise relative);
FP32 tier: products within the elementwise dot-product bound
(s+16) 2^-24 sum_j |x_j a_j|, estimates and gradients within 2e-5 relative
(the FP32 arithmetic of s + tau accumulated terms: about (s + tau) 2^-24 relative
for sums of like-signed terms, with room for the row sums' cancellation)."""
import json
import os

import numpy as np
import pytest
import torch

from oracle import qmc_oracle as O
from paper_2305_11645_gb300 import api
from paper_2305_11645_gb300 import inputs as I
from tests.gpu_common import fp32_product_bound, integrand, need_gpu, norm_rel, u32

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


# ----------------------------------------------------------------------------- points (bit-exact)

@pytest.mark.parametrize("kind", [I.LATTICE, I.DIGITAL_NET])
@pytest.mark.parametrize("seed", range(8))
def test_points_bit_exact(kind, seed):
    p = I.random_problem(seed, kind=kind)
    rule = api.Rule.from_problem(p)
    for r in range(p.R_eff):
        got = u32(api.gen_points(rule, "full", shift_idx=r, device=DEV))
        assert np.array_equal(got, O.x32_points(p, r))
        dist = u32(api.gen_points(rule, "distinct", shift_idx=r, device=DEV))
        want = np.concatenate([O.x32_points(p, r)[: 2 ** (p.m - min(int(w), p.m)), j] for j, w in enumerate(p.w)])
        assert np.array_equal(dist, want)


@pytest.mark.parametrize("seed", range(6))
def test_poly_lattice_points_bit_exact(seed):
    """Reduced polynomial lattices (carry-less products on the GPU) against the oracle's polynomial
    arithmetic, every shift and both layouts."""
    transform = [I.T_IDENTITY, I.T_INV_NORMAL, I.T_CENTER][seed % 3]
    p = I.random_problem(60 + seed, kind=I.POLY_LATTICE, transform=transform,
                         R=max(1, seed % 4) if transform == I.T_INV_NORMAL else seed % 4)
    rule = api.Rule.from_problem(p)
    for r in range(p.R_eff):
        X = O.x32_points(p, r)
        assert np.array_equal(u32(api.gen_points(rule, "full", shift_idx=r, device=DEV)), X)
        dist = u32(api.gen_points(rule, "distinct", shift_idx=r, device=DEV))
        assert np.array_equal(dist, np.concatenate([X[: 2 ** (p.m - min(int(w), p.m)), j] for j, w in enumerate(p.w)]))


@pytest.mark.parametrize("seed", range(6))
def test_mc_points_bit_exact(seed):
    """Reduced MC (Sec. 5): point n of column j is the sample y_{j, n mod N_j} of its replica."""
    transform = [I.T_IDENTITY, I.T_INV_NORMAL, I.T_CENTER][seed % 3]
    p = I.random_problem(40 + seed, kind=I.REDUCED_MC, transform=transform, R=seed % 4)
    rule = api.Rule.from_problem(p)
    for r in range(p.R_eff):
        got = u32(api.gen_points(rule, "full", shift_idx=r, device=DEV))
        assert np.array_equal(got, O.x32_points(p, r))
        assert np.array_equal(u32(api.gen_points(rule, "distinct", shift_idx=r, device=DEV)), p.y[r])


def test_points_worked_examples():
    with open(os.path.join(GOLD, "p3_shifts_b2_m3.json")) as fh:
        g = json.load(fh)
    D = np.array([[int(d, 16) for d in g["D"]]], dtype=np.uint32)
    lat = api.Rule(I.LATTICE, 3, [0, 1, 2], z=[1, 3, 1], shifts=D)
    net = api.Rule(I.DIGITAL_NET, 3, [0, 1, 2], C=[[4, 2, 1], [4, 6, 0], [4, 0, 0]], shifts=D)
    want_l = np.array([[int(v, 16) for v in row] for row in g["lattice_X32"]], dtype=np.uint32)
    want_n = np.array([[int(v, 16) for v in row] for row in g["net_X32"]], dtype=np.uint32)
    assert np.array_equal(u32(api.gen_points(lat, device=DEV)), want_l)
    assert np.array_equal(u32(api.gen_points(net, device=DEV)), want_n)
    A = torch.tensor([[1.0, 2.0], [4.0, -1.0], [8.0, 3.0]], dtype=torch.float64, device=DEV)
    P = api.reduced_matmul(api.Rule(I.LATTICE, 3, [0, 1, 2], z=[1, 3, 1]), A)[0].cpu().numpy()
    with open(os.path.join(GOLD, "p1_lattice_b2_m3.json")) as fh:
        assert np.array_equal(P * 8, np.array(json.load(fh)["XA_times_8"], dtype=float))


# ----------------------------------------------------------------------------- products

TRANSFORMS = [I.T_IDENTITY, I.T_CENTER, I.T_INV_NORMAL, I.T_TENT]


@pytest.mark.parametrize("kind", [I.LATTICE, I.DIGITAL_NET])
@pytest.mark.parametrize("transform", TRANSFORMS)
@pytest.mark.parametrize("seed", range(4))
def test_reduced_matmul_fp64(kind, transform, seed):
    p = I.random_problem(10 * seed + transform, kind=kind, transform=transform,
                         R=max(1, seed % 3) if transform == I.T_INV_NORMAL else seed % 3)
    rule = api.Rule.from_problem(p)
    P = api.reduced_matmul(rule, torch.from_numpy(p.A).to(DEV)).cpu().numpy()
    for r in range(p.R_eff):
        want = O.reduced_matmul(p, r)
        assert norm_rel(P[r], want) <= 1e-12


@pytest.mark.parametrize("kind", [I.LATTICE, I.DIGITAL_NET])
@pytest.mark.parametrize("transform", TRANSFORMS)
@pytest.mark.parametrize("seed", range(4))
def test_reduced_matmul_fp32(kind, transform, seed):
    p = I.random_problem(10 * seed + transform + 500, kind=kind, transform=transform, dtype=np.float32,
                         R=max(1, seed % 3) if transform == I.T_INV_NORMAL else seed % 3)
    rule = api.Rule.from_problem(p)
    P = api.reduced_matmul(rule, torch.from_numpy(p.A).to(DEV)).cpu().numpy()
    for r in range(p.R_eff):
        X = O.points(p, r)
        want = O.product(X, p.A)
        assert np.all(np.abs(P[r] - want) <= fp32_product_bound(X, p.A) + 1e-30)


# shapes that exercise each fine band (S4 dyadic, S1 uniform, S0 fallback), several
# root blocks and column groups, ragged tau, constant columns (w >= m) and gaps in w
SHAPES = [
    dict(m=12, w=I.log2_weights(64, 12), tau=37),          # S4 band, ragged tau
    dict(m=9, w=np.array([j // 16 for j in range(64)]), tau=64),   # S1 band (c1-like)
    dict(m=7, w=np.array([0] * 40 + [3] * 5 + [9] * 3), tau=21),  # S0 fallback (tau_0 > 16), constant columns
    dict(m=6, w=np.array([0, 1, 1, 2, 2, 2, 2, 5, 5, 6, 7]), tau=130),  # S4 with empty levels 3,4
]


def shaped_problem(sh, kind, seed, transform=I.T_IDENTITY, R=2, dtype=np.float64, f_kind=I.F_NONE, f_params=(0,) * 4):
    g = np.random.default_rng(seed)
    w = np.asarray(sh["w"], dtype=np.uint32)
    s = len(w)
    A = (g.standard_normal((s, sh["tau"])) / np.sqrt(s)).astype(dtype)
    if kind == I.REDUCED_MC:        # R independent replicas of the caller's samples
        y = I.mc_samples(g, sh["m"], w, R, force_odd=transform == I.T_INV_NORMAL)
        return I.Problem(kind, sh["m"], w, A, y=y, transform=transform, f_kind=f_kind, f_params=f_params)
    D = I.random_shifts(g, R, s, force_odd=transform == I.T_INV_NORMAL) if R else None
    if kind in (I.LATTICE, I.POLY_LATTICE):
        return I.Problem(kind, sh["m"], w, A, z=I.odd_z(g, sh["m"], w), shifts=D, transform=transform,
                         f_kind=f_kind, f_params=f_params)
    return I.Problem(kind, sh["m"], w, A, C=I.periodic_net_masks(g, sh["m"], w), shifts=D, transform=transform,
                     f_kind=f_kind, f_params=f_params)


@pytest.mark.parametrize("shape", range(len(SHAPES)))
@pytest.mark.parametrize("kind", [I.LATTICE, I.DIGITAL_NET])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_reduced_matmul_band_shapes(shape, kind, dtype):
    p = shaped_problem(SHAPES[shape], kind, 7 + shape, transform=I.T_CENTER, dtype=dtype)
    P = api.reduced_matmul(api.Rule.from_problem(p), torch.from_numpy(p.A).to(DEV)).cpu().numpy()
    for r in range(p.R_eff):
        X = O.points(p, r)
        want = O.product(X, p.A)
        if dtype == np.float64:
            assert norm_rel(P[r], want) <= 1e-12
        else:
            assert np.all(np.abs(P[r] - want) <= fp32_product_bound(X, p.A))


@pytest.mark.parametrize("kind", [I.LATTICE, I.DIGITAL_NET])
@pytest.mark.parametrize("tau", [600, 601])
def test_reduced_matmul_fp32_passes_and_groups(kind, tau):
    """The materialised S4 band over several 256-column passes and many root groups, with a
    ragged last pass; an even tau takes the paired 8-byte stores, an odd one the scalar ones."""
    sh = dict(m=14, w=I.log2_weights(300, 14), tau=tau)
    p = shaped_problem(sh, kind, 31 + tau, transform=I.T_CENTER, R=2, dtype=np.float32)
    P = api.reduced_matmul(api.Rule.from_problem(p), torch.from_numpy(p.A).to(DEV)).cpu().numpy()
    assert P.shape == (2, 1 << 14, tau)
    for r in range(p.R_eff):
        X = O.points(p, r)
        want = O.product(X, p.A)
        assert np.all(np.abs(P[r] - want) <= fp32_product_bound(X, p.A))


# ----------------------------------------------------------------------------- estimates and gradients

FKINDS = [(I.F_LINEAR_MEAN, (0, 0, 0, 0)), (I.F_MEAN_COS, (0, 0, 0, 0)), (I.F_CALL_MEAN_EXP, (0.2, 1.0, 0, 0)),
          (I.F_GAUSS_NORM2, (0, 0, 0, 0)), (I.F_PDE_INV_SQ, (0.5, 0, 0, 0)), (I.F_LOGSUMEXP, (0, 0, 0, 0))]


def rel(got, want):
    return abs(got - want) / max(abs(want), 1e-300)


@pytest.mark.parametrize("fk", range(len(FKINDS)))
@pytest.mark.parametrize("shape", range(len(SHAPES)))
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_integrate_and_backward(fk, shape, dtype):
    f_kind, f_params = FKINDS[fk]
    kind = I.LATTICE if (fk + shape) % 2 == 0 else I.DIGITAL_NET
    transform = I.T_CENTER if f_kind == I.F_PDE_INV_SQ else I.T_IDENTITY
    if f_kind == I.F_CALL_MEAN_EXP:
        f_params = (0.2, 0.9, 0, 0)
    p = shaped_problem(SHAPES[shape], kind, 100 + 7 * fk + shape, transform=transform, R=2, dtype=dtype,
                       f_kind=f_kind, f_params=f_params)
    rule = api.Rule.from_problem(p)
    A = torch.from_numpy(p.A).to(DEV)
    f = integrand(p)
    est, rowf = api.integrate(rule, A, f, rowf=True)
    est = est.cpu().numpy()
    Q, mean = O.estimate(p)
    tol = 1e-12 if dtype == np.float64 else 2e-5
    for r in range(p.R_eff):
        assert rel(est[r], Q[r]) <= tol, (r, est[r], Q[r])
        want_rows = O.integrand(p.f_kind, p.f_params, O.reduced_matmul(p, r))
        assert norm_rel(rowf[0][r].cpu().numpy(), want_rows) <= (1e-12 if dtype == np.float64 else 2e-5)
    assert rel(est[-1], mean) <= tol
    # gradient of the mean estimate, with an upstream factor, reusing and not reusing the forward
    up = torch.tensor([1.7], dtype=torch.float64, device=DEV)
    G = api.integrate_backward(rule, A, f, up)[0].cpu().numpy()
    want = 1.7 * O.grad(p)
    gtol = 1e-12 if dtype == np.float64 else 2e-5
    assert norm_rel(G, want) <= gtol
    ws = torch.empty(api.workspace_size(3, [rule], [p.tau], [f], 0 if dtype == np.float64 else 1),
                     dtype=torch.uint8, device=DEV)
    api.integrate(rule, A, f, ws=ws)
    G2 = api.integrate_backward(rule, A, f, up, ws=ws, reuse_forward=True)[0].cpu().numpy()
    assert np.array_equal(G, G2)          # deterministic, and reuse gives the identical result


@pytest.mark.parametrize("fk", range(len(FKINDS)))
@pytest.mark.parametrize("shape", range(len(SHAPES)))
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_mc_integrate_and_backward(fk, shape, dtype):
    """Reduced MC replicas through the whole path: per-replica estimates, their mean, the rows'
    integrand values, the product (FP64) and the gradient of the mean, against the oracle."""
    f_kind, f_params = FKINDS[fk]
    transform = I.T_CENTER if f_kind == I.F_PDE_INV_SQ else (I.T_INV_NORMAL if fk % 2 else I.T_IDENTITY)
    if f_kind == I.F_CALL_MEAN_EXP:
        f_params = (0.2, 0.9, 0, 0)
    p = shaped_problem(SHAPES[shape], I.REDUCED_MC, 500 + 7 * fk + shape, transform=transform, R=3, dtype=dtype,
                       f_kind=f_kind, f_params=f_params)
    rule = api.Rule.from_problem(p)
    A = torch.from_numpy(p.A).to(DEV)
    f = integrand(p)
    est, rowf = api.integrate(rule, A, f, rowf=True)
    est = est.cpu().numpy()
    Q, mean = O.estimate(p)
    tol = 1e-12 if dtype == np.float64 else 2e-5
    for r in range(p.R_eff):
        assert rel(est[r], Q[r]) <= tol, (r, est[r], Q[r])
        want_rows = O.integrand(p.f_kind, p.f_params, O.reduced_matmul(p, r))
        assert norm_rel(rowf[0][r].cpu().numpy(), want_rows) <= tol
    assert rel(est[-1], mean) <= tol
    if dtype == np.float64 and fk == 0:
        P = api.reduced_matmul(rule, A).cpu().numpy()
        for r in range(p.R_eff):
            assert norm_rel(P[r], O.reduced_matmul(p, r)) <= 1e-12
    up = torch.tensor([0.6], dtype=torch.float64, device=DEV)
    G = api.integrate_backward(rule, A, f, up)[0].cpu().numpy()
    assert norm_rel(G, 0.6 * O.grad(p)) <= (1e-12 if dtype == np.float64 else 2e-5)


@pytest.mark.parametrize("fk", [0, 2, 5])
@pytest.mark.parametrize("shape", range(len(SHAPES)))
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_poly_lattice_integrate_and_backward(fk, shape, dtype):
    """Reduced polynomial lattices with digital shifts through the estimate and the adjoint."""
    f_kind, f_params = FKINDS[fk]
    if f_kind == I.F_CALL_MEAN_EXP:
        f_params = (0.2, 0.9, 0, 0)
    p = shaped_problem(SHAPES[shape], I.POLY_LATTICE, 700 + 7 * fk + shape, transform=I.T_INV_NORMAL, R=2,
                       dtype=dtype, f_kind=f_kind, f_params=f_params)
    rule = api.Rule.from_problem(p)
    A = torch.from_numpy(p.A).to(DEV)
    f = integrand(p)
    est = api.integrate(rule, A, f).cpu().numpy()
    Q, mean = O.estimate(p)
    tol = 1e-12 if dtype == np.float64 else 2e-5
    for r in range(p.R_eff):
        assert rel(est[r], Q[r]) <= tol, (r, est[r], Q[r])
    assert rel(est[-1], mean) <= tol
    G = api.integrate_backward(rule, A, f, torch.ones(1, dtype=torch.float64, device=DEV))[0].cpu().numpy()
    assert norm_rel(G, O.grad(p)) <= (1e-12 if dtype == np.float64 else 2e-5)


def test_autograd_function_matches_oracle():
    p = shaped_problem(SHAPES[0], I.LATTICE, 3, transform=I.T_CENTER, R=3, dtype=np.float64,
                       f_kind=I.F_LOGSUMEXP)
    rule = api.Rule.from_problem(p)
    A = torch.from_numpy(p.A).to(DEV).requires_grad_(True)
    Q = api.qmc_estimate(A, rule, integrand(p))
    (2.0 * Q).backward()
    assert rel(Q.item(), O.estimate(p)[1]) <= 1e-12
    assert norm_rel(A.grad.cpu().numpy(), 2.0 * O.grad(p)) <= 1e-12


def test_multiple_problems_one_call():
    ps = [shaped_problem(SHAPES[i], I.LATTICE if i % 2 else I.DIGITAL_NET, 40 + i, R=i % 3, dtype=np.float32,
                         f_kind=I.F_GAUSS_NORM2) for i in range(len(SHAPES))]
    rules = [api.Rule.from_problem(p) for p in ps]
    As = [torch.from_numpy(p.A).to(DEV) for p in ps]
    fs = [integrand(p) for p in ps]
    est = api.integrate(rules, As, fs).cpu().numpy()
    off = 0
    for p in ps:
        Q, mean = O.estimate(p)
        assert np.all(np.abs(est[off:off + p.R_eff] - Q) <= 2e-5 * np.abs(Q))
        assert rel(est[off + p.R_eff], mean) <= 2e-5
        off += p.R_eff + 1
    ups = torch.tensor([1.0, -2.0, 0.5, 3.0], dtype=torch.float64, device=DEV)
    Gs = api.integrate_backward(rules, As, fs, ups)
    for p, G, u in zip(ps, Gs, ups.cpu().numpy()):
        assert norm_rel(G.cpu().numpy(), u * O.grad(p)) <= 2e-5


def test_edge_sizes():
    # m = 1, s = 1, tau = 1; all columns constant (w >= m) with shifts; tau not a multiple of 4
    for m, w, tau, R in [(1, [0], 1, 0), (1, [0, 5, 5], 3, 2), (2, [3, 3], 5, 1), (4, [0, 0, 1], 6, 0)]:
        for kind in (I.LATTICE, I.DIGITAL_NET):
            g = np.random.default_rng(m * 10 + tau)
            w = np.array(w, dtype=np.uint32)
            A = g.standard_normal((len(w), tau))
            D = I.random_shifts(g, R, len(w)) if R else None
            p = (I.Problem(kind, m, w, A, z=I.odd_z(g, m, w), shifts=D, f_kind=I.F_MEAN_COS) if kind == I.LATTICE
                 else I.Problem(kind, m, w, A, C=I.periodic_net_masks(g, m, w), shifts=D, f_kind=I.F_MEAN_COS))
            rule = api.Rule.from_problem(p)
            At = torch.from_numpy(A).to(DEV)
            P = api.reduced_matmul(rule, At).cpu().numpy()
            for r in range(p.R_eff):
                assert norm_rel(P[r], O.reduced_matmul(p, r)) <= 1e-12
            est = api.integrate(rule, At, integrand(p)).cpu().numpy()
            assert rel(est[-1], O.estimate(p)[1]) <= 1e-12
            G = api.integrate_backward(rule, At, integrand(p), torch.ones(1, dtype=torch.float64, device=DEV))[0]
            assert norm_rel(G.cpu().numpy(), O.grad(p)) <= 1e-12


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_graph_integrator_matches_eager_and_oracle(dtype):
    """api.Integrator replays the forward + backward launches as one CUDA graph; with A
    overwritten between replays it must give exactly the eager results."""
    p = shaped_problem(SHAPES[0], I.LATTICE, 9, transform=I.T_INV_NORMAL, R=2, dtype=dtype,
                       f_kind=I.F_CALL_MEAN_EXP, f_params=(0.2, 0.9, 0, 0))
    rule = api.Rule.from_problem(p)
    A = torch.from_numpy(p.A).to(DEV)
    f = integrand(p)
    graphed = api.Integrator(rule, A, f, backward=True, graph=True)
    eager = api.Integrator(rule, A, f, backward=True, graph=False)
    tol = 1e-12 if dtype == np.float64 else 2e-5
    for scale in (1.0, 0.5):
        A2 = A * scale
        graphed.A.copy_(A2)
        eager.A.copy_(A2)
        eg, gg = [t.clone() for t in graphed.run()]
        ee, ge = [t.clone() for t in eager.run()]
        assert torch.equal(eg, ee) and torch.equal(gg, ge)
        p2 = shaped_problem(SHAPES[0], I.LATTICE, 9, transform=I.T_INV_NORMAL, R=2, dtype=dtype,
                            f_kind=I.F_CALL_MEAN_EXP, f_params=(0.2, 0.9, 0, 0))
        p2.A = A2.cpu().numpy()
        Q, mean = O.estimate(p2)
        assert rel(eg[-1].item(), mean) <= tol
        assert norm_rel(gg.double().cpu().numpy(), O.grad(p2)) <= (1e-12 if dtype == np.float64 else 2e-5)
