"""Pins for the CPU oracle: each test checks the oracle against something other
than itself -- hand-worked examples, textbook closed forms, invariants the paper
states, brute force in exact rational arithmetic, or an independent library
routine (Python's libm erfc for the normal CDF).  CPU only."""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import qmc_oracle as O
from paper_2305_11645_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def load(name):
    with open(os.path.join(GOLD, name)) as fh:
        return json.load(fh)


def lattice_problem(m, w, z, A, shifts=None, transform=I.T_IDENTITY, f_kind=I.F_NONE, f_params=(0, 0, 0, 0)):
    return I.Problem(I.LATTICE, m, np.array(w, dtype=np.uint32), np.array(A, dtype=np.float64),
                     z=np.array(z, dtype=np.uint32), shifts=shifts, transform=transform,
                     f_kind=f_kind, f_params=f_params)


def net_problem(m, w, C, A, shifts=None, transform=I.T_IDENTITY, f_kind=I.F_NONE, f_params=(0, 0, 0, 0)):
    return I.Problem(I.DIGITAL_NET, m, np.array(w, dtype=np.uint32), np.array(A, dtype=np.float64),
                     C=np.array(C, dtype=np.uint32), shifts=shifts, transform=transform,
                     f_kind=f_kind, f_params=f_params)


# ----------------------------------------------------------------------------- P1-P3 hand-worked examples

def test_p1_lattice_worked_example():
    g = load("p1_lattice_b2_m3.json")
    p = lattice_problem(g["m"], g["w"], g["z"], g["A"])
    X = O.points(p)
    assert np.array_equal(X * 8, np.array(g["points_times_8"], dtype=float))
    assert np.array_equal(O.reduced_matmul(p) * 8, np.array(g["XA_times_8"], dtype=float))
    assert np.array_equal(X.sum(axis=0), np.array(g["column_sums"], dtype=float))


def test_p1_algorithm_1_intermediates():
    """The hand-worked intermediates of Algorithm 1 (Sec. 3.1) on the P1 example: P_3 has the two
    distinct rows of column 3, P_2 the four of columns 2-3, and P_1 is X A."""
    g = load("p1_lattice_b2_m3.json")
    p = lattice_problem(g["m"], g["w"], g["z"], g["A"])
    Afr = [[Fraction(v) for v in row] for row in g["A"]]
    trace = {}
    P = alg1(p, Afr, trace)
    as_fr = lambda rows: [[Fraction(v) for v in row] for row in rows]
    assert trace[3] == as_fr(g["alg1_P3"])
    assert trace[2] == as_fr(g["alg1_P2"])
    assert P == [[Fraction(v, 8) for v in row] for row in g["XA_times_8"]]
    assert trace[1] == P


def test_p2_net_worked_example():
    g = load("p2_net_b2_m3.json")
    p = net_problem(g["m"], g["w"], g["C"], g["A"])
    X = O.points(p)
    assert np.array_equal(X * 8, np.array(g["points_times_8"], dtype=float))
    assert np.array_equal(O.reduced_matmul(p) * 8, np.array(g["XA_times_8"], dtype=float))


def test_p3_shifts_worked_example():
    g = load("p3_shifts_b2_m3.json")
    D = np.array([[int(d, 16) for d in g["D"]]], dtype=np.uint32)
    g1, g2 = load("p1_lattice_b2_m3.json"), load("p2_net_b2_m3.json")
    pl = lattice_problem(g1["m"], g1["w"], g1["z"], g1["A"], shifts=D)
    pn = net_problem(g2["m"], g2["w"], g2["C"], g2["A"], shifts=D)
    want_l = np.array([[int(v, 16) for v in row] for row in g["lattice_X32"]], dtype=np.uint32)
    want_n = np.array([[int(v, 16) for v in row] for row in g["net_X32"]], dtype=np.uint32)
    assert np.array_equal(O.x32_points(pl, 0), want_l)
    assert np.array_equal(O.x32_points(pn, 0), want_n)


def test_repetition_example_periods():
    """Sec. 1: with N_1=4, N_2=2, N_3=1 coordinate j takes N_j values and repeats
    with period N_j (the listed points (y_{1,k}, y_{2,k mod 2}, y_{3,0}))."""
    p = lattice_problem(2, [0, 1, 2], [1, 1, 1], np.eye(3))
    X = O.points(p)
    for j, Nj in enumerate([4, 2, 1]):
        col = X[:, j]
        assert len(set(col.tolist())) == Nj
        assert all(col[k] == col[k % Nj] for k in range(4))


# ----------------------------------------------------------------------------- P4 reduced = unreduced (brute force)

@pytest.mark.parametrize("b,mmax", [(2, 9), (3, 5), (5, 3)])
def test_p4_reduced_form_equals_unreduced_definition(b, mmax):
    """{k b^w z / b^m} = (k z mod b^(m-w)) / b^(m-w) for every k, every unit z
    and every w (Sec. 1.3), checked in exact integers for all small cases."""
    for m in range(1, mmax + 1):
        N = b ** m
        for w in range(0, m + 2):
            q = m - min(w, m)
            units = [z for z in range(1, max(b ** q, 2)) if math.gcd(z, b) == 1] if q > 0 else [1]
            for z in units:
                num = O.lattice_numerators(b, m, [w], [z])[:, 0]
                for k in range(N):
                    red = Fraction((k * z) % (b ** q), b ** q) if q > 0 else Fraction(0)
                    assert Fraction(int(num[k]), N) == red


def alg1(p, Afr, trace=None):
    """Algorithm 1 (Sec. 3.1) in exact rationals, lattice, b = 2.  With a dict `trace`, the
    intermediate P_j of every step is recorded under the paper's 1-based j."""
    m, w, z = p.m, [int(v) for v in p.w], [int(v) for v in p.z]
    s, tau = len(w), len(Afr[0])
    sstar = max([j + 1 for j in range(s) if w[j] < m], default=0)
    P = [[Fraction(0)] * tau]
    for j in range(sstar - 1, -1, -1):
        n = 2 ** (m - w[j])
        wnext = m if j + 1 >= sstar else min(w[j + 1], m)
        reps = 2 ** (wnext - w[j])
        assert reps * len(P) == n
        Xj = [Fraction((k * z[j]) % n, n) for k in range(n)]
        P = [[P[k % len(P)][t] + Xj[k] * Afr[j][t] for t in range(tau)] for k in range(n)]
        if trace is not None:
            trace[j + 1] = P
    N = 2 ** m
    return [[P[k % len(P)][t] for t in range(tau)] for k in range(N)]


def alg2(p, Afr):
    """Algorithm 2 (Sec. 3.2) in exact rationals, lattice, b = 2."""
    m, w, z = p.m, [int(v) for v in p.w], [int(v) for v in p.z]
    tau = len(Afr[0])
    P = [[Fraction(0)] * tau]
    for Ilev in range(m - 1, -1, -1):
        cols = [j for j in range(len(w)) if w[j] == Ilev]
        n = 2 ** (m - Ilev)
        P = [[P[k % len(P)][t] for t in range(tau)] for k in range(n)]   # b copies of P_{I+1}
        for j in cols:
            for k in range(n):
                x = Fraction((k * z[j]) % n, n)
                for t in range(tau):
                    P[k][t] += x * Afr[j][t]
    return P


@pytest.mark.parametrize("seed", range(6))
def test_p4_algorithms_1_and_2_return_XA(seed):
    """Both algorithms return exactly P = X A (Sec. 3), compared in exact
    arithmetic with the oracle's dense product of the unreduced points."""
    g = np.random.default_rng(seed)
    m = int(g.integers(1, 6)); s = int(g.integers(1, 9)); tau = int(g.integers(1, 4))
    w = np.sort(g.integers(0, m + 2, size=s)); w[0] = 0
    z = I.odd_z(g, m, w)
    A = g.integers(-8, 9, size=(s, tau))
    p = lattice_problem(m, w, z, A)
    Afr = [[Fraction(int(v)) for v in row] for row in A]
    dense = O.reduced_matmul(p)              # exact: dyadic rationals times small integers
    for P in (alg1(p, Afr), alg2(p, Afr)):
        assert np.array_equal(np.array([[float(v) for v in row] for row in P]), dense)


def test_p4_shift_is_addition_mod_one():
    """{x + Delta} in exact rationals equals the oracle's 32-bit shift."""
    g = np.random.default_rng(7)
    p = lattice_problem(5, [0, 0, 1, 3, 5, 6], I.odd_z(g, 5, np.array([0, 0, 1, 3, 5, 6])), np.eye(6)[:, :1],
                        shifts=I.random_shifts(g, 1, 6))
    X32 = O.x32_points(p, 0)
    base = O.lattice_numerators(2, 5, p.w, p.z)
    for k in range(32):
        for j in range(6):
            v = Fraction(int(base[k, j]), 32) + Fraction(int(p.shifts[0, j]), 2 ** 32)
            v -= math.floor(v)
            assert Fraction(int(X32[k, j]), 2 ** 32) == v


def test_p4_digital_shift_is_digitwise_addition():
    """A digital shift adds base-2 digits mod 2 (y_p + Delta_p mod b)."""
    g = np.random.default_rng(8)
    w = np.array([0, 1, 2, 4], dtype=np.uint32)
    C = I.periodic_net_masks(g, 6, w)
    D = I.random_shifts(g, 1, 4)
    p = net_problem(6, w, C, np.eye(4)[:, :1], shifts=D)
    y32 = O.x32_points(net_problem(6, w, C, np.eye(4)[:, :1]), 0)
    x32 = O.x32_points(p, 0)
    for k in range(64):
        for j in range(4):
            dig_y = [(int(y32[k, j]) >> (31 - p_)) & 1 for p_ in range(32)]
            dig_d = [(int(D[0, j]) >> (31 - p_)) & 1 for p_ in range(32)]
            val = sum(((a + b) % 2) * Fraction(1, 2 ** (p_ + 1)) for p_, (a, b) in enumerate(zip(dig_y, dig_d)))
            assert Fraction(int(x32[k, j]), 2 ** 32) == val


def test_van_der_corput_identity_matrix():
    """C = identity gives the radical inverse of n in base 2 (textbook)."""
    m = 7
    C = np.array([[1 << (m - 1 - q) for q in range(m)]], dtype=np.uint32)
    p = net_problem(m, [0], C, np.eye(1))
    X = O.points(p)[:, 0]
    for n in range(2 ** m):
        rev = int(format(n, f"0{m}b")[::-1], 2)
        assert X[n] == rev / 2 ** m


# ----------------------------------------------------------------------------- P5 permutation, column sums, closed forms

def closed_form_column_sums(p, shift_idx):
    """sum_k x_{k,j} = 2^{w_j} [ (2^q - 1)/2 + 2^q D_lo 2^-32 ], q = m - min(w_j, m),
    D_lo = D_j mod 2^(32-q): the period is a permutation of the grid (Sec. 1.3, Sec. 4)."""
    out = []
    for j, wj in enumerate(p.w):
        wj = min(int(wj), p.m); q = p.m - wj
        D = 0 if p.shifts is None else int(p.shifts[shift_idx, j])
        Dlo = D % (1 << (32 - q))
        out.append(Fraction(2 ** wj) * (Fraction(2 ** q - 1, 2) + Fraction(2 ** q * Dlo, 2 ** 32)))
    return out


@pytest.mark.parametrize("kind", [I.LATTICE, I.DIGITAL_NET])
@pytest.mark.parametrize("seed", range(5))
def test_p5_permutation_and_exact_column_sums(kind, seed):
    p = I.random_problem(seed, kind=kind, R=2 if seed % 2 else 0)
    for r in range(p.R_eff):
        X32 = O.x32_points(p, r).astype(np.int64)
        for j, wj in enumerate(p.w):
            q = p.m - min(int(wj), p.m)
            period = X32[: 2 ** q, j]
            D = 0 if p.shifts is None else int(p.shifts[r, j])
            Dlo = D % (1 << (32 - q))
            grid = sorted(((v - Dlo) >> (32 - q)) if q > 0 else 0 for v in period)
            assert grid == list(range(2 ** q))                       # a permutation of the grid
            assert all(X32[k, j] == X32[k % 2 ** q, j] for k in range(p.N))   # periodic
        sums = [Fraction(int(v), 2 ** 32) for v in X32.sum(axis=0)]
        assert sums == closed_form_column_sums(p, r)


@pytest.mark.parametrize("seed", range(4))
def test_p5_linear_mean_estimate_closed_form(seed):
    """f = mean_t y_t: Q = (N tau)^-1 sum_j c_j sum_t A_jt with c_j the exact column sums."""
    p = I.random_problem(seed, kind=I.LATTICE if seed % 2 else I.DIGITAL_NET, R=seed % 3,
                         f_kind=I.F_LINEAR_MEAN)
    Q, mean = O.estimate(p)
    for r in range(p.R_eff):
        c = closed_form_column_sums(p, r)
        want = sum(float(cj) * p.A[j].sum() for j, cj in enumerate(c)) / (p.N * p.tau)
        assert abs(Q[r] - want) <= 1e-13 * max(1.0, abs(want))


# ----------------------------------------------------------------------------- transforms

def Phi(x):
    return 0.5 * math.erfc(-x / math.sqrt(2.0))


def test_inverse_normal_round_trip_and_known_values():
    ps = [2.0 ** -32, 1e-9, 1e-5, 0.01, 0.02425, 0.1, 0.3, 0.5, 0.7, 0.9, 0.97575, 0.99, 1 - 1e-5, 1 - 2.0 ** -32]
    x32 = np.array([round(p_ * 2 ** 32) for p_ in ps], dtype=np.uint64).astype(np.uint32)
    xs = O.transform(x32, O.T_INV_NORMAL)
    for v, x in zip(x32, xs):
        p_ = int(v) / 2 ** 32
        if p_ < 0.5:
            assert abs(Phi(x) - p_) <= 1e-14 * p_
        else:
            assert abs(0.5 * math.erfc(x / math.sqrt(2.0)) - (1 - p_)) <= 1e-13 * (1 - p_)
    # textbook quantiles
    q975 = O.transform(np.array([int(0.975 * 2 ** 32)], dtype=np.uint32), O.T_INV_NORMAL)[0]
    assert abs(q975 - 1.959963984540054) < 1e-8
    assert O.transform(np.array([1 << 31], dtype=np.uint32), O.T_INV_NORMAL)[0] == 0.0
    assert O.transform(np.array([0], dtype=np.uint32), O.T_INV_NORMAL)[0] == -np.inf


def test_center_and_tent_transforms():
    x32 = np.array([0, 1 << 30, 1 << 31, 3 << 30, 0xFFFFFFFF], dtype=np.uint32)
    assert np.array_equal(O.transform(x32, O.T_CENTER), np.array([-0.5, -0.25, 0.0, 0.25, 0.5 - 2.0 ** -32]))
    assert np.array_equal(O.transform(x32, O.T_TENT), np.array([0.0, 0.5, 1.0, 0.5, 2.0 ** -31]))


# ----------------------------------------------------------------------------- integrands and gradients

FKINDS = [(I.F_LINEAR_MEAN, (0, 0, 0, 0)), (I.F_MEAN_COS, (0, 0, 0, 0)), (I.F_CALL_MEAN_EXP, (0.2, 1.0, 0, 0)),
          (I.F_GAUSS_NORM2, (0, 0, 0, 0)), (I.F_PDE_INV_SQ, (0.5, 0, 0, 0)), (I.F_LOGSUMEXP, (0, 0, 0, 0))]


def test_integrand_values_at_hand_points():
    tau = 4
    Y0 = np.zeros((1, tau))
    assert O.integrand(I.F_LINEAR_MEAN, (0,) * 4, Y0)[0] == 0.0
    assert O.integrand(I.F_MEAN_COS, (0,) * 4, Y0)[0] == 1.0
    assert O.integrand(I.F_CALL_MEAN_EXP, (0.2, 1.0, 0, 0), Y0)[0] == 0.0
    assert O.integrand(I.F_CALL_MEAN_EXP, (0.2, 0.5, 0, 0), Y0)[0] == 0.5
    assert O.integrand(I.F_GAUSS_NORM2, (0,) * 4, Y0)[0] == 1.0
    assert O.integrand(I.F_PDE_INV_SQ, (0.5,) + (0,) * 3, Y0)[0] == 1.0
    assert abs(O.integrand(I.F_LOGSUMEXP, (0,) * 4, Y0)[0] - math.log(4)) < 1e-15
    Y = np.array([[1.0, -1.5, 0.5, 3.0]])
    assert abs(O.integrand(I.F_MEAN_COS, (0,) * 4, Y)[0] - sum(math.cos(v) for v in Y[0]) / 4) < 1e-15
    assert abs(O.integrand(I.F_GAUSS_NORM2, (0,) * 4, Y)[0] - math.exp(-12.5 / 8)) < 1e-15
    assert abs(O.integrand(I.F_PDE_INV_SQ, (0.5,) + (0,) * 3, Y)[0] -
               sum(1 / (1 + 0.5 * v) ** 2 for v in Y[0]) / 4) < 1e-14
    assert abs(O.integrand(I.F_LOGSUMEXP, (0,) * 4, Y)[0] - math.log(sum(math.exp(v) for v in Y[0]))) < 1e-14


@pytest.mark.parametrize("f_kind,params", FKINDS)
def test_integrand_gradient_matches_finite_differences(f_kind, params):
    g = np.random.default_rng(11)
    Y = g.standard_normal((5, 7)) * 0.7
    G = O.integrand_grad(f_kind, params, Y)
    h = 1e-6
    for t in range(7):
        E = np.zeros_like(Y); E[:, t] = h
        fd = (O.integrand(f_kind, params, Y + E) - O.integrand(f_kind, params, Y - E)) / (2 * h)
        assert np.allclose(G[:, t], fd, rtol=1e-6, atol=1e-9)


def test_p6_gradient_invariants():
    """LSE: sum_t dQ/dA_jt = mean_k x_kj = c_j / N; linear f: dQ/dA_jt = c_j / (N tau)."""
    for kind in (I.LATTICE, I.DIGITAL_NET):
        p = I.random_problem(3, kind=kind, m=6, s=9, tau=5, R=2, f_kind=I.F_LOGSUMEXP)
        G = O.grad(p)
        c = np.mean([[float(v) for v in closed_form_column_sums(p, r)] for r in range(p.R_eff)], axis=0)
        assert np.allclose(G.sum(axis=1), c / p.N, rtol=1e-13, atol=1e-15)
        p.f_kind = I.F_LINEAR_MEAN
        G = O.grad(p)
        assert np.allclose(G, (c / (p.N * p.tau))[:, None], rtol=1e-13, atol=1e-16)


@pytest.mark.parametrize("f_kind,params", FKINDS[1:])
def test_p6_oracle_gradient_matches_central_differences(f_kind, params):
    p = I.random_problem(5, kind=I.LATTICE, m=5, s=7, tau=4, R=2, transform=I.T_CENTER,
                         f_kind=f_kind, f_params=params, a_scale=0.8)
    G = O.grad(p)
    pairs = np.array([(j, t) for j in range(7) for t in range(4)])
    fd = O.fd_grad(p, pairs, 1e-5)
    want = np.array([G[j, t] for j, t in pairs])
    assert np.allclose(fd, want, rtol=2e-7, atol=1e-10)


@pytest.mark.parametrize("f_kind,params", FKINDS)
def test_separable_form_is_the_integrand(f_kind, params):
    """f(y) = g(sum_t h(y_t)) for every integrand (log-sum-exp for any row shift M)."""
    g = np.random.default_rng(13)
    Y = g.standard_normal((6, 9)) * 0.8
    hf, gf = O.separable(f_kind, params, Y.shape[1])
    for M in (np.zeros(6), Y.max(axis=1), np.full(6, -2.5)):
        got = gf(hf(Y, M[:, None]).sum(axis=1), M)
        assert np.allclose(got, O.integrand(f_kind, params, Y), rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("f_kind,params", FKINDS[1:])
@pytest.mark.parametrize("kind", [I.LATTICE, I.DIGITAL_NET, I.REDUCED_MC])
def test_o8_one_pass_differences_match_reevaluation(kind, f_kind, params):
    """O8 in one pass over the rows (only entry t of every y_k moves with A_jt) gives the central
    differences of the full re-evaluation, and both match the analytic gradient to O(h^2)."""
    p = I.random_problem(6, kind=kind, m=6, s=9, tau=5, R=3, transform=I.T_CENTER if kind != I.REDUCED_MC
                         else I.T_IDENTITY, f_kind=f_kind, f_params=params, a_scale=0.4)
    pairs = np.array([(j, t) for j in range(9) for t in range(5)])
    h = 1e-5 * np.abs(p.A).max()
    rows = O.fd_grad_rows(p, pairs, h)
    full = O.fd_grad(p, pairs, h)
    scale = np.abs(full).max()
    assert np.all(np.abs(rows - full) <= 1e-8 * scale)
    G = O.grad(p)
    assert np.allclose(rows, [G[j, t] for j, t in pairs], rtol=2e-7, atol=1e-9 * scale)


def test_p7_gaussian_expectation_closed_form():
    """Sec. 1: E[mean_t exp(0.2 y_t)] with y = L x, x ~ N(0, I) equals
    mean_t exp(0.02 Sigma_tt); the shifted, inverse-normal reduced lattice must
    approach it (integration sanity of the transform and of A = L^T)."""
    p = I.c2(m=13, s=32)
    p.f_params = (0.2, 0.0, 0.0, 0.0)                     # K = 0: no kink
    Q, _ = O.estimate(p)
    S = p.A.T @ p.A
    exact = np.exp(0.02 * np.diag(S)).mean()
    assert abs(Q[0] - exact) < 2e-3 * exact


# ----------------------------------------------------------------------------- O9 reduced Monte Carlo (Sec. 5)

def mc_problem(m, w, A, R, seed, transform=I.T_IDENTITY, f_kind=I.F_NONE, f_params=(0, 0, 0, 0)):
    w = np.array(w, dtype=np.uint32)
    y = I.mc_samples(np.random.default_rng(seed), m, w, R, force_odd=transform == I.T_INV_NORMAL)
    return I.Problem(I.REDUCED_MC, m, w, np.array(A, dtype=np.float64), y=y, transform=transform,
                     f_kind=f_kind, f_params=f_params)


@pytest.mark.parametrize("seed", range(6))
def test_mc_mixed_radix_index_is_n_mod_Nj(seed):
    """eq. randpts keeps the digits m_s..m_j of n's mixed-radix form, which is n mod N_j: checked
    for every n by brute force (w_1 = 0 as in the paper, and with w_1 > 0 and w_j >= m)."""
    g = np.random.default_rng(300 + seed)
    m = int(g.integers(1, 11))
    w = np.sort(g.integers(0, m + 3, size=int(g.integers(1, 12))))
    if seed % 2 == 0:
        w[0] = 0
    idx = O.mc_sample_index(m, w)
    n = np.arange(1 << m)
    for j, wj in enumerate(w):
        assert np.array_equal(idx[:, j], n % (1 << (m - min(int(wj), m))))


def test_mc_one_period_is_the_given_samples():
    """Points n < N_j of column j are the column's samples in order (the distinct layout)."""
    m, w = 5, [0, 1, 1, 3, 5, 9]
    p = mc_problem(m, w, np.ones((len(w), 2)), R=3, seed=7)
    off = np.cumsum([0] + [1 << (m - min(wj, m)) for wj in w])
    for r in range(3):
        X = O.x32_points(p, r)
        for j in range(len(w)):
            Nj = off[j + 1] - off[j]
            assert np.array_equal(X[:Nj, j], p.y[r, off[j]:off[j + 1]])


def test_mc_linear_estimate_unbiased_with_closed_form_variance():
    """Sec. 5: the reduced MC estimator is unbiased, and for an additive integrand its variance
    (the theorem's sum with the cross terms zero) is sum_j c_j^2 Var(x) / N_j, c_j = tau^-1 sum_t A_jt.
    Over 3000 replicas: the sample mean within 5 standard errors, the sample variance within 15 %
    (5.8 standard errors).  Positive c_j make a wrong sharing of samples between columns visible."""
    m, w = 6, [0, 1, 1, 2, 3, 4, 7]
    A = np.linspace(0.5, 2.0, 3 * len(w)).reshape(len(w), 3)
    R = 3000
    p = mc_problem(m, w, A, R=R, seed=11, f_kind=I.F_LINEAR_MEAN)
    Q, _ = O.estimate(p)
    c = A.sum(axis=1) / A.shape[1]
    Nj = np.array([1 << (m - min(wj, m)) for wj in w], dtype=np.float64)
    mean_x = 0.5 - 2.0 ** -33                      # X32 uniform on {0, ..., 2^32 - 1}
    var_x = (1.0 - 2.0 ** -64) / 12.0
    EQ = c.sum() * mean_x
    VQ = float((c ** 2 * var_x / Nj).sum())
    assert abs(Q.mean() - EQ) <= 5 * math.sqrt(VQ / R)
    assert 0.85 <= Q.var(ddof=1) / VQ <= 1.15


# ----------------------------------------------------------------------------- O10 polynomial lattices (Sec. 1.3)

def test_poly_lattice_worked_example():
    """b=2, m=3, w=(0,1,2), gt=(1+x, 1, 1), worked by hand from the definition.  Column 1:
    k(x)(1+x) mod x^3 has coefficients (k0, k0+k1, k1+k2), read as k0/8 + (k0+k1)/4 + (k1+k2)/2.
    Column 2: k(x) x mod x^3 = k0 x + k1 x^2, i.e. k0/4 + k1/2.  Column 3: k(x) x^2 mod x^3 = k0 x^2."""
    X = O.poly_lattice_x32(3, [0, 1, 2], [0b11, 1, 1]).astype(np.float64) / 2.0 ** 32
    want = np.array([[0, 0, 0], [3, 2, 4], [6, 4, 0], [5, 6, 4], [4, 0, 0], [7, 2, 4], [2, 4, 0], [1, 6, 4]]) / 8.0
    assert np.array_equal(X, want)


def hankel_masks(m, wj, gt):
    """Generating matrix of x -> nu(k(x) g(x)/x^m) as a digital net: digit p (1-based, of 2^-p) is the
    coefficient of x^(m-p) of k(x) g(x), i.e. C[p][q] = g_(m-p-(q-1)) for digit q-1 of k.  Returned
    as column masks (word q-1 holds row p at bit m-p)."""
    wcl = min(wj, m)
    g = [0] * wcl + [(gt >> i) & 1 for i in range(m)] + [0] * m
    masks = []
    for q in range(1, m + 1):
        word = 0
        for p in range(1, m + 1):
            r = m - p - (q - 1)
            if r >= 0 and g[r]:
                word |= 1 << (m - p)
        masks.append(word)
    return masks


@pytest.mark.parametrize("seed", range(6))
def test_poly_lattice_is_a_digital_net(seed):
    """A polynomial lattice point set is the digital net of its (Hankel) generating matrices: the
    polynomial-product oracle (O10) and the matrix-vector oracle (O2, pinned by P2) agree, shifts
    included.  The reduced g_j = x^w gt_j also makes the rows beyond m-w_j zero, as eq.
    reduced_genmat_net2 does for nets."""
    g = np.random.default_rng(900 + seed)
    m = int(g.integers(1, 11))
    w = np.sort(g.integers(0, m + 2, size=int(g.integers(1, 9)))).astype(np.uint32)
    gt = I.odd_z(g, m, w)
    D = I.random_shifts(g, 1, len(w))[0]
    C = np.array([hankel_masks(m, int(wj), int(t)) for wj, t in zip(w, gt)], dtype=np.uint32)
    assert np.array_equal(O.poly_lattice_x32(m, w, gt), O.net_x32(m, w, C))
    assert np.array_equal(O.poly_lattice_x32(m, w, gt, D), O.net_x32(m, w, C, D))


@pytest.mark.parametrize("seed", range(4))
def test_poly_lattice_periodic_permutation(seed):
    """With gt_j(0) = 1, column j depends only on k mod 2^(m-w_j) and one period is a permutation
    of the grid {0, ..., 2^(m-w_j) - 1} / 2^(m-w_j) (brute force)."""
    g = np.random.default_rng(950 + seed)
    m = int(g.integers(2, 11))
    w = np.sort(g.integers(0, m + 1, size=6)).astype(np.uint32)
    X = O.poly_lattice_x32(m, w, I.odd_z(g, m, w)).astype(np.uint64)
    k = np.arange(1 << m)
    for j, wj in enumerate(w):
        q = m - min(int(wj), m)
        per = X[:, j][k % (1 << q)]
        assert np.array_equal(X[:, j], per)
        grid = np.sort(X[: 1 << q, j] >> np.uint64(32 - q)) if q else X[:1, j]
        assert np.array_equal(grid, np.arange(1 << q, dtype=np.uint64)) if q else grid[0] == 0


# ----------------------------------------------------------------------------- O11 Algorithm 4 (Sec. 4)

def nonperiodic_reduced_masks(g, m, w):
    """Random generating matrices whose reduced form (last w_j rows zeroed) keeps full row rank
    m - w_j but, in general, nonzero columns beyond m - w_j: reduced nets that are not periodic."""
    C = np.zeros((len(w), m), dtype=np.uint32)
    for j, wj in enumerate(w):
        q = m - min(int(wj), m)
        while True:
            B = g.integers(0, 2, size=(m, m))
            B[q:, :] = 0
            if q == 0 or np.linalg.matrix_rank(B[:q].astype(float)) == q:
                # (a real-valued rank >= the GF(2) rank; full GF(2) rank is checked below)
                rows = [int(sum(int(B[p, c]) << c for c in range(m))) for p in range(q)]
                basis, ok = [0] * 32, True
                for x in rows:
                    while x:
                        b = x.bit_length() - 1
                        if not basis[b]:
                            basis[b] = x
                            break
                        x ^= basis[b]
                    else:
                        ok = False
                if ok:
                    break
        for col in range(m):
            C[j, col] = sum(int(B[p, col]) << (m - 1 - p) for p in range(m))
    return C


@pytest.mark.parametrize("seed", range(4))
def test_alg4_returns_XA_exactly(seed):
    """Algorithm 4 in exact rationals equals the dense definition X A (Sec. 4: 'Return: P = X A'),
    on reduced nets that are not periodic, with a constant column (w_j >= m) skipped."""
    g = np.random.default_rng(1200 + seed)
    m = int(g.integers(2, 6))
    w = np.sort(np.append(g.integers(0, m, size=3), m + 1)).astype(np.uint32)
    C = nonperiodic_reduced_masks(g, m, w)
    A = [[Fraction(int(v), 7) for v in g.integers(-9, 10, size=3)] for _ in range(len(w))]
    P = O.alg4_product(m, w, C, A, exact=True)
    X = [[Fraction(int(v), 1 << 32) for v in row] for row in O.net_x32(m, w, C)]
    for n in range(1 << m):
        for t in range(3):
            assert P[n][t] == sum(X[n][j] * A[j][t] for j in range(len(w)))


@pytest.mark.parametrize("seed", range(4))
def test_reduced_net_values_repeat_exactly_2_to_the_w(seed):
    """Sec. 4: in a reduced net whose reduced matrix keeps rank m - w_j, column j takes the values
    k / 2^(m-w_j) only, each exactly 2^(w_j) times, also when it is not periodic."""
    g = np.random.default_rng(1300 + seed)
    m = int(g.integers(2, 9))
    w = np.sort(g.integers(0, m + 1, size=5)).astype(np.uint32)
    C = nonperiodic_reduced_masks(g, m, w)
    X = O.net_x32(m, w, C).astype(np.uint64)
    for j, wj in enumerate(w):
        q = m - min(int(wj), m)
        v = X[:, j] >> np.uint64(32 - q) if q else np.zeros(1 << m, dtype=np.uint64)
        assert np.array_equal(v << np.uint64(32 - q) if q else X[:, j], X[:, j])      # on the 2^-q grid
        assert np.array_equal(np.bincount(v.astype(np.int64), minlength=1 << q), np.full(1 << q, 1 << min(int(wj), m)))


# ----------------------------------------------------------------------------- O2 in a prime base b

@pytest.mark.parametrize("b,m", [(3, 4), (5, 3), (7, 2)])
def test_base_b_identity_net_is_the_radical_inverse(b, m):
    """C = identity over F_b gives the van der Corput sequence in base b: the digits of n mirrored
    about the radix point (a textbook closed form)."""
    X = O.net_points_base(b, m, [0], [np.eye(m, dtype=np.int64)])
    for n in range(b ** m):
        d, v, scale = n, Fraction(0), Fraction(1, b)
        while d:
            v += (d % b) * scale
            d //= b
            scale /= b
        assert X[n, 0] == float(v)


@pytest.mark.parametrize("seed", range(4))
def test_base_b_net_reduces_like_base_2(seed):
    """For b = 2 the general-base net equals O2 on random reduced nets; for b = 3 a reduced column
    takes each of its b^(m-w_j) grid values exactly b^(w_j) times when the leading block is invertible."""
    g = np.random.default_rng(1400 + seed)
    m = int(g.integers(2, 8))
    w = np.sort(g.integers(0, m + 1, size=4)).astype(np.uint32)
    C2 = I.periodic_net_masks(g, m, w)
    mats = [[[(int(C2[j, q]) >> (m - 1 - p)) & 1 for q in range(m)] for p in range(m)] for j in range(len(w))]
    assert np.array_equal(O.net_points_base(2, m, w, mats), O.net_x32(m, w, C2).astype(np.float64) / 2.0 ** 32)
    b, m3 = 3, 4
    for wj in range(m3 + 1):
        q = m3 - wj
        while True:
            B = g.integers(0, b, size=(q, q))
            if q == 0 or round(abs(np.linalg.det(B))) % b != 0:
                break
        Cm = np.zeros((m3, m3), dtype=np.int64)
        Cm[:q, :q] = B
        x = O.net_points_base(b, m3, [wj], [Cm])[:, 0]
        vals, counts = np.unique(np.round(x * b ** q).astype(np.int64), return_counts=True)
        assert np.array_equal(vals, np.arange(b ** q)) and np.all(counts == b ** wj)


def test_pde_assembly_pins():
    """Sec. 1's D_k = sum_j x_{j,k} C_j: with C_j = delta_{j,j0} I every D_k is x_{k,j0} I, and over
    the whole point set sum_k D_k = sum_j c_j C_j with the exact column sums c_j (P5)."""
    p = I.pde_assembly(m=7, s=12, M=5, R=1)
    C = I.stiffness_terms(12, 5)
    for j0 in (0, 5, 11):
        E = np.zeros_like(C)
        E[j0] = np.eye(5)
        D = O.assemble(p, E)
        X = O.points(p)
        assert np.array_equal(D, X[:, j0][:, None, None] * np.eye(5)[None])
    D = O.assemble(p, C)
    c = np.array([float(v) for v in closed_form_column_sums(p, 0)])
    assert np.allclose(D.sum(axis=0), np.einsum("j,juv->uv", c, C), rtol=1e-13, atol=1e-12)
    # the stiffness terms are symmetric and their rows sum to zero away from the boundary
    assert np.allclose(C, C.transpose(0, 2, 1))
    assert np.allclose(C[:, 1:-1, :].sum(axis=2), 0.0, atol=1e-9)


# ----------------------------------------------------------------------------- prime bases b > 2

@pytest.mark.parametrize("b,m", [(3, 4), (5, 3), (7, 2)])
def test_base_b_lattice_points_exact(b, m):
    """Base-b lattice points (Sec. 1.3) against exact rationals: x = {k b^w z / b^m} from the
    unreduced definition equals the reduced (k z mod b^q)/b^q, the shifted {x + D 2^-32} is within
    two roundings of the exact value, and every column over one period is a permutation of the grid."""
    w = np.array([0, 0, 1, min(2, m), m, m + 1], dtype=np.uint32)
    p = I.base_b_problem(b * 10 + m, b, m, len(w), 2, R=2, w=w)
    X0 = O.lattice_points_base(b, m, p.w, p.z)
    N = b ** m
    for j, wj in enumerate(p.w):
        q = m - min(int(wj), m)
        for k in range(N):
            red = Fraction((k * int(p.z[j])) % (b ** q), b ** q) if q else Fraction(0)
            assert abs(Fraction(float(X0[k, j])) - red) <= Fraction(1, 2 ** 53)      # one rounding
        per = sorted(Fraction(int(round(float(X0[k, j]) * b ** q)), b ** q) for k in range(b ** q))
        assert per == [Fraction(u, b ** q) for u in range(b ** q)]
    for r in range(2):
        Xs = O.points(p, r)
        for j in range(len(w)):
            for k in range(N):
                q = m - min(int(p.w[j]), m)
                red = Fraction((k * int(p.z[j])) % (b ** q), b ** q) if q else Fraction(0)
                exact = red + Fraction(int(p.shifts[r, j]), 2 ** 32)
                exact -= math.floor(exact)
                assert abs(Fraction(float(Xs[k, j])) - exact) <= Fraction(2, 2 ** 53)


@pytest.mark.parametrize("b", [3, 5])
def test_base_b_mc_index_is_n_mod_Nj(b):
    m = 4 if b == 3 else 3
    w = np.array([0, 1, 1, 2, m], dtype=np.uint32)
    idx = O.mc_sample_index(m, w, b=b)
    for j, wj in enumerate(w):
        Nj = b ** (m - min(int(wj), m))
        assert np.array_equal(idx[:, j], np.arange(b ** m) % Nj)


@pytest.mark.parametrize("b", [3, 5])
def test_base_b_linear_closed_form(b):
    """Unshifted: column j sums to b^w (b^q - 1)/2 over the N points, so the linear integrand's
    estimate is sum_j c_j sum_t a_jt / (N tau) exactly (up to float rounding)."""
    m = 5 if b == 3 else 3
    p = I.base_b_problem(7 + b, b, m, 9, 4, R=0, f_kind=I.F_LINEAR_MEAN)
    c = np.array([b ** min(int(wj), m) * (b ** (m - min(int(wj), m)) - 1) / 2 for wj in p.w])
    want = c @ np.asarray(p.A, dtype=np.float64).sum(axis=1) / (p.N * p.tau)
    Q, _ = O.estimate(p)
    assert abs(Q[0] - want) <= 1e-14 * max(1.0, abs(want))
    assert np.allclose(O.points(p).sum(axis=0), c, rtol=1e-14, atol=1e-12)
