"""CPU FP64 oracle for the reduced QMC matrix-vector product.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
module.  The library in ``paper_2305_11645_gb300`` never calls it and shares no
code with it.

What it computes is the plain definition of every quantity, in float64 (exact
integers where the definition is integer), with no blocking, reuse or
reordering beyond what the definitions state:

  O1  rank-1 lattice points from the *unreduced* generating vector
      (b^{w_j} z_j) (Sec. 1.3): x_{k,j} = {k b^{w_j} z_j / N}, in integers.
      The reduced form (k z_j mod b^{m-w_j}) / b^{m-w_j} is deliberately not
      used here: it is what the fast method exploits and is checked against
      this definition by the tests.
  O2  digital-net points (Sec. 4, eq. def:digital with the reduced generating
      matrices of eq. reduced_genmat_net2): digits of n least significant
      first, the last min(w_j, m) rows of C^(j) set to zero, y digits as the
      matrix-vector product over GF(2), y = sum_p y_p b^-p; net_points_base
      does the same over F_b for any prime b.
  O3  random shifts as 32-bit fixed point D_j * 2^-32 (Sec. 2.3):
      lattice {x + Delta} = (X32 + D) mod 2^32, nets (digital shift)
      X32 XOR D, with X32 = x * 2^32.  Lattices in a prime base b > 2 have points
      u / b^q that 32 bits cannot hold: they are float64, x = num / b^m, and
      {x + Delta} is the rounded sum, less 1 if it reaches 1 (lattice_points_base).
  O4  coordinate transforms applied elementwise (Sec. 2.3): identity,
      centring x - 1/2, inverse normal CDF (scipy.special.ndtri), tent
      1 - |1 - 2x| (Sec. 1.2).
  O5  the dense product Y = X A (eq. Eq_XA_product), numpy matmul; and Sec. 1's
      PDE assembly D_k = sum_j x_{j,k} C_j summed matrix by matrix (assemble).
  O6  the QMC rule Q_N(f) = N^-1 sum_k f(x_k^T A) (eq. (2)) per shift, and
      the mean over the R shifts.
  O7  the gradient of the shift-averaged estimate with respect to A:
      (1/(R N)) sum_r X_r^T grad f(Y_r).
  O8  central finite differences of the estimate in single entries of A: by
      re-evaluating the estimate (fd_grad), or in one pass over the rows
      (fd_grad_rows), since only entry t of every y_k moves with A_jt.
  O11 the product of Sec. 4 (Algorithm 4) for reduced nets, unshifted: coordinate
      j takes only the grid values v / 2^(m-w_j), so x_{n,j} a_j is a row of the
      table of multiples (v / 2^(m-w_j)) a_j selected by v = floor(x_{n,j}
      2^(m-w_j)); X A is the sum of the selected rows over j (exact rationals
      on request).  It holds for any reduced net, periodic or not.
  O10 reduced polynomial lattice points (Sec. 1.3): x_{k,j} = nu(k(x) g_j(x) / x^m)
      over F_2 with g_j = x^{w_j} gt_j, the product of the coefficient arrays
      written out mod 2 and mod x^m, the coefficient of x^i the digit of 2^(i-m);
      digital shifts as for nets.
  O9  reduced Monte Carlo points (Sec. 5, eq. randpts): with N_j = 2^(m-w_j),
      N_{s+1} = 1 and M_j = N_j / N_{j+1}, write n in the mixed radix
      n = m_s N_{s+1} + m_{s-1} N_s + ... + m_1 N_2 (0 <= m_j < M_j) and take
      x_{j,n} = y_{j, m_s N_{s+1} + ... + m_j N_{j+1}}, the samples y given as
      32-bit words (the caller's draws).

Parity pins for every function live in tests/test_oracle_pins.py.  Nothing in
this file is "parity unpinned".
"""
from __future__ import annotations

import math
from typing import Iterable, Optional, Sequence

import numpy as np
from scipy import special as _sp

LATTICE, DIGITAL_NET, REDUCED_MC, POLY_LATTICE = 0, 1, 2, 3
T_IDENTITY, T_CENTER, T_INV_NORMAL, T_TENT = 0, 1, 2, 3
F_NONE, F_LINEAR_MEAN, F_MEAN_COS, F_CALL_MEAN_EXP, F_GAUSS_NORM2, F_PDE_INV_SQ, F_LOGSUMEXP = range(7)

TWO32 = 1 << 32


# ----------------------------------------------------------------------------- O1 lattice points

def lattice_numerators(b: int, m: int, w: Sequence[int], z: Sequence[int],
                       ks: Optional[np.ndarray] = None) -> np.ndarray:
    """Integers (k * b^{min(w_j,m)} * z_j) mod b^m, i.e. N * x_{k,j} of the
    unreduced lattice x_k = {k z / N} with z = (b^{w_1} z_1, ..., b^{w_s} z_s)."""
    N = b ** m
    gens = [(b ** min(int(wj), m)) * int(zj) for wj, zj in zip(w, z)]   # unreduced generating vector
    exact_in_int64 = (N - 1) * max(gens + [1]) < (1 << 63)
    dt = np.int64 if exact_in_int64 else object
    ks = np.arange(N, dtype=dt) if ks is None else np.asarray(ks).astype(dt)
    out = np.empty((len(ks), len(w)), dtype=dt)
    for j, gen in enumerate(gens):
        out[:, j] = (ks * gen) % N
    return out


def lattice_x32(m: int, w, z, shift: Optional[np.ndarray] = None, ks=None) -> np.ndarray:
    """b = 2 lattice points as 32-bit fixed point X32 = x * 2^32 (x exact, m <= 32),
    optionally shifted: (X32 + D_j) mod 2^32."""
    num = lattice_numerators(2, m, w, z, ks).astype(np.uint64)      # < 2^m
    x32 = (num * np.uint64(1 << (32 - m))).astype(np.uint32)       # x * 2^32, < 2^32
    return x32 if shift is None else apply_shift(LATTICE, x32, shift)


# ----------------------------------------------------------------------------- O2 digital nets

def net_matrix(masks: Sequence[int], m: int) -> np.ndarray:
    """Column masks -> m x m 0/1 matrix C[p, q] (0-based p, q), row p at bit m-1-p."""
    col = np.array([int(v) for v in masks[:m]], dtype=np.int64)[None, :]
    row_bit = np.array([m - 1 - p for p in range(m)], dtype=np.int64)[:, None]
    return (col >> row_bit) & 1


def reduced_net_matrix(masks: Sequence[int], m: int, wj: int) -> np.ndarray:
    """eq. reduced_genmat_net2: zero the last min(w_j, m) rows of C^(j)."""
    C = net_matrix(masks, m)
    C[m - min(int(wj), m):, :] = 0
    return C


def digits_lsb_first(ks: np.ndarray, m: int) -> np.ndarray:
    ks = np.asarray(ks, dtype=np.int64)
    return np.stack([(ks >> q) & 1 for q in range(m)], axis=1)   # n = digits . (1, 2, 4, ...)


def net_x32(m: int, w, C: np.ndarray, shift: Optional[np.ndarray] = None, ks=None) -> np.ndarray:
    """b = 2 reduced digital net (Algorithm 3) as X32 = y * 2^32, optionally XOR-shifted."""
    N = 1 << m
    ks = np.arange(N, dtype=np.int64) if ks is None else np.asarray(ks, dtype=np.int64)
    # (the integer sums below are at most m ones, or y 2^m < 2^m: exact in float64, so the
    # products run through the float BLAS, a block of columns per call)
    dig = digits_lsb_first(ks, m).astype(np.float64)      # len(ks) x m
    out = np.empty((len(ks), len(w)), dtype=np.uint64)
    place = np.array([1 << (m - 1 - p) for p in range(m)], dtype=np.float64)   # y_p b^-p, scaled by 2^m
    blk = 64
    for j0 in range(0, len(w), blk):
        cols = range(j0, min(len(w), j0 + blk))
        Chats = np.concatenate([reduced_net_matrix(C[j], m, int(w[j])).astype(np.float64).T for j in cols], axis=1)
        ydig = ((dig @ Chats).astype(np.int64) & 1).astype(np.float64)   # y digits = Chat n over GF(2)
        ydig = ydig.reshape(len(ks), len(cols), m)
        y_int = (ydig @ place).astype(np.uint64)                        # y * 2^m, per column
        out[:, j0:j0 + len(cols)] = y_int << np.uint64(32 - m)
    x32 = out.astype(np.uint32)
    return x32 if shift is None else apply_shift(DIGITAL_NET, x32, shift)


# ----------------------------------------------------------------------------- O10 polynomial lattices

def poly_lattice_x32(m: int, w, gt, shift: Optional[np.ndarray] = None, ks=None) -> np.ndarray:
    """b = 2 reduced polynomial lattice points as X32 = x * 2^32: k(x) has the binary digits of k as
    coefficients, g_j(x) = x^{min(w_j,m)} gt_j(x) (gt_j's coefficient of x^i at bit i), the product
    k(x) g_j(x) is taken mod 2 and mod x^m, and nu reads coefficient a_i as the digit of 2^(i-m)."""
    N = 1 << m
    ks = np.arange(N, dtype=np.int64) if ks is None else np.asarray(ks, dtype=np.int64)
    kd = digits_lsb_first(ks, m)                                  # coefficients of k(x), degree < m
    out = np.empty((len(ks), len(w)), dtype=np.uint64)
    for j, (wj, gj) in enumerate(zip(w, gt)):
        wcl = min(int(wj), m)
        g = [0] * wcl + [(int(gj) >> i) & 1 for i in range(m)]     # coefficients of x^w gt(x)
        c = np.zeros((len(ks), m), dtype=np.int64)
        for i in range(m):                                        # c_i = sum_{l <= i} k_l g_{i-l} mod 2
            for l in range(i + 1):
                if g[i - l]:
                    c[:, i] ^= kd[:, l]
        y_int = (c.astype(np.uint64) * (np.uint64(1) << np.arange(m, dtype=np.uint64))[None, :]).sum(axis=1)
        out[:, j] = y_int << np.uint64(32 - m)                    # nu: y 2^m = sum_i a_i 2^i
    x32 = out.astype(np.uint32)
    return x32 if shift is None else apply_shift(POLY_LATTICE, x32, shift)


# ----------------------------------------------------------------------------- O11 Algorithm 4

def alg4_product(m: int, w, C: np.ndarray, A, exact: bool = False):
    """X A for the unshifted reduced net with column masks C (b = 2), as Sec. 4 obtains it without
    multiplying every entry: coordinate j of every point lies on the grid {v / 2^(m - w_j)}, v <
    2^(m - w_j), so the products x_{n,j} a_j are drawn from a table of the 2^(m - w_j) multiples
    (v / 2^(m - w_j)) a_j, indexed by v = floor(x_{n,j} 2^(m - w_j)), and X A is the sum over the
    coordinates j with w_j < m of the table rows each point selects (coordinates with w_j >= m are
    zero).  Columns are taken in ascending j.  It holds for any reduced net, periodic or not.  With
    exact=True, A's entries and the result are Fractions (an N x tau list of lists)."""
    from fractions import Fraction
    N = 1 << m
    X32 = net_x32(m, w, C)                                      # y_{n,j} 2^32, O2
    tau = len(A[0])
    P = [[Fraction(0)] * tau for _ in range(N)] if exact else np.zeros((N, tau))
    for j in range(len(w)):
        q = m - min(int(w[j]), m)                               # grid of 2^q values
        if q == 0:
            continue                                            # the coordinate is 0
        v = (X32[:, j].astype(np.uint64) >> np.uint64(32 - q)).astype(np.int64)   # x 2^q, exact
        if exact:
            a = [Fraction(x) for x in A[j]]
            table = [[Fraction(k, 1 << q) * x for x in a] for k in range(1 << q)]
            for n in range(N):
                P[n] = [p + c for p, c in zip(P[n], table[v[n]])]
        else:
            table = (np.arange(1 << q, dtype=np.float64) / (1 << q))[:, None] * np.asarray(A[j], dtype=np.float64)
            P = P + table[v]
    return P


# ----------------------------------------------------------------------------- O9 reduced Monte Carlo

def mc_sample_index(m: int, w, ks=None, b: int = 2) -> np.ndarray:
    """Index of the sample that point n uses in coordinate j (eq. randpts), by the mixed-radix
    digits of n (N_j = b^(m-w_j)).  The paper starts from w_1 = 0; a first column with w_1 > 0 is
    handled by a leading virtual coordinate of weight 0, so that n < N is always representable."""
    N = b ** m
    ks = np.arange(N, dtype=np.int64) if ks is None else np.asarray(ks, dtype=np.int64)
    wl = [0] + [min(int(wj), m) for wj in w] + [m]          # virtual w_0 = 0, ..., w_{s+1} = m
    Nl = [b ** (m - wj) for wj in wl]                       # N_0 = N, N_1, ..., N_{s+1} = 1
    Ml = [Nl[i] // Nl[i + 1] for i in range(len(Nl) - 1)]  # M_i = N_i / N_{i+1}
    digits = [(ks // Nl[i + 1]) % Ml[i] for i in range(len(Ml))]     # m_i, place value N_{i+1}
    out = np.empty((len(ks), len(w)), dtype=np.int64)
    for j in range(len(w)):
        jj = j + 1                                           # index in the extended sequence
        idx = np.zeros(len(ks), dtype=np.int64)
        for i in range(jj, len(Ml)):                         # m_{jj} N_{jj+1} + ... + m_s N_{s+1}
            idx += digits[i] * Nl[i + 1]
        out[:, j] = idx
    return out


def mc_x32(m: int, w, y: np.ndarray, ks=None, b: int = 2) -> np.ndarray:
    """X32 of the reduced MC points of one replica: x_{j,n} = y_{j, index}, where replica row y
    holds column j's samples at offset sum_{j' < j} N_{j'}."""
    idx = mc_sample_index(m, w, ks, b)
    off = np.cumsum([0] + [b ** (m - min(int(wj), m)) for wj in w])[:-1]
    return np.asarray(y, dtype=np.uint32)[idx + off[None, :]]


def net_points_base(b: int, m: int, w, C: np.ndarray, ks=None) -> np.ndarray:
    """Digital net in a prime base b (Sec. 4, eq. def:digital) with the reduced matrices of eq.
    reduced_genmat_net2, as float64 points: C[j] is the m x m matrix over F_b (entries 0..b-1,
    row p-1 the digit of b^-p, column q-1 digit q-1 of n, least significant first), the last
    min(w_j, m) rows are zeroed, y digits = C n mod b, y = sum_p y_p b^-p.  (b = 2 agrees with O2.)"""
    N = b ** m
    ks = np.arange(N, dtype=np.int64) if ks is None else np.asarray(ks, dtype=np.int64)
    dig = np.stack([(ks // b ** q) % b for q in range(m)], axis=1)          # len(ks) x m, n's digits
    out = np.empty((len(ks), len(w)), dtype=np.float64)
    place = np.array([b ** (m - 1 - p) for p in range(m)], dtype=np.int64)     # y_p b^-p, scaled by b^m
    for j, wj in enumerate(w):
        Chat = np.array(C[j], dtype=np.int64) % b
        Chat[m - min(int(wj), m):, :] = 0
        ydig = (dig @ Chat.T) % b
        out[:, j] = (ydig @ place) / float(N)       # one rounding: the integer y b^m over b^m
    return out


# ----------------------------------------------------------------------------- O3/O4 shifts and transforms

def apply_shift(kind: int, x32: np.ndarray, shift) -> np.ndarray:
    """O3 on 32-bit fixed-point rows: a lattice adds D mod 2^32 ({x + Delta}); nets and
    polynomial lattices XOR it (the digital shift)."""
    # (uint32 array addition wraps modulo 2^32)
    D = np.asarray(shift, dtype=np.uint32)[None, :]
    if kind == LATTICE:
        return np.asarray(x32, dtype=np.uint32) + D
    return np.asarray(x32, dtype=np.uint32) ^ D


def unshifted_x32(problem, ks=None) -> np.ndarray:
    """The rule's points before any shift (O1, O2 or O10)."""
    if problem.kind == POLY_LATTICE:
        return poly_lattice_x32(problem.m, problem.w, problem.z, None, ks)
    if problem.kind == LATTICE:
        return lattice_x32(problem.m, problem.w, problem.z, None, ks)
    return net_x32(problem.m, problem.w, problem.C, None, ks)


def lattice_points_base(b: int, m: int, w, z, shift=None, ks=None) -> np.ndarray:
    """Rank-1 lattice points in base b as float64 (O1 with the 32-bit shift of O3): x = num / b^m
    with num = (k b^{min(w_j,m)} z_j) mod b^m from the unreduced generating vector, one rounded
    division; shifted, {x + D_j 2^-32} = x + D_j 2^-32, less 1 if it reaches 1 (one rounded
    addition, the subtraction exact)."""
    x = lattice_numerators(b, m, w, z, ks).astype(np.float64) / float(b ** m)
    if shift is not None:
        x = x + np.asarray(shift, dtype=np.float64)[None, :] * (1.0 / TWO32)
        x = np.where(x >= 1.0, x - 1.0, x)
    return x


def shifted_rows(problem, ks):
    """(r, X) for every shift r (reduced MC: every replica) of the rows ks, X the transformed
    points (O4): the unshifted points of the rows are formed once and each shift is applied to
    them (O3)."""
    if problem.kind == REDUCED_MC:
        for r in range(problem.R_eff):
            yield r, transform(mc_x32(problem.m, problem.w, problem.y[r], ks, problem.b), problem.transform)
        return
    if problem.b != 2:
        if problem.kind != LATTICE:
            raise ValueError("base b > 2: lattices and reduced MC only")
        for r in range(problem.R_eff):
            shift = None if problem.shifts is None else problem.shifts[r]
            yield r, transform_x(lattice_points_base(problem.b, problem.m, problem.w, problem.z, shift, ks),
                                 problem.transform)
        return
    base = unshifted_x32(problem, ks)
    for r in range(problem.R_eff):
        x32 = base if problem.shifts is None else apply_shift(problem.kind, base, problem.shifts[r])
        yield r, transform(x32, problem.transform)


def x32_points(problem, shift_idx: int = 0, ks=None) -> np.ndarray:
    if problem.kind == REDUCED_MC:
        return mc_x32(problem.m, problem.w, problem.y[shift_idx], ks)
    shift = None if problem.shifts is None else problem.shifts[shift_idx]
    if problem.kind == POLY_LATTICE:
        return poly_lattice_x32(problem.m, problem.w, problem.z, shift, ks)
    if problem.kind == LATTICE:
        return lattice_x32(problem.m, problem.w, problem.z, shift, ks)
    return net_x32(problem.m, problem.w, problem.C, shift, ks)


def transform(x32: np.ndarray, kind: int) -> np.ndarray:
    return transform_x(np.asarray(x32, dtype=np.float64) * (1.0 / TWO32), kind)   # exact: 32 bits < 53


def transform_x(x: np.ndarray, kind: int) -> np.ndarray:
    """O4 on points given as float64."""
    x = np.asarray(x, dtype=np.float64)
    if kind == T_IDENTITY:
        return x
    if kind == T_CENTER:
        return x - 0.5
    if kind == T_INV_NORMAL:
        with np.errstate(divide="ignore"):
            return _sp.ndtri(x)
    if kind == T_TENT:
        return 1.0 - np.abs(1.0 - 2.0 * x)
    raise ValueError(kind)


def points(problem, shift_idx: int = 0, ks=None) -> np.ndarray:
    """Rows x_k^T (after shift and transform) as float64, for k in ks (default all)."""
    if problem.b != 2 and problem.kind != REDUCED_MC:
        if problem.kind != LATTICE:
            raise ValueError("base b > 2: lattices and reduced MC only")
        shift = None if problem.shifts is None else problem.shifts[shift_idx]
        return transform_x(lattice_points_base(problem.b, problem.m, problem.w, problem.z, shift, ks),
                           problem.transform)
    if problem.kind == REDUCED_MC:
        return transform(mc_x32(problem.m, problem.w, problem.y[shift_idx], ks, problem.b), problem.transform)
    return transform(x32_points(problem, shift_idx, ks), problem.transform)


# ----------------------------------------------------------------------------- O5 product

def product(X: np.ndarray, A: np.ndarray) -> np.ndarray:
    return np.asarray(X, dtype=np.float64) @ np.asarray(A, dtype=np.float64)


def row_chunks(N: int, chunk: int) -> Iterable[np.ndarray]:
    for k0 in range(0, N, chunk):
        yield np.arange(k0, min(N, k0 + chunk), dtype=np.int64)


def reduced_matmul(problem, shift_idx: int = 0, ks=None) -> np.ndarray:
    """Rows of P = X A for the given shift (all N rows by default)."""
    return product(points(problem, shift_idx, ks), problem.A)


def assemble(problem, C: np.ndarray, shift_idx: int = 0, ks=None) -> np.ndarray:
    """Sec. 1's PDE assembly, D_k = sum_j x_{j,k} C_j (C: s x M x M), for the rows ks of the given
    shift, summed over j directly (not through X A)."""
    X = points(problem, shift_idx, ks)
    C = np.asarray(C, dtype=np.float64)
    D = np.zeros((X.shape[0],) + C.shape[1:])
    for j in range(C.shape[0]):
        D += X[:, j][:, None, None] * C[j][None, :, :]
    return D


# ----------------------------------------------------------------------------- O6 integrands

def integrand(f_kind: int, params, Y: np.ndarray) -> np.ndarray:
    """f(y) for every row y of Y (float64)."""
    Y = np.asarray(Y, dtype=np.float64)
    tau = Y.shape[1]
    if f_kind == F_LINEAR_MEAN:
        return Y.mean(axis=1)
    if f_kind == F_MEAN_COS:
        return np.cos(Y).mean(axis=1)
    if f_kind == F_CALL_MEAN_EXP:
        c, K = params[0], params[1]
        return np.maximum(np.exp(c * Y).mean(axis=1) - K, 0.0)
    if f_kind == F_GAUSS_NORM2:
        return np.exp(-(Y * Y).sum(axis=1) / (2.0 * tau))
    if f_kind == F_PDE_INV_SQ:
        c = params[0]
        return (1.0 / (1.0 + c * Y) ** 2).mean(axis=1)
    if f_kind == F_LOGSUMEXP:
        M = Y.max(axis=1)
        return M + np.log(np.exp(Y - M[:, None]).sum(axis=1))
    raise ValueError(f_kind)


def integrand_grad(f_kind: int, params, Y: np.ndarray) -> np.ndarray:
    """df/dy_t for every row (float64), the analytic derivative of integrand()."""
    Y = np.asarray(Y, dtype=np.float64)
    tau = Y.shape[1]
    if f_kind == F_LINEAR_MEAN:
        return np.full_like(Y, 1.0 / tau)
    if f_kind == F_MEAN_COS:
        return -np.sin(Y) / tau
    if f_kind == F_CALL_MEAN_EXP:
        c, K = params[0], params[1]
        E = np.exp(c * Y)
        active = (E.mean(axis=1) - K) > 0.0
        return np.where(active[:, None], c * E / tau, 0.0)
    if f_kind == F_GAUSS_NORM2:
        f = np.exp(-(Y * Y).sum(axis=1) / (2.0 * tau))
        return -f[:, None] * Y / tau
    if f_kind == F_PDE_INV_SQ:
        c = params[0]
        return -2.0 * c / (1.0 + c * Y) ** 3 / tau
    if f_kind == F_LOGSUMEXP:
        M = Y.max(axis=1)
        E = np.exp(Y - M[:, None])
        return E / E.sum(axis=1)[:, None]
    raise ValueError(f_kind)


# ----------------------------------------------------------------------------- O6/O7 estimate and gradient

def estimate(problem, chunk: int = 1 << 16):
    """Per-shift Q_N(f) (eq. (2)) and their mean; R = 0 counts as one unshifted rule.  Each shift's
    sum over the rows is taken chunk by chunk in increasing row order."""
    Q = np.zeros(problem.R_eff)
    for ks in row_chunks(problem.N, chunk):
        for r, X in shifted_rows(problem, ks):
            Q[r] += integrand(problem.f_kind, problem.f_params, product(X, problem.A)).sum()
    Q /= problem.N
    return Q, Q.mean()


def grad(problem, chunk: int = 1 << 16) -> np.ndarray:
    """d(mean_r Q_r)/dA = (1/(R N)) sum_r X_r^T grad f(X_r A)."""
    G = np.zeros((problem.s, problem.tau))
    for ks in row_chunks(problem.N, chunk):
        for r, X in shifted_rows(problem, ks):
            G += X.T @ integrand_grad(problem.f_kind, problem.f_params, product(X, problem.A))
    return G / (problem.R_eff * problem.N)


def estimate_with_A(problem, A: np.ndarray, chunk: int = 1 << 16) -> float:
    Q = 0.0
    for ks in row_chunks(problem.N, chunk):
        for r, X in shifted_rows(problem, ks):
            Q += integrand(problem.f_kind, problem.f_params, product(X, A)).sum()
    return Q / (problem.R_eff * problem.N)


def fd_grad(problem, pairs: np.ndarray, h: float) -> np.ndarray:
    """O8: central differences (Q(A + h e_jt) - Q(A - h e_jt)) / (2h), one full
    re-evaluation of the estimate per perturbed matrix."""
    out = np.zeros(len(pairs))
    A = np.asarray(problem.A, dtype=np.float64)
    for i, (j, t) in enumerate(pairs):
        Ap = A.copy(); Ap[j, t] += h
        Am = A.copy(); Am[j, t] -= h
        out[i] = (estimate_with_A(problem, Ap) - estimate_with_A(problem, Am)) / (2.0 * h)
    return out


# ----------------------------------------------------------------------------- O8 in one pass over the rows

def separable(f_kind: int, params, tau: int):
    """The integrands as f(y) = g(u), u = sum_t h(y_t) (row-separable).  Returns (h, g), where h
    and g also take the row's shift M (used by log-sum-exp only: h = exp(y - M), g = M + log u,
    the same value for any M)."""
    c, K = params[0], params[1]
    if f_kind == F_LINEAR_MEAN:
        return (lambda y, M: y), (lambda u, M: u / tau)
    if f_kind == F_MEAN_COS:
        return (lambda y, M: np.cos(y)), (lambda u, M: u / tau)
    if f_kind == F_CALL_MEAN_EXP:
        return (lambda y, M: np.exp(c * y)), (lambda u, M: np.maximum(u / tau - K, 0.0))
    if f_kind == F_GAUSS_NORM2:
        return (lambda y, M: y * y), (lambda u, M: np.exp(-u / (2.0 * tau)))
    if f_kind == F_PDE_INV_SQ:
        return (lambda y, M: 1.0 / (1.0 + c * y) ** 2), (lambda u, M: u / tau)
    if f_kind == F_LOGSUMEXP:
        return (lambda y, M: np.exp(y - M)), (lambda u, M: M + np.log(u))
    raise ValueError(f_kind)


def fd_grad_rows(problem, pairs: np.ndarray, h: float, chunk: int = 1 << 16) -> np.ndarray:
    """O8 without re-evaluating the estimate: moving A_jt by +-h moves only entry t of every
    y_k = x_k^T A, by +-h x_kj, so with f = g(u), u_k = sum_t h(y_kt), the perturbed row values are
    g(u_k - h(y_kt) + h(y_kt +- h x_kj)).  Returns (1/(2 h R N)) sum_r sum_k (f_k^+ - f_k^-) for
    every (j, t) in pairs: the same central differences as fd_grad, in one pass over the rows."""
    A = np.asarray(problem.A, dtype=np.float64)
    hf, gf = separable(problem.f_kind, problem.f_params, problem.tau)
    acc = np.zeros(len(pairs))
    for ks in row_chunks(problem.N, chunk):
        for r, X in shifted_rows(problem, ks):
            Y = product(X, A)
            M = Y.max(axis=1) if problem.f_kind == F_LOGSUMEXP else np.zeros(len(ks))
            u = hf(Y, M[:, None]).sum(axis=1)
            for i, (j, t) in enumerate(pairs):
                y, d = Y[:, t], h * X[:, j]
                rest = u - hf(y, M)
                acc[i] += (gf(rest + hf(y + d, M), M) - gf(rest + hf(y - d, M), M)).sum()
    return acc / (2.0 * h * problem.R_eff * problem.N)
