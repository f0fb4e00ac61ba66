"""Seeded synthetic workloads for the reduced QMC matrix-vector product.

This module only draws the numbers that define a problem instance: reduction
indices w, generating vectors z, generating matrices C, the matrix A, random
(digital) shifts and finite-difference sample positions.  It contains none of
the method's arithmetic (no point generation, no products, no integrands), so
both the CPU oracle and the CUDA path can be fed from it without sharing any
computation.

Every array comes from ``numpy.random.Generator(PCG64(SeedSequence([230511645,
config_id, purpose])))``; the purposes are fixed below, so a workload is a pure
function of its identifiers.

The five named workloads restate the synthetic configurations of the reduced
QMC product (Sec. 3 and Sec. 6 of the paper set the shapes: N=b^m points,
s dimensions, tau output columns, decaying reduction indices w_j):

  c1  reduced rank-1 lattice, b=2, m=10, s=tau=64, w_j=floor(j/16), FP64,
      unshifted, f(y)=mean_t cos(y_t)
  c2  Gaussian expectation: lattice, m=16, s=tau=512,
      w_j=min(floor(log2(j+1)),10), one random shift with odd D_j,
      inverse-normal transform, A=L^T with L the Cholesky factor of
      exp(-|t_i-t_j|/0.1)+1e-10 I on t_i=i/(tau-1), f=max(mean exp(0.2y)-1,0)
  c3  reduced periodic digital net, m=20, s=tau=1024,
      w_j=min(floor(log2(j+1)),12), C_j=[[B_j,0],[0,0]] with B_j a random
      nonsingular (m-w_j)x(m-w_j) GF(2) matrix, A~N(0,1/s) FP32, R=16 XOR
      shifts, f=exp(-|y|^2/(2 tau))
  c4  8 uneven PDE-like lattice instances, centred points, R=4 shifts each,
      A_{j,i}=(j+1)^-2 sin((j+1) pi t_i), t_i=(i+1)/(tau+1),
      f=mean 1/(1+0.5y)^2
  c5  adjoint workload: lattice, m=20, s=tau=1024, w as c3, A~N(0,1/s) FP32,
      R=8 shifts, f=log sum exp(y), 64 sampled (j,t) entries for
      finite differences
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

SEED_ROOT = 230511645

# purpose identifiers of the seed sequence
P_Z, P_C, P_A, P_SHIFT, P_FD, P_MISC = 0, 1, 2, 3, 4, 5

LATTICE, DIGITAL_NET, REDUCED_MC, POLY_LATTICE = 0, 1, 2, 3
T_IDENTITY, T_CENTER, T_INV_NORMAL, T_TENT = 0, 1, 2, 3

F_NONE, F_LINEAR_MEAN, F_MEAN_COS, F_CALL_MEAN_EXP, F_GAUSS_NORM2, F_PDE_INV_SQ, F_LOGSUMEXP = range(7)
F_NAMES = {F_NONE: "none", F_LINEAR_MEAN: "linear_mean", F_MEAN_COS: "mean_cos",
           F_CALL_MEAN_EXP: "call_mean_exp", F_GAUSS_NORM2: "gauss_norm2",
           F_PDE_INV_SQ: "pde_inv_sq", F_LOGSUMEXP: "logsumexp"}


def rng(config_id: int, purpose: int, extra: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([SEED_ROOT, config_id, purpose, extra])))


@dataclasses.dataclass
class Problem:
    """One reduced-QMC instance: the rule (points), the matrix A and the integrand."""
    kind: int                 # LATTICE, DIGITAL_NET, REDUCED_MC or POLY_LATTICE
    m: int                    # N = 2^m points
    w: np.ndarray             # uint32[s], nondecreasing reduction indices
    A: np.ndarray             # s x tau, float64 or float32
    z: Optional[np.ndarray] = None      # uint32[s], lattice generating vector (reduced z_j), or the reduced
                                        # generating polynomials gt_j (coefficient of x^i at bit i)
    C: Optional[np.ndarray] = None      # uint32[s, m], net column masks (column q, bit m-1-p = row p)
    shifts: Optional[np.ndarray] = None  # uint32[R, s], 32-bit shifts (add mod 2^32 / XOR)
    y: Optional[np.ndarray] = None       # uint32[R, T], reduced MC samples per replica (X32 words; column j's
                                         # N_j = 2^(m-min(w_j,m)) samples, columns in order, T = sum_j N_j)
    transform: int = T_IDENTITY
    f_kind: int = F_NONE
    f_params: tuple = (0.0, 0.0, 0.0, 0.0)
    b: int = 2
    name: str = ""

    @property
    def s(self) -> int:
        return int(self.w.shape[0])

    @property
    def tau(self) -> int:
        return int(self.A.shape[1])

    @property
    def N(self) -> int:
        return self.b ** self.m

    @property
    def R(self) -> int:
        if self.kind == REDUCED_MC:
            return int(self.y.shape[0])          # independent replicas
        return 0 if self.shifts is None else int(self.shifts.shape[0])

    @property
    def R_eff(self) -> int:
        return max(self.R, 1)


# ----------------------------------------------------------------------------- draws

def odd_z(g: np.random.Generator, m: int, w: np.ndarray) -> np.ndarray:
    """z_j odd and uniform in [1, 2^(m-w_j)); z_j = 1 where w_j >= m."""
    z = np.ones(len(w), dtype=np.uint32)
    for j, wj in enumerate(w):
        q = m - int(wj)
        if q >= 1:
            z[j] = 2 * int(g.integers(0, 1 << (q - 1))) + 1
    return z


def gf2_nonsingular(g: np.random.Generator, q: int) -> np.ndarray:
    """A random nonsingular q x q matrix over GF(2): P * L * U with L unit lower and
    U unit upper triangular (both invertible), P a random row permutation."""
    if q == 0:
        return np.zeros((0, 0), dtype=np.uint8)
    L = np.tril(g.integers(0, 2, size=(q, q)), -1) + np.eye(q, dtype=np.int64)
    U = np.triu(g.integers(0, 2, size=(q, q)), 1) + np.eye(q, dtype=np.int64)
    B = (L @ U) % 2
    return B[g.permutation(q)].astype(np.uint8)


def periodic_net_masks(g: np.random.Generator, m: int, w: np.ndarray) -> np.ndarray:
    """Column masks of C_j = [[B_j, 0], [0, 0]] with B_j nonsingular of size q=m-w_j.

    Mask word q' (0-based column q'+1) holds row p (1-based) at bit m-p.  Columns
    q' >= m-w_j are zero, rows p > m-w_j are zero."""
    s = len(w)
    C = np.zeros((s, m), dtype=np.uint32)
    for j, wj in enumerate(w):
        q = m - min(int(wj), m)
        B = gf2_nonsingular(g, q)
        for col in range(q):
            word = 0
            for p in range(q):           # 0-based row p <-> bit m-1-p
                if B[p, col]:
                    word |= 1 << (m - 1 - p)
            C[j, col] = word
    return C


def nonsingular_net_masks(g: np.random.Generator, m: int, s: int) -> np.ndarray:
    """Column masks of s random nonsingular m x m GF(2) generating matrices: the nets of Sec. 4
    before the row reduction, which the library applies (the last min(w_j, m) rows zeroed).  The
    reduced matrices then generally have nonzero columns beyond m - w_j: a non-periodic reduced
    net (Algorithm 4's case), whose first m - w_j rows stay linearly independent."""
    C = np.zeros((s, m), dtype=np.uint32)
    for j in range(s):
        B = gf2_nonsingular(g, m)
        for col in range(m):
            C[j, col] = sum(1 << (m - 1 - p) for p in range(m) if B[p, col])
    return C


def random_shifts(g: np.random.Generator, R: int, s: int, force_odd: bool = False) -> np.ndarray:
    D = g.integers(0, 1 << 32, size=(R, s), dtype=np.uint64).astype(np.uint32)
    if force_odd:
        D |= np.uint32(1)
    return D


def mc_samples(g: np.random.Generator, m: int, w: np.ndarray, R: int, force_odd: bool = False) -> np.ndarray:
    """Reduced MC draws (Sec. 5): per replica, N_j = 2^(m-min(w_j,m)) i.i.d. uniform 32-bit words for
    every column j, columns in order.  Odd words (force_odd) keep x = X32 2^-32 away from 0 for the
    inverse-normal transform."""
    T = sum(1 << (m - min(int(wj), m)) for wj in w)
    y = g.integers(0, 1 << 32, size=(max(R, 1), T), dtype=np.uint64).astype(np.uint32)
    if force_odd:
        y |= np.uint32(1)
    return y


def log2_weights(s: int, cap: int) -> np.ndarray:
    return np.array([min(int(math.floor(math.log2(j + 1))), cap) for j in range(s)], dtype=np.uint32)


# ----------------------------------------------------------------------------- named workloads

def c1() -> Problem:
    m, s, tau = 10, 64, 64
    w = np.array([j // 16 for j in range(s)], dtype=np.uint32)
    z = odd_z(rng(1, P_Z), m, w)
    A = rng(1, P_A).standard_normal((s, tau))
    return Problem(LATTICE, m, w, A, z=z, transform=T_IDENTITY, f_kind=F_MEAN_COS, name="c1")


def exp_cov_cholesky_T(tau: int, ell: float = 0.1, nugget: float = 1e-10) -> np.ndarray:
    t = np.arange(tau) / (tau - 1)
    S = np.exp(-np.abs(t[:, None] - t[None, :]) / ell) + nugget * np.eye(tau)
    return np.linalg.cholesky(S).T.copy()


def c2(m: int = 16, s: int = 512, dtype=np.float64) -> Problem:
    w = log2_weights(s, 10)
    z = odd_z(rng(2, P_Z), m, w)
    D = random_shifts(rng(2, P_SHIFT), 1, s, force_odd=True)
    A = exp_cov_cholesky_T(s).astype(dtype)
    return Problem(LATTICE, m, w, A, z=z, shifts=D, transform=T_INV_NORMAL,
                   f_kind=F_CALL_MEAN_EXP, f_params=(0.2, 1.0, 0.0, 0.0), name="c2")


def c3(m: int = 20, s: int = 1024, R: int = 16) -> Problem:
    w = log2_weights(s, 12)
    C = periodic_net_masks(rng(3, P_C), m, w)
    A = (rng(3, P_A).standard_normal((s, s)) / math.sqrt(s)).astype(np.float32)
    D = random_shifts(rng(3, P_SHIFT), R, s)
    return Problem(DIGITAL_NET, m, w, A, C=C, shifts=D, transform=T_IDENTITY,
                   f_kind=F_GAUSS_NORM2, name="c3")


C4_INSTANCES = [(14, 256, 1024), (14, 2048, 4096), (16, 1024, 2048), (16, 256, 4096),
                (16, 2048, 1024), (18, 1024, 1024), (18, 256, 2048), (18, 2048, 4096)]


def pde_matrix(s: int, tau: int) -> np.ndarray:
    t = (np.arange(tau) + 1.0) / (tau + 1.0)
    j = np.arange(s)[:, None] + 1.0
    return (j ** -2.0) * np.sin(j * math.pi * t[None, :])


def c4(instance: int, R: int = 4) -> Problem:
    m, s, tau = C4_INSTANCES[instance]
    w = log2_weights(s, 12)
    z = odd_z(rng(4, P_Z, instance), m, w)
    D = random_shifts(rng(4, P_SHIFT, instance), R, s)
    A = pde_matrix(s, tau).astype(np.float32)
    return Problem(LATTICE, m, w, A, z=z, shifts=D, transform=T_CENTER,
                   f_kind=F_PDE_INV_SQ, f_params=(0.5, 0.0, 0.0, 0.0), name=f"c4.{instance}")


def c5(m: int = 20, s: int = 1024, R: int = 8) -> Problem:
    w = log2_weights(s, 12)
    z = odd_z(rng(5, P_Z), m, w)
    A = (rng(5, P_A).standard_normal((s, s)) / math.sqrt(s)).astype(np.float32)
    D = random_shifts(rng(5, P_SHIFT), R, s)
    return Problem(LATTICE, m, w, A, z=z, shifts=D, transform=T_IDENTITY,
                   f_kind=F_LOGSUMEXP, name="c5")


def stiffness_terms(s: int, M: int) -> np.ndarray:
    """Matrices C_j (s x M x M) of a PDE with an affine random coefficient (Sec. 1's assembly
    example): the 1-D P1 finite-element stiffness matrix on M interior nodes of a uniform mesh of
    (0, 1), h = 1/(M+1), for the coefficient term psi_j(t) = (j+1)^-2 sin((j+1) pi t) taken at each
    element's midpoint.  Element e (nodes e-1, e in 0-based interior numbering) adds
    psi_j(t_e)/h [[1, -1], [-1, 1]]; the boundary elements touch one interior node."""
    h = 1.0 / (M + 1)
    mid = (np.arange(M + 1) + 0.5) * h                     # element midpoints, elements 0..M
    C = np.zeros((s, M, M))
    for j in range(s):
        k = psi_coeff(j) * np.sin((j + 1) * math.pi * mid) / h
        for e in range(M + 1):
            a, b = e - 1, e                                # the element's interior nodes (-1, M: none)
            if a >= 0:
                C[j, a, a] += k[e]
            if b < M:
                C[j, b, b] += k[e]
            if a >= 0 and b < M:
                C[j, a, b] -= k[e]
                C[j, b, a] -= k[e]
    return C


def psi_coeff(j: int) -> float:
    return (j + 1.0) ** -2


def pde_assembly(m: int = 16, s: int = 256, M: int = 32, R: int = 1) -> Problem:
    """The PDE matrix-assembly workload: a reduced lattice (w_j = min(floor(log2(j+1)), 12), random odd
    z, R random shifts) and A whose row j is C_j flattened, so that row k of X A is D_k flattened
    (tau = M^2)."""
    w = log2_weights(s, 12)
    z = odd_z(rng(7, P_Z), m, w)
    D = random_shifts(rng(7, P_SHIFT), R, s) if R else None
    A = stiffness_terms(s, M).reshape(s, M * M).astype(np.float32)
    return Problem(LATTICE, m, w, A, z=z, shifts=D, transform=T_IDENTITY, f_kind=F_NONE, name="pde_assembly")


def fd_pairs(config_id: int, s: int, tau: int, count: int = 64) -> np.ndarray:
    g = rng(config_id, P_FD)
    return np.stack([g.integers(0, s, size=count), g.integers(0, tau, size=count)], axis=1)


# ----------------------------------------------------------------------------- random small cases

def random_weights(g: np.random.Generator, m: int, s: int, allow_ge_m: bool = True) -> np.ndarray:
    top = m + 2 if allow_ge_m else max(m - 1, 0)
    steps = g.integers(0, 2, size=s) * g.integers(0, 3, size=s)
    w = np.minimum(np.cumsum(steps) - steps[0], top)
    if g.random() < 0.3:
        w = w + int(g.integers(0, 2))
    return np.sort(np.maximum(w, 0)).astype(np.uint32)


def random_problem(seed: int, kind: int = LATTICE, m: Optional[int] = None, s: Optional[int] = None,
                   tau: Optional[int] = None, R: Optional[int] = None, transform: int = T_IDENTITY,
                   f_kind: int = F_NONE, f_params=(0.0, 0.0, 0.0, 0.0), dtype=np.float64,
                   a_scale: Optional[float] = None) -> Problem:
    g = rng(100, P_MISC, seed)
    m = int(g.integers(1, 11)) if m is None else m
    s = int(g.integers(1, 70)) if s is None else s
    tau = int(g.integers(1, 70)) if tau is None else tau
    R = int(g.integers(0, 4)) if R is None else R
    w = random_weights(g, m, s)
    if a_scale is None:
        a_scale = 1.0 / math.sqrt(max(s, 1))
    A = (g.standard_normal((s, tau)) * a_scale).astype(dtype)
    if kind == REDUCED_MC:
        return Problem(REDUCED_MC, m, w, A, y=mc_samples(g, m, w, R, force_odd=(transform == T_INV_NORMAL)),
                       transform=transform, f_kind=f_kind, f_params=tuple(f_params), name=f"rand{seed}")
    shifts = random_shifts(g, R, s, force_odd=(transform == T_INV_NORMAL)) if R > 0 else None
    if kind in (LATTICE, POLY_LATTICE):     # odd z_j < 2^(m-w_j): also gt_j(0) = 1, deg gt_j < m - w_j
        return Problem(kind, m, w, A, z=odd_z(g, m, w), shifts=shifts, transform=transform,
                       f_kind=f_kind, f_params=tuple(f_params), name=f"rand{seed}")
    return Problem(DIGITAL_NET, m, w, A, C=periodic_net_masks(g, m, w), shifts=shifts, transform=transform,
                   f_kind=f_kind, f_params=tuple(f_params), name=f"rand{seed}")


def units_z(g: np.random.Generator, b: int, m: int, w: np.ndarray) -> np.ndarray:
    """z_j uniform in U_{b^q} (prime b: not divisible by b, 1 <= z_j < b^q), z_j = 1 where w_j >= m."""
    z = np.ones(len(w), dtype=np.uint32)
    for j, wj in enumerate(w):
        q = m - min(int(wj), m)
        if q >= 1:
            while True:
                v = int(g.integers(1, b ** q))
                if v % b:
                    z[j] = v
                    break
    return z


def base_b_problem(seed: int, b: int, m: int, s: int, tau: int, R: int = 0, kind: int = LATTICE,
                   transform: int = T_IDENTITY, f_kind: int = F_NONE, f_params=(0.0, 0.0, 0.0, 0.0),
                   dtype=np.float64, w=None) -> Problem:
    """A reduced lattice (Sec. 1.3, N = b^m) or reduced MC point set (Sec. 5, N_j = b^(m-w_j)) in a
    prime base b, with A ~ N(0, 1/s)."""
    g = rng(101, P_MISC, seed)
    w = random_weights(g, m, s) if w is None else np.asarray(w, dtype=np.uint32)
    A = (g.standard_normal((s, tau)) / math.sqrt(s)).astype(dtype)
    if kind == REDUCED_MC:
        T = sum(b ** (m - min(int(wj), m)) for wj in w)
        y = g.integers(0, 1 << 32, size=(max(R, 1), T), dtype=np.uint64).astype(np.uint32)
        if transform == T_INV_NORMAL:
            y |= np.uint32(1)
        return Problem(REDUCED_MC, m, w, A, y=y, transform=transform, f_kind=f_kind, f_params=tuple(f_params), b=b,
                       name=f"b{b}mc{seed}")
    D = random_shifts(g, R, s, force_odd=transform == T_INV_NORMAL) if R else None
    return Problem(LATTICE, m, w, A, z=units_z(g, b, m, w), shifts=D, transform=transform, f_kind=f_kind,
                   f_params=tuple(f_params), b=b, name=f"b{b}lat{seed}")


def named(name: str) -> List[Problem]:
    if name == "c1":
        return [c1()]
    if name == "c2":
        return [c2()]
    if name == "c3":
        return [c3()]
    if name == "c4":
        return [c4(i) for i in range(len(C4_INSTANCES))]
    if name == "c5":
        return [c5()]
    raise KeyError(name)
