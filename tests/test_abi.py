"""C ABI checks that need no GPU: the library builds and loads, exports every
function include/qmc.h declares, and rejects invalid arguments (with an error
status and a message, never an abort) before any CUDA call is made."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2305_11645_gb300 import _lib as L
from paper_2305_11645_gb300 import build as B
from paper_2305_11645_gb300 import inputs as I
from paper_2305_11645_gb300.api import Integrand, Rule

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return L.load()


def declared_functions():
    with open(os.path.join(ROOT, "include", "qmc.h")) as fh:
        text = fh.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(qmc_\w+)\s*\(", text, flags=re.M)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert set(names) == set(L.EXPORTS), names
    for n in names:
        assert hasattr(lib, n)
    assert lib.qmc_version().decode().startswith("qmc_gb300")


def status(lib, rule):
    return lib.qmc_validate_rule(ctypes.byref(rule.struct()))


def test_valid_rules_pass(lib):
    for kind in (I.LATTICE, I.DIGITAL_NET):
        for seed in range(5):
            p = I.random_problem(seed, kind=kind)
            assert status(lib, Rule.from_problem(p)) == L.QMC_OK, lib.qmc_last_error()
    for p in (I.c1(), I.c2(m=8, s=64)):
        assert status(lib, Rule.from_problem(p)) == L.QMC_OK


def test_invalid_base_and_sizes(lib):
    p = I.random_problem(1, kind=I.DIGITAL_NET)
    r = Rule.from_problem(p)
    r.b = 3                                   # nets over F_b, b > 2, are not built
    assert status(lib, r) == L.QMC_ERR_UNSUPPORTED
    p = I.random_problem(1)
    r.b = 1
    assert status(lib, r) == L.QMC_ERR_INVALID_ARG
    r = Rule.from_problem(p)
    r.m = 0
    assert status(lib, r) == L.QMC_ERR_INVALID_ARG
    r.m = 31
    assert status(lib, r) == L.QMC_ERR_UNSUPPORTED
    assert "m=31" in lib.qmc_last_error().decode()


def test_nonmonotone_weights(lib):
    r = Rule(I.LATTICE, 5, [0, 2, 1], z=[1, 1, 1])
    assert status(lib, r) == L.QMC_ERR_INVALID_ARG
    assert "nondecreasing" in lib.qmc_last_error().decode()


@pytest.mark.parametrize("z", [[2, 1, 1], [1, 9, 1], [1, 0, 1], [1, 1, 3]])
def test_z_outside_units(lib, z):
    # m=4, w=(0,1,4): z_0 in U_16 (odd < 16), z_1 in U_8 (odd < 8), z_2 in U_1 = {1}
    assert status(lib, Rule(I.LATTICE, 4, [0, 1, 4], z=z)) == L.QMC_ERR_INVALID_ARG


def test_singular_and_nonperiodic_nets(lib):
    m = 3
    # singular (two equal columns, the third row alone cannot make rank 3)
    C = np.array([[4, 4, 1]], dtype=np.uint32)
    assert status(lib, Rule(I.DIGITAL_NET, m, [0], C=C)) == L.QMC_ERR_INVALID_ARG
    assert "rank" in lib.qmc_last_error().decode()
    # w=1 and column 3 (beyond m-w) nonzero after the row reduction: a non-periodic reduced net
    # (Algorithm 4's case), accepted; its first two rows [[1,0,1],[0,1,0]] have rank 2
    C = np.array([[4, 2, 4]], dtype=np.uint32)
    assert status(lib, Rule(I.DIGITAL_NET, m, [1], C=C)) == L.QMC_OK
    # w=1 with the first two reduced rows dependent ([[1,0,1],[1,0,1]]): rejected
    C = np.array([[6, 0, 6]], dtype=np.uint32)
    assert status(lib, Rule(I.DIGITAL_NET, m, [1], C=C)) == L.QMC_ERR_INVALID_ARG
    # bits above row 1
    C = np.array([[8, 2, 1]], dtype=np.uint32)
    assert status(lib, Rule(I.DIGITAL_NET, m, [0], C=C)) == L.QMC_ERR_INVALID_ARG
    # rows beyond m-w are zeroed by the library (eq. reduced_genmat_net2): accepted
    C = np.array([[4 | 1, 2, 0]], dtype=np.uint32)
    assert status(lib, Rule(I.DIGITAL_NET, m, [1], C=C)) == L.QMC_OK


def test_null_pointers_and_shift_rules(lib):
    r = Rule(I.LATTICE, 3, [0, 1], z=[1, 1])
    st = r.struct()
    st.z = None
    assert lib.qmc_validate_rule(ctypes.byref(st)) == L.QMC_ERR_INVALID_ARG
    st = r.struct()
    st.w = None
    assert lib.qmc_validate_rule(ctypes.byref(st)) == L.QMC_ERR_INVALID_ARG
    assert lib.qmc_validate_rule(None) == L.QMC_ERR_INVALID_ARG
    st = r.struct()
    st.R = 2
    assert lib.qmc_validate_rule(ctypes.byref(st)) == L.QMC_ERR_INVALID_ARG
    r = Rule(I.LATTICE, 3, [0, 1], z=[1, 1], transform=I.T_INV_NORMAL)
    assert status(lib, r) == L.QMC_ERR_INVALID_ARG
    assert "shift" in lib.qmc_last_error().decode()


@pytest.mark.parametrize("kind", [I.LATTICE, I.DIGITAL_NET, I.POLY_LATTICE])
def test_inverse_normal_rejects_shifts_that_reach_zero(lib, kind):
    """Under the inverse normal a shift word whose low 32 - q_j bits vanish puts a point at x = 0
    (the column takes every value u 2^(32-q_j) over its period), which maps to -inf: rejected.
    One set bit among those low bits keeps every point away from 0."""
    from oracle import qmc_oracle as O
    m, w = 6, np.array([0, 1, 2, 6], dtype=np.uint32)
    g = np.random.default_rng(7)
    z = I.odd_z(I.rng(9, I.P_Z), m, w)
    C = I.periodic_net_masks(I.rng(9, I.P_C), m, w)
    base = np.array([1 << 31, 3 << 29, 5 << 28, 0x80000000], dtype=np.uint32)   # low bits of each zero
    for j in range(len(w)):
        q = m - min(int(w[j]), m)
        D = (g.integers(0, 1 << 32, size=len(w), dtype=np.uint64) | 1).astype(np.uint32)
        D[j] = base[j] & np.uint32(~((1 << (32 - q)) - 1) & 0xFFFFFFFF)
        r = Rule(kind, m, w, z=z if kind != I.DIGITAL_NET else None, C=C if kind == I.DIGITAL_NET else None,
                 shifts=D[None, :], transform=I.T_INV_NORMAL)
        assert status(lib, r) == L.QMC_ERR_INVALID_ARG, (j, lib.qmc_last_error())
        assert "low" in lib.qmc_last_error().decode()
        # the oracle's points of that column indeed reach 0 over one period
        p = I.Problem(kind, m, w, np.zeros((len(w), 1)), z=z if kind != I.DIGITAL_NET else None,
                      C=C if kind == I.DIGITAL_NET else None, shifts=D[None, :], transform=I.T_IDENTITY)
        assert np.any(O.x32_points(p, 0)[:, j] == 0)
        D[j] |= np.uint32(1 << (32 - q - 1))               # one low bit set: accepted
        r = Rule(kind, m, w, z=z if kind != I.DIGITAL_NET else None, C=C if kind == I.DIGITAL_NET else None,
                 shifts=D[None, :], transform=I.T_INV_NORMAL)
        assert status(lib, r) == L.QMC_OK, lib.qmc_last_error()


def ws_size(lib, op, rule, tau, f, prec):
    out = ctypes.c_size_t(0)
    fa = None if f is None else ctypes.byref(f.struct())
    st = lib.qmc_workspace_size(op, ctypes.byref(rule.struct()), ctypes.byref(ctypes.c_uint32(tau)), 1, fa, prec,
                                ctypes.byref(out))
    return st, out.value


def test_workspace_size_and_its_errors(lib):
    p = I.c2(m=10, s=64)
    r = Rule.from_problem(p)
    f = Integrand(I.F_CALL_MEAN_EXP, (0.2, 1.0))
    st, fwd = ws_size(lib, L.QMC_OP_INTEGRATE, r, 64, f, L.QMC_FP32)
    assert st == L.QMC_OK and fwd > 0
    st, bwd = ws_size(lib, L.QMC_OP_INTEGRATE_BWD, r, 64, f, L.QMC_FP32)
    assert st == L.QMC_OK and bwd > fwd
    st, _ = ws_size(lib, L.QMC_OP_INTEGRATE, r, 0, f, L.QMC_FP32)
    assert st == L.QMC_ERR_INVALID_ARG
    st, _ = ws_size(lib, L.QMC_OP_INTEGRATE, r, 64, Integrand(I.F_NONE), L.QMC_FP32)
    assert st == L.QMC_ERR_INVALID_ARG
    for tier in (L.QMC_SPLIT, L.QMC_BF16):          # the tensor-core tiers plan like FP32 (float data)
        st, tc = ws_size(lib, L.QMC_OP_INTEGRATE, r, 64, f, tier)
        assert st == L.QMC_OK and tc > 0
    st, _ = ws_size(lib, L.QMC_OP_INTEGRATE, r, 64, f, 9)
    assert st == L.QMC_ERR_INVALID_ARG


def test_unaligned_product_rejected_before_any_cuda_call(lib):
    p = I.random_problem(3)
    r = Rule.from_problem(p)
    fake = ctypes.c_void_p(0x1000)
    unaligned = ctypes.c_void_p(0x1004)     # never dereferenced: the alignment check fails first
    for prec in (L.QMC_FP64, L.QMC_FP32):
        st = lib.qmc_reduced_matmul(ctypes.byref(r.struct()), fake, p.tau, prec, unaligned, fake, 1 << 30, None)
        assert st == L.QMC_ERR_INVALID_ARG
        assert b"16-byte aligned" in lib.qmc_last_error()


def test_too_small_workspace_rejected_before_any_cuda_call(lib):
    p = I.random_problem(2, f_kind=I.F_MEAN_COS)
    r = Rule.from_problem(p)
    f = Integrand(I.F_MEAN_COS)
    fake = ctypes.c_void_p(0x1000)          # never dereferenced: the size check fails first
    st = lib.qmc_integrate(ctypes.byref(r.struct()), ctypes.byref(fake), ctypes.byref(ctypes.c_uint32(p.tau)), 1,
                           ctypes.byref(f.struct()), L.QMC_FP64, fake, None, None, 0, None)
    assert st == L.QMC_ERR_NO_MEMORY
    st = lib.qmc_reduced_matmul(ctypes.byref(r.struct()), fake, p.tau, L.QMC_FP64, fake, None, 0, None)
    assert st == L.QMC_ERR_NO_MEMORY
    st = lib.qmc_gen_points(ctypes.byref(r.struct()), 0, L.QMC_LAYOUT_FULL, fake, 1, None, 0, None)
    assert st == L.QMC_ERR_INVALID_ARG      # output capacity checked
    st = lib.qmc_integrate_backward(ctypes.byref(r.struct()), ctypes.byref(fake),
                                    ctypes.byref(ctypes.c_uint32(p.tau)), 1, ctypes.byref(f.struct()), L.QMC_FP64,
                                    fake, ctypes.byref(fake), 7, fake, 1 << 30, None)
    assert st == L.QMC_ERR_INVALID_ARG      # unknown flags


def test_reduced_mc_rules(lib):
    """Reduced MC (Sec. 5): valid rules pass; C, a shift, a missing sample array or, with the
    inverse-normal transform, a zero sample word are rejected on the host."""
    for seed in range(4):
        p = I.random_problem(seed, kind=I.REDUCED_MC, transform=I.T_INV_NORMAL if seed % 2 else I.T_IDENTITY)
        assert status(lib, Rule.from_problem(p)) == L.QMC_OK, lib.qmc_last_error()
    p = I.random_problem(5, kind=I.REDUCED_MC, m=4, s=3, R=2)
    r = Rule.from_problem(p)
    st = r.struct()
    keep = (ctypes.c_uint32 * 4)(1, 2, 3, 4)
    st.C = ctypes.cast(keep, ctypes.POINTER(ctypes.c_uint32))
    assert lib.qmc_validate_rule(ctypes.byref(st)) == L.QMC_ERR_INVALID_ARG
    st = r.struct()
    st.shift = ctypes.cast(keep, ctypes.POINTER(ctypes.c_uint32))
    assert lib.qmc_validate_rule(ctypes.byref(st)) == L.QMC_ERR_INVALID_ARG
    st = r.struct()
    st.z = None
    assert lib.qmc_validate_rule(ctypes.byref(st)) == L.QMC_ERR_INVALID_ARG
    y = p.y.copy()
    y[1, 5] = 0
    r0 = Rule(I.REDUCED_MC, p.m, p.w, y=y, transform=I.T_INV_NORMAL)
    assert status(lib, r0) == L.QMC_ERR_INVALID_ARG
    assert "sample word" in lib.qmc_last_error().decode()
    r0 = Rule(I.REDUCED_MC, p.m, p.w, y=y, transform=I.T_IDENTITY)      # a zero word is a valid sample
    assert status(lib, r0) == L.QMC_OK


def test_reduced_mc_workspace_holds_every_replica(lib):
    """Without a device copy the samples of all replicas are uploaded into the workspace."""
    p = I.random_problem(6, kind=I.REDUCED_MC, m=9, s=20, R=3)
    r = Rule.from_problem(p)
    T = sum(1 << (p.m - min(int(wj), p.m)) for wj in p.w)
    nbytes = ctypes.c_size_t(0)
    assert lib.qmc_workspace_size(L.QMC_OP_GEN_POINTS, ctypes.byref(r.struct()), None, 1, None, L.QMC_FP32,
                                  ctypes.byref(nbytes)) == L.QMC_OK
    assert nbytes.value >= 3 * T * 4


def test_poly_lattice_rules(lib):
    """Reduced polynomial lattices: gt_j(0) = 1 and deg gt_j < m - w_j (as z_j for lattices)."""
    for seed in range(4):
        p = I.random_problem(seed, kind=I.POLY_LATTICE)
        assert status(lib, Rule.from_problem(p)) == L.QMC_OK, lib.qmc_last_error()
    assert status(lib, Rule(I.POLY_LATTICE, 4, [0, 1], z=[0b1010, 1])) == L.QMC_ERR_INVALID_ARG   # gt(0) = 0
    assert status(lib, Rule(I.POLY_LATTICE, 4, [0, 1], z=[0b10011, 1])) == L.QMC_ERR_INVALID_ARG  # degree 4
    assert status(lib, Rule(I.POLY_LATTICE, 4, [0, 9], z=[0b1011, 3])) == L.QMC_ERR_INVALID_ARG   # w >= m: 1
    assert status(lib, Rule(I.POLY_LATTICE, 4, [0, 9], z=[0b1011, 1])) == L.QMC_OK


def test_selftest_wait_arguments_checked_on_the_host(lib):
    """The wait self-test's poll count is checked before anything is enqueued."""
    assert lib.qmc_selftest_wait_timeout(0, None) == L.QMC_ERR_INVALID_ARG
    assert lib.qmc_selftest_wait_timeout((1 << 20) + 1, None) == L.QMC_ERR_INVALID_ARG


@pytest.mark.parametrize("seed", range(40))
def test_planner_never_fails_uncleanly(lib, seed):
    """The host planner (workspace query: validation, block schedule, grids, workspace layout) on
    random rules of every kind, operation and tier: a status and a size, no abort, and a workspace
    that at least holds the point table of every shift."""
    g = np.random.default_rng(4000 + seed)
    kind = [I.LATTICE, I.DIGITAL_NET, I.REDUCED_MC, I.POLY_LATTICE][seed % 4]
    m = int(g.integers(1, 21))
    s = int(g.integers(1, 300))
    p = I.random_problem(seed, kind=kind, m=m, s=s, tau=int(g.integers(1, 600)), R=int(g.integers(0, 4)))
    r = Rule.from_problem(p)
    f = Integrand([I.F_LINEAR_MEAN, I.F_MEAN_COS, I.F_CALL_MEAN_EXP, I.F_GAUSS_NORM2, I.F_PDE_INV_SQ,
                   I.F_LOGSUMEXP][seed % 6], (0.2, 0.9, 0, 0))
    T = sum(1 << (m - min(int(wj), m)) for wj in p.w)
    for op in (L.QMC_OP_GEN_POINTS, L.QMC_OP_REDUCED_MATMUL, L.QMC_OP_INTEGRATE, L.QMC_OP_INTEGRATE_BWD):
        for prec in (L.QMC_FP64, L.QMC_FP32, L.QMC_SPLIT, L.QMC_BF16):
            nbytes = ctypes.c_size_t(0)
            st = lib.qmc_workspace_size(op, ctypes.byref(r.struct()), ctypes.byref(ctypes.c_uint32(p.tau)), 1,
                                        ctypes.byref(f.struct()) if op >= L.QMC_OP_INTEGRATE else None, prec,
                                        ctypes.byref(nbytes))
            assert st == L.QMC_OK, (op, prec, lib.qmc_last_error())
            if op != L.QMC_OP_GEN_POINTS:
                elt = 8 if prec == L.QMC_FP64 else 4
                assert nbytes.value >= elt * T * p.R_eff


def gf2_rank_reference(rows):
    """Row echelon form over GF(2) with numpy (an independent restatement for the test)."""
    M = np.array(rows, dtype=np.uint8) % 2
    rank = 0
    for col in range(M.shape[1]):
        piv = next((i for i in range(rank, M.shape[0]) if M[i, col]), None)
        if piv is None:
            continue
        M[[rank, piv]] = M[[piv, rank]]
        for i in range(M.shape[0]):
            if i != rank and M[i, col]:
                M[i] ^= M[rank]
        rank += 1
    return rank


@pytest.mark.parametrize("seed", range(30))
def test_net_leading_block_rank_check(lib, seed):
    """The library accepts a periodic reduced net exactly when every leading (m-w_j) x (m-w_j)
    block is nonsingular over GF(2): random blocks, about half of them singular."""
    g = np.random.default_rng(7000 + seed)
    m = int(g.integers(2, 13))
    w = np.sort(g.integers(0, m, size=int(g.integers(1, 6)))).astype(np.uint32)
    C = np.zeros((len(w), m), dtype=np.uint32)
    expect_ok = True
    bad = int(g.integers(0, len(w))) if seed % 2 else -1     # one singular block in odd seeds
    for j, wj in enumerate(w):
        q = m - int(wj)
        B = I.gf2_nonsingular(g, q).astype(np.int64)
        if j == bad:                                       # make a column depend on the others
            B[:, -1] = B[:, 0] ^ (B[:, 1] if q > 2 else 0) if q > 1 else 0
        expect_ok &= gf2_rank_reference(B) == q
        for col in range(q):
            C[j, col] = sum(int(B[p, col]) << (m - 1 - p) for p in range(q))
    st = status(lib, Rule(I.DIGITAL_NET, m, w, C=C))
    assert st == (L.QMC_OK if expect_ok else L.QMC_ERR_INVALID_ARG), lib.qmc_last_error()


def tune_key(p, precision, f_kind, tau):
    """The schedule cache's shape key: m, precision, integrand, tau padded to 4, shifts, and the
    column count of every level min(w_j, m) = 0..m."""
    lev = [int(np.sum(np.minimum(p.w, p.m) == I)) for I in range(p.m + 1)]
    return (f"m{p.m} p{precision} f{f_kind} t{(tau + 3) // 4 * 4} r{max(p.R, 1)} L" + ",".join(map(str, lev)))


def test_schedule_cache_file_and_planner(lib, tmp_path):
    """A loaded schedule changes the plan (in the FP32 tier the forward's column groups size the row
    partials, the largest area of this workspace, so the workspace changes with them); save writes
    what was loaded; a malformed file is rejected."""
    p = I.c2(m=10, s=64, dtype=np.float32)
    r = Rule.from_problem(p)
    f = Integrand(I.F_CALL_MEAN_EXP, (0.2, 1.0))
    assert lib.qmc_tune_clear() == L.QMC_OK
    st, base = ws_size(lib, L.QMC_OP_INTEGRATE, r, 64, f, L.QMC_FP32)
    assert st == L.QMC_OK
    key = tune_key(p, L.QMC_FP32, I.F_CALL_MEAN_EXP, 64)
    path = tmp_path / "sched.txt"
    path.write_text(f"# comment\n{key}|16|6\n")              # 64 columns per CTA: one column group
    n = ctypes.c_uint32(0)
    assert lib.qmc_tune_load(str(path).encode(), ctypes.byref(n)) == L.QMC_OK and n.value == 1
    st, tuned = ws_size(lib, L.QMC_OP_INTEGRATE, r, 64, f, L.QMC_FP32)
    assert st == L.QMC_OK and tuned != base                  # (the cost model takes 16 groups of 4 columns)
    out = tmp_path / "saved.txt"
    assert lib.qmc_tune_save(str(out).encode()) == L.QMC_OK
    assert f"{key}|16|6|0|0|0|0" in out.read_text().splitlines()  # (missing fields read as 0)
    assert lib.qmc_tune_clear() == L.QMC_OK
    assert ws_size(lib, L.QMC_OP_INTEGRATE, r, 64, f, L.QMC_FP32)[1] == base
    # the tensor-core tiers' coarse path is part of the schedule: this shape's coarse partial sums
    # are small, so the model takes the block products; forcing the level passes adds their areas
    q = I.c2(m=12, s=1024, dtype=np.float32)                 # (wide: the passes' A pieces dominate)
    rq = Rule.from_problem(q)
    fq = Integrand(I.F_CALL_MEAN_EXP, (0.2, 1.0))
    st, products = ws_size(lib, L.QMC_OP_INTEGRATE, rq, 1024, fq, L.QMC_SPLIT)
    kq = tune_key(q, L.QMC_SPLIT, I.F_CALL_MEAN_EXP, 1024)
    path.write_text(f"{kq}|0|0|1\n{kq.replace('p2', 'p3')}|0|0|2\n")
    assert lib.qmc_tune_load(str(path).encode(), ctypes.byref(n)) == L.QMC_OK and n.value == 2
    st, passes = ws_size(lib, L.QMC_OP_INTEGRATE, rq, 1024, fq, L.QMC_SPLIT)
    assert st == L.QMC_OK and passes != products
    assert lib.qmc_tune_clear() == L.QMC_OK
    bad = tmp_path / "bad.txt"
    bad.write_text("no separators here\n")
    assert lib.qmc_tune_load(str(bad).encode(), ctypes.byref(n)) == L.QMC_ERR_INVALID_ARG
    assert lib.qmc_tune_load(str(tmp_path / "missing.txt").encode(), ctypes.byref(n)) == L.QMC_ERR_INVALID_ARG
    assert lib.qmc_tune_clear() == L.QMC_OK


def test_schedule_set_adjoint_path(lib, tmp_path):
    """qmc_tune_set caches a schedule for a problem's shape without a GPU: forcing the fused
    fold-gradient and TMA gradient kernels on a small split-tier problem (the model takes the one-fold
    path below 2^24 root-gradient elements) adds their pre-split table buffer to the backward's
    workspace; the entry is what qmc_tune_save writes; values out of range are rejected."""
    p = I.c5(m=14, s=256, R=2)
    r = Rule.from_problem(p)
    f = Integrand(I.F_LOGSUMEXP, ())
    tau = int(p.A.shape[1])
    assert lib.qmc_tune_clear() == L.QMC_OK
    st, compact = ws_size(lib, L.QMC_OP_INTEGRATE_BWD, r, tau, f, L.QMC_SPLIT)
    assert st == L.QMC_OK
    assert lib.qmc_tune_set(ctypes.byref(r.struct()), tau, ctypes.byref(f.struct()), L.QMC_SPLIT, 0, 0, 0, 2) == L.QMC_OK
    st, fused = ws_size(lib, L.QMC_OP_INTEGRATE_BWD, r, tau, f, L.QMC_SPLIT)
    assert st == L.QMC_OK and fused > compact
    out = tmp_path / "saved.txt"
    assert lib.qmc_tune_save(str(out).encode()) == L.QMC_OK
    key = tune_key(p, L.QMC_SPLIT, I.F_LOGSUMEXP, tau)
    assert f"{key}|0|0|0|2|0|0" in out.read_text().splitlines()
    for bad in ((129, 0, 0, 0), (0, -1, 0, 0), (0, 0, 3, 0), (0, 0, 0, 3)):
        assert lib.qmc_tune_set(ctypes.byref(r.struct()), tau, ctypes.byref(f.struct()), L.QMC_SPLIT,
                                *bad) == L.QMC_ERR_INVALID_ARG
    assert lib.qmc_tune_clear() == L.QMC_OK
    assert ws_size(lib, L.QMC_OP_INTEGRATE_BWD, r, tau, f, L.QMC_SPLIT)[1] == compact


def test_base_b_rules_checked_on_the_host(lib):
    """Base b > 2 (lattices, reduced MC): a zero shift under the inverse normal (the point u = 0
    stays 0), z_j divisible by b, a composite base and a net over F_b are rejected; valid rules pass."""
    for b, m in ((3, 7), (5, 5), (7, 4)):
        for kind in (I.LATTICE, I.REDUCED_MC):
            p = I.base_b_problem(1 + b, b, m, 29, 3, R=2, kind=kind)
            assert status(lib, Rule.from_problem(p)) == L.QMC_OK, lib.qmc_last_error()
    assert status(lib, Rule(I.LATTICE, 4, [0, 1], z=[1, 1], b=9)) == L.QMC_ERR_INVALID_ARG      # 9 = 3^2
    assert status(lib, Rule(I.LATTICE, 30, [0], z=[1], b=3)) == L.QMC_ERR_UNSUPPORTED         # 3^30 > 2^31
    p = I.base_b_problem(3, 3, 5, 8, 4, R=1, transform=I.T_INV_NORMAL)
    r = Rule.from_problem(p)
    r.shifts = r.shifts.copy()
    r.shifts[0, 0] = 0                         # x = u/b^q + 0 reaches 0 at k = 0
    assert status(lib, r) == L.QMC_ERR_INVALID_ARG
    r = Rule(I.LATTICE, 4, [0, 1], z=[3, 1], b=3)    # z_0 = 3 is divisible by b
    assert status(lib, r) == L.QMC_ERR_INVALID_ARG
    r = Rule(I.DIGITAL_NET, 3, [0], C=[[1, 0, 0]], b=3)
    assert status(lib, r) == L.QMC_ERR_UNSUPPORTED
