"""Python binding of libqmc_gb300 (argument marshalling only).

Every computation runs in the library's CUDA kernels; torch supplies device
memory (inputs, outputs, workspace) and the current CUDA stream.

    rule = Rule(LATTICE, m, w, z=z, shifts=D, transform=T_INV_NORMAL)
    est  = integrate(rule, A, Integrand(F_CALL_MEAN_EXP, (0.2, 1.0)))   # [Q_0..Q_{R-1}, mean]
    P    = reduced_matmul(rule, A)                                        # (R_eff, N, tau)
    X    = gen_points(rule)                                               # (N, s) uint32 as int32
    Q    = qmc_estimate(A, rule, f)                                       # differentiable in A
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from typing import List, Optional, Sequence, Tuple, Union

import numpy as np
import torch

from . import _lib as L
from .inputs import (DIGITAL_NET, LATTICE, POLY_LATTICE, REDUCED_MC, T_CENTER, T_IDENTITY, T_INV_NORMAL,  # noqa: F401
                     T_TENT,
                     F_CALL_MEAN_EXP, F_GAUSS_NORM2, F_LINEAR_MEAN, F_LOGSUMEXP, F_MEAN_COS, F_NONE,
                     F_PDE_INV_SQ)


@dataclass(frozen=True)
class Integrand:
    kind: int
    params: Tuple[float, ...] = (0.0, 0.0, 0.0, 0.0)

    def struct(self) -> L.QmcIntegrand:
        p = tuple(self.params) + (0.0,) * (4 - len(self.params))
        return L.QmcIntegrand(self.kind, (ctypes.c_double * 4)(*p[:4]))


def _u32(a) -> Optional[np.ndarray]:
    if a is None:
        return None
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint64).astype(np.uint32))


class Rule:
    """A reduced QMC rule: lattice (z), polynomial lattice (z: the reduced generating polynomials) or
    periodic reduced digital net (C) with optional shifts, or reduced Monte Carlo (y: the replicas'
    samples, uint32 [R, sum_j N_j] in the distinct layout)."""

    def __init__(self, kind: int, m: int, w, z=None, C=None, shifts=None, transform: int = T_IDENTITY, b: int = 2,
                 y=None):
        self.kind, self.m, self.b, self.transform = int(kind), int(m), int(b), int(transform)
        self.w = _u32(w)
        self.s = int(self.w.shape[0])
        self.z = _u32(z)
        self.C = None if C is None else _u32(np.asarray(C).reshape(-1))
        self.shifts = None if shifts is None else _u32(np.asarray(shifts).reshape(-1, self.s))
        self.R = 0 if self.shifts is None else int(self.shifts.shape[0])
        self.y = None
        if self.kind == REDUCED_MC:
            if y is None:
                raise ValueError("a reduced MC rule needs its samples y")
            T = sum(self.b ** (self.m - min(int(wj), self.m)) for wj in self.w)
            self.y = _u32(np.asarray(y).reshape(-1, T))
            self.R = int(self.y.shape[0])        # independent replicas
        self._dev = {}

    @classmethod
    def from_problem(cls, p) -> "Rule":
        return cls(p.kind, p.m, p.w, z=p.z, C=p.C, shifts=p.shifts, transform=p.transform, b=p.b,
                   y=getattr(p, "y", None))

    @property
    def N(self) -> int:
        return self.b ** self.m

    def nonperiodic(self) -> bool:
        """A net whose reduced generating matrices (last min(w_j, m) rows zeroed) have a nonzero
        column beyond m - w_j: its columns do not repeat periodically (Sec. 4, Algorithm 4's case)."""
        if self.kind != DIGITAL_NET:
            return False
        C = self.C.reshape(self.s, self.m)
        for j in range(self.s):
            wcl = min(int(self.w[j]), self.m)
            rowmask = (0xFFFFFFFF << wcl) & 0xFFFFFFFF
            if any(int(C[j, c]) & rowmask for c in range(self.m - wcl, self.m)):
                return True
        return False

    def distinct_rows(self) -> int:
        """Entries of the distinct layout: one period of every column, or all N rows of every column
        of a non-periodic net."""
        if self.nonperiodic():
            return self.s * self.N
        return int(sum(self.b ** (self.m - min(int(w), self.m)) for w in self.w))

    @property
    def R_eff(self) -> int:
        return max(self.R, 1)

    def _device_arrays(self, device: torch.device):
        key = str(device)
        if key not in self._dev:
            gen = {LATTICE: self.z, POLY_LATTICE: self.z, DIGITAL_NET: self.C,
                   REDUCED_MC: None if self.y is None else self.y.reshape(-1)}[self.kind]
            d_gen = None if gen is None else torch.from_numpy(gen.view(np.int32).copy()).to(device)
            d_shift = None if self.shifts is None else torch.from_numpy(
                self.shifts.reshape(-1).view(np.int32).copy()).to(device)
            self._dev[key] = (d_gen, d_shift)
        return self._dev[key]

    def struct(self, device: Optional[torch.device] = None) -> L.QmcRule:
        def ptr(a):
            return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))
        r = L.QmcRule()
        r.kind, r.b, r.m, r.s = self.kind, self.b, self.m, self.s
        r.w, r.z, r.C = ptr(self.w), ptr(self.y.reshape(-1) if self.kind == REDUCED_MC else self.z), ptr(self.C)
        r.R = self.R
        r.shift = ptr(None if self.shifts is None else self.shifts.reshape(-1))
        r.transform = self.transform
        if device is not None:
            d_gen, d_shift = self._device_arrays(device)
            r.d_gen = None if d_gen is None else d_gen.data_ptr()
            r.d_shift = None if d_shift is None else d_shift.data_ptr()
        return r

    def validate(self) -> None:
        L.check(L.load().qmc_validate_rule(ctypes.byref(self.struct())))


def _precision(A: torch.Tensor, precision: Optional[str] = None) -> int:
    """The tier of a call: float64 A -> FP64; float32 A -> FP32, or the tensor-core tiers
    'split' (bf16x6 block products, FP32-level accuracy) and 'bf16' (one bf16 product)."""
    if A.dtype not in (torch.float32, torch.float64):
        raise TypeError(f"A must be float32 or float64 (got {A.dtype})")
    if precision is None:
        return L.QMC_FP64 if A.dtype == torch.float64 else L.QMC_FP32
    if precision not in L.PRECISIONS:
        raise ValueError(f"precision must be one of {sorted(L.PRECISIONS)} (got {precision!r})")
    want = torch.float64 if precision == "fp64" else torch.float32
    if A.dtype != want:
        raise TypeError(f"precision {precision!r} takes A as {want} (got {A.dtype})")
    return L.PRECISIONS[precision]


def _stream(device: torch.device) -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _as_list(x):
    return list(x) if isinstance(x, (list, tuple)) else [x]


def workspace_size(op: int, rules: Sequence[Rule], taus: Sequence[int], fs: Optional[Sequence[Integrand]],
                   precision: int) -> int:
    n = len(rules)
    rs = (L.QmcRule * n)(*[r.struct() for r in rules])
    ts = (ctypes.c_uint32 * n)(*[int(t) for t in taus])
    fa = None if fs is None else (L.QmcIntegrand * n)(*[f.struct() for f in fs])
    out = ctypes.c_size_t(0)
    L.check(L.load().qmc_workspace_size(op, rs, ts, n, fa, precision, ctypes.byref(out)))
    return int(out.value)


def _workspace(nbytes: int, device: torch.device, ws: Optional[torch.Tensor]) -> torch.Tensor:
    if ws is not None and ws.numel() >= nbytes:
        return ws
    return torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device)


def gen_points(rule: Rule, layout: str = "full", shift_idx: int = 0, device="cuda") -> torch.Tensor:
    """Bit-exact points X32 (uint32 stored in an int32 tensor): (N, s) for layout='full',
    or one period of every column concatenated for layout='distinct'."""
    device = torch.device(device)
    lay = L.QMC_LAYOUT_FULL if layout == "full" else L.QMC_LAYOUT_DISTINCT
    if lay == L.QMC_LAYOUT_FULL:
        out = torch.empty((rule.N, rule.s), dtype=torch.int32, device=device)
    else:
        out = torch.empty(rule.distinct_rows(), dtype=torch.int32, device=device)
    r = rule.struct(device)
    L.check(L.load().qmc_gen_points(ctypes.byref(r), shift_idx, lay, out.data_ptr(), out.numel(), None, 0,
                                    _stream(device)))
    return out


def reduced_matmul(rule: Rule, A: torch.Tensor, ws: Optional[torch.Tensor] = None,
                   precision: Optional[str] = None, out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """P = X A for every shift: (R_eff, N, tau), dtype of A (float64 -> FP64 tier, float32 -> FP32
    tier unless `precision` names a tensor-core tier), written into `out` when given."""
    A = A.contiguous()
    prec = _precision(A, precision)
    tau = A.shape[1]
    nbytes = workspace_size(L.QMC_OP_REDUCED_MATMUL, [rule], [tau], None, prec)
    ws = _workspace(nbytes, A.device, ws)
    shape = (rule.R_eff, rule.N, tau)
    if out is not None:
        if tuple(out.shape) != shape or out.dtype != A.dtype or not out.is_contiguous() or out.device != A.device:
            raise ValueError(f"out must be a contiguous {A.dtype} tensor of shape {shape} on {A.device}")
        P = out
    else:
        P = torch.empty(shape, dtype=A.dtype, device=A.device)
    r = rule.struct(A.device)
    L.check(L.load().qmc_reduced_matmul(ctypes.byref(r), A.data_ptr(), tau, prec, P.data_ptr(), ws.data_ptr(),
                                        ws.numel(), _stream(A.device)))
    return P


def assemble(rule: Rule, C: torch.Tensor, ws: Optional[torch.Tensor] = None,
             precision: Optional[str] = None) -> torch.Tensor:
    """The matrices D_k = sum_j x_{k,j} C_j for every point k and shift (Sec. 1's PDE assembly), as the
    reduced product X A with A's row j the flattened C_j (tau = M^2): (R_eff, N, M, M)."""
    if C.dim() != 3 or C.shape[1] != C.shape[2] or C.shape[0] != rule.s:
        raise ValueError(f"C must be (s, M, M) with s = {rule.s} (got {tuple(C.shape)})")
    M = C.shape[1]
    P = reduced_matmul(rule, C.reshape(rule.s, M * M), ws=ws, precision=precision)
    return P.view(rule.R_eff, rule.N, M, M)


def integrate(rules: Union[Rule, Sequence[Rule]], As, fs, rowf: bool = False,
              ws: Optional[torch.Tensor] = None, precision: Optional[str] = None):
    """QMC estimates for one or several problems.  Returns a float64 tensor holding, per problem,
    the R_eff per-shift estimates followed by their mean (and, with rowf=True, the per-point
    integrand values of every problem as (R_eff, N) tensors)."""
    rules, As, fs = _as_list(rules), [a.contiguous() for a in _as_list(As)], _as_list(fs)
    n = len(rules)
    prec = _precision(As[0], precision)
    device = As[0].device
    taus = [a.shape[1] for a in As]
    nbytes = workspace_size(L.QMC_OP_INTEGRATE, rules, taus, fs, prec)
    ws = _workspace(nbytes, device, ws)
    est = torch.empty(sum(r.R_eff + 1 for r in rules), dtype=torch.float64, device=device)
    rs = (L.QmcRule * n)(*[r.struct(device) for r in rules])
    ap = (ctypes.c_void_p * n)(*[a.data_ptr() for a in As])
    ts = (ctypes.c_uint32 * n)(*taus)
    fa = (L.QmcIntegrand * n)(*[f.struct() for f in fs])
    rowf_t = None
    rp = None
    if rowf:
        rowf_t = [torch.empty((r.R_eff, r.N), dtype=a.dtype, device=device) for r, a in zip(rules, As)]
        rp = (ctypes.c_void_p * n)(*[t.data_ptr() for t in rowf_t])
    L.check(L.load().qmc_integrate(rs, ap, ts, n, fa, prec, est.data_ptr(), rp, ws.data_ptr(), ws.numel(),
                                   _stream(device)))
    return (est, rowf_t) if rowf else est


def integrate_backward(rules, As, fs, upstream: torch.Tensor, ws: Optional[torch.Tensor] = None,
                       reuse_forward: bool = False, precision: Optional[str] = None) -> List[torch.Tensor]:
    """d(upstream_p * mean estimate_p)/dA_p for every problem p."""
    rules, As, fs = _as_list(rules), [a.contiguous() for a in _as_list(As)], _as_list(fs)
    n = len(rules)
    prec = _precision(As[0], precision)
    device = As[0].device
    taus = [a.shape[1] for a in As]
    nbytes = workspace_size(L.QMC_OP_INTEGRATE_BWD, rules, taus, fs, prec)
    if reuse_forward and (ws is None or ws.numel() < nbytes):
        raise ValueError("reuse_forward needs the workspace of the forward call, sized for the backward")
    ws = _workspace(nbytes, device, ws)
    up = upstream.to(device=device, dtype=torch.float64).reshape(-1).contiguous()
    grads = [torch.empty_like(a) for a in As]
    rs = (L.QmcRule * n)(*[r.struct(device) for r in rules])
    ap = (ctypes.c_void_p * n)(*[a.data_ptr() for a in As])
    ts = (ctypes.c_uint32 * n)(*taus)
    fa = (L.QmcIntegrand * n)(*[f.struct() for f in fs])
    gp = (ctypes.c_void_p * n)(*[g.data_ptr() for g in grads])
    flags = L.QMC_BWD_REUSE_FORWARD if reuse_forward else 0
    L.check(L.load().qmc_integrate_backward(rs, ap, ts, n, fa, prec, up.data_ptr(), gp, flags, ws.data_ptr(),
                                            ws.numel(), _stream(device)))
    return grads


def autotune(rule: Rule, A: torch.Tensor, f: Integrand, precision: Optional[str] = None) -> int:
    """Time the fine band's schedules for this problem shape on the GPU and cache the fastest (the
    library's planner then uses it for every call of this shape).  Returns the candidates timed.
    Synchronises the current stream; call it before sizing workspaces and before graph capture."""
    A = A.contiguous()
    prec = _precision(A, precision)
    nbytes = workspace_size(L.QMC_OP_INTEGRATE_BWD, [rule], [A.shape[1]], [f], prec)
    ws = torch.empty(max(2 * nbytes, 256), dtype=torch.uint8, device=A.device)
    est = torch.empty(rule.R_eff + 1, dtype=torch.float64, device=A.device)
    grad = torch.empty_like(A)
    n = ctypes.c_uint32(0)
    r = rule.struct(A.device)
    L.check(L.load().qmc_autotune(ctypes.byref(r), A.data_ptr(), A.shape[1], ctypes.byref(f.struct()), prec,
                                  est.data_ptr(), grad.data_ptr(), ws.data_ptr(), ws.numel(), _stream(A.device),
                                  ctypes.byref(n)))
    return int(n.value)


def tune_set(rule: Rule, tau: int, f: Integrand, precision: str, fwd_qpg: int = 0, bwd_rpc: int = 0,
             coarse: int = 0, bwd_path: int = 0) -> None:
    """Cache a schedule for this problem's shape (host only): forward columns per CTA / 4, adjoint
    roots per CTA, the coarse forward's path (1 level passes, 2 block products) and the coarse
    adjoint's path (1 one fold and the cp.async gradient kernel, 2 the fused fold-gradient and TMA
    gradient kernels); 0 keeps the cost model's choice of that value."""
    if precision not in L.PRECISIONS:
        raise ValueError(f"precision must be one of {sorted(L.PRECISIONS)} (got {precision!r})")
    r = rule.struct()
    L.check(L.load().qmc_tune_set(ctypes.byref(r), int(tau), ctypes.byref(f.struct()), L.PRECISIONS[precision],
                                  int(fwd_qpg), int(bwd_rpc), int(coarse), int(bwd_path)))


def tune_save(path: str) -> None:
    L.check(L.load().qmc_tune_save(str(path).encode()))


def tune_load(path: str) -> int:
    n = ctypes.c_uint32(0)
    L.check(L.load().qmc_tune_load(str(path).encode(), ctypes.byref(n)))
    return int(n.value)


def tune_clear() -> None:
    L.check(L.load().qmc_tune_clear())


class QMCEstimate(torch.autograd.Function):
    """Randomised QMC estimate (mean over shifts) of N^-1 sum_k f(x_k^T A), differentiable in A.
    The backward reuses the forward's workspace (no recomputation of the forward pass)."""

    @staticmethod
    def forward(ctx, A: torch.Tensor, rule: Rule, f: Integrand, precision: Optional[str] = None):
        A = A.contiguous()
        prec = _precision(A, precision)
        nbytes = workspace_size(L.QMC_OP_INTEGRATE_BWD, [rule], [A.shape[1]], [f], prec)
        ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=A.device)
        est = integrate(rule, A, f, ws=ws, precision=precision)
        ctx.save_for_backward(A)
        ctx.rule, ctx.f, ctx.ws, ctx.precision = rule, f, ws, precision
        return est[-1].to(A.dtype)

    @staticmethod
    def backward(ctx, grad_out):
        (A,) = ctx.saved_tensors
        g = integrate_backward(ctx.rule, A, ctx.f, grad_out.detach().reshape(1), ws=ctx.ws, reuse_forward=True,
                               precision=ctx.precision)[0]
        return g, None, None, None


def qmc_estimate(A: torch.Tensor, rule: Rule, f: Integrand, precision: Optional[str] = None) -> torch.Tensor:
    return QMCEstimate.apply(A, rule, f, precision)


class Integrator:
    """Fixed problems (rules, A's shapes and dtype, integrands) evaluated repeatedly: the estimates
    and, with ``backward=True``, dQ/dA, through one CUDA graph of the library's launches.

    Pass one problem (rule, A, f) or lists of them: several problems go to the library in one call,
    which runs them on parallel internal streams joined back to the caller's stream, so the graph
    holds every instance's launches as concurrent branches and one replay runs them all.
    The C structures, the workspace and the input/output buffers are built once; ``A`` (a tensor,
    or ``As``, a list) are static device tensors the caller overwrites before each ``run()``, which
    replays the graph on the current stream and returns the static outputs ``(est, grad)``: est holds,
    per problem, the R_eff per-shift estimates and their mean; grad is dQ/dA (a list for several
    problems).
    """

    def __init__(self, rule, A, f, backward: bool = True, graph: bool = True,
                 precision: Optional[str] = None):
        self.single = not isinstance(rule, (list, tuple))
        rules, As, fs = _as_list(rule), _as_list(A), _as_list(f)
        if not (len(rules) == len(As) == len(fs)):
            raise ValueError("rules, As and fs must have the same length")
        self.rules, self.fs, self.backward = rules, fs, backward
        self.device = As[0].device
        self.As = [a.detach().contiguous().clone() for a in As]
        self.prec = _precision(self.As[0], precision)
        n = len(rules)
        op = L.QMC_OP_INTEGRATE_BWD if backward else L.QMC_OP_INTEGRATE
        self.ws = torch.empty(max(workspace_size(op, rules, [a.shape[1] for a in self.As], fs, self.prec), 256),
                              dtype=torch.uint8, device=self.device)
        self.est = torch.empty(sum(r.R_eff + 1 for r in rules), dtype=torch.float64, device=self.device)
        self.grads = [torch.empty_like(a) for a in self.As]
        self.upstream = torch.ones(n, dtype=torch.float64, device=self.device)
        self._r = (L.QmcRule * n)(*[r.struct(self.device) for r in rules])
        self._ap = (ctypes.c_void_p * n)(*[a.data_ptr() for a in self.As])
        self._ts = (ctypes.c_uint32 * n)(*[a.shape[1] for a in self.As])
        self._fa = (L.QmcIntegrand * n)(*[x.struct() for x in fs])
        self._gp = (ctypes.c_void_p * n)(*[g.data_ptr() for g in self.grads])
        self._n = n
        self._lib = L.load()
        self.graph = None
        if graph:
            self._eager(torch.cuda.current_stream(self.device))          # loads modules, checks arguments
            torch.cuda.synchronize(self.device)
            g = torch.cuda.CUDAGraph()
            s = torch.cuda.Stream(self.device)
            s.wait_stream(torch.cuda.current_stream(self.device))
            with torch.cuda.stream(s):
                with torch.cuda.graph(g, stream=s):
                    self._eager(s)
            torch.cuda.current_stream(self.device).wait_stream(s)
            self.graph = g

    @property
    def A(self) -> torch.Tensor:
        return self.As[0]

    @property
    def grad(self) -> torch.Tensor:
        return self.grads[0]

    def _eager(self, stream) -> None:
        st = ctypes.c_void_p(stream.cuda_stream)
        L.check(self._lib.qmc_integrate(self._r, self._ap, self._ts, self._n, self._fa, self.prec, self.est.data_ptr(),
                                        None, self.ws.data_ptr(), self.ws.numel(), st))
        if self.backward:
            L.check(self._lib.qmc_integrate_backward(self._r, self._ap, self._ts, self._n, self._fa, self.prec,
                                                     self.upstream.data_ptr(), self._gp, L.QMC_BWD_REUSE_FORWARD,
                                                     self.ws.data_ptr(), self.ws.numel(), st))

    def run(self):
        if self.graph is not None:
            self.graph.replay()
        else:
            self._eager(torch.cuda.current_stream(self.device))
        return self.est, (self.grad if self.single else self.grads)
