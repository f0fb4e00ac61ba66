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
            T = sum(1 << (self.m - min(int(wj), self.m)) for wj in self.w)
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
        n = int(sum(2 ** (rule.m - min(int(w), rule.m)) for w in rule.w))
        out = torch.empty(n, dtype=torch.int32, device=device)
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
    """A fixed problem (rule, A's shape and dtype, f) evaluated repeatedly: the estimate and,
    with ``backward=True``, dQ/dA, through one CUDA graph of the library's launches.

    The C structures, the workspace and the input/output buffers are built once; ``A`` is a
    static device tensor the caller overwrites (``integrator.A.copy_(...)``) before each
    ``run()``, which replays the graph on the current stream and returns the static outputs
    ``(est, grad)`` -- est holds the R_eff per-shift estimates and their mean.
    """

    def __init__(self, rule: Rule, A: torch.Tensor, f: Integrand, backward: bool = True, graph: bool = True,
                 precision: Optional[str] = None):
        self.rule, self.f, self.backward = rule, f, backward
        self.device = A.device
        self.A = A.detach().contiguous().clone()
        self.prec = _precision(self.A, precision)
        op = L.QMC_OP_INTEGRATE_BWD if backward else L.QMC_OP_INTEGRATE
        self.ws = torch.empty(max(workspace_size(op, [rule], [self.A.shape[1]], [f], self.prec), 256),
                              dtype=torch.uint8, device=self.device)
        self.est = torch.empty(rule.R_eff + 1, dtype=torch.float64, device=self.device)
        self.grad = torch.empty_like(self.A)
        self.upstream = torch.ones(1, dtype=torch.float64, device=self.device)
        self._rs = L.QmcRule * 1
        self._r = self._rs(rule.struct(self.device))
        self._ap = (ctypes.c_void_p * 1)(self.A.data_ptr())
        self._ts = (ctypes.c_uint32 * 1)(self.A.shape[1])
        self._fa = (L.QmcIntegrand * 1)(f.struct())
        self._gp = (ctypes.c_void_p * 1)(self.grad.data_ptr())
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

    def _eager(self, stream) -> None:
        st = ctypes.c_void_p(stream.cuda_stream)
        L.check(self._lib.qmc_integrate(self._r, self._ap, self._ts, 1, self._fa, self.prec, self.est.data_ptr(),
                                        None, self.ws.data_ptr(), self.ws.numel(), st))
        if self.backward:
            L.check(self._lib.qmc_integrate_backward(self._r, self._ap, self._ts, 1, self._fa, self.prec,
                                                     self.upstream.data_ptr(), self._gp, L.QMC_BWD_REUSE_FORWARD,
                                                     self.ws.data_ptr(), self.ws.numel(), st))

    def run(self):
        if self.graph is not None:
            self.graph.replay()
        else:
            self._eager(torch.cuda.current_stream(self.device))
        return self.est, self.grad
