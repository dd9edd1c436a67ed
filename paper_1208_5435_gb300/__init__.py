"""GB300 matrix-free primal-dual IPM for  min tau*||x||_1 + 1/2*||A x - b||^2
(arXiv:1208.5435).  Thin Python binding over the C ABI of include/mfipm.h: torch
tensors supply device memory and the stream; every step of the solve runs in the
library's CUDA kernels (libmfipm.so, built by build.py)."""
from __future__ import annotations

import ctypes
import dataclasses
from typing import List, Optional, Sequence

from . import _capi as C
from ._capi import MfipmError, lib

__all__ = ["Dense", "DenseBF16", "PartialDCT", "PartialHaar", "SolverParams", "solve", "solve_batched", "workspace_bytes",
           "apply_A", "apply_At", "kkt_residual", "autotune", "clear_tuning", "MfipmError", "lib"]


def _torch():
    import torch
    return torch


@dataclasses.dataclass
class SolverParams:
    """Mirror of mfipm_params (defaults of mfipm_params_default)."""
    tol: float = 1e-10
    max_iter: int = 100
    tol_pcg: float = 1e-2
    max_iter_pcg: int = 200
    sigma1: float = 0.1
    sigma2: float = 0.5
    sigma3: float = 0.8
    alpha_bar: float = 0.5
    alpha_tilde: float = 0.1
    eta: float = 0.995
    precision: Optional[int] = None   # None: FP32 PCG for the DCT, FP64 for dense A
    equal_steps: int = 0
    cluster_size: int = 0
    outer: int = 0                    # partial DCT outer loop: 0 double-float, 1 native float64
    outer_f32_gap: float = 1e-8       # partial DCT: float32 outer residual while the gap exceeds this
    centrality_correctors: int = 0    # 0: the single corrector; K: up to K centrality correctors

    def to_c(self, default_precision: int) -> C.Params:
        p = C.Params()
        for f in dataclasses.fields(self):
            v = getattr(self, f.name)
            if f.name == "precision" and v is None:
                v = default_precision
            setattr(p, f.name, v)
        return p


class PartialDCT:
    """A = the sampled rows `rows` (int64 CUDA tensor, ascending, distinct) of the
    orthonormal n x n DCT-II."""

    def __init__(self, n: int, rows):
        torch = _torch()
        self.n = int(n)
        self.rows = rows.to(device="cuda", dtype=torch.int64).contiguous()
        self.m = int(self.rows.numel())
        self.default_precision = C.PREC_FP32_PCG

    def c_op(self) -> C.Operator:
        op = C.Operator()
        op.kind, op.a_dtype, op.m, op.n = C.OP_PARTIAL_DCT, 0, self.m, self.n
        op.A, op.a_scale, op.lda = None, 1.0, 0
        op.rows = self.rows.data_ptr() if self.m else None
        return op


class PartialHaar:
    """A = the sampled rows `rows` (int64, ascending, distinct) of the orthonormal n x n Haar
    matrix: row 0 the constant 1/sqrt(n), row 2^j + k the wavelet of scale j, position k."""

    def __init__(self, n: int, rows):
        torch = _torch()
        self.n = int(n)
        self.rows = rows.to(device="cuda", dtype=torch.int64).contiguous()
        self.m = int(self.rows.numel())
        self.default_precision = C.PREC_FP32_PCG

    def c_op(self) -> C.Operator:
        op = C.Operator()
        op.kind, op.a_dtype, op.m, op.n = C.OP_PARTIAL_HAAR, 0, self.m, self.n
        op.A, op.a_scale, op.lda = None, 1.0, 0
        op.rows = self.rows.data_ptr() if self.m else None
        return op


class Dense:
    """Explicit A (float64 CUDA tensor, m x n, row-major)."""

    def __init__(self, A, a_scale: float = 1.0):
        torch = _torch()
        self.A = A.to(device="cuda", dtype=torch.float64).contiguous()
        self.m, self.n = (int(s) for s in self.A.shape)
        self.a_scale = float(a_scale)
        self.default_precision = C.PREC_FP64

    def c_op(self) -> C.Operator:
        op = C.Operator()
        op.kind, op.a_dtype, op.m, op.n = C.OP_DENSE, C.A_F64, self.m, self.n
        op.A, op.a_scale, op.lda = self.A.data_ptr(), self.a_scale, self.n
        op.rows = None
        return op


class DenseBF16:
    """A = a_scale * A_bf16 with A_bf16 an m x n bfloat16 CUDA tensor (or its uint16 bit
    patterns), shared by the right-hand sides of one mfipm_solve_batched call
    (MFIPM_PREC_BF16_A: tensor-core products, float64 outer loop)."""

    def __init__(self, A_bf16, a_scale: float = 1.0):
        torch = _torch()
        if A_bf16.dtype == torch.uint16 if hasattr(torch, "uint16") else False:
            A_bf16 = A_bf16.view(torch.bfloat16)
        if A_bf16.dtype == torch.int16:
            A_bf16 = A_bf16.view(torch.bfloat16)
        self.A = A_bf16.to(device="cuda").contiguous()
        assert self.A.dtype == torch.bfloat16
        self.m, self.n = (int(s) for s in self.A.shape)
        self.a_scale = float(a_scale)
        self.default_precision = C.PREC_BF16_A

    def c_op(self) -> C.Operator:
        op = C.Operator()
        op.kind, op.a_dtype, op.m, op.n = C.OP_DENSE, C.A_BF16, self.m, self.n
        op.A, op.a_scale, op.lda = self.A.data_ptr(), self.a_scale, self.n
        op.rows = None
        return op


def _stream_handle(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def workspace_bytes(ops: Sequence, params: Optional[SolverParams] = None) -> int:
    params = params or SolverParams()
    arr = (C.Operator * len(ops))(*[o.c_op() for o in ops])
    p = params.to_c(ops[0].default_precision)
    nbytes = ctypes.c_size_t(0)
    C.check(lib().mfipm_workspace_size(arr, len(ops), ctypes.byref(p), ctypes.byref(nbytes)))
    return int(nbytes.value)


def _alloc_ws(nbytes: int):
    torch = _torch()
    return torch.empty(max(nbytes, 256), dtype=torch.uint8, device="cuda")


def solve(op, b, tau: float, params: Optional[SolverParams] = None, return_zs: bool = False, ws=None,
          stream=None, raise_on_failure: bool = True):
    """Solve one problem.  Returns (x, info dict[, zs]) with x a float64 CUDA tensor."""
    torch = _torch()
    params = params or SolverParams()
    b = b.to(device="cuda", dtype=torch.float64).contiguous()
    x = torch.empty(op.n, dtype=torch.float64, device="cuda")
    zs = torch.empty(4 * op.n, dtype=torch.float64, device="cuda") if return_zs else None
    p = params.to_c(op.default_precision)
    cop = op.c_op()
    if ws is None:
        ws = _alloc_ws(workspace_bytes([op], params))
    info = C.Info()
    rc = lib().mfipm_solve(ctypes.byref(cop), b.data_ptr() if op.m else None, float(tau), ctypes.byref(p),
                           x.data_ptr(), zs.data_ptr() if zs is not None else None, ws.data_ptr(), ws.numel(),
                           ctypes.byref(info), _stream_handle(stream))
    if raise_on_failure:
        C.check(rc, allow=(C.MFIPM_OK, C.MFIPM_NOT_CONVERGED))
    d = info.as_dict()
    d["return_code"] = rc
    return (x, d, zs) if return_zs else (x, d)


def solve_batched(ops: Sequence, bs: Sequence, taus: Sequence[float], params: Optional[SolverParams] = None,
                  return_zs: bool = False, ws=None, stream=None, raise_on_failure: bool = True):
    """Solve independent problems in one persistent launch.  Returns (xs, infos[, zss])."""
    torch = _torch()
    params = params or SolverParams()
    B = len(ops)
    bs = [bb.to(device="cuda", dtype=torch.float64).contiguous() for bb in bs]
    xs = [torch.empty(o.n, dtype=torch.float64, device="cuda") for o in ops]
    zss = [torch.empty(4 * o.n, dtype=torch.float64, device="cuda") for o in ops] if return_zs else None
    arr = (C.Operator * B)(*[o.c_op() for o in ops])
    bp = (ctypes.c_void_p * B)(*[bb.data_ptr() for bb in bs])
    xp = (ctypes.c_void_p * B)(*[xx.data_ptr() for xx in xs])
    zp = (ctypes.c_void_p * B)(*[z.data_ptr() for z in zss]) if return_zs else None
    tp = (ctypes.c_double * B)(*[float(t) for t in taus])
    p = params.to_c(ops[0].default_precision)
    if ws is None:
        ws = _alloc_ws(workspace_bytes(ops, params))
    infos = (C.Info * B)()
    rc = lib().mfipm_solve_batched(B, arr, bp, tp, ctypes.byref(p), xp, zp, ws.data_ptr(), ws.numel(), infos,
                                   _stream_handle(stream))
    out = [i.as_dict() for i in infos]
    # a problem of the batch that ended MFIPM_NUMERIC is reported in its info, like one that
    # did not converge; anything else (bad arguments, CUDA errors, non-finite b: the calls
    # that leave a message in mfipm_last_error) raises
    per_problem = rc == C.MFIPM_NUMERIC and not C.last_error() and any(i["status"] == rc for i in out)
    if raise_on_failure and not per_problem:
        C.check(rc, allow=(C.MFIPM_OK, C.MFIPM_NOT_CONVERGED))
    return (xs, out, zss) if return_zs else (xs, out)


def backward(ops, bs, taus, xs, zss, grad_xs, params: Optional[SolverParams] = None, want_A: bool = False,
             ws=None, stream=None):
    """mfipm_backward for a list of problems (forward outputs xs and zss from solve(...,
    return_zs=True)).  Returns (grad_bs, grad_taus, grad_As or None, infos)."""
    torch = _torch()
    params = params or SolverParams()
    B = len(ops)
    bs = [bb.to(device="cuda", dtype=torch.float64).contiguous() for bb in bs]
    gxs = [g.to(device="cuda", dtype=torch.float64).contiguous() for g in grad_xs]
    gbs = [torch.empty(o.m, dtype=torch.float64, device="cuda") for o in ops]
    gAs = [torch.empty(o.m, o.n, dtype=torch.float64, device="cuda") for o in ops] if want_A else None
    arr = (C.Operator * B)(*[o.c_op() for o in ops])
    ptrs = lambda ts: (ctypes.c_void_p * B)(*[t.data_ptr() for t in ts])
    tp = (ctypes.c_double * B)(*[float(t) for t in taus])
    gtau = (ctypes.c_double * B)()
    p = params.to_c(ops[0].default_precision)
    if ws is None:
        ws = _alloc_ws(workspace_bytes(ops, params))
    infos = (C.Info * B)()
    rc = lib().mfipm_backward(B, arr, ptrs(bs), tp, ptrs(xs), ptrs(zss), ptrs(gxs), ptrs(gbs), gtau,
                              ptrs(gAs) if want_A else None, ctypes.byref(p), ws.data_ptr(), ws.numel(), infos,
                              _stream_handle(stream))
    C.check(rc)
    return gbs, [gtau[i] for i in range(B)], gAs, [i.as_dict() for i in infos]


def solve_differentiable(op, b, tau, params: Optional[SolverParams] = None):
    """x* as a differentiable function of b, tau (and of A for a Dense operator whose A requires
    grad): torch.autograd calls mfipm_backward, which solves the adjoint KKT system at the
    solution with the same PCG (no unrolling of iterations)."""
    from .autograd import MfipmFunction
    torch = _torch()
    tau_t = tau if torch.is_tensor(tau) else torch.tensor(float(tau), dtype=torch.float64)
    A = op.A if isinstance(op, Dense) else None
    return MfipmFunction.apply(b, tau_t, A, op, params or SolverParams())


def apply_A(op, x, ws=None, stream=None):
    """y = A x (float64 CUDA tensors) through mfipm_apply_A."""
    torch = _torch()
    x = x.to(device="cuda", dtype=torch.float64).contiguous()
    y = torch.empty(op.m, dtype=torch.float64, device="cuda")
    ws = ws if ws is not None else _alloc_ws(workspace_bytes([op]))
    cop = op.c_op()
    C.check(lib().mfipm_apply_A(ctypes.byref(cop), x.data_ptr(), y.data_ptr(), ws.data_ptr(), ws.numel(),
                                _stream_handle(stream)))
    return y


def apply_At(op, y, ws=None, stream=None):
    """x = A^T y (float64 CUDA tensors) through mfipm_apply_At."""
    torch = _torch()
    y = y.to(device="cuda", dtype=torch.float64).contiguous()
    x = torch.empty(op.n, dtype=torch.float64, device="cuda")
    ws = ws if ws is not None else _alloc_ws(workspace_bytes([op]))
    cop = op.c_op()
    C.check(lib().mfipm_apply_At(ctypes.byref(cop), y.data_ptr(), x.data_ptr(), ws.data_ptr(), ws.numel(),
                                 _stream_handle(stream)))
    return x


def kkt_residual(op, b, tau: float, x, ws=None, stream=None) -> float:
    """kkt_rel(x) = ||x - S_tau(x - A^T(Ax - b))|| / (1 + ||x||) through mfipm_kkt_residual."""
    torch = _torch()
    b = b.to(device="cuda", dtype=torch.float64).contiguous()
    x = x.to(device="cuda", dtype=torch.float64).contiguous()
    ws = ws if ws is not None else _alloc_ws(workspace_bytes([op]))
    out = ctypes.c_double(0.0)
    cop = op.c_op()
    C.check(lib().mfipm_kkt_residual(ctypes.byref(cop), b.data_ptr(), float(tau), x.data_ptr(), ws.data_ptr(),
                                     ws.numel(), ctypes.byref(out), _stream_handle(stream)))
    return float(out.value)


def autotune(ops: Sequence, bs: Sequence, taus: Sequence[float], params: Optional[SolverParams] = None, ws=None,
             stream=None):
    """mfipm_autotune: time the candidate decompositions on this batch and keep the fastest for
    later solves of this process.  Returns (xs, infos, tuning dict)."""
    torch = _torch()
    params = params or SolverParams()
    B = len(ops)
    bs = [bb.to(device="cuda", dtype=torch.float64).contiguous() for bb in bs]
    xs = [torch.empty(o.n, dtype=torch.float64, device="cuda") for o in ops]
    arr = (C.Operator * B)(*[o.c_op() for o in ops])
    bp = (ctypes.c_void_p * B)(*[bb.data_ptr() for bb in bs])
    xp = (ctypes.c_void_p * B)(*[xx.data_ptr() for xx in xs])
    tp = (ctypes.c_double * B)(*[float(t) for t in taus])
    p = params.to_c(ops[0].default_precision)
    ws = ws if ws is not None else _alloc_ws(workspace_bytes(ops, params))
    infos = (C.Info * B)()
    tun = C.Tuning()
    C.check(lib().mfipm_autotune(B, arr, bp, tp, ctypes.byref(p), xp, ws.data_ptr(), ws.numel(), infos,
                                 ctypes.byref(tun), _stream_handle(stream)), allow=(C.MFIPM_OK, C.MFIPM_NOT_CONVERGED))
    return xs, [i.as_dict() for i in infos], tun.as_dict()


def clear_tuning():
    C.check(lib().mfipm_clear_tuning())
