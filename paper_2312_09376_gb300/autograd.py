"""Differentiable RBT solve: X = solve(A, B) with a hand-written adjoint.

Forward: ``rbt_solve`` (Eq. precond with refinement, Sec. 5).  Backward
reuses the factors of A~ = U^T A V that the forward call left in its
workspace:

    grad_B = A^{-T} grad_X = U A~^{-T} V^T grad_X     (rbt_solve_adjoint)
    grad_A = -grad_B X^T                               (rbt_outer)

Both run in the library's kernels; this module only marshals tensors.
Matrices are float64 CUDA tensors; a non-column-major input is copied to a
column-major layout first (a layout change, no arithmetic).
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib


def _colmajor(t):
    if t.dim() == 1:
        return t.contiguous()
    if t.stride(0) == 1 and t.stride(1) >= max(1, t.shape[0]):
        return t
    return t.T.contiguous().T


class _RBTSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A, B, depth, seed, prec, refine_max, tol, fallback, kind="scaled"):
        A = _colmajor(A.detach())
        vec = B.dim() == 1
        Bm = _colmajor(B.detach().reshape(-1, 1) if vec else B.detach())
        n, nrhs = Bm.shape
        opts = _lib.make_opts(depth, seed, prec, refine_max, tol, fallback, kind=kind)
        X = _lib.colmajor(n, nrhs, device=A.device)
        work = torch.empty(max(_lib.rbt_solve_workspace(opts, n, nrhs), 1), dtype=torch.uint8, device=A.device)
        info = _lib.rbt_info()
        lib = _lib.load()
        pa, lda, _, _ = _lib._mat(A, "A", torch.float64)
        pb, ldb, _, _ = _lib._mat(Bm, "B", torch.float64)
        px, ldx, _, _ = _lib._mat(X, "X", torch.float64)
        code = lib.rbt_solve(ctypes.byref(opts), n, nrhs, pa, lda, pb, ldb, px, ldx,
                             ctypes.c_void_p(work.data_ptr()), work.numel(), ctypes.byref(info), _lib._stream())
        _lib._check("rbt_solve", code, (_lib.RBT_OK, _lib.RBT_NOT_CONVERGED))
        ctx.opts, ctx.work, ctx.info, ctx.vec = opts, work, info, vec
        ctx.save_for_backward(A, X)
        ctx.fwd_info = info.as_dict()
        return X[:, 0] if vec else X

    @staticmethod
    def backward(ctx, gX):
        A, X = ctx.saved_tensors
        n, nrhs = X.shape
        G = _colmajor(gX.reshape(-1, 1) if ctx.vec else gX)
        if G.dtype != torch.float64:
            G = G.double()
        Y = _lib.colmajor(n, nrhs, device=A.device)
        info = _lib.rbt_info()
        lib = _lib.load()
        pa, lda, _, _ = _lib._mat(A, "A", torch.float64)
        pg, ldg, _, _ = _lib._mat(G, "G", torch.float64)
        py, ldy, _, _ = _lib._mat(Y, "Y", torch.float64)
        code = lib.rbt_solve_adjoint(ctypes.byref(ctx.opts), ctypes.byref(ctx.info), n, nrhs, pa, lda, pg, ldg,
                                     py, ldy, ctypes.c_void_p(ctx.work.data_ptr()), ctx.work.numel(),
                                     ctypes.byref(info), _lib._stream())
        _lib._check("rbt_solve_adjoint", code, (_lib.RBT_OK, _lib.RBT_NOT_CONVERGED))
        gA = None
        if ctx.needs_input_grad[0]:
            gA = _lib.colmajor(n, n, device=A.device)
            px, ldx, _, _ = _lib._mat(X, "X", torch.float64)
            pga, ldga, _, _ = _lib._mat(gA, "gA", torch.float64)
            _lib._check("rbt_outer", lib.rbt_outer(n, n, nrhs, -1.0, py, ldy, px, ldx, pga, ldga, _lib._stream()))
        gB = Y[:, 0] if ctx.vec else Y
        ctx.adj_info = info.as_dict()
        return gA, gB, None, None, None, None, None, None, None


def solve(A, B, depth=2, seed=1, prec="f64", refine_max=30, tol=1e-13, fallback=True, kind="scaled"):
    """Differentiable X = A^{-1} B through the RBT solver (float64 CUDA tensors);
    kind = "rotation" takes the orthogonal block-rotation butterflies."""
    return _RBTSolve.apply(A, B, depth, seed, prec, refine_max, tol, fallback, kind)


def solve_batched(As, Bs, depth=2, seed=1000, prec="f32", refine_max=30, tol=1e-13, seeds=None, fallback=True):
    """Batched forward (one persistent launch).  Returns (Xs, plan); pass the
    plan to ``solve_batched_backward``."""
    opts = _lib.make_opts(depth, seed, prec, refine_max, tol, fallback)
    As = [_colmajor(a) for a in As]
    Bs = [_colmajor(b.reshape(-1, 1) if b.dim() == 1 else b) for b in Bs]
    Xs = [_lib.colmajor(b.shape[0], b.shape[1], device=b.device) for b in Bs]
    plan = _lib.rbt_solve_batched_plan(opts, As, Bs, Xs, seeds=seeds)
    _lib.rbt_solve_batched_run(plan)
    plan.As, plan.Xs = As, Xs
    return Xs, plan


def solve_batched_backward(plan, gXs, want_grad_A=True):
    """Batched adjoint on a planned and run batch: returns (grad_Bs, grad_As)."""
    gXs = [_colmajor(g.reshape(-1, 1) if g.dim() == 1 else g) for g in gXs]
    Ys = [_lib.colmajor(x.shape[0], x.shape[1], device=x.device) for x in plan.Xs]
    GAs = [_lib.colmajor(a.shape[0], a.shape[0], device=a.device) for a in plan.As] if want_grad_A else None
    lib = _lib.load()
    b = len(gXs)
    g_arr = _lib._ptr_array(gXs)
    y_arr = _lib._ptr_array(Ys)
    ldg = _lib._i64_array([g.stride(1) if g.shape[1] > 1 else g.shape[0] for g in gXs])
    ldy = _lib._i64_array([y.stride(1) if y.shape[1] > 1 else y.shape[0] for y in Ys])
    ga_arr = _lib._ptr_array(GAs) if GAs else None
    ldga = _lib._i64_array([a.stride(1) for a in GAs]) if GAs else None
    code = lib.rbt_solve_batched_adjoint(ctypes.byref(plan.opts), ctypes.c_void_p(plan.work.data_ptr()), b, g_arr,
                                         ldg, y_arr, ldy, ga_arr, ldga, ctypes.c_void_p(plan.infos.data_ptr()),
                                         _lib._stream())
    _lib._check("rbt_solve_batched_adjoint", code)
    return Ys, GAs
