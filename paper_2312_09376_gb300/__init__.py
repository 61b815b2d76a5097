"""gb300-rbt: generalized random butterfly transform + GENP solver on GB300 (sm_103a).

Method: Lindquist, Luszczek, Dongarra, "Generalizing Random Butterfly
Transforms to Arbitrary Matrix Sizes" (arXiv 2312.09376).  The compute path is
the C-ABI library ``libgb300rbt.so`` (``include/rbt.h``); this package holds
its ctypes binding (``_lib``), its in-tree build (``_build``), the seeded
synthetic inputs (``inputs``) and the autograd wrapper (``autograd``).
"""
from __future__ import annotations

from . import _build  # noqa: F401


def solve(A, B, depth=2, seed=1, prec="f64", refine_max=30, tol=1e-13, fallback=True, nb=0, stream=None, align=1,
          refine="stationary", restart=0, kind="scaled", grid=(1, 1)):
    """X = A^{-1} B through ``rbt_solve``; A (n x n) and B (n x nrhs or n) are
    column-major float64 CUDA tensors; align = n_b selects the tiled reference
    size of the butterflies; refine = "gmres" refines by restarted GMRES
    (restart = basis size, 0 = 30) instead of stationary steps; kind =
    "rotation" takes the orthogonal block-rotation butterflies instead of the
    scaled ones; grid = (p, q) aligns the butterflies for a p x q process grid
    (the communication-free size of Sec. 6, with tiles of align rows).
    Returns (X, info dict)."""
    import torch

    from . import _lib
    n = A.shape[0]
    opts = _lib.make_opts(depth, seed, prec, refine_max, tol, fallback, nb, align, refine, restart, kind, grid)
    nrhs = 1 if B.dim() == 1 else B.shape[1]
    X = torch.empty_like(B) if B.dim() == 1 else _lib.colmajor(n, nrhs, device=B.device)
    ws = _lib.rbt_solve_workspace(opts, n, nrhs)
    work = torch.empty(max(ws, 1), dtype=torch.uint8, device=A.device)
    code, info = _lib.rbt_solve(opts, n, A, B, X, work, stream=stream)
    info["code"] = code
    return X, info
