"""rbt_residual_noalloc: the residual / backward-error check for callers that
cannot allocate device memory (inside someone else's graph capture, plugins
whose framework owns the allocator, C callers without a device allocator).

It must give the results of rbt_residual (the workspace-taking entry point)
on two calls in a row, since all calls share one fixed scratch array in the
library, and refuse sizes beyond that array before touching the GPU.  This
file is collected last so that a run stopping at the first failure has run
every other test first; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2312_09376_gb300 import _lib, inputs
from tests import _bounds

pytestmark = pytest.mark.gpu


def _with_workspace(n, A, X, B):
    nrhs = X.shape[1] if X.dim() == 2 else 1
    R = _lib.colmajor(n, nrhs)
    berr = torch.zeros(1, dtype=torch.float64, device="cuda")
    work = torch.empty(_lib.rbt_residual_workspace(n, nrhs), dtype=torch.uint8, device="cuda")
    _lib.rbt_residual(n, A, X, B, R, d_berr=berr, work=work)
    return R, berr


def _without_workspace(n, A, X, B):
    nrhs = X.shape[1] if X.dim() == 2 else 1
    R = _lib.colmajor(n, nrhs)
    berr = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    _lib.rbt_residual_noalloc(n, A, X, B, R, d_berr=berr)
    return R, berr


def test_noalloc_matches_workspace_entry_point_twice_in_a_row():
    cases = [(1003, 1, 1), (2000, 3, 2)]          # (n, nrhs, seed): the second call sees new data
    for n, nrhs, seed in cases:
        A = _lib.to_device(inputs.gaussian(n, seed=40 + seed))
        X = _lib.to_device(inputs.rhs(n, nrhs, seed=50 + seed))
        B = _lib.to_device(inputs.rhs(n, nrhs, seed=60 + seed))
        Rw, bw = _with_workspace(n, A, X, B)
        Rn, bn = _without_workspace(n, A, X, B)
        torch.cuda.synchronize()
        # same tolerance as the residual parity test: 2 gamma_(n+1) (|A||x| + |b|)
        scale = (A.abs() @ X.abs().reshape(n, nrhs)) + B.abs().reshape(n, nrhs)
        tol = 2 * _bounds.gamma(n + 1, _bounds.U64) * scale
        assert torch.all((Rn - Rw).abs() <= tol)
        assert abs(float(bn.item()) - float(bw.item())) <= 1e-10 * float(bw.item())
        assert float(bn.item()) > 0


def test_noalloc_with_given_norm_and_without_backward_error():
    """The other two branches: a caller-supplied ||A|| (from rbt_norm_inf), and
    a residual-only call (d_berr = NULL), each twice in a row against
    rbt_residual with the same arguments."""
    for n, nrhs, seed in [(1500, 2, 3), (777, 1, 4)]:
        A = _lib.to_device(inputs.gaussian(n, seed=70 + seed))
        X = _lib.to_device(inputs.rhs(n, nrhs, seed=80 + seed))
        B = _lib.to_device(inputs.rhs(n, nrhs, seed=90 + seed))
        anorm = torch.zeros(1, dtype=torch.float64, device="cuda")
        work = torch.empty(_lib.rbt_residual_workspace(n, nrhs), dtype=torch.uint8, device="cuda")
        _lib.rbt_norm_inf(n, A, anorm, work)
        scale = (A.abs() @ X.abs().reshape(n, nrhs)) + B.abs().reshape(n, nrhs)
        tol = 2 * _bounds.gamma(n + 1, _bounds.U64) * scale
        # given norm
        Rw, bw = _lib.colmajor(n, nrhs), torch.zeros(1, dtype=torch.float64, device="cuda")
        _lib.rbt_residual(n, A, X, B, Rw, d_berr=bw, d_anorm=anorm, work=work)
        Rn, bn = _lib.colmajor(n, nrhs), torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        _lib.rbt_residual_noalloc(n, A, X, B, Rn, d_berr=bn, d_anorm=anorm)
        torch.cuda.synchronize()
        assert torch.all((Rn - Rw).abs() <= tol)
        assert abs(float(bn.item()) - float(bw.item())) <= 1e-10 * float(bw.item())
        # residual only: R matches, nothing else is written
        Rw2 = _lib.colmajor(n, nrhs)
        _lib.rbt_residual(n, A, X, B, Rw2, work=work)
        Rn2 = _lib.colmajor(n, nrhs)
        _lib.rbt_residual_noalloc(n, A, X, B, Rn2)
        torch.cuda.synchronize()
        assert torch.all((Rn2 - Rw2).abs() <= tol)


def test_noalloc_refuses_sizes_beyond_its_scratch():
    lib = _lib.load()
    cap = lib.rbt_residual_noalloc_max_bytes()
    assert cap >= 16 << 20
    n, nrhs = 50000, 8                              # needs far more than the fixed array
    assert lib.rbt_residual_workspace(n, nrhs) > cap
    P = ctypes.c_void_p(16)                          # never dereferenced: refused before any launch
    code = lib.rbt_residual_noalloc(n, nrhs, P, n, P, n, P, n, P, n, None, P, None)
    assert code == _lib.RBT_ERR_WORKSPACE
