"""Bounded device waits run out cleanly and are reported: failure detection
without any GPU fault.

Every spin-wait of the library's kernels gives up after a time limit.  These
tests shorten that limit to a few milliseconds (rbt_debug_wait_limit), make
one kind of wait run out on purpose (rbt_debug_stall, a host setting: the
chained solves' block queue starts at block 1, so block 0 is never solved; or
the sliced update's copy warp issues no copy, so nothing ever fills the
stage the tensor-core warp waits for), and check that
  1. the call reports the timeout through its documented status,
  2. it comes back within a bounded time (the waits really end),
  3. the next normal call on the same stream is correct: the context and
     the library stay usable.
"""
import time

import numpy as np
import pytest
import torch

from paper_2312_09376_gb300 import _lib, inputs, solve
from paper_2312_09376_gb300 import autograd as ag
from tests._df64 import from_df64, to_df64

pytestmark = pytest.mark.gpu

LIMIT_NS = 2_000_000        # 2 ms per wait
BOUND_S = 20.0              # a whole call with every wait running out, generously


@pytest.fixture
def stall():
    _lib.load()
    _lib.rbt_debug_wait_limit(LIMIT_NS)
    yield _lib.rbt_debug_stall
    _lib.rbt_debug_stall("none")
    _lib.rbt_debug_wait_limit(0)


def _berr(A, X, B):
    r = np.abs(B - A @ X).max(axis=0)
    return float((r / (np.abs(A).sum(axis=1).max() * np.abs(X).max(axis=0) + np.abs(B).max(axis=0))).max())


def _flag(work):
    return int(work[:4].view(torch.int32).item())


def _f64_factors(n, seed):
    A = inputs.gaussian(n, seed=seed)
    LU = _lib.to_device(A)
    info = torch.empty(1, dtype=torch.int64, device="cuda")
    _lib.genp_factor(n, "f64", LU, info)
    torch.cuda.synchronize()
    assert int(info.item()) == -1
    return A, LU


@pytest.mark.parametrize("trans", [0, 1])
def test_chained_solve_wait_runs_out_then_recovers(stall, trans):
    n, nrhs = 700, 2                      # 11 row blocks of 64, the chained form (< 4 right-hand sides)
    A, LU = _f64_factors(n, 3)
    B = _lib.to_device(inputs.rhs(n, nrhs, seed=4))
    work = torch.empty(_lib.genp_solve_workspace(n, nrhs, "f64"), dtype=torch.uint8, device="cuda")
    Xref = B.clone()
    _lib.genp_solve(n, "f64", LU, trans, Xref, work)
    torch.cuda.synchronize()
    assert _flag(work) == 0

    stall("chain")
    X = B.clone()
    t0 = time.perf_counter()
    _lib.genp_solve(n, "f64", LU, trans, X, work)
    torch.cuda.synchronize()
    assert time.perf_counter() - t0 < BOUND_S
    assert _flag(work) != 0                # reported in the first int of work

    stall("none")
    X2 = B.clone()
    _lib.genp_solve(n, "f64", LU, trans, X2, work)
    torch.cuda.synchronize()
    assert _flag(work) == 0                # cleared on entry, not set again
    assert torch.equal(X2, Xref)           # the chained solve is bitwise reproducible


@pytest.mark.parametrize("prec,refine,nrhs", [("f64", "stationary", 1), ("f32", "gmres", 2)])
def test_solve_reports_chain_timeout_then_recovers(stall, prec, refine, nrhs):
    n = 500
    A = inputs.gaussian(n, seed=5)
    B = inputs.rhs(n, nrhs, seed=6)
    Ad, Bd = _lib.to_device(A), _lib.to_device(B)
    opts = _lib.make_opts(depth=2, seed=1, prec=prec, refine=refine, fallback=True)
    work = torch.empty(_lib.rbt_solve_workspace(opts, n, nrhs), dtype=torch.uint8, device="cuda")
    X = _lib.colmajor(n, nrhs)

    stall("chain")
    t0 = time.perf_counter()
    code, _ = _lib.rbt_solve(opts, n, Ad, Bd, X, work, ok=(_lib.RBT_ERR_TIMEOUT,))
    assert code == _lib.RBT_ERR_TIMEOUT
    assert time.perf_counter() - t0 < BOUND_S

    stall("none")
    code, info = _lib.rbt_solve(opts, n, Ad, Bd, X, work)
    assert code == _lib.RBT_OK and info["berr"] <= 1e-13
    assert _berr(A, _lib.to_host(X), B) <= 1e-13


def test_adjoint_reports_chain_timeout(stall):
    n, k = 300, 3
    A = _lib.to_device(inputs.gaussian(n, seed=8)).requires_grad_(True)
    B = _lib.to_device(inputs.rhs(n, k, seed=9)).requires_grad_(True)
    X = ag.solve(A, B, depth=2, seed=1, prec="f64")
    stall("chain")                          # the forward solve ran normally; the adjoint's waits run out
    with pytest.raises(_lib.RbtError) as e:
        X.sum().backward()
    assert e.value.code == _lib.RBT_ERR_TIMEOUT
    stall("none")
    A.grad = B.grad = None
    X = ag.solve(A, B, depth=2, seed=1, prec="f64")
    X.sum().backward()
    assert torch.isfinite(B.grad).all()


def test_sliced_update_wait_runs_out_then_recovers(stall):
    M, N, K = 300, 200, 64
    rng = np.random.default_rng(10)
    Ah, Bh, Ch = rng.standard_normal((M, K)), rng.standard_normal((K, N)), rng.standard_normal((M, N))
    Ad, Av = to_df64(Ah)
    Bd, Bv = to_df64(Bh)
    status = torch.empty(1, dtype=torch.int64, device="cuda")
    work = torch.empty(_lib.genp_update_workspace(M, N, K, "df64tc"), dtype=torch.uint8, device="cuda")

    stall("oz_copy")
    Cd, _ = to_df64(Ch)
    t0 = time.perf_counter()
    _lib.genp_update("df64tc", Ad, Bd, Cd, status, work)
    torch.cuda.synchronize()
    assert time.perf_counter() - t0 < BOUND_S
    assert int(status.item()) == -2         # the documented timeout status

    stall("none")
    Cd, Cv = to_df64(Ch)
    _lib.genp_update("df64tc", Ad, Bd, Cd, status, work)
    torch.cuda.synchronize()
    assert int(status.item()) == -1
    got = from_df64(Cd)
    S = np.abs(Av) @ np.abs(Bv)
    assert np.abs(got - (Cv - Av @ Bv)).max() <= 2.0 ** -40 * (S.max() + np.abs(Cv).max())


def test_df64tc_solve_reports_update_timeout_then_recovers(stall):
    n = 600                                 # two 512-column panels: inner and outer sliced updates
    A = inputs.gaussian(n, seed=11)
    B = inputs.rhs(n, 1, seed=12)
    Ad, Bd = _lib.to_device(A), _lib.to_device(B)
    opts = _lib.make_opts(depth=2, seed=1, prec="df64tc", fallback=True)
    work = torch.empty(_lib.rbt_solve_workspace(opts, n, 1), dtype=torch.uint8, device="cuda")
    stall("oz_copy")
    t0 = time.perf_counter()
    code, _ = _lib.rbt_solve(opts, n, Ad, Bd, _lib.colmajor(n, 1), work, ok=(_lib.RBT_ERR_TIMEOUT,))
    assert code == _lib.RBT_ERR_TIMEOUT
    assert time.perf_counter() - t0 < BOUND_S
    stall("none")
    X, info = solve(Ad, Bd, depth=2, seed=1, prec="df64tc", fallback=True)
    assert info["code"] == _lib.RBT_OK and info["berr"] <= 1e-13 and info["fell_back"] == 0
    assert _berr(A, _lib.to_host(X), B) <= 1e-13
