"""End-to-end RBT solves on the GPU against the oracle (Eq. precond with the
refinement of Sec. 5).  Pass criterion: backward error (Eq. inf-norm-backerr)
<= 1e-13 with refinement, as the oracle reaches; the solutions themselves are
compared with a condition-number-scaled bound (x is unique, its rounding is
not)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2312_09376_gb300 import _lib, inputs, solve
from tests import _bounds

pytestmark = pytest.mark.gpu


def _run(A, B, **kw):
    X, info = solve(_lib.to_device(A), _lib.to_device(B), **kw)
    torch.cuda.synchronize()
    return _lib.to_host(X), info


@pytest.mark.parametrize("n,d,nrhs", [(1, 2, 1), (2, 1, 1), (67, 2, 1), (1003, 2, 1), (1003, 1, 3), (1003, 3, 1),
                                      (2048, 2, 8)])
def test_solve_f64_matches_oracle(n, d, nrhs):
    A = inputs.gaussian(n)
    B = inputs.rhs(n, nrhs)
    X, info = _run(A, B, depth=d, seed=1, prec="f64", refine_max=10, tol=1e-13)
    assert info["code"] == 0 and info["status"] == 0
    berr = _bounds.berr(A, X, B)
    assert berr <= 1e-13 and info["berr"] <= 1e-13
    # two evaluations of a residual at rounding level agree to within a few ulps of |A||x|
    assert abs(berr - info["berr"]) <= 8 * n * 2.2e-16
    Xo, st, b0, bo, it = oracle.rbt_solve(A, B, d, seed=1, refine_max=10, tol=1e-13)
    assert st == -1 and bo <= 1e-13
    kappa = np.linalg.cond(A, np.inf) if n <= 2048 else 1e8
    assert np.abs(X - Xo).max() <= 100 * n * kappa * 2.2e-16 * np.abs(Xo).max()


def test_solve_config1_unrefined_matches_oracle_scale():
    n, d = 1003, 2
    A = inputs.gaussian(n)
    B = inputs.rhs(n, 1)
    X, info = _run(A, B, depth=d, seed=1, prec="f64", refine_max=0, tol=0.0)
    Xo, st, b0, bo, it = oracle.rbt_solve(A, B, d, seed=1, refine_max=0, tol=0.0)
    # same factorization up to rounding: unrefined backward errors of one order
    assert info["berr_unrefined"] <= 10 * b0 + 1e-15 and b0 <= 10 * info["berr_unrefined"] + 1e-15


def test_zero_corner_needs_the_transform():
    n = 1003
    A = inputs.zero_corner(inputs.gaussian(n))
    B = inputs.rhs(n, 1)
    X, info = _run(A, B, depth=0, prec="f64")
    assert info["code"] == 1 and info["zero_pivot"] == 0
    X, info = _run(A, B, depth=2, prec="f64")
    assert info["code"] == 0 and _bounds.berr(A, X, B) <= 1e-13


def test_nonfinite_input_reports():
    n = 100
    A = inputs.gaussian(n)
    A[3, 3] = np.inf
    X, info = _run(A, inputs.rhs(n, 1), depth=0, prec="f64")
    assert info["code"] == 2 and info["zero_pivot"] == 3


def test_theorem3_full_depth_on_gpu():
    """Permutation-like matrices that defeat plain GENP are solved at full depth."""
    for n in (5, 8, 11, 16):
        d = int(np.ceil(np.log2(n))) + 1
        A = np.fliplr(np.eye(n))
        B = inputs.rhs(n, 1)
        X, info = _run(A, B, depth=d, prec="f64", refine_max=5)
        assert info["code"] == 0
        # a backward-stable solve: normwise backward error O(n u), u = 2^-53
        assert _bounds.berr(A, X, B) <= 2 * n * 2.0 ** -53


def test_solve_f32_refined_to_double():
    n = 1003
    A = inputs.gaussian(n)
    B = inputs.rhs(n, 2)
    X, info = _run(A, B, depth=2, prec="f32", refine_max=30, tol=1e-13, fallback=False)
    assert info["code"] == 0 and info["fell_back"] == 0
    assert _bounds.berr(A, X, B) <= 1e-13


def test_solve_f32_slow_refinement_falls_back():
    """At n = 4000 the float factors of RBT+GENP refine slowly (growth after a
    depth-2 transform times the float unit roundoff is close to one); given two
    steps the float attempt misses the tolerance, and the double factorization
    of the same A~ then reaches it."""
    n = 4000
    A = inputs.gaussian(n)
    B = inputs.rhs(n, 1)
    X, info = _run(A, B, depth=2, prec="f32", refine_max=2, tol=1e-13, fallback=False)
    assert info["code"] == 3 and info["fell_back"] == 0
    X, info = _run(A, B, depth=2, prec="f32", refine_max=2, tol=1e-13, fallback=True)
    assert info["code"] == 0 and info["fell_back"] == 1
    assert _bounds.berr(A, X, B) <= 1e-13


@pytest.mark.parametrize("n,d,nrhs", [(67, 2, 1), (1003, 2, 1), (4000, 2, 3)])
def test_solve_df64_refined_to_double(n, d, nrhs):
    A, _, _ = inputs.scaled_gaussian(n)
    B = inputs.rhs(n, nrhs)
    X, info = _run(A, B, depth=d, prec="df64", refine_max=30, tol=1e-13, fallback=False)
    assert info["code"] == 0 and info["fell_back"] == 0
    assert _bounds.berr(A, X, B) <= 1e-13


def test_f32_fallback_when_refinement_is_forbidden_to_converge():
    """refine_max = 0 on the low-precision path: the stall rule hands over to
    the double refactorization, which then reaches the tolerance."""
    n = 500
    A = inputs.gaussian(n)
    B = inputs.rhs(n, 1)
    X, info = _run(A, B, depth=2, prec="f32", refine_max=0, tol=1e-13, fallback=True)
    assert info["fell_back"] == 1
    assert _bounds.berr(A, X, B) <= 1e-13 or info["code"] == 3


def test_empty_system():
    X, info = solve(torch.zeros((0, 0), dtype=torch.float64, device="cuda"),
                    torch.zeros(0, dtype=torch.float64, device="cuda"))
    assert info["code"] == 0


def _host_colmajor(a, pinned, ld=None):
    """A column-major float64 CPU tensor holding a (rows x cols), leading dimension ld."""
    rows, cols = a.shape
    ld = ld or rows
    buf = torch.empty((cols, ld), dtype=torch.float64, pin_memory=pinned)
    buf[:, :rows] = torch.from_numpy(np.ascontiguousarray(a.T))
    return buf.T[:rows]


@pytest.mark.parametrize("pinned,pad", [(True, 0), (True, 5), (False, 0)])
def test_solve_host_matches_device_solve(pinned, pad):
    """rbt_solve_host (A, B, X in host memory: SM-driven copies of pinned
    memory, contiguous or with a padded leading dimension, and the copy-engine
    path for pageable memory) returns bit for bit the X of rbt_solve on device
    copies of the same inputs."""
    n, nrhs = 1003, 2
    A = inputs.scaled_gaussian(n)[0]
    B = inputs.rhs(n, nrhs)
    opts = _lib.make_opts(depth=2, seed=1, prec="df64tc7", refine_max=30, tol=1e-13, fallback=True)
    Xd = _lib.colmajor(n, nrhs)
    work = torch.empty(_lib.rbt_solve_workspace(opts, n, nrhs), dtype=torch.uint8, device="cuda")
    code_d, info_d = _lib.rbt_solve(opts, n, _lib.to_device(A), _lib.to_device(B), Xd, work)
    torch.cuda.synchronize()
    Ah = _host_colmajor(A, pinned, n + pad)
    Bh = _host_colmajor(B, pinned, n + pad)
    Xh = _host_colmajor(np.full((n, nrhs), np.nan), pinned, n + pad)
    hwork = torch.empty(_lib.rbt_solve_host_workspace(opts, n, nrhs), dtype=torch.uint8, device="cuda")
    code_h, info_h = _lib.rbt_solve_host(opts, n, Ah, Bh, Xh, hwork)
    assert code_h == code_d == 0
    assert info_h["iters"] == info_d["iters"] and info_h["berr"] == info_d["berr"]
    assert torch.equal(Xh.contiguous(), Xd.cpu().contiguous())
    assert _bounds.berr(A, Xh.numpy(), B) <= 1e-13
