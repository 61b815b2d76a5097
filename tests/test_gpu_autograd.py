"""Hand-written adjoint of X = solve(A, B) against finite differences and
against the oracle's gradient (grad_B = A^{-T} grad_X, grad_A = -grad_B X^T
computed from the oracle's own solves)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2312_09376_gb300 import _lib, inputs
from paper_2312_09376_gb300.autograd import solve, solve_batched, solve_batched_backward

pytestmark = pytest.mark.gpu


def _oracle_grads(A, B, W):
    """Loss L = sum(W * X), X = A^{-1} B: grad_X = W, grad_B = A^{-T} W (oracle
    GENP solve of A^T after its RBT: solve (A^T) with the oracle), grad_A = -grad_B X^T."""
    X, st, _, _, _ = oracle.rbt_solve(A, B, 2, seed=1, refine_max=30, tol=1e-15)
    gB, st2, _, _, _ = oracle.rbt_solve(np.asfortranarray(A.T), W, 2, seed=2, refine_max=30, tol=1e-15)
    assert st == -1 and st2 == -1
    return X, gB, -gB @ X.T


def test_finite_differences_n67():
    n, k = 67, 3
    A = inputs.gaussian(n, seed=3)
    B = inputs.rhs(n, k, seed=4)
    W = inputs.rhs(n, k, seed=5)
    Ad = _lib.to_device(A).requires_grad_(True)
    Bd = _lib.to_device(B).requires_grad_(True)
    Wd = _lib.to_device(W)
    X = solve(Ad, Bd, depth=2, prec="f64")
    (X * Wd).sum().backward()
    gA, gB = _lib.to_host(Ad.grad), _lib.to_host(Bd.grad)
    rng = np.random.default_rng(0)
    h = 1e-6
    for _ in range(12):
        i, j = rng.integers(0, n, 2)
        Ap, Am = A.copy(), A.copy()
        Ap[i, j] += h
        Am[i, j] -= h
        Lp = (oracle.rbt_solve(Ap, B, 2, 1, 30, 1e-15)[0] * W).sum()
        Lm = (oracle.rbt_solve(Am, B, 2, 1, 30, 1e-15)[0] * W).sum()
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - gA[i, j]) <= 1e-6 * max(1.0, abs(fd)), (i, j, fd, gA[i, j])
    for _ in range(6):
        i, c = rng.integers(0, n), rng.integers(0, k)
        Bp, Bm = B.copy(), B.copy()
        Bp[i, c] += h
        Bm[i, c] -= h
        fd = ((oracle.rbt_solve(A, Bp, 2, 1, 30, 1e-15)[0] - oracle.rbt_solve(A, Bm, 2, 1, 30, 1e-15)[0]) * W).sum() / (2 * h)
        assert abs(fd - gB[i, c]) <= 1e-6 * max(1.0, abs(fd))


@pytest.mark.parametrize("prec", ["f64", "df64", "df64tc", "df64tc7", "f32"])
def test_gradients_match_oracle(prec):
    n, k = 1200, 8
    A = inputs.gaussian(n, seed=6)
    B = inputs.rhs(n, k, seed=7)
    W = inputs.rhs(n, k, seed=8)
    Ad = _lib.to_device(A).requires_grad_(True)
    Bd = _lib.to_device(B).requires_grad_(True)
    X = solve(Ad, Bd, depth=2, prec=prec, fallback=True)
    (X * _lib.to_device(W)).sum().backward()
    Xo, gBo, gAo = _oracle_grads(A, B, W)
    kappa = np.linalg.cond(A, np.inf)
    tol = 100 * n * kappa * 2.2e-16
    assert np.abs(_lib.to_host(X.detach()) - Xo).max() <= tol * np.abs(Xo).max()
    assert np.abs(_lib.to_host(Bd.grad) - gBo).max() <= tol * np.abs(gBo).max()
    assert np.abs(_lib.to_host(Ad.grad) - gAo).max() <= tol * np.abs(gAo).max()


def test_adjoint_backward_error():
    """grad_B solves A^T y = w to the refinement tolerance."""
    n = 8197
    g = torch.Generator(device="cuda").manual_seed(9)
    A = torch.randn((n, n), generator=g, device="cuda", dtype=torch.float64).T.requires_grad_(True)
    B = torch.randn((32, n), generator=g, device="cuda", dtype=torch.float64).T.requires_grad_(True)
    W = torch.randn((32, n), generator=g, device="cuda", dtype=torch.float64).T
    X = solve(A, B, depth=2, prec="df64")
    (X * W).sum().backward()
    Y = B.grad
    R = W - A.detach().T @ Y        # check only (torch GEMM on the test side)
    berr = R.abs().max(0).values / (A.detach().abs().sum(0).max() * Y.abs().max(0).values + W.abs().max(0).values)
    assert float(berr.max()) <= 1e-13
    # grad_A = -grad_B X^T on a sample of entries
    rng = np.random.default_rng(1)
    idx = rng.integers(0, n, (50, 2))
    for i, j in idx:
        want = -(Y[i] * X.detach()[j]).sum()
        assert abs(float(A.grad[i, j] - want)) <= 1e-12 * (Y[i].abs() * X.detach()[j].abs()).sum().item()


def test_batched_backward_matches_per_system():
    ns = inputs.batch_sizes(256, 32, 256, seed=21)
    As = [inputs.gaussian(int(n), seed=100 + i) for i, n in enumerate(ns)]
    Bs = [inputs.rhs(int(n), 2, seed=300 + i) for i, n in enumerate(ns)]
    Ws = [inputs.rhs(int(n), 2, seed=500 + i) for i, n in enumerate(ns)]
    Ad = [_lib.to_device(a) for a in As]
    Bd = [_lib.to_device(b) for b in Bs]
    Xs, plan = solve_batched(Ad, Bd, prec="f32", seeds=[1000 + i for i in range(len(ns))])
    Ys, GAs = solve_batched_backward(plan, [_lib.to_device(w) for w in Ws])
    torch.cuda.synchronize()
    infos = plan.infos_host()
    assert np.all(infos["status"] == 0)
    for i in np.random.default_rng(2).choice(len(ns), 10, replace=False):
        A, W = As[i], Ws[i]
        Y = _lib.to_host(Ys[i])
        # adjoint backward error of A^T y = w
        R = W - A.T @ Y
        berr = (np.abs(R).max(0) / (np.abs(A).sum(0).max() * np.abs(Y).max(0) + np.abs(W).max(0))).max()
        assert berr <= 1e-13
        X = _lib.to_host(Xs[i])
        assert np.allclose(_lib.to_host(GAs[i]), -Y @ X.T, rtol=1e-12, atol=1e-12 * np.abs(Y).max() * np.abs(X).max())
