"""GMRES-based refinement on the GPU (restarted GMRES right preconditioned
by the transformed low-precision factors, the preconditioner applied in
double) against the oracle's GMRES-IR: both reach the double backward-error
target where stationary refinement with the same kind of factors does not."""
import numpy as np
import pytest
import torch

import oracle
from paper_2312_09376_gb300 import _lib, inputs, solve
from tests import _bounds, _df64

pytestmark = pytest.mark.gpu


def _oracle_float_factors(A, d, seed):
    """The oracle's butterflies and its GENP factors of U^T A V rounded to float (exact in double)."""
    U, V = oracle.generate(A.shape[0], d, seed)
    At = oracle.transform_2sided(A, U, V, d)
    LU, st = oracle.genp(At.astype(np.float32).astype(np.float64))
    assert st == -1
    return U, V, LU.astype(np.float32).astype(np.float64)


def _oracle_gmres(A, b, d, seed, restart=30, max_iter=300):
    """The oracle's GMRES-IR with its own float factors, from the double substitution's x0."""
    U, V, LU = _oracle_float_factors(A, d, seed)
    x0 = oracle.transform_vec(oracle.genp_solve(LU, oracle.transform_vec(b, U, d, True)), V, d, False)
    _, _, berr, used, _, _ = oracle.gmres_ir(A, b, U, V, d, LU, x0, restart=restart, max_iter=max_iter)
    return berr, used


@pytest.mark.parametrize("n,nrhs", [(1, 1), (129, 1), (1003, 1), (2000, 3)])
@pytest.mark.parametrize("trans", [False, True])
@pytest.mark.parametrize("prec", ["f32", "df64"])
def test_genp_solve_wp_parity(prec, n, nrhs, trans):
    """The working-precision solve with low-precision factors (the oracle's,
    rounded to float or split into float pairs, uploaded) is a double
    substitution with those factors (their entries are exact in double): its
    residual meets the double bound of a forward and a back substitution,
    |b - L U x| <= c gamma_3n |L| |U| |x| (Higham, Thm. 8.5, the factors
    taken as exact), which a float-arithmetic solve misses by a factor of
    2^29, and it matches the oracle's substitution with the same factors to
    the conditioning of those triangles."""
    U, V = oracle.generate(n, 2, 1)
    At = oracle.transform_2sided(inputs.gaussian(n, seed=31), U, V, 2)
    if prec == "f32":
        LU, st = oracle.genp(At.astype(np.float32).astype(np.float64))
        LU = LU.astype(np.float32).astype(np.float64)
        LUd = _lib.to_device(LU).to(torch.float32)
    else:
        LU, st = oracle.genp(At)
        LUd, LU = _df64.to_df64(LU)
    assert st == -1
    B = inputs.rhs(n, nrhs, seed=9)
    Bd = _lib.to_device(B)
    work = torch.empty(_lib.genp_solve_wp_workspace(n, nrhs), dtype=torch.uint8, device="cuda")
    _lib.genp_solve_wp(n, prec, LUd, trans, Bd, work)
    torch.cuda.synchronize()
    assert int(work[:4].view(torch.int32).item()) == 0
    X = _lib.to_host(Bd)
    L = np.tril(LU, -1) + np.eye(n)
    Uu = np.triu(LU)
    M = (L @ Uu).T if trans else L @ Uu
    absM = (np.abs(L) @ np.abs(Uu)).T if trans else np.abs(L) @ np.abs(Uu)
    R = np.abs(B - M @ X)
    assert np.all(R <= 4 * _bounds.gamma(3 * n, _bounds.U64) * (absM @ np.abs(X))), float(
        (R / np.maximum(absM @ np.abs(X), 1e-300)).max() / _bounds.U64)
    # two double substitutions in different orders differ by the triangles'
    # conditioning times u (1e-10 at n = 2000 here); a float solve, by 1e-4
    Xo = oracle.genp_solve(LU, B, trans=trans)
    assert np.abs(X - Xo).max() <= 1e-8 * np.abs(Xo).max()


def test_genp_solve_wp_arguments():
    LU = _lib.colmajor(8, 8)
    B = _lib.colmajor(8, 1)
    with pytest.raises(_lib.RbtError):   # workspace too short
        _lib.genp_solve_wp(8, "f64", LU, False, B, torch.empty(16, dtype=torch.uint8, device="cuda"))
    assert _lib.genp_solve_wp_workspace(0, 1) == 0
    assert _lib.genp_solve_wp_workspace(8, 0) == 0


def test_gmres_refinement_float_factors():
    """Float factors of the depth-2 transform at n = 4000 (GENP growth about
    1e5 on this matrix): stationary refinement stalls far above the target,
    GMRES reaches 1e-13 without the double fallback, in about as many
    preconditioned products as the oracle's GMRES-IR with its own float
    factors of the same transformed matrix."""
    n = 4000
    A = inputs.gaussian(n, seed=31)
    B = inputs.rhs(n, 1)
    Ad, Bd = _lib.to_device(A), _lib.to_device(B)
    X, info = solve(Ad, Bd, depth=2, seed=1, prec="f32", refine="gmres", restart=30, refine_max=10)
    torch.cuda.synchronize()
    print("gpu", info)
    assert info["code"] == 0 and info["berr"] <= 1e-13, info
    assert _bounds.berr(A, _lib.to_host(X), B) <= 1e-13
    assert info["fell_back"] == 0 and 0 < info["iters"] <= 120, info
    _, st_info = solve(Ad, Bd, depth=2, seed=1, prec="f32", refine_max=10, fallback=False)
    assert st_info["berr"] > 1e-13   # the stationary steps do not get there
    berr, used = _oracle_gmres(A, B[:, 0], 2, 1)
    print("oracle", berr, used)
    assert berr <= 1e-13
    assert info["iters"] <= 3 * used + 10, (info["iters"], used)


@pytest.mark.parametrize("prec,n", [("f32", 2000), ("tf32", 1003), ("bf16", 1003)])
def test_gmres_refinement_reaches_target(prec, n):
    """Factors whose first solution is too poor for GMRES(30) as well (TF32
    and BF16 updates; float factors of the n = 2000 matrix, whose float
    working copy leaves a backward error near 1e-2 even with double
    substitutions, the GENP growth being 2e4): GMRES stalls by the 10 %-per-
    cycle rule and the double fallback reaches the target."""
    A = inputs.gaussian(n, seed=31)
    B = inputs.rhs(n, 1)
    X, info = solve(_lib.to_device(A), _lib.to_device(B), depth=2, seed=1, prec=prec, refine="gmres", restart=30,
                    refine_max=10)
    torch.cuda.synchronize()
    print(prec, n, info)
    assert info["code"] == 0 and info["berr"] <= 1e-13, info
    assert _bounds.berr(A, _lib.to_host(X), B) <= 1e-13
    assert info["iters"] > 0


def test_gmres_refinement_several_rhs_and_double_path():
    n = 1003
    A = inputs.gaussian(n, seed=2)
    B = inputs.rhs(n, 3)
    for prec in ("f64", "df64tc", "f32"):
        X, info = solve(_lib.to_device(A), _lib.to_device(B), depth=2, prec=prec, refine="gmres")
        torch.cuda.synchronize()
        assert info["code"] == 0 and info["berr"] <= 1e-13, (prec, info)
        assert _bounds.berr(A, _lib.to_host(X), B) <= 1e-13


def test_gmres_matches_oracle_gmres_ir():
    """Float factors on both sides (each side's own, of the same transformed
    matrix): the oracle's GMRES-IR and the GPU's converge in a similar number
    of products."""
    n, d = 1003, 2
    A = inputs.gaussian(n, seed=4)
    b = inputs.rhs(n, 1)[:, 0]
    X, info = solve(_lib.to_device(A), _lib.to_device(b.reshape(-1, 1)), depth=d, seed=1, prec="f32",
                    refine="gmres", restart=30)
    torch.cuda.synchronize()
    assert info["code"] == 0 and info["fell_back"] == 0 and info["berr"] <= 1e-13
    berr, used = _oracle_gmres(A, b, d, 1)
    assert berr <= 1e-13
    assert info["iters"] <= 3 * used + 10


def test_gmres_argument_checks():
    with pytest.raises(_lib.RbtError):
        solve(_lib.to_device(np.eye(10)), _lib.to_device(np.ones((10, 1))), refine="gmres", restart=65)


def test_gmres_refinement_with_tiled_reference_size():
    """GMRES refinement on the tiled reference size (n_b = 64) with float
    factors: the target without the fallback."""
    n = 1003
    A = inputs.gaussian(n, seed=4)
    B = inputs.rhs(n, 2)
    X, info = solve(_lib.to_device(A), _lib.to_device(B), depth=2, seed=1, prec="f32", refine="gmres", align=64)
    torch.cuda.synchronize()
    assert info["code"] == 0 and info["berr"] <= 1e-13 and info["fell_back"] == 0, info
    assert _bounds.berr(A, _lib.to_host(X), B) <= 1e-13
