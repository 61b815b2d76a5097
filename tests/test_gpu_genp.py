"""GPU parity of GENP (factor and triangular solves) and of the residual.

Criterion for the factors (rigorous, any summation order): the computed
factors of GENP satisfy L U = A + E with |E| <= gamma_n |L| |U| elementwise
(Higham, Thm. 9.3), gamma_n = n u / (1 - n u).  The check forms L U in
numpy, which adds at most another gamma_n |L||U|, hence the factor 2.  The
factors are also compared with the oracle's normwise, as a guard against a
result that is a valid factorization of the wrong matrix.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2312_09376_gb300 import _lib, inputs
from tests import _bounds, _df64

pytestmark = pytest.mark.gpu


def _factor(A, prec, nb=0):
    """Factor the working copy of A in precision prec; returns (factors as float64 on the device, info)."""
    n = A.shape[0]
    if prec == "df64":
        Ad = _lib.colmajor(n, n)
        if n > 0:
            _lib.rbt_apply_2sided_wp(n, 0, _lib.colmajor(n, 1), _lib.colmajor(n, 1), _lib.to_device(A), Ad, "df64")
    else:
        dt = torch.float64 if prec == "f64" else torch.float32
        Ad = _lib.to_device(A).to(dt)
    info = torch.empty(1, dtype=torch.int64, device="cuda")
    ws = _lib.genp_factor_workspace(n, prec, nb)
    work = torch.empty(max(ws, 1), dtype=torch.uint8, device="cuda")
    _lib.genp_factor(n, prec, Ad, info, work, nb)
    torch.cuda.synchronize()
    if prec == "df64":
        Ad = _lib.df64_to_double(Ad)
    return Ad, int(info.item())


def _check_lu(A, LU, u):
    n = A.shape[0]
    L = np.tril(LU, -1) + np.eye(n)
    U = np.triu(LU)
    E = np.abs(A - L @ U)
    B = np.abs(L) @ np.abs(U)
    assert np.all(E <= 2 * _bounds.gamma(n, u) * B), float((E / np.maximum(B, 1e-300)).max() / u)


def _rbt_matrix(n, d=2, seed=1, a_seed=42):
    A = inputs.gaussian(n, seed=a_seed)
    U, V = oracle.generate(n, d, seed)
    return oracle.transform_2sided(A, U, V, d)


SIZES = [1, 2, 3, 17, 63, 64, 65, 127, 128, 129, 300, 1003]


@pytest.mark.parametrize("n", SIZES)
def test_genp_f64_parity(n):
    At = _rbt_matrix(n)
    LUd, st = _factor(At, "f64")
    assert st == -1
    LU = _lib.to_host(LUd)
    _check_lu(At, LU, _bounds.U64)
    LUo, sto = oracle.genp(At)
    assert sto == -1
    assert np.abs(LU - LUo).max() <= 1e-8 * np.abs(LUo).max()


@pytest.mark.parametrize("n,nb", [(1003, 16), (1003, 128), (257, 32), (500, 100)])
def test_genp_f64_block_sizes(n, nb):
    At = _rbt_matrix(n, seed=3)
    LUd, st = _factor(At, "f64", nb)
    assert st == -1
    _check_lu(At, _lib.to_host(LUd), _bounds.U64)


@pytest.mark.parametrize("n", [1, 5, 64, 129, 1003])
def test_genp_f32_parity(n):
    At = _rbt_matrix(n).astype(np.float32).astype(np.float64)   # the float working copy, exactly
    LUd, st = _factor(At, "f32")
    assert st == -1
    _check_lu(At, _lib.to_host(LUd).astype(np.float64), _bounds.U32)


U_DF64 = 2.0 ** -44   # per-operation relative error of the double-float kernels (Dekker/Knuth forms)


@pytest.mark.parametrize("n", [1, 5, 64, 129, 1003, 2500])   # 2500: trailing updates on 128 x 128 tiles
def test_genp_df64_parity(n):
    At = _rbt_matrix(n)
    LUd, st = _factor(At, "df64")
    assert st == -1
    LU = _lib.to_host(LUd)
    _check_lu(At, LU, U_DF64)
    LUo, _ = oracle.genp(At)
    if n <= 1024:
        assert np.abs(LU - LUo).max() <= 1e-6 * np.abs(LUo).max()
    else:
        # Without pivoting the factors of a large matrix differ from the
        # double ones by the working precision times the elimination's
        # growth (max |U| is about 1e5 here), so the whole-factor comparison
        # is left to the backward-error bound above.  The first four block
        # columns of L and block rows of U (three trailing updates on the
        # 128 x 128 tiles) still match the oracle to 1e-5 of their largest
        # entry: perturbing A alone by 6e-14 moves them by 4.5e-10, the
        # double-float roundings along the way by a few hundred times that,
        # while a wrong index or tile offset shows as an O(1) difference.
        w = 256
        for got, ref in ((LU[:, :w], LUo[:, :w]), (LU[:w, :], LUo[:w, :])):
            assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()


def test_genp_reports_zero_and_nonfinite_pivots():
    n = 300
    A = inputs.zero_corner(inputs.gaussian(n))
    _, st = _factor(A, "f64")
    assert st == 0
    _, st = _factor(A, "f32")
    assert st == 0
    _, st = _factor(A, "df64")
    assert st == 0
    B = inputs.gaussian(n, seed=3)
    B[:, 200] = np.nan                       # pivot 200 becomes NaN first
    _, st = _factor(B, "f64")
    assert st == 200
    # singular leading minor deep inside a later block: pivot 150 exactly zero
    L = np.tril(np.random.default_rng(1).standard_normal((n, n)) * 0.01, -1) + np.eye(n)
    Uu = np.triu(np.random.default_rng(2).standard_normal((n, n)) * 0.01, 1) + np.eye(n)
    Uu[150, 150] = 0.0
    Uu[150, 151:] = 0.0
    M = L @ Uu
    _, sto = oracle.genp(M)
    _, st = _factor(M, "f64")
    assert st == sto


def _solve_bound_ok(LU, X, B, trans, u, c=4):
    """|B - op(L U) X| <= c gamma_3n op(|L| |U|) |X|: a forward and a back
    substitution with the given factors, each backward stable (Higham, Thm.
    8.5), the factors taken as exact."""
    n = LU.shape[0]
    L = np.tril(LU, -1) + np.eye(n)
    Uu = np.triu(LU)
    M = L @ Uu
    absM = np.abs(L) @ np.abs(Uu)
    if trans:
        M, absM = M.T, absM.T
    R = np.abs(B - M @ X)
    bound = c * _bounds.gamma(3 * n, u) * (absM @ np.abs(X))
    return bool(np.all(R <= bound)), float((R / np.maximum(absM @ np.abs(X), 1e-300)).max() / u)


@pytest.mark.parametrize("n,nrhs", [(1, 1), (7, 3), (129, 1), (1003, 1), (1003, 8), (2000, 32)])
@pytest.mark.parametrize("trans", [False, True])
def test_genp_solve_f64(n, nrhs, trans):
    """Solves with the oracle's factors (uploaded): the device result meets
    the substitution bound in double and matches the oracle's substitution."""
    LU, st = oracle.genp(_rbt_matrix(n, seed=5))
    assert st == -1
    B = inputs.rhs(n, nrhs)
    Bd = _lib.to_device(B)
    work = torch.empty(_lib.genp_solve_workspace(n, nrhs, "f64"), dtype=torch.uint8, device="cuda")
    _lib.genp_solve(n, "f64", _lib.to_device(LU), trans, Bd, work)
    torch.cuda.synchronize()
    X = _lib.to_host(Bd)
    ok, ratio = _solve_bound_ok(LU, X, B, trans, _bounds.U64)
    assert ok, ratio
    Xo = oracle.genp_solve(LU, B, trans=trans)
    assert np.abs(X - Xo).max() <= 1e-9 * np.abs(Xo).max()


@pytest.mark.parametrize("n,nrhs", [(1003, 5), (1003, 40), (130, 33), (1003, 1)])
@pytest.mark.parametrize("trans", [False, True])
@pytest.mark.parametrize("prec", ["df64", "f32"])
def test_genp_solve_many_rhs(prec, n, nrhs, trans):
    """Low-precision factors (the oracle's, rounded to float or split into
    float pairs, uploaded).  Many right-hand sides take the blocked solve
    (inverse of each diagonal block plus one correction step, then one wide
    update per block), one the chained solve; both meet the substitution
    bound in the working precision, and match the oracle's double
    substitution with the same factors to that precision times the
    triangles' conditioning."""
    LU, st = oracle.genp(_rbt_matrix(n, seed=6))
    assert st == -1
    if prec == "f32":
        LU = LU.astype(np.float32).astype(np.float64)
        LUd = _lib.to_device(LU).to(torch.float32)
    else:
        LUd, LU = _df64.to_df64(LU)
    B = inputs.rhs(n, nrhs)
    Bd = _lib.to_device(B)
    work = torch.empty(_lib.genp_solve_workspace(n, nrhs, prec), dtype=torch.uint8, device="cuda")
    _lib.genp_solve(n, prec, LUd, trans, Bd, work)
    torch.cuda.synchronize()
    X = _lib.to_host(Bd)
    u = U_DF64 if prec == "df64" else _bounds.U32
    ok, ratio = _solve_bound_ok(LU, X, B, trans, u, c=8)
    assert ok, ratio
    Xo = oracle.genp_solve(LU, B, trans=trans)
    assert np.abs(X - Xo).max() <= (1e-6 if prec == "df64" else 1e-1) * np.abs(Xo).max()


@pytest.mark.parametrize("n,nrhs", [(1, 1), (129, 2), (1003, 1), (3001, 4)])
def test_residual_and_backward_error(n, nrhs):
    A = inputs.gaussian(n)
    X = inputs.rhs(n, nrhs, seed=3)
    B = inputs.rhs(n, nrhs, seed=64)
    Ad, Xd, Bd = _lib.to_device(A), _lib.to_device(X), _lib.to_device(B)
    Rd = _lib.colmajor(n, nrhs)
    berr = torch.zeros(1, dtype=torch.float64, device="cuda")
    work = torch.empty(_lib.rbt_residual_workspace(n, nrhs), dtype=torch.uint8, device="cuda")
    _lib.rbt_residual(n, Ad, Xd, Bd, Rd, d_berr=berr, work=work)
    torch.cuda.synchronize()
    Ro = oracle.residual(A, X, B)
    scale = np.abs(A) @ np.abs(X) + np.abs(B)
    assert np.all(np.abs(_lib.to_host(Rd) - Ro) <= 2 * _bounds.gamma(n + 1, _bounds.U64) * scale)
    bo = oracle.backward_error(A, X, B)
    assert abs(float(berr.item()) - bo) <= 1e-10 * bo
    an = torch.zeros(1, dtype=torch.float64, device="cuda")
    _lib.rbt_norm_inf(n, Ad, an, work)
    torch.cuda.synchronize()
    assert abs(float(an.item()) - oracle.norm_inf_mat(A)) <= 2 * _bounds.gamma(n, _bounds.U64) * oracle.norm_inf_mat(A)


@pytest.mark.parametrize("prec", ["f64", "f32", "df64"])
def test_chained_solve_bitwise_reproducible(prec):
    """The chained solves' summation order does not depend on which earlier
    blocks had finished when a block read them: repeated solves with the same
    factors agree bit for bit (both triangles, both orientations), and so do
    repeated full solves."""
    n = 6000
    rng = np.random.default_rng(7)               # well-conditioned triangles, built directly
    LU = np.tril(0.01 * rng.standard_normal((n, n)), -1) + np.triu(0.01 * rng.standard_normal((n, n)), 1)
    LU[np.arange(n), np.arange(n)] = 1.0 + np.abs(rng.standard_normal(n))
    if prec == "f32":
        LUd = _lib.to_device(LU).to(torch.float32)
    elif prec == "df64":
        LUd, _ = _df64.to_df64(LU)
    else:
        LUd = _lib.to_device(LU)
    work = torch.empty(_lib.genp_solve_workspace(n, 2, prec), dtype=torch.uint8, device="cuda")
    for nrhs in (1, 2):                          # the one-column kernel and the multi-column one
        B = inputs.rhs(n, nrhs, seed=3)
        for trans in (False, True):
            outs = []
            for _ in range(4):
                Bd = _lib.to_device(B)
                _lib.genp_solve(n, prec, LUd, trans, Bd, work)
                torch.cuda.synchronize()
                outs.append(_lib.to_host(Bd))
            for o in outs[1:]:
                assert np.array_equal(o, outs[0])
    A = inputs.gaussian(3001, seed=9)
    b = inputs.rhs(3001, 1)
    from paper_2312_09376_gb300 import solve
    xs = [_lib.to_host(solve(_lib.to_device(A), _lib.to_device(b), depth=2, prec="f64" if prec == "f64" else "df64tc",
                             refine_max=0, fallback=False)[0]) for _ in range(3)]
    assert np.array_equal(xs[0], xs[1]) and np.array_equal(xs[0], xs[2])
