"""GPU parity of the rotation-form butterflies (the block-rotation variant of
Sec. 3: [[C, 0, S], [0, I, 0], [S, 0, -C]] blocks, R_k = I) against the
oracle: generator, two-sided transform in every working precision, one-sided
transforms, the full solve and its adjoint.

Tolerances (derived as for the scaled form): a rotated pair costs two
products and a sum per layer and side, each relative to the entry's share of
(|U|^T |A| |V|)_ij; in double 1e-14 of that scale (about 90 u) covers the
6 d roundings of a path for d <= 5; the float copy 64 float ulps; the
double-float copy (7 d + 1) 2^-46.  For n <= 1100 the scale is formed from the
dense rotation butterflies; above, through the group-sum bound (every entry
of |U| is at most 1 here)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2312_09376_gb300 import _lib, inputs, solve
from paper_2312_09376_gb300 import autograd as ag
from tests import _bounds
from tests import _explicit as ex

pytestmark = pytest.mark.gpu

REL = 1e-14


def _coefs(n, d, seed, align=1):
    """The oracle's rotation coefficients, host and uploaded."""
    U, V = oracle.generate_rot(n, d, seed, align=align)
    return U, V, _lib.to_device(U), _lib.to_device(V)


def _scale(A, U, V, d, align):
    n = A.shape[0]
    if n <= 1100:
        Ua = np.abs(ex.dense_rot_rbt(n, d, U, align))
        Va = np.abs(ex.dense_rot_rbt(n, d, V, align))
        return Ua.T @ np.abs(A) @ Va
    return _bounds.group_bound(A, d)


@pytest.mark.parametrize("n,d,align,seed", [(1, 1, 1, 0), (7, 3, 1, 5), (67, 4, 3, 2), (1003, 2, 64, 1),
                                            (20001, 3, 1, 1), (40003, 2, 1, 99)])
def test_rot_generator_matches_oracle(n, d, align, seed):
    U = _lib.colmajor(n, d)
    V = _lib.colmajor(n, d)
    _lib.rbt_generate_rot(n, d, align, seed, U, V)
    torch.cuda.synchronize()
    Uo, Vo = oracle.generate_rot(n, d, seed, align=align)
    for g, o in ((U, Uo), (V, Vo)):
        g = _lib.to_host(g)
        # the same angle on both sides; cos and sin of libm and of CUDA may
        # differ by an ulp of values at most 1
        assert np.all(np.abs(g - o) <= 4 * 2.0 ** -53), np.abs(g - o).max()
        assert np.array_equal(g == 1.0, o == 1.0)


SMALL = [(n, d, a) for n in (1, 2, 3, 5, 8, 17, 31, 64, 67, 100, 251) for d in (1, 2, 3, 4, 5) for a in (1, 8)]


@pytest.mark.parametrize("n,d,align", SMALL)
def test_rot_transform_small(n, d, align):
    A = inputs.gaussian(n, seed=n * 10 + d)
    U, V, Ud, Vd = _coefs(n, d, 3, align)
    out = _lib.colmajor(n, n)
    _lib.rbt_transform_2sided(n, d, align, "rotation", "f64", Ud, Vd, _lib.to_device(A), out)
    torch.cuda.synchronize()
    want = oracle.transform_2sided_rot(A, U, V, d, align=align)
    err = np.abs(_lib.to_host(out) - want)
    scale = _scale(A, U, V, d, align)
    assert np.all(err <= REL * scale), float((err / np.maximum(scale, 1e-300)).max())


@pytest.mark.parametrize("n,d", [(1003, 2), (2048, 3), (4099, 7)])
def test_rot_transform_in_place_and_multipass(n, d):
    """In place, and d_s > 3 (two passes over the matrix)."""
    A = inputs.gaussian(n, seed=4)
    U, V, Ud, Vd = _coefs(n, d, 8)
    Ad = _lib.to_device(A)
    _lib.rbt_transform_2sided(n, d, 1, "rotation", "f64", Ud, Vd, Ad, Ad)
    torch.cuda.synchronize()
    want = oracle.transform_2sided_rot(A, U, V, d)
    err = np.abs(_lib.to_host(Ad) - want)
    scale = _scale(A, U, V, d, 1)
    assert np.all(err <= REL * scale), float((err / np.maximum(scale, 1e-300)).max())


@pytest.mark.parametrize("n,d", [(1003, 2), (67, 3), (8197, 2)])
@pytest.mark.parametrize("prec", ["f32", "df64"])
def test_rot_working_copy(n, d, prec):
    A = inputs.gaussian(n, seed=5)
    U, V, Ud, Vd = _coefs(n, d, 1)
    dt = torch.float32 if prec == "f32" else torch.float64
    out = _lib.colmajor(n, n, dtype=dt, ld=n + 3)
    _lib.rbt_transform_2sided(n, d, 1, "rotation", prec, Ud, Vd, _lib.to_device(A), out)
    torch.cuda.synchronize()
    want = oracle.transform_2sided_rot(A, U, V, d)
    scale = _scale(A, U, V, d, 1)
    if prec == "f32":
        err = np.abs(_lib.to_host(out).astype(np.float64) - want)
        assert np.all(err <= 64 * 2.0 ** -24 * scale), float((err / scale).max() / 2.0 ** -24)
    else:
        err = np.abs(_lib.to_host(_lib.df64_to_double(out)) - want)
        assert np.all(err <= (7 * d + 1) * 2.0 ** -46 * scale), float((err / scale).max() / 2.0 ** -46)


@pytest.mark.parametrize("n,d,align,nrhs", [(1, 2, 1, 1), (1003, 2, 1, 3), (1003, 3, 64, 2), (20001, 3, 1, 1)])
def test_rot_vec_transforms(n, d, align, nrhs):
    B = inputs.rhs(n, nrhs)
    U, _, Ud, _ = _coefs(n, d, 4, align)
    for trans in (True, False):
        Bd = _lib.to_device(B)
        _lib.rbt_transform_vec(n, d, align, "rotation", Ud, trans, Bd)
        torch.cuda.synchronize()
        want = oracle.transform_vec_rot(B, U, d, trans, align=align)
        # |W| |b| <= (group sum of |b|) for coefficients at most 1
        scale = (2 ** min(d, 20)) * np.abs(B).max(axis=0)[None, :]
        assert np.all(np.abs(_lib.to_host(Bd) - want) <= REL * scale)


def test_rot_full_size_sampled_and_norm():
    """n = 40003, d = 2, the transform of the benchmark's size: sampled entries
    A~_ij = (U e_i)^T A (V e_j) with the oracle's columns of U and V, and the
    Frobenius norm, which an orthogonal transform keeps."""
    n, d = 40003, 2
    g = torch.Generator(device="cuda").manual_seed(42)
    Ad = torch.randn((n, n), generator=g, device="cuda", dtype=torch.float64).T
    norm_in = float(torch.linalg.norm(Ad))
    U, V, Ud, Vd = _coefs(n, d, 1)
    rng = np.random.default_rng(0)
    ii = rng.integers(0, n, 200)
    jj = rng.integers(0, n, 200)
    ii[:2] = [0, n - 1]
    jj[:2] = [n - 1, 0]

    def cols(W, idx):
        E = np.zeros((n, len(idx)))
        E[idx, np.arange(len(idx))] = 1.0
        return oracle.transform_vec_rot(E, W, d, False)

    Uc, Vc = cols(U, ii), cols(V, jj)
    rows = [np.nonzero(Uc[:, k])[0] for k in range(len(ii))]
    cs = [np.nonzero(Vc[:, k])[0] for k in range(len(jj))]
    blocks = [Ad[torch.as_tensor(rows[k], device="cuda")][:, torch.as_tensor(cs[k], device="cuda")].cpu().numpy()
              for k in range(len(ii))]
    out = _lib.colmajor(n, n)
    _lib.rbt_transform_2sided(n, d, 1, "rotation", "f64", Ud, Vd, Ad, out)
    torch.cuda.synchronize()
    got = out[torch.as_tensor(ii, device="cuda"), torch.as_tensor(jj, device="cuda")].cpu().numpy()
    for k in range(len(ii)):
        u, v = Uc[rows[k], k], Vc[cs[k], k]
        want = u @ blocks[k] @ v
        assert abs(got[k] - want) <= REL * (np.abs(u) @ np.abs(blocks[k]) @ np.abs(v)), (ii[k], jj[k])
    assert abs(float(torch.linalg.norm(out)) - norm_in) <= 1e-12 * norm_in


@pytest.mark.parametrize("prec", ["f64", "df64tc", "df64", "f32"])
@pytest.mark.parametrize("n", [301, 1003])
def test_rot_solve_matches_oracle(prec, n):
    A = inputs.gaussian(n, seed=12)
    A[0, 0] = 0.0                       # GENP without a transform stops at once
    B = inputs.rhs(n, 2)
    X, info = solve(_lib.to_device(A), _lib.to_device(B), depth=2, seed=3, prec=prec, kind="rotation")
    torch.cuda.synchronize()
    assert info["code"] == 0 and info["berr"] <= 1e-13, info
    assert _bounds.berr(A, _lib.to_host(X), B) <= 1e-13
    Xo, st, b0, bo, _ = oracle.rbt_solve(A, B, 2, seed=3, kind="rotation")
    assert st == -1 and bo <= 1e-13
    kappa = np.linalg.cond(A, np.inf)
    assert np.abs(_lib.to_host(X) - Xo).max() <= 100 * n * kappa * 2.0 ** -53 * np.abs(Xo).max()
    if prec == "f64":
        # the first solution: the same transform and GENP up to rounding order
        g = info["berr_unrefined"]
        assert g <= 10 * b0 + 1e-15 and b0 <= 10 * g + 1e-15


def test_rot_solve_tiled_and_gmres():
    n = 1003
    A = inputs.gaussian(n, seed=13)
    B = inputs.rhs(n, 1)
    for kw in ({"align": 64}, {"refine": "gmres", "prec": "f32"}):
        X, info = solve(_lib.to_device(A), _lib.to_device(B), depth=2, seed=2, kind="rotation", **kw)
        torch.cuda.synchronize()
        assert info["code"] == 0 and info["berr"] <= 1e-13, (kw, info)
        assert _bounds.berr(A, _lib.to_host(X), B) <= 1e-13


def test_rot_adjoint_matches_oracle_gradient():
    """grad_B = A^{-T} W and grad_A = -grad_B X^T through the rotation-form
    solver, against the oracle's solves of A and A^T (rotation form too)."""
    n, k = 257, 3
    A = inputs.gaussian(n, seed=21)
    B = inputs.rhs(n, k, seed=22)
    W = inputs.rhs(n, k, seed=23)
    Ad = _lib.to_device(A).requires_grad_(True)
    Bd = _lib.to_device(B).requires_grad_(True)
    X = ag.solve(Ad, Bd, depth=2, prec="f64", kind="rotation")
    (X * _lib.to_device(W)).sum().backward()
    Xo, st, _, _, _ = oracle.rbt_solve(A, B, 2, seed=1, kind="rotation", tol=1e-15)
    gB, st2, _, _, _ = oracle.rbt_solve(np.asfortranarray(A.T), W, 2, seed=2, kind="rotation", tol=1e-15)
    assert st == -1 and st2 == -1
    gA = -gB @ Xo.T
    kappa = np.linalg.cond(A, np.inf)
    tol = 100 * n * kappa * 2.0 ** -53
    assert np.abs(_lib.to_host(Bd.grad) - gB).max() <= tol * np.abs(gB).max()
    assert np.abs(_lib.to_host(Ad.grad) - gA).max() <= tol * np.abs(gA).max()


def test_rot_arguments_and_batched_unsupported():
    n = 16
    U, V = _lib.colmajor(n, 2), _lib.colmajor(n, 2)
    with pytest.raises(_lib.RbtError):
        _lib.rbt_generate_rot(n, 2, -1, 1, U, V)
    A = _lib.to_device(np.eye(n))
    with pytest.raises(_lib.RbtError):
        _lib.rbt_transform_2sided(n, 2, 1, 7, "f64", U, V, A, _lib.colmajor(n, n))
    with pytest.raises(_lib.RbtError):
        solve(A, _lib.to_device(np.ones((n, 1))), kind=5)
    opts = _lib.make_opts(depth=2, prec="f64", kind="rotation")
    with pytest.raises(_lib.RbtError):
        _lib.rbt_solve_batched_plan(opts, [A], [_lib.to_device(np.ones((n, 1)))], [_lib.colmajor(n, 1)])
