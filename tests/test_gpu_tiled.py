"""GPU parity of the tiled reference size (Sec. 3, Algorithm 1: m chosen so
that every butterfly is aligned to n_b-row tiles) against the oracle's tiled
transforms and solve.  Tolerances as for the non-tiled transforms: relative
1e-14 of (|U|^T |A| |V|)_ij for the double transform (about 90 u for at most
4 d roundings per path), with the explicit tiled butterfly matrices giving
|U| and |V|; solves by the backward-error bound."""
import numpy as np
import pytest
import torch

import oracle
from paper_2312_09376_gb300 import _lib, inputs, solve
from tests import _bounds
from tests import _explicit as ex

pytestmark = pytest.mark.gpu

REL = 1e-14


def _gen(n, d, seed):
    """The oracle's butterflies for (n, d, seed), uploaded: the device
    transform and the oracle transform the same inputs (the device generator
    has its own parity test)."""
    U, V = oracle.generate(n, d, seed)
    return _lib.to_device(U), _lib.to_device(V)


@pytest.mark.parametrize("n,d,nb", [(13, 2, 3), (67, 3, 5), (257, 3, 8), (1003, 2, 64), (1003, 1, 100)])
def test_tiled_transform_matches_oracle(n, d, nb):
    A = inputs.gaussian(n, seed=n + nb)
    Ud, Vd = _gen(n, d, seed=5)
    U, V = _lib.to_host(Ud), _lib.to_host(Vd)
    out = _lib.colmajor(n, n)
    _lib.rbt_apply_2sided_tiled(n, d, nb, Ud, Vd, _lib.to_device(A), out)
    torch.cuda.synchronize()
    want = oracle.transform_2sided(A, U, V, d, align=nb)
    scale = np.abs(ex.dense_rbt(n, d, U, align=nb).T) @ np.abs(A) @ np.abs(ex.dense_rbt(n, d, V, align=nb))
    err = np.abs(_lib.to_host(out) - want)
    assert np.all(err <= REL * scale), float((err / scale).max())
    # the tiled transform differs from the non-tiled one unless 2^d n_b divides n
    if n % (2 ** oracle.depth_eff(n, d) * nb):
        plain = oracle.transform_2sided(A, U, V, d)
        assert np.abs(plain - want).max() > 1e-3 * np.abs(want).max()


@pytest.mark.parametrize("n,d,nb,nrhs", [(1003, 2, 64, 3), (20001, 3, 512, 1)])
def test_tiled_vec_transforms(n, d, nb, nrhs):
    B = inputs.rhs(n, nrhs)
    Ud, _ = _gen(n, d, seed=4)
    U = _lib.to_host(Ud)
    for trans in (True, False):
        Bd = _lib.to_device(B)
        _lib.rbt_apply_vec_tiled(n, d, nb, Ud, trans, Bd)
        torch.cuda.synchronize()
        want = oracle.transform_vec(B, U, d, trans=trans, align=nb)
        scale = np.exp(d / 20) * (2 ** d) * np.abs(B).max(axis=0)[None, :]
        assert np.all(np.abs(_lib.to_host(Bd) - want) <= REL * scale)


@pytest.mark.parametrize("prec", ["f64", "df64tc", "df64", "f32"])
def test_tiled_solve(prec):
    """A tiled solve (its working copy in every precision follows the tiled
    layout) meets the backward-error bound, as the oracle's does."""
    n, d, nb = 1003, 2, 64
    A = inputs.gaussian(n, seed=17)
    B = inputs.rhs(n, 2)
    X, info = solve(_lib.to_device(A), _lib.to_device(B), depth=d, seed=1, prec=prec, align=nb)
    torch.cuda.synchronize()
    assert info["code"] == 0 and info["berr"] <= 1e-13, info
    assert _bounds.berr(A, _lib.to_host(X), B) <= 1e-13
    _, st, b0, berr, _ = oracle.rbt_solve(A, B, d, 1, align=nb)
    assert st == -1 and berr <= 1e-13
    if prec == "f64":
        # same transform and factorization in double: the same first solve up to rounding order
        assert info["berr_unrefined"] <= 100 * max(b0, 1e-16)


def test_tiled_argument_checks():
    n = 10
    U = _lib.colmajor(n, 2)
    V = _lib.colmajor(n, 2)
    A = _lib.colmajor(n, n)
    with pytest.raises(_lib.RbtError):
        _lib.rbt_apply_2sided_tiled(n, 2, -1, U, V, A, A)
    opts = _lib.make_opts(depth=2, prec="f32", align=64)
    with pytest.raises(_lib.RbtError):
        _lib.rbt_solve_batched_plan(opts, [A], [_lib.colmajor(n, 1)], [_lib.colmajor(n, 1)])


@pytest.mark.parametrize("prec", ["f64", "df64tc"])
@pytest.mark.parametrize("n,d,nb,grid", [(1003, 2, 16, (4, 4)), (2500, 2, 64, (2, 3)), (777, 3, 8, (3, 1))])
def test_comm_free_size_solve(prec, n, d, nb, grid):
    """rbt_opts.grid_p/grid_q (Sec. 6, Eq. comm-free-rbt-size): the solve uses
    the reference size of the p x q grid, i.e. the tiled rule with tiles of
    lcm(p, q) n_b rows.  Its first solution in double equals the solve with
    that alignment bit for bit (the same kernels on the same butterfly
    structure), both meet the backward-error bound, and so does the oracle's
    solve on that size."""
    p, q = grid
    l = int(np.lcm(p, q))
    assert _lib.rbt_reference_size(n, d, nb, grid) == oracle.ref_size_comm_free(n, d, nb, p, q) \
        == oracle.ref_size(n, d, nb * l)
    A = inputs.gaussian(n, seed=23)
    B = inputs.rhs(n, 1, seed=24)
    Ad, Bd = _lib.to_device(A), _lib.to_device(B)
    X1, i1 = solve(Ad, Bd, depth=d, seed=1, prec=prec, align=nb, grid=grid, refine_max=0, fallback=False)
    X2, i2 = solve(Ad, Bd, depth=d, seed=1, prec=prec, align=nb * l, refine_max=0, fallback=False)
    torch.cuda.synchronize()
    assert torch.equal(X1, X2) and i1["berr_unrefined"] == i2["berr_unrefined"]
    X, info = solve(Ad, Bd, depth=d, seed=1, prec=prec, align=nb, grid=grid)
    assert info["code"] == 0 and info["berr"] <= 1e-13, info
    assert _bounds.berr(A, _lib.to_host(X), B) <= 1e-13
    _, st, _, berr, _ = oracle.rbt_solve(A, B, d, 1, align=nb * l)
    assert st == -1 and berr <= 1e-13


def test_comm_free_transform_matches_oracle():
    """The working matrix of the communication-free size against the oracle's
    transform on that size (the explicit tiled matrices give the scale)."""
    n, d, nb, p, q = 1003, 2, 16, 4, 4
    a = nb * int(np.lcm(p, q))
    A = inputs.gaussian(n, seed=25)
    Ud, Vd = _gen(n, d, seed=5)
    U, V = _lib.to_host(Ud), _lib.to_host(Vd)
    out = _lib.colmajor(n, n)
    _lib.rbt_apply_2sided_tiled(n, d, a, Ud, Vd, _lib.to_device(A), out)
    torch.cuda.synchronize()
    want = oracle.transform_2sided(A, U, V, d, align=a)
    scale = np.abs(ex.dense_rbt(n, d, U, align=a).T) @ np.abs(A) @ np.abs(ex.dense_rbt(n, d, V, align=a))
    err = np.abs(_lib.to_host(out) - want)
    assert np.all(err <= REL * scale), float((err / scale).max())
