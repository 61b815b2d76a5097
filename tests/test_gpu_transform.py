"""GPU parity of the butterfly generator and transforms against the CPU oracle.

Tolerance (derived, not fitted): a structured evaluation of U^T A V in double
has elementwise error at most a small multiple of u (|U|^T |A| |V|) with
u = 2^-53 and one rounding per butterfly add, per pair normalization and per
diagonal scaling (at most 4 d roundings on each path).  The transformed-entry
target is relative 1e-14 of that scale, i.e. about 90 u, which covers 4 d <= 12
roundings on each of the two sides with room to spare.  Entries are compared
against (|U|^T|A||V|)_ij, exactly for n <= 1100 and through the group-sum
upper bound above that.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2312_09376_gb300 import _lib, inputs
from tests import _bounds

pytestmark = pytest.mark.gpu

REL = 1e-14


def _gen(n, d, seed):
    """The oracle's butterflies for (n, d, seed), uploaded: the device
    transform and the oracle transform the same inputs (the device generator
    has its own parity test)."""
    U, V = oracle.generate(n, d, seed)
    return _lib.to_device(U), _lib.to_device(V)


@pytest.mark.parametrize("n,d,seed", [(1, 1, 0), (7, 3, 5), (1003, 2, 1), (20001, 3, 1), (40003, 2, 99)])
def test_generator_matches_oracle(n, d, seed):
    U = _lib.colmajor(n, d)
    V = _lib.colmajor(n, d)
    _lib.rbt_generate(n, d, seed, U, V)
    torch.cuda.synchronize()
    Uo, Vo = oracle.generate(n, d, seed)
    for g, o in ((U, Uo), (V, Vo)):
        g = _lib.to_host(g)
        # same 53-bit uniform on both sides; exp() of libm and of CUDA may differ by an ulp
        assert np.all(np.abs(g - o) <= 2 * np.spacing(o)), np.abs(g - o).max()


def _check_transform(n, d, A, got, U, V):
    want = oracle.transform_2sided(A, U, V, d)
    scale = _bounds.abs_transform_bound(A, U, V, d) if n <= 1100 else _bounds.group_bound(A, d)
    err = np.abs(got - want)
    ok = err <= REL * scale
    assert ok.all(), (n, d, float((err / np.maximum(scale, 1e-300)).max()))


SMALL = [(n, d) for n in (1, 2, 3, 4, 5, 8, 17, 31, 64, 67, 100, 251) for d in (1, 2, 3, 4, 5)]


@pytest.mark.parametrize("n,d", SMALL)
def test_fused_transform_small(n, d):
    A = inputs.gaussian(n, seed=n * 10 + d)
    Ud, Vd = _gen(n, d, seed=3)
    U, V = _lib.to_host(Ud), _lib.to_host(Vd)
    Ad = _lib.to_device(A)
    out = _lib.colmajor(n, n)
    _lib.rbt_apply_2sided(n, d, Ud, Vd, Ad, out)           # out of place
    _lib.rbt_apply_2sided(n, d, Ud, Vd, Ad)                # in place
    lay = _lib.to_device(A)
    _lib.rbt_apply_2sided_layered(n, d, Ud, Vd, lay)       # one pass per layer
    torch.cuda.synchronize()
    for g in (out, Ad, lay):
        _check_transform(n, d, A, _lib.to_host(g), U, V)
    assert np.array_equal(_lib.to_host(out), _lib.to_host(Ad))


@pytest.mark.parametrize("n,d", [(1003, 2), (1003, 1), (1003, 3), (1024, 2), (1001, 6), (2047, 3), (4099, 2)])
def test_fused_transform_medium(n, d):
    A = inputs.gaussian(n, seed=42)
    Ud, Vd = _gen(n, d, seed=1)
    U, V = _lib.to_host(Ud), _lib.to_host(Vd)
    Ad = _lib.to_device(A)
    _lib.rbt_apply_2sided(n, d, Ud, Vd, Ad)
    torch.cuda.synchronize()
    _check_transform(n, d, A, _lib.to_host(Ad), U, V)


def test_fused_transform_padded_leading_dimension():
    n, d, lda = 1003, 2, 1040
    A = inputs.gaussian(n, seed=7)
    Ud, Vd = _gen(n, d, seed=2)
    Ad = _lib.colmajor(n, n, ld=lda)
    Ad.copy_(_lib.to_device(A))
    sentinel = Ad.as_strided((lda - n, n), (1, lda), storage_offset=n)
    sentinel.fill_(123.0)
    out = _lib.colmajor(n, n, ld=1030)
    _lib.rbt_apply_2sided(n, d, Ud, Vd, Ad, out)
    _lib.rbt_apply_2sided(n, d, Ud, Vd, Ad)
    torch.cuda.synchronize()
    assert torch.all(sentinel == 123.0)                    # padding rows untouched
    _check_transform(n, d, A, _lib.to_host(Ad), _lib.to_host(Ud), _lib.to_host(Vd))
    assert np.array_equal(_lib.to_host(out), _lib.to_host(Ad))


@pytest.mark.parametrize("n,d", [(20001, 3), (20000, 2), (20480, 1)])
def test_fused_transform_large_full(n, d):
    A = inputs.gaussian(n, seed=42)
    Ud, Vd = _gen(n, d, seed=1)
    Ad = _lib.to_device(A)
    _lib.rbt_apply_2sided(n, d, Ud, Vd, Ad)
    torch.cuda.synchronize()
    _check_transform(n, d, A, _lib.to_host(Ad), _lib.to_host(Ud), _lib.to_host(Vd))


def _oracle_columns(n, d, W, idx):
    """Columns idx of the dense W, each from the oracle's one-sided transform of e_i."""
    E = np.zeros((n, len(idx)))
    E[idx, np.arange(len(idx))] = 1.0
    return oracle.transform_vec(E, W, d, trans=False)


@pytest.mark.parametrize("n,d", [(40003, 2), (40000, 2)])
def test_fused_transform_full_size_sampled(n, d):
    """Full-size launch (the benchmark's): sampled entries A~_ij = (U e_i)^T A (V e_j),
    the columns of U and V taken from the oracle."""
    g = torch.Generator(device="cuda").manual_seed(42)
    Ad = torch.randn((n, n), generator=g, device="cuda", dtype=torch.float64).T  # column-major view
    rng = np.random.default_rng(0)
    ii = rng.integers(0, n, 400)
    jj = rng.integers(0, n, 400)
    ii[:4] = [0, n - 1, n - 1, 0]
    jj[:4] = [0, n - 1, 0, n - 1]
    Ud, Vd = _gen(n, d, seed=1)
    U, V = _lib.to_host(Ud), _lib.to_host(Vd)
    Ucols = _oracle_columns(n, d, U, ii)
    Vcols = _oracle_columns(n, d, V, jj)
    rows = [np.nonzero(Ucols[:, k])[0] for k in range(len(ii))]
    cols = [np.nonzero(Vcols[:, k])[0] for k in range(len(jj))]
    blocks = []
    for k in range(len(ii)):
        r = torch.as_tensor(rows[k], device="cuda")
        c = torch.as_tensor(cols[k], device="cuda")
        blocks.append(Ad[r][:, c].cpu().numpy())
    _lib.rbt_apply_2sided(n, d, Ud, Vd, Ad)
    torch.cuda.synchronize()
    got = Ad[torch.as_tensor(ii, device="cuda"), torch.as_tensor(jj, device="cuda")].cpu().numpy()
    for k in range(len(ii)):
        u = Ucols[rows[k], k]
        v = Vcols[cols[k], k]
        want = u @ blocks[k] @ v
        scale = np.abs(u) @ np.abs(blocks[k]) @ np.abs(v)
        assert abs(got[k] - want) <= REL * scale, (ii[k], jj[k], got[k], want)


@pytest.mark.parametrize("n,d,align", [(1003, 2, 1), (67, 3, 1), (8197, 2, 1), (5, 5, 1), (2500, 3, 1),
                                       (2500, 2, 512), (1003, 3, 64)])
@pytest.mark.parametrize("prec", ["f32", "df64"])
def test_working_copy_transform(n, d, align, prec):
    """The working copies (row a4: the float and double-float outputs of the
    transform pass) against the oracle's double transform of the same A with
    the same coefficients."""
    A = inputs.gaussian(n, seed=5)
    U, V = oracle.generate(n, d, 1)
    Ud, Vd = _lib.to_device(U), _lib.to_device(V)
    Ad = _lib.to_device(A)
    dt = torch.float32 if prec == "f32" else torch.float64
    out = _lib.colmajor(n, n, dtype=dt, ld=n + 3)
    if min(d, int(np.ceil(np.log2(n)))) > 3:
        with pytest.raises(_lib.RbtError):
            _lib.rbt_transform_2sided(n, d, align, "scaled", prec, Ud, Vd, Ad, out)
        return
    _lib.rbt_transform_2sided(n, d, align, "scaled", prec, Ud, Vd, Ad, out)
    torch.cuda.synchronize()
    want = oracle.transform_2sided(A, U, V, d, align=align)
    scale = (_bounds.abs_transform_bound(A, U, V, d, align=align) if n <= 1100
             else _bounds.group_bound(A, d, align=align))
    # the oracle's own double rounding: at most 4 d roundings of 2^-53 per path
    oracle_err = 8 * d * 2.0 ** -53
    if prec == "f32":
        # float arithmetic from the double input: a double -> float rounding of
        # each input entry and each coefficient, then 4 d float roundings per
        # path, all relative to (|U|^T |A| |V|)_ij; 64 ulps of float covers them
        err = np.abs(_lib.to_host(out).astype(np.float64) - want)
        tol = (64 * 2.0 ** -24 + oracle_err) * scale
        assert np.all(err <= tol), float((err / scale).max() / 2.0 ** -24)
    else:
        # double-float arithmetic from the double input: the input and each
        # coefficient split into a pair within 2^-48; each pair sum errs by at
        # most 2^-46 (|a| + |b|) and each pair product by 2^-46 of its size;
        # a path meets at most 2 d sums, 2 d products and 3 d + 1 splits, so
        # (7 d + 1) 2^-46 of (|U|^T |A| |V|)_ij bounds it
        val = _lib.to_host(_lib.df64_to_double(out))
        err = np.abs(val - want)
        tol = ((7 * d + 1) * 2.0 ** -46 + oracle_err) * scale
        assert np.all(err <= tol), float((err / scale).max() / 2.0 ** -46)
        # and far below float accuracy
        assert err.max() <= 2.0 ** -40 * scale.max()
    assert torch.equal(Ad, _lib.to_device(A))              # input untouched


@pytest.mark.parametrize("n,d,nrhs", [(1, 2, 1), (5, 4, 3), (67, 2, 32), (1003, 2, 1), (1003, 3, 8), (8197, 2, 32),
                                      (40003, 2, 1)])
def test_vec_transforms(n, d, nrhs):
    B = inputs.rhs(n, nrhs)
    Ud, _ = _gen(n, d, seed=4)
    U = _lib.to_host(Ud)
    for trans in (True, False):
        Bd = _lib.to_device(B)
        _lib.rbt_apply_vec(n, d, Ud, trans, Bd)
        torch.cuda.synchronize()
        want = oracle.transform_vec(B, U, d, trans=trans)
        # |W| |b| <= e^(d/20) * (group sum of |b|): same argument as the matrix bound
        scale = np.exp(d / 20) * (2 ** min(d, 20)) * np.abs(B).max(axis=0)[None, :]
        assert np.all(np.abs(_lib.to_host(Bd) - want) <= REL * scale)


def test_vec_transforms_are_adjoint():
    """The two one-sided GPU transforms are transposes of each other:
    (U^T b) . y == b . (U y) up to rounding."""
    n, d = 1003, 2
    Ud, _ = _gen(n, d, seed=11)
    b = inputs.rhs(n, 1, seed=1)[:, 0]
    y = inputs.rhs(n, 1, seed=2)[:, 0]
    bd, yd = _lib.to_device(b), _lib.to_device(y)
    _lib.rbt_apply_vec(n, d, Ud, True, bd)
    _lib.rbt_apply_vec(n, d, Ud, False, yd)
    torch.cuda.synchronize()
    lhs = float(_lib.to_host(bd) @ y)
    rhs = float(b @ _lib.to_host(yd))
    assert abs(lhs - rhs) <= 1e-12 * (np.abs(b).sum() * np.abs(y).max() * 4)
