"""Tensor-core trailing update (tcgen05, TF32 / BF16 operands, FP32
accumulation) against float64 products, and the TF32 / BF16 factorizations.

Tolerances (derived): a product of operands rounded to p significant bits has
relative error at most 2^(1-p) + 2^(2-2p) (two roundings); FP32 accumulation
of K terms adds at most K 2^-24 of sum |a||b|; the final subtraction from C
one more 2^-24 |C - AB|.  With p = 8 (BF16) or p = 11 (TF32; the tensor cores
may also truncate instead of rounding, which doubles the first term) the
elementwise bound is (2^(2-p) + (K + 1) 2^-24) (|A||B|)_ij + 2^-24 |C|_ij.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2312_09376_gb300 import _lib, inputs
from tests import _bounds

pytestmark = pytest.mark.gpu

P_BITS = {"bf16": 8, "tf32": 11}


def _update(prec, A, B, C):
    Ad, Bd, Cd = (_lib.to_device(x.astype(np.float32)) for x in (A, B, C))
    M, K = A.shape
    N = B.shape[1]
    st = torch.empty(1, dtype=torch.int64, device="cuda")
    ws = _lib.genp_update_workspace(M, N, K, prec)
    work = torch.empty(max(ws, 1), dtype=torch.uint8, device="cuda")
    _lib.genp_update(prec, Ad, Bd, Cd, st, work)
    torch.cuda.synchronize()
    return _lib.to_host(Cd).astype(np.float64), int(st.item())


SHAPES = [(5, 7, 3), (128, 256, 64), (129, 257, 65), (300, 517, 128), (1000, 1100, 1024), (4099, 300, 128),
          (256, 4100, 200)]


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
@pytest.mark.parametrize("M,N,K", SHAPES)
def test_update_matches_float64(prec, M, N, K):
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    A = rng.standard_normal((M, K)).astype(np.float32).astype(np.float64)
    B = rng.standard_normal((K, N)).astype(np.float32).astype(np.float64)
    C = rng.standard_normal((M, N)).astype(np.float32).astype(np.float64)
    got, st = _update(prec, A, B, C)
    assert st == -1
    want = C - A @ B
    scale = np.abs(A) @ np.abs(B)
    p = P_BITS[prec]
    tol = (2.0 ** (2 - p) + (K + 1) * 2.0 ** -24) * scale + 2.0 ** -24 * np.abs(C)
    err = np.abs(got - want)
    assert np.all(err <= tol), float((err / np.maximum(tol, 1e-30)).max())
    # and the operands really were rounded (the result is not a float SIMT product)
    if K >= 64:
        assert np.abs(got - want).max() > 2.0 ** -20 * scale.max()


def test_update_is_exact_for_small_integers():
    """Integer operands with |a|,|b| <= 15 are exact in BF16 and TF32 and their
    K-term sums are exact in FP32: the result must equal the exact product."""
    rng = np.random.default_rng(1)
    M, N, K = 200, 300, 256
    A = rng.integers(-15, 16, (M, K)).astype(np.float64)
    B = rng.integers(-15, 16, (K, N)).astype(np.float64)
    C = rng.integers(-1000, 1000, (M, N)).astype(np.float64)
    for prec in ("bf16", "tf32"):
        got, st = _update(prec, A, B, C)
        assert st == -1
        assert np.array_equal(got, C - A @ B), prec


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
@pytest.mark.parametrize("n", [1, 100, 129, 1003, 2500])
def test_tc_factorization_backward_error(prec, n):
    A = inputs.gaussian(n, seed=11)
    U, V = oracle.generate(n, 2, 1)
    At = oracle.transform_2sided(A, U, V, 2).astype(np.float32).astype(np.float64)
    Ad = _lib.to_device(At.astype(np.float32))
    info = torch.empty(1, dtype=torch.int64, device="cuda")
    work = torch.empty(max(_lib.genp_factor_workspace(n, prec), 1), dtype=torch.uint8, device="cuda")
    _lib.genp_factor(n, prec, Ad, info, work)
    torch.cuda.synchronize()
    assert int(info.item()) == -1
    LU = _lib.to_host(Ad).astype(np.float64)
    L = np.tril(LU, -1) + np.eye(n)
    Uu = np.triu(LU)
    E = np.abs(At - L @ Uu)
    p = P_BITS[prec]
    tol = (2.0 ** (2 - p) + 3 * n * 2.0 ** -24) * (np.abs(L) @ np.abs(Uu))
    assert np.all(E <= tol), float((E / np.maximum(tol, 1e-30)).max())


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
def test_tc_solve_reaches_tolerance_through_fallback(prec):
    """Low-precision factors after a depth-2 transform do not refine to 1e-13 at
    this size; the stall hands over to the double factorization."""
    n = 1500
    A = inputs.gaussian(n)
    B = inputs.rhs(n, 1)
    from paper_2312_09376_gb300 import solve
    X, info = solve(_lib.to_device(A), _lib.to_device(B), depth=2, prec=prec, refine_max=10, tol=1e-13,
                    fallback=True)
    torch.cuda.synchronize()
    assert info["code"] == 0
    assert _bounds.berr(A, _lib.to_host(X), B) <= 1e-13
