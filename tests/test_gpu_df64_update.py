"""Double-float trailing update C <- C - A B on the FP32 pipes (RBT_DF64),
the kernel behind every GENP step of the double-float working precision,
against float64 products.

Tolerance, derived from the accumulation the kernel performs per output
(S = sum_k |a_k| |b_k|): the hi accumulator is exact (TwoSum, exact
product error by FMA); the lo accumulator gathers the rounding terms and
the two cross products, so |lo| <= (K + 3) 2^-24 S, and each of its four
float roundings per k costs at most 2^-24 |lo|; the dropped lo x lo term is
at most 2^-48 |a||b|.  Total at most 4 K (K + 3) 2^-48 S + 2^-48 S, plus
the double-float subtraction from C, below 2^-44 (|C| + S).
"""
import numpy as np
import pytest
import torch

from paper_2312_09376_gb300 import _lib
from tests._df64 import from_df64, to_df64

pytestmark = pytest.mark.gpu


def _update(A, B, C):
    Ad, Av = to_df64(A)
    Bd, Bv = to_df64(B)
    Cd, Cv = to_df64(C)
    st = torch.empty(1, dtype=torch.int64, device="cuda")
    assert _lib.genp_update_workspace(A.shape[0], B.shape[1], A.shape[1], "df64") == 0
    _lib.genp_update("df64", Ad, Bd, Cd, st)
    torch.cuda.synchronize()
    return from_df64(Cd), int(st.item()), Av, Bv, Cv


# both tilings: 64 x 64 below 2048 rows or columns, 128 x 128 from there on,
# with ragged edges in M, N and K
@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (5, 7, 3), (64, 64, 16), (65, 129, 17), (300, 517, 64),
                                   (2048, 2048, 64), (2049, 2111, 64), (2500, 2177, 37), (4099, 2048, 128)])
def test_df64_update_matches_float64(M, N, K):
    rng = np.random.default_rng(M + 5 * N + 11 * K)
    A = rng.standard_normal((M, K)) * np.exp(rng.uniform(-3, 3, (M, 1)))
    B = rng.standard_normal((K, N)) * np.exp(rng.uniform(-3, 3, (1, N)))
    C = rng.standard_normal((M, N))
    got, st, Av, Bv, Cv = _update(A, B, C)
    assert st == -1
    want = Cv - Av @ Bv
    S = np.abs(Av) @ np.abs(Bv)
    tol = (4 * K * (K + 3) + 1) * 2.0 ** -48 * S + 2.0 ** -44 * (np.abs(Cv) + S)
    err = np.abs(got - want)
    assert np.all(err <= tol), float((err / tol).max())
    # in practice the rounding terms cancel: close to double-float accuracy
    assert err.max() <= 2.0 ** -40 * S.max()


def test_df64_update_is_exact_for_small_integers():
    """Products of integers below 2^11 are exact floats, and every partial sum
    stays an integer below 2^48: each step of the accumulation is exact."""
    rng = np.random.default_rng(5)
    M, N, K = 2100, 2050, 64
    A = rng.integers(-2000, 2001, (M, K)).astype(np.float64)
    B = rng.integers(-2000, 2001, (K, N)).astype(np.float64)
    C = rng.integers(-10**9, 10**9, (M, N)).astype(np.float64)
    got, st, _, _, _ = _update(A, B, C)
    assert st == -1
    assert np.array_equal(got, C - A @ B)


def test_df64_update_empty_sets_status():
    st = torch.zeros(1, dtype=torch.int64, device="cuda")
    A = _lib.colmajor(0, 4)
    B = _lib.colmajor(4, 3)
    C = _lib.colmajor(0, 3)
    _lib.genp_update("df64", A, B, C, st)
    torch.cuda.synchronize()
    assert int(st.item()) == -1
