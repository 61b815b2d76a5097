"""The sliced double-float update (RBT_DF64TC, the benchmark's trailing-update
kernel) is exact only if the tensor cores' FP32 accumulation of integer digit
products is exact.  Each digit is an integer of at most 7 bits plus sign, a
product is at most 64 * 64 = 2^12, and the weight class p + q = t (0-based
digits) collects t + 1 products per k: with K <= 512 every sum, and every
partial sum in any order, stays within 8 * 512 * 2^12 = 2^24, where FP32
holds every integer.  These tests run the update kernel's own TMA and
tcgen05 pipeline on given digits (rbt_debug_oz_products) and require the
eight accumulators to equal the exact integer sums bit for bit, with every
digit at +-64 so that the top class reaches the 2^24 bound itself.

Expected values: float64 matrix products of the digit matrices (every
product and partial sum is an integer below 2^53, so they are exact).
"""
import numpy as np
import pytest
import torch

from paper_2312_09376_gb300 import _lib

pytestmark = pytest.mark.gpu

S = 8


def _exact(da, db):
    a = da.astype(np.float64)
    b = db.astype(np.float64)
    M, N = a.shape[1], b.shape[1]
    out = np.zeros((S, M, N))
    for t in range(S):
        for p in range(t + 1):
            out[t] += a[p] @ b[t - p].T
    return out


def _run(da, db):
    acc = _lib.rbt_debug_oz_products(torch.from_numpy(da).cuda(), torch.from_numpy(db).cuda())
    torch.cuda.synchronize()
    return acc.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("sign_a,sign_b", [(1, 1), (-1, 1), (-1, -1)])
def test_every_class_at_its_bound(sign_a, sign_b):
    # all digits +-64, K = 512: class t holds (t + 1) 2^21, class 7 exactly +-2^24
    M, N, K = 130, 70, 512                    # ragged in M and N: 2 x 2 output tiles
    da = np.full((S, M, K), 64 * sign_a, dtype=np.int8)
    db = np.full((S, N, K), 64 * sign_b, dtype=np.int8)
    got = _run(da, db)
    want = np.array([(t + 1) * 2.0 ** 21 * sign_a * sign_b for t in range(S)])[:, None, None] * np.ones((S, M, N))
    assert abs(want[S - 1]).max() == 2.0 ** 24
    assert np.array_equal(got, want)


def test_random_signs_at_full_magnitude():
    # every product is +-2^12; partial sums wander but stay within 2^24
    rng = np.random.default_rng(1)
    M, N, K = 200, 190, 512
    da = (rng.integers(0, 2, (S, M, K)) * 128 - 64).astype(np.int8)
    db = (rng.integers(0, 2, (S, N, K)) * 128 - 64).astype(np.int8)
    assert np.array_equal(_run(da, db), _exact(da, db))


def test_aligned_signs_keep_the_top_class_at_the_bound_with_mixed_other_classes():
    # signs per digit position chosen so that every product of class 7 is
    # +2^12 (a_p and b_(7-p) of equal sign) while the lower classes mix signs
    signs = np.array([1, -1, -1, 1, -1, 1, 1, -1])
    M, N, K = 129, 65, 512
    da = np.broadcast_to((64 * signs)[:, None, None], (S, M, K)).astype(np.int8)
    db = np.broadcast_to((64 * signs[::-1])[:, None, None], (S, N, K)).astype(np.int8)
    got = _run(da, db)
    want = _exact(da, db)
    assert want[S - 1].max() == 2.0 ** 24
    assert np.array_equal(got, want)


@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (257, 129, 500), (128, 64, 32), (300, 200, 97)])
def test_random_digits_ragged_shapes(M, N, K):
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    da = rng.integers(-64, 65, (S, M, K)).astype(np.int8)
    db = rng.integers(-64, 65, (S, N, K)).astype(np.int8)
    assert np.array_equal(_run(da, db), _exact(da, db))


def test_refuses_k_beyond_the_exactness_bound():
    da = torch.zeros((S, 4, 513), dtype=torch.int8, device="cuda")
    db = torch.zeros((S, 4, 513), dtype=torch.int8, device="cuda")
    with pytest.raises(_lib.RbtError) as e:
        _lib.rbt_debug_oz_products(da, db)
    assert e.value.code == _lib.RBT_ERR_UNSUPPORTED
