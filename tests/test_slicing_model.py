"""The error bound the sliced-update tests use, checked on an exact model of
the slicing (CPU, rational arithmetic; no GPU code involved).

Model, from the construction of the update: each k is balanced by
2^t_k, t_k = floor((E_B(k) - E_A(k)) / 2) with E the binary exponent of the
largest |entry| of column k of A or row k of B (|x| < 2^E <= 2|x|); row i of
A 2^t is held relative to 2^e_i (e_i one above the largest exponent of the
row) as the integer rint(hi 2^(7S - e_i)) + rint(lo 2^(7S - e_i)) of its
double-float parts, written as S balanced base-128 digits, likewise column j
of B 2^-t with f_j; only digit products of weight p + q <= S + 1 are kept.
The claim the GPU tests rely on: per entry, |computed - exact| <=
K 2^(e_i + f_j - (7S - 4))."""
from fractions import Fraction

import numpy as np
import pytest


def _exp(x):
    """E with 2^(E-1) <= |x| < 2^E (x != 0)."""
    return int(np.frexp(x)[1])


def _df(x):
    """The double-float pair (hi, lo) of a double: hi = fl32(x), lo = fl32(x - hi)."""
    hi = np.float32(x)
    lo = np.float32(x - float(hi))
    return float(hi), float(lo)


def _digits(v_hi, v_lo, e, s):
    """Balanced base-128 digits (most significant first) of the model's integer."""
    y = int(round(v_hi * 2.0 ** (7 * s - e))) + int(round(v_lo * 2.0 ** (7 * s - e)))
    d = []
    for _ in range(s):
        r = ((y % 128) + 64) % 128 - 64
        d.append(r)
        y = (y - r) // 128
    d.append(y)            # what is left goes into the leading digit
    d = d[::-1]
    lead = d[0] * 128 + d[1]
    return [lead] + d[2:]  # the remainder joins the leading digit (|y| < 2^(7S - 1) keeps it in range)


def _sliced_product(A, B, s):
    M, K = A.shape
    N = B.shape[1]
    Ahl = [[_df(A[i, k]) for k in range(K)] for i in range(M)]
    Bhl = [[_df(B[k, j]) for j in range(N)] for k in range(K)]
    EA = [max(_exp(Ahl[i][k][0]) for i in range(M)) for k in range(K)]
    EB = [max(_exp(Bhl[k][j][0]) for j in range(N)) for k in range(K)]
    t = [(EB[k] - EA[k]) // 2 for k in range(K)]
    e = [max(_exp(Ahl[i][k][0]) + t[k] for k in range(K)) + 1 for i in range(M)]
    f = [max(_exp(Bhl[k][j][0]) - t[k] for k in range(K)) + 1 for j in range(N)]
    da = [[_digits(Ahl[i][k][0] * 2.0 ** t[k], Ahl[i][k][1] * 2.0 ** t[k], e[i], s) for k in range(K)]
          for i in range(M)]
    db = [[_digits(Bhl[k][j][0] * 2.0 ** -t[k], Bhl[k][j][1] * 2.0 ** -t[k], f[j], s) for j in range(N)]
          for k in range(K)]
    out = np.empty((M, N), dtype=object)
    for i in range(M):
        for j in range(N):
            acc = 0
            for k in range(K):
                for p in range(1, s + 1):
                    for q in range(1, s + 2 - p):
                        acc += da[i][k][p - 1] * db[k][j][q - 1] * Fraction(1, 128 ** (p + q))
            out[i, j] = acc * Fraction(2) ** (e[i] + f[j])
    exact = np.empty((M, N), dtype=object)
    for i in range(M):
        for j in range(N):
            exact[i, j] = sum((Fraction(Ahl[i][k][0]) + Fraction(Ahl[i][k][1]))
                              * (Fraction(Bhl[k][j][0]) + Fraction(Bhl[k][j][1])) for k in range(K))
    return out, exact, e, f


@pytest.mark.parametrize("s", [7, 8])
@pytest.mark.parametrize("seed", [0, 1])
def test_slicing_error_bound(s, seed):
    rng = np.random.default_rng(seed)
    M, N, K = 5, 4, 12
    c = rng.integers(-12, 13, K)
    # GENP-like binade mixing across k (column k of A times 2^c_k, row k of B times 2^-c_k)
    A = rng.standard_normal((M, K)) * np.exp2(c)[None, :] * np.exp(rng.uniform(-2, 2, (M, 1)))
    B = rng.standard_normal((K, N)) * np.exp2(-c)[:, None]
    got, exact, e, f = _sliced_product(A, B, s)
    worst = 0.0
    for i in range(M):
        for j in range(N):
            err = abs(got[i, j] - exact[i, j])
            bound = K * Fraction(2) ** (e[i] + f[j] - (7 * s - 4))
            assert err <= bound, (s, i, j, float(err), float(bound))
            worst = max(worst, float(err / bound))
    # the bound is not vacuous: seven digits use a visible part of it
    if s == 7:
        assert worst > 1e-4


def test_digits_reassemble_and_stay_balanced():
    rng = np.random.default_rng(3)
    for _ in range(200):
        x = rng.standard_normal() * 2.0 ** rng.integers(-20, 20)
        hi, lo = _df(x)
        e = _exp(hi) + 1
        for s in (7, 8):
            d = _digits(hi, lo, e, s)
            y = int(round(hi * 2.0 ** (7 * s - e))) + int(round(lo * 2.0 ** (7 * s - e)))
            assert sum(dp * 128 ** (s - 1 - p) for p, dp in enumerate(d)) == y
            assert all(-64 <= dp <= 64 for dp in d)
