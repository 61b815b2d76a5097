"""Double-float GENP update on the BF16 tensor cores by exact digit slicing
(RBT_DF64TC, eight digits; RBT_DF64TC7, seven) against float64 products, and
the factorization / solve built on it.

Tolerance of the update (derived from the construction): each k is first
balanced by an exact power of two, A_ik B_kj = (A_ik 2^t_k)(B_kj 2^-t_k) with
t_k = floor((E_B(k) - E_A(k)) / 2), E the binary exponent of the largest |hi|
of column k of A or row k of B.  Entry A_ik 2^t_k is then held as 7S
fractional bits of 2^e_i (S 7-bit digits; e_i one above the largest exponent
of row i after the shift), so its error is at most 2^(e_i - 7S) and its size
below 2^(e_i - 1), likewise for B with f_j; the dropped digit products have
weights 2^-7t, t >= S + 2 (at most S - 1 of weight S + 2, each at most 2^12,
fewer at each later weight).  Per k the product error is at most
2^(e_i + f_j) (2^-7S + 1.02 (S - 1) 2^(12 - 7(S + 2))) < 2^(e_i + f_j - (7S - 4))
(S = 8: 2^-52, S = 7: 2^-45); the double-float fold and update add
2^-46 (|C| + |A||B|).
"""

import numpy as np
import pytest
import torch

import oracle
from paper_2312_09376_gb300 import _lib, inputs, solve
from tests import _bounds
from tests._df64 import from_df64, to_df64

pytestmark = pytest.mark.gpu


NOEXP = -(1 << 30)


def _exps(h):
    """Binary exponents E (|h| < 2^E <= 2|h|) of float32 values, NOEXP for zeros."""
    e = np.frexp(h.astype(np.float64))[1].astype(np.int64)
    return np.where(h == 0, NOEXP, e)


def _balanced_exponents(Av, Bv):
    """(e_i, f_j) of the sliced update, with the k-balancing shifts t_k."""
    ea = _exps(Av.astype(np.float32))            # M x K
    eb = _exps(Bv.astype(np.float32))            # K x N
    EA, EB = ea.max(0), eb.max(1)
    t = np.where((EA == NOEXP) | (EB == NOEXP), 0, np.floor_divide(EB - EA, 2))
    er = np.where(ea == NOEXP, NOEXP, ea + t[None, :]).max(1)
    fc = np.where(eb == NOEXP, NOEXP, eb - t[:, None]).max(0)
    return np.where(er == NOEXP, 0, er + 1).astype(float), np.where(fc == NOEXP, 0, fc + 1).astype(float)


DIGITS = {"df64tc": 8, "df64tc7": 7}


def _slice_bits(prec):
    """7S - 4: the per-k slicing error is below 2^(e_i + f_j - (7S - 4))."""
    return 7 * DIGITS[prec] - 4


def _update(A, B, C, prec="df64tc"):
    Ad, Av = to_df64(A)
    Bd, Bv = to_df64(B)
    Cd, Cv = to_df64(C)
    M, K = A.shape
    N = B.shape[1]
    st = torch.empty(1, dtype=torch.int64, device="cuda")
    work = torch.empty(_lib.genp_update_workspace(M, N, K, prec), dtype=torch.uint8, device="cuda")
    _lib.genp_update(prec, Ad, Bd, Cd, st, work)
    torch.cuda.synchronize()
    return from_df64(Cd), int(st.item()), Av, Bv, Cv


@pytest.mark.parametrize("prec", ["df64tc", "df64tc7"])
@pytest.mark.parametrize("M,N,K", [(5, 7, 3), (128, 96, 32), (129, 97, 33), (300, 517, 64), (1000, 700, 512),
                                   (4099, 200, 128), (200, 3000, 511)])
def test_sliced_update_matches_float64(M, N, K, prec):
    rng = np.random.default_rng(M + 3 * N + 7 * K)
    A = rng.standard_normal((M, K)) * np.exp(rng.uniform(-3, 3, (M, 1)))
    B = rng.standard_normal((K, N)) * np.exp(rng.uniform(-3, 3, (1, N)))
    C = rng.standard_normal((M, N))
    got, st, Av, Bv, Cv = _update(A, B, C, prec)
    assert st == -1
    want = Cv - Av @ Bv
    ea, fb = _balanced_exponents(Av, Bv)
    tol = K * np.exp2(ea[:, None] + fb[None, :] - _slice_bits(prec)) + 2.0 ** -46 * (np.abs(Cv) + np.abs(Av) @ np.abs(Bv))
    err = np.abs(got - want)
    assert np.all(err <= tol), float((err / tol).max())
    # well beyond float: 7 bits per digit of relative accuracy where the scales allow
    if K >= 64:
        assert np.abs(got - want).max() < 2.0 ** -(7 * DIGITS[prec] - 16) * (np.abs(Av) @ np.abs(Bv)).max()


def test_seven_digits_lose_accuracy_against_eight():
    """The digit count is live: on the same operands the seven-digit update's
    error exceeds the eight-digit one's (a dropped or repeated digit weight in
    either would show as an O(1) error, a wrong count as equal errors)."""
    rng = np.random.default_rng(5)
    M, N, K = 512, 384, 512
    A = rng.standard_normal((M, K))
    B = rng.standard_normal((K, N))
    C = rng.standard_normal((M, N))
    errs = {}
    for prec in ("df64tc", "df64tc7"):
        got, st, Av, Bv, Cv = _update(A, B, C, prec)
        assert st == -1
        errs[prec] = np.abs(got - (Cv - Av @ Bv)).max() / (np.abs(Av) @ np.abs(Bv)).max()
    assert errs["df64tc7"] > 2 * errs["df64tc"], errs
    assert errs["df64tc7"] < 2.0 ** -38, errs


@pytest.mark.parametrize("prec", ["df64tc", "df64tc7"])
def test_sliced_update_is_exact_for_small_integers(prec):
    """Integers below 2^10 have at most two nonzero base-128 digits: every digit
    product is exact, so the update is exact."""
    rng = np.random.default_rng(3)
    M, N, K = 300, 200, 512
    A = rng.integers(-1000, 1001, (M, K)).astype(np.float64)
    B = rng.integers(-1000, 1001, (K, N)).astype(np.float64)
    C = rng.integers(-10**6, 10**6, (M, N)).astype(np.float64)
    got, st, Av, Bv, Cv = _update(A, B, C, prec)
    assert st == -1
    assert np.array_equal(got, C - A @ B)


@pytest.mark.parametrize("prec", ["df64tc", "df64tc7"])
def test_sliced_update_balances_each_k(prec):
    """GENP's panels: column k of L21 carries 1/u_kk and row k of U12 carries
    u_kk.  Here A_ik = g 2^c_k and B_kj = g 2^-c_k with c_k over +-20 binades,
    so every product is of order one while each row of A spans 40 binades.
    Slicing relative to the row maxima alone would keep about 2^-12 of the
    result; with the power-of-two balancing of each k the error stays at the
    double-float level."""
    rng = np.random.default_rng(11)
    M, N, K = 700, 600, 512
    c = rng.integers(-20, 21, K)
    A = rng.standard_normal((M, K)) * np.exp2(c)[None, :]
    B = rng.standard_normal((K, N)) * np.exp2(-c)[:, None]
    C = rng.standard_normal((M, N))
    got, st, Av, Bv, Cv = _update(A, B, C, prec)
    assert st == -1
    S = np.abs(Av) @ np.abs(Bv)
    err = np.abs(got - (Cv - Av @ Bv))
    ea, fb = _balanced_exponents(Av, Bv)
    tol = K * np.exp2(ea[:, None] + fb[None, :] - _slice_bits(prec)) + 2.0 ** -46 * (np.abs(Cv) + S)
    assert np.all(err <= tol), float((err / tol).max())
    assert err.max() <= 2.0 ** -(7 * DIGITS[prec] - 16) * S.max()


def _digit_slack(prec):
    """2^(7 (8 - S)): how much larger the seven-digit slicing error is."""
    return 2.0 ** (7 * (8 - DIGITS[prec]))


@pytest.mark.parametrize("prec", ["df64tc", "df64tc7"])
@pytest.mark.parametrize("n", [1, 65, 300, 1003, 2500])
def test_df64tc_factorization(n, prec):
    A = inputs.gaussian(n, seed=13)
    U, V = oracle.generate(n, 2, 1)
    At = oracle.transform_2sided(A, U, V, 2)
    Ad, Av = to_df64(At)
    info = torch.empty(1, dtype=torch.int64, device="cuda")
    work = torch.empty(max(_lib.genp_factor_workspace(n, prec), 1), dtype=torch.uint8, device="cuda")
    _lib.genp_factor(n, prec, Ad, info, work)
    torch.cuda.synchronize()
    assert int(info.item()) == -1
    LU = from_df64(Ad)
    L = np.tril(LU, -1) + np.eye(n)
    Uu = np.triu(LU)
    E = np.abs(Av - L @ Uu).max()
    scale = np.abs(L).max() * np.abs(Uu).max()
    assert E <= (n * 2.0 ** -44 + 2.0 ** -44) * scale * 4 * _digit_slack(prec)


U_DF64 = 2.0 ** -44   # per-operation relative error of the double-float panel kernels and C updates


def _sliced_lu_bound(L, U, prec="df64tc"):
    """Elementwise bound on |A - L U| for the two-level sliced factorization
    (512-column panels in 64-column steps): the double-float part as for the
    plain double-float factorization, 2 gamma_n(2^-44) (|L||U|)_ij, plus, for
    every sliced update that touched (i, j), its slicing error
    K 2^(e_i + f_j - (7S - 4)) (see the top of this file) with e_i, f_j the
    balanced exponents of that update's operands, which are blocks of the
    final L and U.  One extra binade on each exponent covers a pair whose
    hi part sits at a power of two."""
    n = L.shape[0]
    bound = 2 * _bounds.gamma(n, U_DF64) * (np.abs(L) @ np.abs(U))

    def add(r0, r1, c0, c1, k0, k1):
        if r1 <= r0 or c1 <= c0:
            return
        ea, fb = _balanced_exponents(L[r0:r1, k0:k1], U[k0:k1, c0:c1])
        bound[r0:r1, c0:c1] += (k1 - k0) * np.exp2(ea[:, None] + fb[None, :] - (_slice_bits(prec) - 2))

    for k in range(0, n, 512):
        kb = min(512, n - k)
        for j in range(k, k + kb, 64):
            jb = min(64, k + kb - j)
            r0 = j + jb
            add(r0, n, r0, k + kb, j, j + jb)            # the panel's remaining columns
            add(r0, k + kb, k + kb, n, j, j + jb)        # the block row right of the panel
        add(k + kb, n, k + kb, n, k, k + kb)             # the trailing matrix
    return bound


@pytest.mark.parametrize("prec", ["df64tc", "df64tc7"])
@pytest.mark.parametrize("n", [1, 65, 300, 1003, 2500])
def test_df64tc_factors_elementwise_and_against_oracle(n, prec):
    """Row a5 on the sliced paths: the sliced factorization satisfies the
    elementwise bound above, and at n = 2500 its first 256 rows and columns
    match the oracle's double GENP as the double-float factors do (seven
    digits: 2^7 times looser)."""
    A = inputs.gaussian(n, seed=13)
    U, V = oracle.generate(n, 2, 1)
    At = oracle.transform_2sided(A, U, V, 2)
    Ad, Av = to_df64(At)
    info = torch.empty(1, dtype=torch.int64, device="cuda")
    work = torch.empty(max(_lib.genp_factor_workspace(n, prec), 1), dtype=torch.uint8, device="cuda")
    _lib.genp_factor(n, prec, Ad, info, work)
    torch.cuda.synchronize()
    assert int(info.item()) == -1
    LU = from_df64(Ad)
    L = np.tril(LU, -1) + np.eye(n)
    Uu = np.triu(LU)
    # forming L U in double adds at most gamma_n(2^-53) |L||U|, inside the margin of the bound
    E = np.abs(Av - L @ Uu)
    bound = _sliced_lu_bound(L, Uu, prec)
    assert np.all(E <= bound), float((E / bound).max())
    LUo, sto = oracle.genp(At)
    assert sto == -1
    if n <= 1024:
        assert np.abs(LU - LUo).max() <= 1e-6 * _digit_slack(prec) * np.abs(LUo).max()
    else:
        # the leading block columns of L and block rows of U: same reasoning
        # and bound as for the double-float factors (a wrong index, tile or
        # digit weight shows as an O(1) difference)
        w = 256
        for got, ref in ((LU[:, :w], LUo[:, :w]), (LU[:w, :], LUo[:w, :])):
            assert np.abs(got - ref).max() <= 1e-5 * _digit_slack(prec) * np.abs(ref).max()


@pytest.mark.parametrize("prec", ["df64tc", "df64tc7"])
@pytest.mark.parametrize("n,nrhs", [(67, 1), (1003, 2), (4000, 1)])
def test_df64tc_solve(n, nrhs, prec):
    A, _, _ = inputs.scaled_gaussian(n)
    B = inputs.rhs(n, nrhs)
    X, info = solve(_lib.to_device(A), _lib.to_device(B), depth=2, prec=prec, refine_max=30, tol=1e-13,
                    fallback=False)
    torch.cuda.synchronize()
    assert info["code"] == 0 and info["fell_back"] == 0, info
    assert _bounds.berr(A, _lib.to_host(X), B) <= 1e-13


def test_seven_digit_fallback_ladder():
    """With a tolerance no factorization meets and no refinement steps, a
    seven-digit attempt falls back to eight digits and then to double: all
    three factorizations run (fell_back = 1: X from the double factors), and
    X still solves the system to a double backward error."""
    n = 600
    A, _, _ = inputs.scaled_gaussian(n)
    B = inputs.rhs(n, 1)
    X, info = solve(_lib.to_device(A), _lib.to_device(B), depth=2, prec="df64tc7", refine_max=0, tol=0.0,
                    fallback=True)
    torch.cuda.synchronize()
    assert info["code"] == _lib.RBT_NOT_CONVERGED and info["fell_back"] == 1, info
    assert _bounds.berr(A, _lib.to_host(X), B) <= 1e-13


def test_seven_digit_attempt_stops_at_eight_digits_and_the_adjoint_uses_them():
    """A tolerance between what one refinement step reaches with seven-digit
    factors and with eight-digit ones: the seven-digit attempt is exhausted,
    the eight-digit refactorization of the same A~ meets the tolerance
    (fell_back = 2), and X is bit for bit the plain eight-digit solve's.  The
    adjoint of that solve uses the eight-digit factors: its grad_B is bit for
    bit the plain eight-digit solve's too."""
    from paper_2312_09376_gb300 import autograd
    n = 3000
    for seed in (21, 22, 23, 24):
        A = inputs.scaled_gaussian(n, seed=seed)[0]
        b = inputs.rhs(n, 1, seed=seed + 100)
        Ad, bd = _lib.to_device(A), _lib.to_device(b)
        _, i7 = solve(Ad, bd, depth=2, prec="df64tc7", refine_max=1, tol=0.0, fallback=False)
        _, i8 = solve(Ad, bd, depth=2, prec="df64tc", refine_max=1, tol=0.0, fallback=False)
        if i8["berr"] < 0.25 * i7["berr"]:
            break
    else:
        pytest.fail("no seed separates one seven-digit step from one eight-digit step")
    tol = float(np.sqrt(i8["berr"] * i7["berr"]))
    X8, j8 = solve(Ad, bd, depth=2, prec="df64tc", refine_max=1, tol=tol, fallback=False)
    X, info = solve(Ad, bd, depth=2, prec="df64tc7", refine_max=1, tol=tol, fallback=True)
    torch.cuda.synchronize()
    assert j8["code"] == 0 and info["code"] == 0 and info["fell_back"] == 2, (info, j8, tol)
    assert torch.equal(X, X8) and info["berr"] == j8["berr"]
    W = inputs.rhs(n, 1, seed=seed + 200)
    grads = {}
    for prec in ("df64tc7", "df64tc"):
        Bg = _lib.to_device(b).requires_grad_(True)
        Xg = autograd.solve(_lib.to_device(A), Bg, depth=2, prec=prec, refine_max=1, tol=tol, fallback=True)
        (Xg * _lib.to_device(W)).sum().backward()
        grads[prec] = Bg.grad.clone()
    torch.cuda.synchronize()
    assert torch.equal(grads["df64tc7"], grads["df64tc"])
