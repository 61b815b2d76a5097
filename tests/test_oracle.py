"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these tests needs a GPU.  Each one checks the oracle against something
other than itself: published generator outputs, the worked example of Sec. 4,
Lemma 1, Theorem 3, closed forms (inverse, orthogonality), explicit dense
matrices assembled from Eq. (O-matrix-definition) and Eq. (rbt-depth-d),
Parker's recursive construction, LAPACK (scipy) factorizations, and a hand
computed backward error.
"""
import itertools
import math
import os

import numpy as np
import pytest
import scipy.linalg

import oracle
from tests import _explicit as ex

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------ generator

def test_splitmix64_published_vectors():
    gamma = 0x9E3779B97F4A7C15
    with open(os.path.join(GOLDEN, "splitmix64.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    for row in rows:
        state = int(row[0])
        for k, want in enumerate(row[1:]):
            # k-th output of a generator started at `state` = mix(state + (k+1) gamma)
            got = oracle.splitmix64((state + k * gamma) % 2**64)
            assert got == int(want), (state, k, got, want)


def test_coefficients_range_and_spread():
    n, d = 4096, 3
    U, V = oracle.generate(n, d, seed=5)
    lo, hi = math.exp(-1 / 20), math.exp(1 / 20)
    for W in (U, V):
        assert np.all(W >= lo) and np.all(W < hi)
        r = 20 * np.log(W)                      # back to r ~ U[-1,1)
        assert abs(r.mean()) < 0.05 and abs(r.var() - 1 / 3) < 0.03
    assert not np.array_equal(U, V)
    assert not np.array_equal(U[:, 0], U[:, 1])
    U2, _ = oracle.generate(n, d, seed=5)
    assert np.array_equal(U, U2)                # deterministic per seed


# ------------------------------------------------- butterfly structure

def _dense_from_oracle(n, d, W, trans):
    """Apply the oracle's one-sided transform to the identity."""
    return oracle.transform_vec(np.eye(n), W, d, trans=trans)


@pytest.mark.parametrize("n", list(range(1, 41)))
def test_structured_matches_explicit_dense(n):
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n))
    for d in range(1, 6):
        U = np.exp(rng.uniform(-1, 1, (n, d)) / 20)
        V = np.exp(rng.uniform(-1, 1, (n, d)) / 20)
        Ud = ex.dense_rbt(n, d, U)
        Vd = ex.dense_rbt(n, d, V)
        want = Ud.T @ A @ Vd
        got = oracle.transform_2sided(A, U, V, d)
        assert np.allclose(got, want, rtol=0, atol=1e-13 * max(1.0, np.abs(want).max())), (n, d)
        assert np.allclose(_dense_from_oracle(n, d, U, False), Ud, rtol=0, atol=1e-14), (n, d)
        assert np.allclose(_dense_from_oracle(n, d, U, True), Ud.T, rtol=0, atol=1e-14), (n, d)


@pytest.mark.parametrize("n,d", [(8, 1), (8, 2), (8, 3), (16, 4), (24, 3), (12, 2), (40, 3), (64, 6)])
def test_generalized_equals_parker_when_power_divides(n, d):
    """Sec. 3: when 2^d divides n every butterfly is a Parker butterfly."""
    rng = np.random.default_rng(100 + n + d)
    W = np.exp(rng.uniform(-1, 1, (n, d)) / 20)
    P = ex.parker_rbt(n, d, W)
    G = _dense_from_oracle(n, d, W, False)
    assert np.allclose(G, P, rtol=0, atol=1e-15)


def _oracle_layer_matrix(n, d, k):
    return oracle.layer_rows(n, d, k, np.eye(n))


@pytest.mark.parametrize("n", [1, 2, 3, 5, 6, 7, 9, 17, 33, 100])
def test_layers_symmetric_and_involutory(n):
    """Eq. (O-matrix-definition): each O is symmetric and orthogonal, so O O = I."""
    for d in (1, 2, 3, 4):
        for k in range(1, d + 1):
            B = _oracle_layer_matrix(n, d, k)
            assert np.allclose(B, B.T, atol=0)
            assert np.allclose(B @ B, np.eye(n), atol=1e-15)
            Bc = oracle.layer_cols(n, d, k, np.eye(n))
            assert np.array_equal(Bc, B)


def test_lemma1_minors_of_single_butterfly():
    """Lemma 1: det O[alpha, gamma] = 0 iff alpha != gamma (mod mu+nu) as
    multisets; otherwise 2^(-|alpha|/2) <= |det| <= 1.  Brute force over every
    pair of index sets for every layer-1 butterfly with n <= 8."""
    seen = set()
    for n in range(2, 9):
        for d in (1, 2, 3):
            O = _oracle_layer_matrix(n, d, 1)
            h = oracle.ref_size(n, d) // 2
            mu, nu = n - h, 2 * h - n
            if mu < 0:
                mu, nu = 0, n
            seen.add((mu, nu))
            assert np.allclose(O, ex.O_block(mu, nu), atol=0)
            mod = mu + nu
            for k in range(1, n + 1):
                for a in itertools.combinations(range(1, n + 1), k):
                    for g in itertools.combinations(range(1, n + 1), k):
                        c = np.linalg.det(O[np.ix_([i - 1 for i in a], [j - 1 for j in g])])
                        cong = sorted(x % mod for x in a) == sorted(x % mod for x in g)
                        if not cong:
                            assert abs(c) < 1e-14, (n, d, a, g, c)
                        else:
                            assert 2 ** (-k / 2) - 1e-12 <= abs(c) <= 1 + 1e-12, (n, d, a, g, c)
    assert {(1, 3), (2, 2), (3, 1), (4, 0)} <= seen


def test_closed_form_inverse():
    """U^{-1} = R_1^{-1} B_1 R_2^{-1} B_2 ... R_d^{-1} B_d since each B_k is its own inverse."""
    for n, d in [(1003 // 17, 2), (37, 3), (64, 3), (5, 4), (100, 1)]:
        rng = np.random.default_rng(n * 7 + d)
        W = np.exp(rng.uniform(-1, 1, (n, d)) / 20)
        U = _dense_from_oracle(n, d, W, False)
        X = np.eye(n)
        for k in range(d, 0, -1):          # rightmost factor B_d acts first
            X = _oracle_layer_matrix(n, d, k) @ X
            X = X / W[:, k - 1][:, None]
        assert np.allclose(X @ U, np.eye(n), atol=1e-13)
        assert np.allclose(U @ X, np.eye(n), atol=1e-13)


def test_orthogonal_when_coefficients_are_one():
    for n, d in [(10, 2), (33, 3), (7, 5), (128, 2)]:
        U = _dense_from_oracle(n, d, np.ones((n, d)), False)
        assert np.allclose(U.T @ U, np.eye(n), atol=1e-14)


def test_worked_example_depth1():
    """Sec. 4, Eq. (example-for-small-d): depth-1 transform of the 4x4 block
    permutation gives the printed matrix (factor 2 -> 1 with normalized O)."""
    with open(os.path.join(GOLDEN, "example_small_depth.txt")) as f:
        lines = [l.split() for l in f if l.strip() and not l.startswith("#")]
    ia, ie = lines.index(["A"]), lines.index(["expect"])
    A = np.array([[float(x) for x in r] for r in lines[ia + 1:ie]])
    expect = lines[ie + 1:]
    r = np.array([0.0, 1.01, 0.97, 1.03, 0.99, 0.96, 1.04, 0.98, 1.02])  # r[1..8]
    U = r[1:5].reshape(4, 1)
    V = r[5:9].reshape(4, 1)
    got = oracle.transform_2sided(A, U, V, 1)
    for i in range(4):
        for j in range(4):
            tok = expect[i][j]
            want = 0.0 if tok == "0" else r[int(tok[1])] * r[int(tok[3])]
            assert got[i, j] == pytest.approx(want, abs=1e-15)
    # and GENP on it stops at the first pivot
    _, st = oracle.genp(got)
    assert st == 0


# ------------------------------------------------------------------ GENP

def test_genp_recovers_known_factors():
    rng = np.random.default_rng(3)
    for n in (1, 2, 7, 64, 150):
        L = np.tril(rng.standard_normal((n, n)) * 0.3, -1) + np.eye(n)
        Uu = np.triu(rng.standard_normal((n, n)) * 0.3, 1) + np.diag(rng.uniform(1, 2, n) * rng.choice([-1, 1], n))
        LU, st = oracle.genp(L @ Uu)
        assert st == -1
        assert np.allclose(np.tril(LU, -1) + np.eye(n), L, atol=1e-10)
        assert np.allclose(np.triu(LU), Uu, atol=1e-10)


def test_genp_matches_lapack_without_swaps():
    """Strict column diagonal dominance: partial pivoting makes no swaps, so
    LAPACK's getrf factors are GENP's."""
    rng = np.random.default_rng(4)
    for n in (5, 50, 200):
        A = rng.standard_normal((n, n))
        A += np.diag(np.abs(A).sum(axis=0) + 1.0)
        lu, piv = scipy.linalg.lu_factor(A)
        assert np.array_equal(piv, np.arange(n))
        LU, st = oracle.genp(A)
        assert st == -1
        assert np.allclose(LU, lu, rtol=1e-13, atol=1e-13)


def test_genp_reports_first_bad_pivot():
    rng = np.random.default_rng(5)
    A = rng.standard_normal((6, 6))
    A[0, 0] = 0.0
    assert oracle.genp(A)[1] == 0
    B = np.array([[1.0, 2.0, 3.0, 1.0], [2.0, 4.0, 1.0, 0.0], [1.0, 0.0, 1.0, 2.0], [0.0, 1.0, 1.0, 1.0]])
    assert oracle.genp(B)[1] == 1                  # 2x2 leading minor is singular
    C = rng.standard_normal((5, 5))
    C[3, 3] = np.nan
    st = oracle.genp(C)[1]
    assert st == 3


def test_genp_solve_both_orientations():
    rng = np.random.default_rng(6)
    n = 80
    A = rng.standard_normal((n, n)) + n * np.eye(n)
    b = rng.standard_normal((n, 3))
    LU, st = oracle.genp(A)
    assert st == -1
    x = oracle.genp_solve(LU, b, trans=False)
    assert np.allclose(A @ x, b, atol=1e-12)
    y = oracle.genp_solve(LU, b, trans=True)
    assert np.allclose(A.T @ y, b, atol=1e-12)


# ------------------------------------------------------- Theorem 3

def _special_matrices(n, rng):
    P = np.eye(n)[rng.permutation(n)]
    J = np.fliplr(np.eye(n))
    Z = rng.standard_normal((n, n))
    Z[0, 0] = 0.0
    return [P, J, Z]


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6, 7, 8, 11, 16])
def test_full_depth_makes_genp_succeed(n):
    """Theorem 3: with depth ceil(log2 n)+1 on both sides, U^T A V is strongly
    nonsingular with probability one, even where GENP on A hits a zero pivot."""
    rng = np.random.default_rng(n)
    d = math.ceil(math.log2(n)) + 1
    for A in _special_matrices(n, rng):
        for seed in range(60):
            U, V = oracle.generate(n, d, seed)
            At = oracle.transform_2sided(A, U, V, d)
            _, st = oracle.genp(At)
            assert st == -1, (n, seed)
            if n <= 8:
                for k in range(1, n + 1):
                    assert abs(np.linalg.det(At[:k, :k])) > 1e-12, (n, seed, k)
    # untransformed GENP fails on the A[0,0] = 0 case
    assert oracle.genp(_special_matrices(n, rng)[2])[1] == 0


def test_depth1_counterexample_fails_for_every_seed():
    """Sec. 4: a depth below ceil(log2 n)+1 guarantees nothing; the block
    permutation stays not strongly nonsingular at depth 1 for any coefficients."""
    A = np.array([[0, 1, 0, 0], [1, 0, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], dtype=float)
    for seed in range(20):
        U, V = oracle.generate(4, 1, seed)
        assert oracle.genp(oracle.transform_2sided(A, U, V, 1))[1] == 0


# -------------------------------------------------- backward error, solve

def test_backward_error_hand_example():
    with open(os.path.join(GOLDEN, "backward_error_2x2.txt")) as f:
        kv = {l.split()[0]: [float(x) for x in l.split()[1:]] for l in f if l.strip() and not l.startswith("#")}
    A = np.array(kv["A"]).reshape(2, 2)
    x = np.array(kv["x"])
    b = np.array(kv["b"])
    assert oracle.backward_error(A, x, b) == kv["berr"][0]


def test_backward_error_properties():
    rng = np.random.default_rng(9)
    A = np.diag([1.0, 2.0, 4.0])
    x = np.array([1.0, -3.0, 0.5])
    assert oracle.backward_error(A, x, A @ x) == 0.0
    A = rng.standard_normal((30, 30))
    x = rng.standard_normal(30)
    b = rng.standard_normal(30)
    e = oracle.backward_error(A, x, b)
    assert e == pytest.approx(oracle.backward_error(8 * A, x, 8 * b), rel=1e-15)
    assert 0 < e <= 1
    X = np.stack([x, 2 * x], axis=1)
    B = np.stack([b, b], axis=1)
    e2 = oracle.backward_error(A, X, B)
    assert e2 == max(oracle.backward_error(A, x, b), oracle.backward_error(A, 2 * x, b))


@pytest.mark.parametrize("n,d", [(1, 2), (2, 1), (67, 2), (200, 2), (203, 3), (256, 1)])
def test_rbt_solve_accuracy(n, d):
    rng = np.random.default_rng(n + d)
    A = rng.standard_normal((n, n))
    if n > 1:
        A[0, 0] = 0.0                              # plain GENP would fail here
    B = rng.standard_normal((n, 2))
    X, st, berr0, berr, it = oracle.rbt_solve(A, B, d, seed=1, refine_max=5, tol=1e-15)
    assert st == -1
    # unrefined RBT+GENP is around 1e-10 at large n in Table 2 (randn); refined to O(eps)
    assert berr <= 1e-15 and berr0 <= 1e-9
    xs = np.linalg.solve(A, B)
    kappa = np.linalg.cond(A, np.inf)
    assert np.abs(X - xs).max() / np.abs(xs).max() <= 100 * n * kappa * 2.2e-16


def test_sizes_rule():
    """Sec. 3 non-tiled rule m = 2^d ceil(n/2^d), with d capped at ceil(log2 n)."""
    assert oracle.ref_size(1003, 2) == 1004
    assert oracle.ref_size(20001, 3) == 20008
    assert oracle.ref_size(40003, 2) == 40004
    assert oracle.ref_size(8197, 2) == 8200
    assert oracle.ref_size(5, 4) == 8 and oracle.depth_eff(5, 4) == 3
    assert oracle.depth_eff(1, 3) == 0 and oracle.ref_size(1, 3) == 1


# ------------------------------------------------- tiled reference size (Sec. 3)

TILED = [(13, 1, 2), (13, 2, 3), (37, 2, 4), (50, 3, 2), (64, 2, 8), (61, 3, 5), (100, 2, 7)]


@pytest.mark.parametrize("n,d,nb", TILED)
def test_tiled_reference_size_aligns_butterflies_to_tiles(n, d, nb):
    """Sec. 3: the tiled rule m = 2^d n_b ceil(n / (2^d n_b)) puts every
    butterfly boundary of every layer on a tile boundary."""
    m = oracle.ref_size(n, d, nb)
    ds = oracle.depth_eff(n, d)
    assert m % (2 ** ds * nb) == 0 and n <= m < n + 2 ** ds * nb
    for k in range(1, ds + 1):
        h = m >> k                      # half size of the layer's butterflies
        assert h % nb == 0
    assert oracle.ref_size(n, d, 1) == oracle.ref_size(n, d)


@pytest.mark.parametrize("n,d,nb", TILED)
def test_tiled_transform_matches_explicit_dense(n, d, nb):
    """Structured tiled transform against explicit butterfly matrices built
    from the block-size recursion with the tiled reference size."""
    rng = np.random.default_rng(n * 31 + d * 7 + nb)
    A = rng.standard_normal((n, n))
    U, V = oracle.generate(n, d, 9)
    got = oracle.transform_2sided(A, U, V, d, align=nb)
    Ue = ex.dense_rbt(n, d, U, align=nb)
    Ve = ex.dense_rbt(n, d, V, align=nb)
    want = Ue.T @ A @ Ve
    scale = np.abs(Ue.T) @ np.abs(A) @ np.abs(Ve)
    assert np.all(np.abs(got - want) <= 1e-13 * scale)
    b = rng.standard_normal((n, 2))
    assert np.allclose(oracle.transform_vec(b, U, d, True, align=nb), Ue.T @ b, rtol=0, atol=1e-13 * n)
    assert np.allclose(oracle.transform_vec(b, V, d, False, align=nb), Ve @ b, rtol=0, atol=1e-13 * n)


@pytest.mark.parametrize("n,d,nb", [(48, 2, 3), (64, 3, 2), (40, 1, 4)])
def test_tiled_equals_non_tiled_when_aligned(n, d, nb):
    """When 2^d n_b divides n both rules give m = n: identical transforms."""
    assert oracle.ref_size(n, d, nb) == n == oracle.ref_size(n, d)
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n))
    U, V = oracle.generate(n, d, 2)
    assert np.array_equal(oracle.transform_2sided(A, U, V, d, align=nb), oracle.transform_2sided(A, U, V, d))


@pytest.mark.parametrize("n,d,nb", [(13, 2, 3), (61, 3, 5)])
def test_tiled_butterflies_orthogonal_with_unit_coefficients(n, d, nb):
    """Each tiled layer is still made of O-blocks (Eq. O-matrix-definition):
    with all random coefficients 1 the transform is orthogonal."""
    M = ex.dense_rbt(n, d, np.ones((n, d)), align=nb)
    assert np.allclose(M.T @ M, np.eye(n), atol=1e-13)
    A = np.eye(n)
    got = oracle.transform_2sided(A, np.ones((n, d)), np.ones((n, d)), d, align=nb)
    assert np.allclose(got, M.T @ M, atol=1e-13)


def test_tiled_solve_accuracy():
    n, d, nb = 301, 2, 16
    rng = np.random.default_rng(21)
    A = rng.standard_normal((n, n))
    B = rng.standard_normal((n, 2))
    X, st, b0, berr, it = oracle.rbt_solve(A, B, d, 1, align=nb)
    assert st == -1 and berr <= 1e-13
    assert oracle.backward_error(A, X, B) == pytest.approx(berr, rel=1e-12)


# ------------------------------------------ communication-free reference size

def test_lcm_textbook_values():
    assert [oracle.lcm(*pq) for pq in [(1, 1), (1, 7), (4, 4), (4, 6), (2, 3), (12, 18), (5, 1)]] == \
        [1, 7, 4, 12, 6, 36, 5]


@pytest.mark.parametrize("d", [1, 2, 3])
def test_comm_free_size_on_one_process_is_the_tiled_rule(d):
    """Eq. (comm-free-rbt-size) with p = q = 1 is the tiled rule of Sec. 3:
    the top half of the first layer is 2^(d-1) ceil(n_t 2^-d) tiles."""
    for nb in (1, 3, 16, 64):
        for n in range(1, 400, 7):
            assert oracle.ref_size_comm_free(n, d, nb, 1, 1) == oracle.ref_size(n, d, nb)


@pytest.mark.parametrize("p,q", [(4, 4), (2, 3), (1, 4), (3, 6), (8, 2)])
def test_comm_free_size_is_the_tiled_rule_with_lcm_tiles(p, q):
    """ceil(ceil(n / n_b) / c) = ceil(n / (n_b c)): the rule equals the tiled
    rule with tiles of lcm(p, q) n_b rows."""
    l = math.lcm(p, q)
    for d in (1, 2, 3):
        for nb in (1, 2, 5, 32):
            for n in range(1, 700, 13):
                m = oracle.ref_size_comm_free(n, d, nb, p, q)
                assert m == oracle.ref_size(n, d, nb * l)
                ds = oracle.depth_eff(n, d)
                assert n <= m and m % (2 ** ds * nb * l) == 0


def _pairs(n, d, align):
    """Row pairs (i, j), i < j, that some butterfly layer combines, from the
    explicit layer matrices of the block-size recursion."""
    out = []
    for blocks in ex.layer_blocks(n, d, align):
        B = ex.layer_matrix(n, blocks)
        ii, jj = np.nonzero(np.triu(B, 1))
        out.extend(zip(ii.tolist(), jj.tolist()))
    return out


def _comm_free(pairs, nb, p, q):
    """True when no butterfly pair crosses process rows (tile row mod p) or,
    for the column butterflies of V, process columns (tile column mod q)."""
    return all((i // nb) % p == (j // nb) % p and (i // nb) % q == (j // nb) % q for i, j in pairs)


@pytest.mark.parametrize("n,d,nb,p,q", [(37, 2, 2, 2, 2), (61, 2, 3, 4, 4), (100, 3, 2, 2, 3), (45, 1, 4, 3, 2),
                                        (130, 2, 4, 4, 2), (97, 3, 1, 3, 3)])
def test_comm_free_size_keeps_every_butterfly_on_one_process(n, d, nb, p, q):
    """Brute force on a p x q block-cyclic grid of n_b x n_b tiles: with the
    reference size of Eq. (comm-free-rbt-size) every pair of every layer
    lies in one tile row class mod p and one tile column class mod q, and
    the transform is still the product of explicit O-block layers."""
    l = math.lcm(p, q)
    m = oracle.ref_size_comm_free(n, d, nb, p, q)
    assert m == oracle.ref_size(n, d, nb * l)
    pairs = _pairs(n, d, nb * l)
    assert pairs                                    # the layers do pair rows
    assert _comm_free(pairs, nb, p, q)
    rng = np.random.default_rng(n + 7 * d)
    A = rng.standard_normal((n, n))
    U, V = oracle.generate(n, d, 3)
    got = oracle.transform_2sided(A, U, V, d, align=nb * l)
    Ue, Ve = ex.dense_rbt(n, d, U, align=nb * l), ex.dense_rbt(n, d, V, align=nb * l)
    assert np.all(np.abs(got - Ue.T @ A @ Ve) <= 1e-13 * (np.abs(Ue.T) @ np.abs(A) @ np.abs(Ve)))


def test_tiled_rule_on_a_4x4_grid_is_comm_free_iff_tile_count_divisible_by_4():
    """Sec. 6 (Performance) on its 4 x 4 grid: with the tiled rule no
    communication is needed if and only if ceil(n_t 2^-d) is divisible by 4.
    Brute force over the number of tile rows n_t, d = 2, 2-row tiles."""
    d, nb, p = 2, 2, 4
    seen = set()
    for nt in range(5, 70):
        n = nt * nb - 1                               # a ragged last tile
        free = _comm_free(_pairs(n, d, nb), nb, p, p)
        assert free == ((-(-nt // 2 ** d)) % 4 == 0), nt
        seen.add(free)
        # the communication-free size never communicates
        assert _comm_free(_pairs(n, d, nb * p), nb, p, p)
    assert seen == {True, False}


# --------------------------------------------------------------- GMRES-IR

def _system(n, d, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n))
    b = rng.standard_normal(n)
    U, V = oracle.generate(n, d, seed)
    At = oracle.transform_2sided(A, U, V, d)
    LU, st = oracle.genp(At)
    assert st == -1
    return A, b, U, V, LU


def test_gmres_ir_with_exact_preconditioner_takes_one_step():
    """With the double factors M^{-1} = A^{-1} up to rounding: the Krylov
    space of A M^{-1} r is one-dimensional, one or two products suffice."""
    n, d = 150, 2
    A, b, U, V, LU = _system(n, d, 3)
    x, b_in, berr, used, cycles, hist = oracle.gmres_ir(A, b, U, V, d, LU, np.zeros(n))
    assert b_in == 1.0 and berr <= 1e-13 and used <= 3 and cycles == 1


def test_gmres_ir_unpreconditioned_is_plain_gmres():
    """d = 0 and identity factors: GMRES itself.  In exact arithmetic it
    terminates within n steps; its residual estimate never increases."""
    n = 40
    rng = np.random.default_rng(8)
    A = rng.standard_normal((n, n)) + 4 * np.eye(n)
    b = rng.standard_normal(n)
    I = np.eye(n)
    x, b_in, berr, used, cycles, hist = oracle.gmres_ir(A, b, np.ones((n, 0)), np.ones((n, 0)), 0, I, np.zeros(n),
                                                        restart=n + 5, max_iter=n + 5)
    assert berr <= 1e-13 and used <= n and cycles == 1
    assert np.all(np.diff(hist) <= 1e-12 * hist[0])
    assert np.allclose(A @ x, b, atol=1e-10)


def test_gmres_ir_recovers_where_stationary_refinement_stalls():
    """Factors with a relative perturbation of 1e-3 (a low working precision
    times growth): stationary refinement x += M^{-1} (b - A x) diverges,
    GMRES-IR reaches the double backward-error target."""
    n, d = 300, 2
    A, b, U, V, LU = _system(n, d, 5)
    rng = np.random.default_rng(9)
    LUp = LU * (1 + 1e-3 * rng.standard_normal(LU.shape))

    def minv(r):
        z = oracle.transform_vec(r, U, d, True)
        z = oracle.genp_solve(LUp, z)
        return oracle.transform_vec(z, V, d, False)

    x = minv(b)
    for _ in range(10):
        x = x + minv(b - A @ x)
    stationary = oracle.backward_error(A, x.reshape(-1, 1), b.reshape(-1, 1))
    xg, b_in, berr, used, cycles, _ = oracle.gmres_ir(A, b, U, V, d, LUp, minv(b), restart=30, max_iter=120)
    assert berr <= 1e-13 < stationary
    assert oracle.backward_error(A, xg.reshape(-1, 1), b.reshape(-1, 1)) == pytest.approx(berr, rel=1e-12)


# ------------------------------------------------- rotation butterflies

ROT_CASES = [(n, d, a) for n in (1, 2, 3, 5, 8, 13, 17, 31, 64, 67) for d in (1, 2, 3, 4) for a in (1, 3)]


def _u_from_splitmix(seed, side, layer, i):
    """The uniform of the pair's angle, recomputed from the pinned SplitMix64 (golden vectors)."""
    key = (seed ^ (side << 62) ^ (layer << 48) ^ i) & (2**64 - 1)
    return (oracle.splitmix64(key) >> 11) * 2.0 ** -53


@pytest.mark.parametrize("n,d,align", [(13, 3, 1), (67, 4, 3), (64, 2, 1), (1003, 3, 64)])
def test_rot_generator_angles_and_identity_rows(n, d, align):
    """Each pair holds (cos 2 pi u, sin 2 pi u) at its (top, bottom) rows with u
    the counter's uniform for (seed, side, layer, top row); nu rows and layers
    past the effective depth hold exactly 1."""
    seed = 77
    U, V = oracle.generate_rot(n, d, seed, align=align)
    for side, W in ((0, U), (1, V)):
        for k, (pairs, nus) in enumerate(ex.rot_pairs(n, d, align), start=1):
            for i in nus:
                assert W[i, k - 1] == 1.0
            paired = set()
            for top, bot in pairs:
                c, s = W[top, k - 1], W[bot, k - 1]
                assert abs(c * c + s * s - 1.0) <= 4 * 2.0 ** -53
                th = math.atan2(s, c) % (2 * math.pi)
                want = 2 * math.pi * _u_from_splitmix(seed, side, k, top)
                diff = abs(th - want)
                assert min(diff, 2 * math.pi - diff) <= 1e-14, (k, top, th, want)
                paired |= {top, bot}
            if not pairs:
                assert np.all(W[:, k - 1] == 1.0)
            assert paired | set(nus) == set(range(n)) or not pairs


@pytest.mark.parametrize("n,d,align", ROT_CASES)
def test_rot_transform_matches_explicit(n, d, align):
    """U^T A V and the one-sided transforms against dense products of the
    block-rotation butterflies built from the block-size recursion."""
    rng = np.random.default_rng(n * 10 + d)
    A = rng.standard_normal((n, n))
    B = rng.standard_normal((n, 2))
    U, V = oracle.generate_rot(n, d, 5, align=align)
    Ud = ex.dense_rot_rbt(n, d, U, align)
    Vd = ex.dense_rot_rbt(n, d, V, align)
    np.testing.assert_allclose(oracle.transform_2sided_rot(A, U, V, d, align=align), Ud.T @ A @ Vd,
                               rtol=0, atol=1e-13 * max(1.0, np.abs(A).max()))
    np.testing.assert_allclose(oracle.transform_vec_rot(B, U, d, True, align=align), Ud.T @ B, rtol=0, atol=1e-13)
    np.testing.assert_allclose(oracle.transform_vec_rot(B, U, d, False, align=align), Ud @ B, rtol=0, atol=1e-13)


@pytest.mark.parametrize("n,d", [(7, 3), (40, 2), (129, 4), (1000, 3)])
def test_rot_orthogonal(n, d):
    """R_k = I and C^2 + S^2 = I make the transform orthogonal: U^T U = I and
    ||U^T A V||_F = ||A||_F."""
    U, V = oracle.generate_rot(n, d, 3)
    Ud = oracle.transform_vec_rot(np.eye(n), U, d, False)
    assert np.abs(Ud.T @ Ud - np.eye(n)).max() <= 8 * d * 2.0 ** -53
    A = np.random.default_rng(1).standard_normal((n, n))
    At = oracle.transform_2sided_rot(A, U, V, d)
    assert abs(np.linalg.norm(At) - np.linalg.norm(A)) <= 1e-13 * np.linalg.norm(A)
    # the one-sided transforms invert each other
    Bv = np.random.default_rng(2).standard_normal((n, 3))
    back = oracle.transform_vec_rot(oracle.transform_vec_rot(Bv, U, d, True), U, d, False)
    assert np.abs(back - Bv).max() <= 1e-13


def test_rot_depth1_two_rows_closed_form():
    """n = 2, d = 1: U = [[c, s], [s, -c]] with angle 2 pi u of (seed, side 0, layer 1, row 0)."""
    U, V = oracle.generate_rot(2, 1, 9)
    th = 2 * math.pi * _u_from_splitmix(9, 0, 1, 0)
    c, s = math.cos(th), math.sin(th)
    A = np.array([[1.0, 2.0], [3.0, 4.0]])
    Uf = np.array([[c, s], [s, -c]])
    th_v = 2 * math.pi * _u_from_splitmix(9, 1, 1, 0)
    Vf = np.array([[math.cos(th_v), math.sin(th_v)], [math.sin(th_v), -math.cos(th_v)]])
    np.testing.assert_allclose(oracle.transform_2sided_rot(A, U, V, 1), Uf.T @ A @ Vf, rtol=0, atol=1e-14)


def test_rot_solve_zero_leading_pivot():
    """A zero leading pivot stops GENP; after the rotation transform the
    system is solved and refined to the target."""
    n = 200
    rng = np.random.default_rng(8)
    A = rng.standard_normal((n, n))
    A[0, 0] = 0.0
    B = rng.standard_normal((n, 2))
    _, st = oracle.genp(A)
    assert st == 0
    X, st, b0, b, it = oracle.rbt_solve(A, B, 2, seed=4, kind="rotation")
    assert st == -1 and b <= 1e-13
    assert oracle.backward_error(A, X, B) <= 1e-13


def test_gmres_ir_uses_the_tiled_reference_size():
    """Exact factors of the tiled transform (n_b = 8): GMRES-IR with the same
    alignment converges at once; with the non-tiled rule the one-sided
    transforms no longer match the factors and it needs many more products."""
    n, d, nb = 150, 2, 8
    rng = np.random.default_rng(12)
    A = rng.standard_normal((n, n))
    b = rng.standard_normal(n)
    U, V = oracle.generate(n, d, 1)
    assert oracle.ref_size(n, d, nb) != oracle.ref_size(n, d)
    LU, st = oracle.genp(oracle.transform_2sided(A, U, V, d, align=nb))
    assert st == -1
    _, _, berr, used, _, _ = oracle.gmres_ir(A, b, U, V, d, LU, np.zeros(n), align=nb)
    assert berr <= 1e-13 and used <= 5
    _, _, berr1, used1, _, _ = oracle.gmres_ir(A, b, U, V, d, LU, np.zeros(n), max_iter=60)
    assert used1 == 60 and berr1 > 1e-3


# ------------------------------------------------- residual, norms, generator scalars

def test_residual_exact_on_small_integers():
    """B - A X on small integers is exact in double: compared entry by entry
    with the integer computation (a sign, index or transposition slip shows)."""
    rng = np.random.default_rng(21)
    n, k = 7, 3
    A = rng.integers(-9, 10, (n, n)).astype(np.int64)
    X = rng.integers(-9, 10, (n, k)).astype(np.int64)
    B = rng.integers(-99, 100, (n, k)).astype(np.int64)
    R = oracle.residual(A.astype(float), X.astype(float), B.astype(float))
    assert np.array_equal(R, (B - A @ X).astype(float))


def test_residual_rounding_bound():
    """|fl(B - A X) - (B - A X)| <= gamma_{n+1} (|A| |X| + |B|) (Higham, Eq. 3.5), the
    exact value formed in long integer arithmetic from integer-scaled inputs."""
    rng = np.random.default_rng(22)
    n = 60
    A = rng.integers(-2**20, 2**20, (n, n)) / 2.0**10
    X = rng.integers(-2**20, 2**20, (n, 2)) / 2.0**10
    B = rng.integers(-2**20, 2**20, (n, 2)) / 2.0**10
    R = oracle.residual(A, X, B)
    exact = (np.round(B * 2**20).astype(object) - (np.round(A * 2**10).astype(object) @ np.round(X * 2**10).astype(object)))
    exact = np.array(exact, dtype=float) / 2.0**20
    gam = (n + 1) * 2.0**-53 / (1 - (n + 1) * 2.0**-53)
    assert np.all(np.abs(R - exact) <= gam * (np.abs(A) @ np.abs(X) + np.abs(B)))


def test_norm_inf_is_max_row_sum():
    """||A||_inf = max_i sum_j |a_ij| (rows, not columns: the example's row and
    column maxima differ)."""
    A = np.array([[1.0, -2.0, 3.0], [-4.0, 0.0, 0.5], [0.0, 7.0, -1.0]])
    assert oracle.norm_inf_mat(A) == 8.0          # row 3 sums to 8; the largest column sum is 9
    assert oracle.norm_inf_mat(A.T) == 9.0


def test_coef_and_ceil_log2_from_their_definitions():
    """coef = exp((2u - 1)/20) with u the top 53 bits of the golden-vector
    SplitMix64 output for the key (seed, side, layer, row); ceil_log2 exact."""
    for seed, side, layer, i in [(0, 0, 1, 0), (42, 1, 2, 999), (2**63 + 5, 0, 7, 123456), (1, 1, 62, 3)]:
        key = (seed ^ (side << 62) ^ (layer << 48) ^ i) & (2**64 - 1)
        u = (oracle.splitmix64(key) >> 11) * 2.0**-53
        assert oracle.coef(seed, side, layer, i) == math.exp((2 * u - 1) / 20)
        assert math.exp(-1 / 20) <= oracle.coef(seed, side, layer, i) <= math.exp(1 / 20)
        assert oracle.rot_u(seed, side, layer, i) == u
    for n in list(range(1, 70)) + [1000, 1024, 1025, 40003, 2**31, 2**31 + 1]:
        assert oracle.ceil_log2(n) == (n - 1).bit_length()
