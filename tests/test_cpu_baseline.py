"""The timed CPU baseline (tier b: cache-blocked OpenMP FP64, oracle/
rbt_cpu_blocked.c) computes the same method as the plain oracle (tier a).

Criteria: its factors satisfy the elementwise backward-error bound of any LU
computed in double (|A - L U| <= gamma_n |L||U|, Higham Thm. 9.3; a factor 2
for forming L U in numpy) and agree with the oracle's factors to rounding;
its pivot-failure status is the oracle's; its solve reaches the same
backward-error target, with a solution that differs from the oracle's by at
most the conditioning-scaled rounding of two double solves.
"""
import numpy as np
import pytest

import oracle
from paper_2312_09376_gb300 import inputs
from tests import _bounds


def _rbt_matrix(n, d=2, seed=1, a_seed=42):
    A = inputs.gaussian(n, seed=a_seed)
    U, V = oracle.generate(n, d, seed)
    return oracle.transform_2sided(A, U, V, d)


def test_uses_the_host_cores():
    assert oracle.cpu_threads() >= 1


@pytest.mark.parametrize("n,nb", [(0, 64), (1, 64), (5, 2), (129, 64), (300, 128), (1003, 128), (1003, 100),
                                  (700, 256)])
def test_blocked_genp_matches_oracle(n, nb):
    At = _rbt_matrix(max(n, 1))[:n, :n] if n else np.zeros((0, 0))
    LU, st = oracle.cpu_genp(At, nb)
    assert st == -1
    if n == 0:
        return
    L = np.tril(LU, -1) + np.eye(n)
    U = np.triu(LU)
    E = np.abs(At - L @ U)
    assert np.all(E <= 2 * _bounds.gamma(n, _bounds.U64) * (np.abs(L) @ np.abs(U)))
    LUo, sto = oracle.genp(At)
    assert sto == -1
    assert np.abs(LU - LUo).max() <= 1e-8 * np.abs(LUo).max()


def test_blocked_genp_reports_the_oracles_pivot_failures():
    n = 300
    A = inputs.zero_corner(inputs.gaussian(n))
    assert oracle.cpu_genp(A, 64)[1] == oracle.genp(A)[1] == 0
    # exactly singular leading minor inside a later block
    rng = np.random.default_rng(1)
    L = np.tril(rng.standard_normal((n, n)) * 0.01, -1) + np.eye(n)
    U = np.triu(rng.standard_normal((n, n)) * 0.01, 1) + np.eye(n)
    U[150, 150] = 0.0
    U[150, 151:] = 0.0
    M = L @ U
    st_o = oracle.genp(M)[1]
    assert oracle.cpu_genp(M, 64)[1] == st_o
    B = inputs.gaussian(n, seed=3)
    B[:, 200] = np.nan
    assert oracle.cpu_genp(B, 64)[1] == oracle.genp(B)[1] == 200


@pytest.mark.parametrize("n,nrhs,d", [(67, 1, 2), (1003, 2, 2), (2000, 1, 2), (777, 3, 3)])
def test_blocked_solve_matches_oracle(n, nrhs, d):
    A, _, _ = inputs.scaled_gaussian(n)
    B = inputs.rhs(n, nrhs)
    X, st, b0, berr, it, tf, tt = oracle.cpu_rbt_solve(A, B, d, 1)
    Xo, sto, b0o, berro, ito = oracle.rbt_solve(A, B, d, 1)
    assert st == sto == -1
    assert berr <= 1e-13 and berro <= 1e-13
    assert oracle.backward_error(A, X, B) == pytest.approx(berr, rel=1e-6, abs=1e-18)
    # same transform and factorization up to rounding order: first backward
    # errors of the same size, solutions within the conditioning-scaled bound
    assert b0 <= 100 * max(b0o, 1e-16) and b0o <= 100 * max(b0, 1e-16)
    kappa = np.linalg.cond(A, np.inf)
    assert np.abs(X - Xo).max() <= 100 * n * kappa * _bounds.U64 * np.abs(Xo).max()
    assert 0.0 <= tf <= tt
