"""Error bounds used by the parity tests (test code; no method arithmetic is
shared with either side).

* ``abs_transform_bound``: (|U|^T |A| |V|)_ij, the natural scale of the
  rounding error of any evaluation order of U^T A V, from the explicit dense
  factors (small n only).
* ``group_bound``: a cheaper elementwise upper bound of the same quantity for
  large n.  Row i of U^T has its nonzeros inside i's group of 2^d rows (the
  rows i' = i mod q congruent under the butterfly pairing), each of magnitude
  at most e^(d/20); so (|U|^T|A||V|)_ij <= e^(2d/20) * sum of |A| over the
  2^d x 2^d group holding (i, j).
* ``berr``: the normwise backward error of a device result.
* ``gamma(n, u)``: n u / (1 - n u), the constant of the standard backward
  error bounds of LU and dot products (Higham, Accuracy and Stability of
  Numerical Algorithms, Thm. 9.3 and Eq. 3.5).
"""
from __future__ import annotations

import math

import numpy as np

from tests import _explicit as ex

U64 = 2.0 ** -53
U32 = 2.0 ** -24


def gamma(n, u):
    return n * u / (1 - n * u)


def abs_transform_bound(A, U, V, d, align=1):
    n = A.shape[0]
    Ud = np.abs(ex.dense_rbt(n, d, U, align))
    Vd = np.abs(ex.dense_rbt(n, d, V, align))
    return Ud.T @ np.abs(A) @ Vd


def group_bound(A, d, align=1):
    """align = n_b: the groups of the tiled reference size (q = m / 2^d_s)."""
    n = A.shape[0]
    ds = ex.eff_depth(n, d)
    p = (2 ** ds) * max(1, align)
    m = p * math.ceil(n / p)
    q = m // (2 ** ds)
    g = 2 ** ds
    P = np.zeros((m, m))
    P[:n, :n] = np.abs(A)
    # group of (i, j) = (i mod q, j mod q); sum over the g x g members
    S = P.reshape(q, g, q, g, order="F").sum(axis=(1, 3))   # [i0, j0], i = i0 + q s
    B = np.tile(S, (g, g))[:n, :n]
    return math.exp(2 * d / 20) * B


def berr(A, X, B):
    """Normwise backward error of a computed solution, the largest over the
    columns of ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf) (Rigal and
    Gaches; the refinement's stopping quantity in Sec. 5), in plain numpy:
    the tests measure device results with this, never with the oracle."""
    A = np.asarray(A, dtype=np.float64)
    X = np.asarray(X, dtype=np.float64).reshape(A.shape[0], -1)
    B = np.asarray(B, dtype=np.float64).reshape(A.shape[0], -1)
    if A.shape[0] == 0 or X.shape[1] == 0:
        return 0.0
    an = np.abs(A).sum(axis=1).max()
    R = np.abs(B - A @ X).max(axis=0)
    den = an * np.abs(X).max(axis=0) + np.abs(B).max(axis=0)
    return float(np.max(np.where(den > 0, R / np.where(den > 0, den, 1.0), np.where(R > 0, np.inf, 0.0))))
