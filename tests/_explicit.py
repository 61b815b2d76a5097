"""Explicit dense butterfly matrices, built straight from the paper's definitions.

Used only to pin the structured oracle (and, through it, the GPU path).  Nothing
here shares code with ``oracle/`` or with the CUDA sources: the block sizes come
from the recursive alignment rule, each block from Eq. (O-matrix-definition),
and U from the product of Eq. (rbt-depth-d), all as dense numpy matrices.
"""
from __future__ import annotations

import math

import numpy as np


def O_block(mu: int, nu: int) -> np.ndarray:
    """Eq. (O-matrix-definition): [[I/r2, 0, I/r2], [0, I_nu, 0], [I/r2, 0, -I/r2]]."""
    m = 2 * mu + nu
    O = np.zeros((m, m))
    s = 1.0 / math.sqrt(2.0)
    for i in range(mu):
        O[i, i] = s
        O[i, mu + nu + i] = s
        O[mu + nu + i, i] = s
        O[mu + nu + i, mu + nu + i] = -s
    for i in range(nu):
        O[mu + i, mu + i] = 1.0
    return O


def eff_depth(n: int, d: int) -> int:
    return min(d, max(0, math.ceil(math.log2(n))) if n > 1 else 0)


def layer_blocks(n: int, d: int, align: int = 1):
    """Block sizes (mu, nu) of every layer 1..d via Eq. (butterfly-alignment).

    Layer 1 is one butterfly on all n rows.  A block of size l whose Parker
    slot is S (S = m / 2^(k-1) at layer k) has a top part of min(l, S/2) rows;
    mu = l - top bottom rows pair with the first mu top rows, nu = top - mu
    rows pass through.  The children are the top part and the bottom part,
    each in a slot of S/2 (l_{k+1,2j} = mu + nu, l_{k+1,2j+1} = mu).
    Layers past the effective depth hold blocks of size one (identity).
    """
    ds = eff_depth(n, d)
    p = (2 ** ds) * align           # align = n_b: the tiled reference size of Sec. 3
    m = p * math.ceil(n / p) if n > 0 else 0
    layers = []
    blocks = [(n, m)]  # (size, slot)
    for k in range(1, d + 1):
        if k > ds:
            layers.append([(0, 1)] * n)
            continue
        this, nxt = [], []
        for size, slot in blocks:
            if size == 0:
                continue
            top = min(size, slot // 2)
            mu = size - top
            nu = top - mu
            this.append((mu, nu))
            if top > 0:
                nxt.append((top, slot // 2))
            if mu > 0:
                nxt.append((mu, slot // 2))
        layers.append(this)
        blocks = nxt
    return layers


def layer_matrix(n: int, blocks) -> np.ndarray:
    B = np.zeros((n, n))
    o = 0
    for mu, nu in blocks:
        s = 2 * mu + nu
        B[o:o + s, o:o + s] = O_block(mu, nu)
        o += s
    assert o == n, (o, n, blocks)
    return B


def dense_rbt(n: int, d: int, W: np.ndarray, align: int = 1) -> np.ndarray:
    """Eq. (rbt-depth-d): W = B_d R_d ... B_1 R_1 with R_k = diag(W[:, k-1])."""
    M = np.eye(n)
    for k, blocks in enumerate(layer_blocks(n, d, align), start=1):
        M = layer_matrix(n, blocks) @ np.diag(W[:, k - 1]) @ M
    return M


def parker_rbt(n: int, d: int, W: np.ndarray, col: int = 0) -> np.ndarray:
    """Parker's recursive RBT of depth d on n = 2^d * q rows.

    Parker's butterfly B^<n> = 1/sqrt(2) [[R0, R1], [R0, -R1]], and a depth-d
    transform is diag(W_top, W_bot) B^<n> with depth-(d-1) transforms on each
    half.  Column ``col`` of W holds this layer's diagonal.
    """
    if d == 0:
        return np.eye(n)
    h = n // 2
    R0 = np.diag(W[:h, col])
    R1 = np.diag(W[h:, col])
    B = np.block([[R0, R1], [R0, -R1]]) / math.sqrt(2.0)
    top = parker_rbt(h, d - 1, W[:h], col + 1)
    bot = parker_rbt(h, d - 1, W[h:], col + 1)
    Z = np.zeros((h, h))
    return np.block([[top, Z], [Z, bot]]) @ B


def rot_block(C: np.ndarray, S: np.ndarray, nu: int) -> np.ndarray:
    """The block-rotation butterfly of Sec. 3: [[C, 0, S], [0, I_nu, 0], [S, 0, -C]]
    with C = diag(C), S = diag(S) (mu = len(C) pairs)."""
    mu = len(C)
    m = 2 * mu + nu
    B = np.zeros((m, m))
    B[:mu, :mu] = np.diag(C)
    B[:mu, mu + nu:] = np.diag(S)
    B[mu:mu + nu, mu:mu + nu] = np.eye(nu)
    B[mu + nu:, :mu] = np.diag(S)
    B[mu + nu:, mu + nu:] = -np.diag(C)
    return B


def dense_rot_rbt(n: int, d: int, W: np.ndarray, align: int = 1) -> np.ndarray:
    """W = B_d ... B_1 (R_k = I), B_k block diagonal with rotation butterflies on
    the block sizes of the alignment rule; each block's C comes from the packed
    column k-1 at its top rows, S at its bottom rows."""
    M = np.eye(n)
    for k, blocks in enumerate(layer_blocks(n, d, align), start=1):
        B = np.zeros((n, n))
        o = 0
        for mu, nu in blocks:
            sz = 2 * mu + nu
            B[o:o + sz, o:o + sz] = rot_block(W[o:o + mu, k - 1], W[o + mu + nu:o + sz, k - 1], nu)
            o += sz
        assert o == n
        M = B @ M
    return M


def rot_pairs(n: int, d: int, align: int = 1):
    """For every layer k (1-based) the (top, bottom) row pairs and the nu rows, from the block sizes."""
    out = []
    for blocks in layer_blocks(n, d, align):
        pairs, nus = [], []
        o = 0
        for mu, nu in blocks:
            pairs += [(o + i, o + mu + nu + i) for i in range(mu)]
            nus += [o + mu + i for i in range(nu)]
            o += 2 * mu + nu
        out.append((pairs, nus))
    return out
