"""Seeded synthetic inputs shared by the CUDA path's tests, the oracle's tests and the benchmark.

This module holds no arithmetic of the method: it only draws matrices and
right-hand sides with numpy's PCG64 generator, so that the GPU path and the CPU
oracle see identical bytes.

The paper evaluates on generated matrices (Sec. 6: the SLATE generator with
``--seed 42 --seedB 64``); the stand-ins here follow that: the system matrix is
drawn from seed 42 and the right-hand sides from seed 64 unless stated
otherwise.  Distributions:

* ``gaussian``          -- i.i.d. N(0, 1) (the ``randn`` analogue);
* ``scaled_gaussian``   -- D_r G D_c with G i.i.d. N(0,1) and diagonal entries
                           10^U(-1.5, 1.5) (seeds 43, 44 for D_r, D_c), a
                           stress case for mixed-precision refinement;
* ``batch_sizes``       -- uniform integer orders for batched solves;
* ``device_system``     -- the same families drawn on a CUDA device with
                           torch's generator, for sizes (n = 40003: 12.8 GB)
                           that should not pass through host memory.
"""
from __future__ import annotations

import numpy as np

SEED_A = 42
SEED_B = 64
SEED_DR = 43
SEED_DC = 44
SEED_RBT = 1


def gaussian(n: int, m: int | None = None, seed: int = SEED_A) -> np.ndarray:
    """n x m (default n x n) column-major float64 matrix with i.i.d. N(0,1) entries."""
    m = n if m is None else m
    g = np.random.Generator(np.random.PCG64(seed))
    # draw column by column so that column-major storage is filled in order
    return np.asfortranarray(g.standard_normal((m, n)).T)


def rhs(n: int, nrhs: int = 1, seed: int = SEED_B) -> np.ndarray:
    return gaussian(n, nrhs, seed)


def scaled_gaussian(n: int, seed: int = SEED_A, seed_r: int = SEED_DR, seed_c: int = SEED_DC):
    """Return (A, dr, dc) with A = diag(dr) G diag(dc)."""
    G = gaussian(n, seed=seed)
    dr = 10.0 ** np.random.Generator(np.random.PCG64(seed_r)).uniform(-1.5, 1.5, n)
    dc = 10.0 ** np.random.Generator(np.random.PCG64(seed_c)).uniform(-1.5, 1.5, n)
    A = np.asfortranarray(G * dr[:, None] * dc[None, :])
    return A, dr, dc


def batch_sizes(count: int, lo: int, hi: int, seed: int = 7) -> np.ndarray:
    """Uniform integer sizes in [lo, hi] (inclusive)."""
    g = np.random.Generator(np.random.PCG64(seed))
    return g.integers(lo, hi + 1, size=count).astype(np.int64)


def batch_nrhs(count: int, lo: int = 1, hi: int = 8, seed: int = 8) -> np.ndarray:
    g = np.random.Generator(np.random.PCG64(seed))
    return g.integers(lo, hi + 1, size=count).astype(np.int64)


def zero_corner(A: np.ndarray) -> np.ndarray:
    """Copy of A with A[0,0] = 0 (untransformed GENP then fails at its first pivot)."""
    B = np.array(A, order="F", copy=True)
    B[0, 0] = 0.0
    return B


def device_system(n: int, scaled: bool = True, seed: int = SEED_A, device="cuda"):
    """(A, b) on a CUDA device: A column-major (a transposed view, lda = n),
    i.i.d. N(0,1), times D_r and D_c with entries 10^U(-1.5, 1.5) when
    ``scaled``; b i.i.d. N(0,1).  Drawn from one torch generator seeded with
    ``seed``, column block by column block to keep temporaries small."""
    import torch

    dev = torch.device(device)
    g = torch.Generator(device=dev).manual_seed(seed)
    A = torch.empty((n, n), dtype=torch.float64, device=dev)
    for c0 in range(0, n, 4096):
        A[c0:min(n, c0 + 4096)].normal_(generator=g)
    A = A.T
    dr = torch.pow(10.0, torch.rand(n, generator=g, device=dev, dtype=torch.float64) * 3 - 1.5)
    dc = torch.pow(10.0, torch.rand(n, generator=g, device=dev, dtype=torch.float64) * 3 - 1.5)
    if scaled:
        A.mul_(dr[:, None]).mul_(dc[None, :])
    b = torch.randn(n, generator=g, device=dev, dtype=torch.float64)
    return A, b
