"""The structure-sensitivity sweep at small sizes: tile 128 and d = 2 make
the multiples of 512 the Parker sizes; every size between them solves (no
zero pivot), and the first backward error of the device solve is that of the
oracle's transform and GENP with the same tiled reference size up to
rounding order (within a factor 10 either way)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2312_09376_gb300 import _lib, inputs, solve, sweep

pytestmark = pytest.mark.gpu


def test_sweep_small_sizes_against_oracle():
    d, tile = 2, 128
    ns = sweep.sizes(1024, 1536, 32)
    res = []
    for n in ns:
        A = inputs.gaussian(n, seed=n)
        b = inputs.rhs(n, 1, seed=n + 1)
        _, info = solve(_lib.to_device(A), _lib.to_device(b), depth=d, seed=1, prec="f64", refine_max=0,
                        fallback=False, align=tile)
        torch.cuda.synchronize()
        assert info["code"] in (0, 3) and info["zero_pivot"] == -1, (n, info)
        res.append((n, info["berr_unrefined"]))
        if n in (1024, 1056, 1536):
            _, st, b0, _, _ = oracle.rbt_solve(A, b, d, seed=1, refine_max=0, tol=0.0, align=tile)
            g = info["berr_unrefined"]
            assert st == -1 and g <= 10 * b0 + 1e-16 and b0 <= 10 * g + 1e-16, (n, g, b0)
    out = sweep.summarize(res, d, tile)
    assert set(out["parker"]) == {"1024", "1536"} and out["non_parker_count"] == len(ns) - 2
    assert np.isfinite(out["non_parker_max"]) and out["non_parker_max"] < 1e-8
