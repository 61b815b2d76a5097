"""Structure-sensitivity sweep of the generalized RBT (Sec. 6.2, the accuracy
study over matrix sizes): solve without refinement at every multiple of 4
between two multiples of 2^d n_b, with the tiled reference size, and compare
the first backward error of the sizes where the generalized transform has
Parker's recursive structure (n a multiple of 2^d n_b, so m = n and no
butterfly is truncated) against the sizes in between, where it does not.

Host logic only; the solves run through ``paper_2312_09376_gb300.solve``.
"""
from __future__ import annotations

import math
import statistics


def ref_size(n: int, d: int, align: int) -> int:
    """Tiled reference size of Sec. 3: m = 2^d_s a ceil(n / (2^d_s a)), d_s = min(d, ceil(log2 n))."""
    if n <= 0:
        return 0
    ds = min(d, (n - 1).bit_length())          # ceil(log2 n), 0 for n = 1
    p = (2 ** ds) * max(align, 1)
    return p * ((n + p - 1) // p)


def is_parker(n: int, d: int, align: int) -> bool:
    """True where no butterfly of the generalized transform is truncated (m = n)."""
    return ref_size(n, d, align) == n


def sizes(lo: int, hi: int, step: int = 4):
    """lo, lo + step, ..., hi (both ends included when step divides hi - lo)."""
    return list(range(lo, hi + 1, step))


def summarize(results, d: int, align: int):
    """results: iterable of (n, backward error).  Splits them into Parker and
    non-Parker sizes and reports, for the non-Parker ones, the fractions below
    every Parker error and above every Parker error (the comparison of Sec. 6.2),
    with the spread of both groups."""
    parker = [(n, e) for n, e in results if is_parker(n, d, align)]
    other = [(n, e) for n, e in results if not is_parker(n, d, align)]
    if not parker or not other:
        raise ValueError("the sweep needs Parker and non-Parker sizes")
    pe = [e for _, e in parker]
    oe = [e for _, e in other]
    lo, hi = min(pe), max(pe)
    return {
        "parker": {str(n): e for n, e in parker},
        "non_parker_count": len(oe),
        "below_all_parker": sum(e < lo for e in oe) / len(oe),
        "above_all_parker": sum(e > hi for e in oe) / len(oe),
        "non_parker_min": min(oe),
        "non_parker_median": statistics.median(oe),
        "non_parker_max": max(oe),
        "max_over_parker_max": max(oe) / hi if hi > 0 else math.inf,
    }


def summarize_paired(results):
    """results: iterable of (n, backward error with the generalized structure,
    backward error of the same matrix and seed with Parker's structure).  At a
    multiple of 2^d the non-tiled reference size is m = n, where the
    generalized transform is Parker's; the tiled one truncates its
    butterflies.  Reports the fraction of sizes where the generalized form is
    at least as accurate, and the spread of the ratio."""
    rs = [(n, g / p) for n, g, p in results if p > 0]
    if not rs:
        raise ValueError("no paired results")
    ratios = sorted(r for _, r in rs)
    logs = [math.log10(r) for r in ratios]
    return {
        "pairs": len(rs),
        "generalized_not_worse": sum(r <= 1.0 for r in ratios) / len(ratios),
        "ratio_median": statistics.median(ratios),
        "ratio_geomean": 10 ** statistics.fmean(logs),
        "ratio_p10": ratios[int(0.1 * (len(ratios) - 1))],
        "ratio_p90": ratios[int(0.9 * (len(ratios) - 1))],
        "ratio_max": ratios[-1],
        "ratio_min": ratios[0],
    }
