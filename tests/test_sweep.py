"""Host logic of the structure-sensitivity sweep: the Parker classification
against the oracle's tiled reference size, and the summary statistics."""
import pytest

import oracle
from paper_2312_09376_gb300 import sweep


@pytest.mark.parametrize("n", [20480, 20484, 21000, 22016, 22528, 1, 2, 3, 2048, 2052, 4096])
@pytest.mark.parametrize("d,align", [(2, 512), (2, 1), (3, 64)])
def test_ref_size_matches_oracle(n, d, align):
    assert sweep.ref_size(n, d, align) == oracle.ref_size(n, d, align)


def test_parker_sizes_of_the_paper_sweep():
    """With tiles of 512 rows and d = 2 only the multiples of 2048 in
    [20480, 22528] keep Parker's structure (the two ends of the sweep)."""
    s = sweep.sizes(20480, 22528, 4)
    assert len(s) == 513 and s[0] == 20480 and s[-1] == 22528
    assert [n for n in s if sweep.is_parker(n, 2, 512)] == [20480, 22528]
    # with the non-tiled rule every multiple of 4 would be a Parker size
    assert all(sweep.is_parker(n, 2, 1) for n in s)


def test_summarize():
    res = [(20480, 2e-16), (20484, 1e-16), (20488, 3e-16), (20492, 5e-16), (22528, 4e-16)]
    out = sweep.summarize(res, 2, 512)
    assert out["non_parker_count"] == 3
    assert out["below_all_parker"] == pytest.approx(1 / 3)
    assert out["above_all_parker"] == pytest.approx(1 / 3)
    assert out["non_parker_median"] == 3e-16
    assert out["max_over_parker_max"] == pytest.approx(1.25)
    with pytest.raises(ValueError):
        sweep.summarize(res[1:4], 2, 512)


def test_summarize_paired():
    res = [(20484, 1e-16, 2e-16), (20488, 4e-16, 2e-16), (20492, 3e-16, 3e-16), (20496, 1e-15, 1e-16)]
    out = sweep.summarize_paired(res)
    assert out["pairs"] == 4
    assert out["generalized_not_worse"] == 0.5
    assert out["ratio_median"] == pytest.approx(1.5)
    assert out["ratio_max"] == pytest.approx(10.0) and out["ratio_min"] == pytest.approx(0.5)
    assert out["ratio_geomean"] == pytest.approx((0.5 * 2 * 1 * 10) ** 0.25)
