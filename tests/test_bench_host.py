"""Host helpers of bench.py: the confidence interval of the step times, the
traffic record lookup (null once the recorded source changed) and the flop
count of the metric."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_ci99(bench):
    # mean 3, sample s.d. sqrt(2.5), t(0.995; 4) = 4.604095 (Student t table)
    lo, hi = bench.ci99([1.0, 2.0, 3.0, 4.0, 5.0])
    h = 4.604095 * 2.5 ** 0.5 / 5 ** 0.5
    assert lo == pytest.approx(3 - h, rel=1e-6) and hi == pytest.approx(3 + h, rel=1e-6)
    assert bench.ci99([7.0]) is None


def test_flops_of_the_metric(bench):
    assert bench.flops(3) == pytest.approx(18.0)
    assert bench.flops(40003) == pytest.approx(2 * 40003 ** 3 / 3)


def test_traffic_records_parse():
    # every committed record: kernel, sha1 prefix, an existing source file, positive byte counts
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    assert rows
    for f in rows:
        assert len(f) >= 6 and len(f[1]) >= 8
        assert os.path.exists(os.path.join(ROOT, f[2]))
        assert float(f[3]) > 0 and float(f[4]) > 0


def test_traffic_lookup(bench, tmp_path, monkeypatch):
    assert bench.traffic_ratio("no_such_kernel") is None
    # a record whose source no longer hashes the same reads as null
    (tmp_path / "profiles").mkdir()
    (tmp_path / "src.cu").write_text("// kernel\n")
    (tmp_path / "profiles" / "traffic.txt").write_text("k deadbeef0000 src.cu 120 100 shape\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_ratio("k") is None
    import hashlib
    sha = hashlib.sha1(b"// kernel\n").hexdigest()[:12]
    (tmp_path / "profiles" / "traffic.txt").write_text("k %s src.cu 120 100 shape\n" % sha)
    assert bench.traffic_ratio("k") == pytest.approx(1.2)


def test_digit_products_of_the_sliced_precisions(bench):
    # S digits per entry keep the products of weight p + q <= S + 1: S (S + 1) / 2 of them
    for prec, s in (("df64tc", 8), ("df64tc7", 7)):
        pairs = [(p, q) for p in range(1, s + 1) for q in range(1, s + 1) if p + q <= s + 1]
        assert bench.DIGIT_PRODUCTS[prec] == len(pairs) == s * (s + 1) // 2
    assert bench.DEFAULT_PREC in bench.DIGIT_PRODUCTS


def test_update_kernel_traffic_records_are_current(bench):
    # the sliced update's records match the committed kernel source, for both digit counts
    for name in ("oz_update_kernel<7>", "oz_update_kernel<8>"):
        r = bench.traffic_ratio(name)
        assert r is not None and 0.9 < r < 1.5, (name, r)


def test_oz_update_bytes_counts_every_update_once(bench):
    # a single 512-column panel (n <= 512): only the inner updates of its 64-column steps
    n = 192
    got = bench.oz_update_bytes(n)
    want = 0.0
    for j in range(0, n, 64):
        r0 = j + 64
        M, N, K = n - r0, n - r0, 64
        if M > 0 and N > 0:
            want += 2 * 8 * M * N + 8 * K * (M + N)
    assert got == pytest.approx(want)
