"""The transform kernels convert double to float (the float working copy) and
split double into a float pair (the double-float working copy) with 32-bit
integer operations on the two halves of each double, since the conversion
instruction runs on the FP64 pipe.  These CPU tests re-run those integer
steps, exactly as the kernels write them, in numpy uint32 arithmetic and
compare them bit for bit with IEEE round-to-nearest-even (numpy's
float64 -> float32 cast) on random doubles over the whole float range,
exact half-way ties, mantissa carries into the exponent, and the edges of
the range the integer path rounds (outside it the kernels select signed
zero below 2^-126, infinity above the float range, NaN for NaN: no FP64
instruction at all)."""
import numpy as np

U32 = np.uint32


def _halves(x):
    b = np.asarray(x, dtype=np.float64).view(np.uint64)
    return (b >> np.uint64(32)).astype(U32), (b & np.uint64(0xFFFFFFFF)).astype(U32)


def d2f_rn_int(x):
    """(in_range, float32 result) of the kernels' integer double -> float
    conversion; in_range marks the doubles it rounds (float exponent 1..254)."""
    hi, lo = _halves(x)
    ex = (hi >> U32(20)) & U32(0x7FF)
    in_range = (ex - U32(897)) < U32(254)                        # unsigned wrap
    t = (hi & U32(0x7FFFFFFF)) - U32(896 << 20)
    f = (t << U32(3)) | (lo >> U32(29))                          # __funnelshift_l(lo, t, 3)
    rem = lo << U32(3)
    f = f + (rem > (U32(0x80000000) - (f & U32(1)))).astype(U32)
    f = np.where(ex < U32(897), U32(0), f)
    nan = (ex == U32(2047)) & (((hi & U32(0xFFFFF)) | lo) != U32(0))
    big = np.where(nan, U32(0x7FC00000), U32(0x7F800000))
    f = np.where(ex > U32(1150), big, f).astype(U32)
    f = f | (hi & U32(0x80000000))
    return in_range, f.view(np.float32)


def _check(x):
    x = np.asarray(x, dtype=np.float64)
    ok, got = d2f_rn_int(x)
    want = x.astype(np.float32)
    assert np.array_equal(got[ok].view(U32), want[ok].view(U32))
    return ok


def test_random_doubles_over_the_float_range():
    rng = np.random.default_rng(1)
    m = rng.uniform(1, 2, 400000) * rng.choice([-1.0, 1.0], 400000)
    e = rng.integers(-126, 128, 400000)
    ok = _check(np.ldexp(m, e))
    assert ok.mean() > 0.999


def test_half_way_ties_round_to_even():
    rng = np.random.default_rng(2)
    f = rng.uniform(1, 2, 20000).astype(np.float32)
    f = f * np.ldexp(1.0, rng.integers(-120, 120, 20000)).astype(np.float32)
    up = np.nextafter(f, np.float32(np.inf))
    mid = (f.astype(np.float64) + up.astype(np.float64)) / 2          # exact in double
    ok = _check(mid)
    assert ok.all()
    # just above and below the tie
    _check(np.nextafter(mid, np.inf))
    _check(np.nextafter(mid, -np.inf))


def test_mantissa_carry_into_the_exponent_and_range_edges():
    vals = []
    for e in (-126, -100, -1, 0, 1, 50, 126, 127):
        top = np.ldexp(2.0 - 2.0 ** -52, e)                          # all mantissa bits set: rounds up a binade
        vals += [top, -top, np.ldexp(1.0, e), np.nextafter(np.ldexp(1.0, e), 0)]
    vals += [np.float64(np.finfo(np.float32).max), np.ldexp(2.0 - 2.0 ** -24, 127), np.ldexp(2.0 - 2.0 ** -25, 127),
             np.float64(np.finfo(np.float32).tiny), np.ldexp(1.0, -126) * (1 - 2.0 ** -30)]
    x = np.array(vals)
    ok = _check(x)
    # values that overflow to infinity in round-to-nearest also do so here
    big = np.array([np.ldexp(2.0 - 2.0 ** -25, 127)])
    assert d2f_rn_int(big)[0].all() and np.isinf(d2f_rn_int(big)[1]).all()
    # outside the rounded range: signed zero for zero and anything below the
    # smallest normal float (flushed), infinity above the float range, NaN kept
    special = np.array([0.0, -0.0, 1e-40, -1e-300, np.inf, -np.inf, np.nan, 1e300, -1e300])
    inr, got = d2f_rn_int(special)
    assert not inr.any()
    assert np.array_equal(got[:4].view(U32), np.array([0.0, -0.0, 0.0, -0.0], dtype=np.float32).view(U32))
    assert got[4] == np.inf and got[5] == -np.inf and np.isnan(got[6]) and got[7] == np.inf and got[8] == -np.inf
    assert ok.sum() >= len(vals) - 2


def split_pair_int(x):
    """The double-float working copy's split of a double into (hi, lo), as the
    kernel writes it: hi = the double rounded to 24 bits by the integer steps
    above; the remainder r (the low 29 mantissa bits, less 2^29 when hi
    rounded up, so |r| <= 2^28) converted to float by the integer-to-float
    unit (round to nearest even) and scaled by the double's unit in the last
    place 2^(E - 1075); below |x| = 2^-74 (E < 949) lo is zero.  Returns
    (in_range, hi, lo); in range for double exponents E in [949, 1149]."""
    hi_w, lo_w = _halves(x)
    ex = (hi_w >> U32(20)) & U32(0x7FF)
    in_range = (ex - U32(949)) < U32(201)
    t = (hi_w & U32(0x7FFFFFFF)) - U32(896 << 20)
    f = (t << U32(3)) | (lo_w >> U32(29))
    up = ((lo_w << U32(3)) > (U32(0x80000000) - (f & U32(1)))).astype(U32)
    f = (f + up) | (hi_w & U32(0x80000000))
    r = (lo_w & U32(0x1FFFFFFF)).astype(np.int64) - (up.astype(np.int64) << 29)
    scale = np.ldexp(np.float32(1.0), np.clip(ex.astype(np.int64) - 1075, -126, 127))  # 2^(E - 1075)
    lo = r.astype(np.float32) * scale.astype(np.float32)                        # I2F (RN), then an exact scaling
    lo = np.where(in_range, lo, np.float32(0))
    lo = np.where(hi_w & U32(0x80000000), -lo, lo).astype(np.float32)
    _, hi = d2f_rn_int(x)
    return in_range, hi, lo


def test_pair_split_is_exact_to_48_bits():
    """hi = RN(x) exactly; hi + lo within 2^-48 |x| (the pair's precision); lo
    is RN(x - hi) whenever x - hi fits 24 bits."""
    rng = np.random.default_rng(3)
    x = rng.standard_normal(200000) * np.ldexp(1.0, rng.integers(-60, 60, 200000))
    x = np.concatenate([x, [1.0, -1.0, 3.0, np.ldexp(2.0 - 2.0 ** -52, 40), np.ldexp(1.0 + 2.0 ** -24, -20)]])
    ok, hi, lo = split_pair_int(x)
    assert ok.all()
    assert np.array_equal(hi.view(U32), x.astype(np.float32).view(U32))
    err = np.abs((hi.astype(np.float64) + lo.astype(np.float64)) - x)
    assert np.all(err <= np.ldexp(np.abs(x), -48))
    exact = (x - hi.astype(np.float64)).astype(np.float32)
    small = np.abs(x - hi.astype(np.float64)) == np.abs(exact.astype(np.float64))
    assert np.array_equal(lo[small], exact[small])
    # |lo| <= ulp(hi) / 2: the pair is normalized
    assert np.all(np.abs(lo.astype(np.float64)) <= np.spacing(np.abs(hi)).astype(np.float64) / 2)


def test_pair_split_of_tiny_values_keeps_the_leading_part():
    x = np.array([np.ldexp(1.0 + 2.0 ** -30, -80), -np.ldexp(1.5, -100), np.ldexp(1.25, -74)])
    ok, hi, lo = split_pair_int(x)
    assert np.array_equal(hi, x.astype(np.float32))
    assert np.all(lo[:2] == 0) and ok[2]
    assert np.all(np.abs(hi.astype(np.float64) + lo.astype(np.float64) - x) <= np.ldexp(np.abs(x), -24))
