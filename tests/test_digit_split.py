"""The sliced update's digit split (S balanced 7-bit digits of a
double-float entry scaled by 2^(7S - e), S = 8 or 7) computed the way the
kernel does it, in 32-bit pieces: each scaled part rounded to an
integer-valued float, split exactly at 2^28, the low four digits from the low
halves with their carry into the high half, the other S - 4 from the high
halves.  Checked against the plain definition (one exact integer
Y = rint(hi 2^(7S-e)) + rint(lo 2^(7S-e)), digits by repeated balanced
remainder mod 128) on random pairs, tiny entries and half-ulp ties."""
import numpy as np
import pytest

f32 = np.float32


def _digits_definition(hi, lo, e, S=8):
    Y = int(np.rint(np.ldexp(np.float64(hi), 7 * S - e))) + int(np.rint(np.ldexp(np.float64(lo), 7 * S - e)))
    d = [0] * S
    for p in range(S - 1, 0, -1):
        r = Y % 128
        if r >= 64:
            r -= 128
        d[p] = r
        Y = (Y - r) // 128
    d[0] = Y
    return d


def _digits_split(hi, lo, e, S=8):
    hs = np.rint(np.ldexp(f32(hi), 7 * S - e).astype(f32)).astype(f32)
    ls = np.rint(np.ldexp(f32(lo), 7 * S - e).astype(f32)).astype(f32)
    hh = np.rint(hs * f32(2.0 ** -28)).astype(f32)
    lh = np.rint(ls * f32(2.0 ** -28)).astype(f32)
    rh = float(hs) - float(hh) * 2.0 ** 28          # the kernel's fma(-hh, 2^28, hs)
    rl = float(ls) - float(lh) * 2.0 ** 28
    assert float(f32(rh)) == rh and float(f32(rl)) == rl   # exact in float
    low, high = int(rh) + int(rl), int(hh) + int(lh)
    assert abs(low) <= 2 ** 28 and abs(high) < 2 ** 31      # 32-bit integers
    d = [0] * S
    for p in range(S - 1, S - 5, -1):
        r = ((low & 127) ^ 64) - 64
        d[p] = r
        low = (low - r) >> 7
    high += low
    for p in range(S - 5, 0, -1):
        r = ((high & 127) ^ 64) - 64
        d[p] = r
        high = (high - r) >> 7
    d[0] = high
    return d


@pytest.mark.parametrize("S", [8, 7])
def test_split_matches_definition(S):
    rng = np.random.default_rng(S)
    for trial in range(20000):
        E = int(rng.integers(-60, 60))                   # exponent of the row's largest entry
        x = np.float64(2.0 ** (E - rng.uniform(0, 45))) * rng.choice([-1, 1])
        x = float(np.clip(x, -0.999 * 2.0 ** E, 0.999 * 2.0 ** E))
        hi = f32(x)
        lo = f32(x - np.float64(hi))
        if trial % 5 == 0:                               # half-ulp ties of the pair
            lo = f32(np.spacing(np.abs(hi)).astype(np.float64) / 2 * rng.choice([-1, 1]))
        e = E + 2                                        # the row exponent plus one bit of headroom
        d = _digits_split(hi, lo, e, S)
        assert d == _digits_definition(hi, lo, e, S), (hi, lo, e, S)
        assert all(-64 <= v <= 63 for v in d[1:]) and -64 <= d[0] <= 64


def test_digit_to_bf16_is_exact():
    # 2^23 + 2^22 + r in float, minus the same constant, is r exactly; its
    # upper 16 bits are the bf16 of r (r has at most 8 significant bits)
    for r in range(-64, 65):
        bits = np.array([0x4B400000 + r], dtype=np.uint32)
        f = bits.view(np.float32)[0] - np.float32(12582912.0)
        assert f == r
        b = np.array([f], dtype=np.float32).view(np.uint32)[0] >> 16
        back = np.array([b << 16], dtype=np.uint32).view(np.float32)[0]
        assert back == r
