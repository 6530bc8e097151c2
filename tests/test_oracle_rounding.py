"""Pins for the oracle's software rounding (IEEE 754 binary16 / binary32,
round-to-nearest-even), against NumPy's independent float16/float32 casts.

The oracle stores every reduced-precision vector of Algorithm 3 through these
two functions, so a wrong exponent bias, tie rule, subnormal spacing or
overflow threshold here would corrupt every mixed-precision result."""
import numpy as np
import pytest

import oracle


def _np16(x):
    with np.errstate(over="ignore"):
        return np.asarray(x, dtype=np.float64).astype(np.float16).astype(np.float64)


def _np32(x):
    with np.errstate(over="ignore"):
        return np.asarray(x, dtype=np.float64).astype(np.float32).astype(np.float64)


def _same(a, b):
    a, b = np.asarray(a), np.asarray(b)
    both_nan = np.isnan(a) & np.isnan(b)
    eq = (a == b) & (np.signbit(a) == np.signbit(b))
    return np.all(eq | both_nan)


def test_round16_fixed_points_all_finite_halves():
    h = np.arange(0, 1 << 16, dtype=np.uint32).astype(np.uint16).view(np.float16)
    v = h.astype(np.float64)
    v = v[np.isfinite(v)]
    assert _same(oracle.round16(v), v)


def test_round16_midpoints_ties_to_even_and_sticky_bits():
    pos = np.arange(0, 0x7BFF, dtype=np.uint16).view(np.float16).astype(np.float64)
    nxt = np.arange(1, 0x7C00, dtype=np.uint16).view(np.float16).astype(np.float64)
    mid = 0.5 * (pos + nxt)                     # exact in binary64
    for sgn in (1.0, -1.0):
        for x in (mid, np.nextafter(mid, np.inf), np.nextafter(mid, -np.inf),
                  mid + (nxt - pos) * 2.0 ** -30, mid - (nxt - pos) * 2.0 ** -30):
            assert _same(oracle.round16(sgn * x), _np16(sgn * x))
    # ties go to the neighbour with an even significand
    even = (np.arange(0, 0x7BFF) % 2 == 0)
    got = oracle.round16(mid)
    assert np.all(np.where(even, got == pos, got == nxt))


def test_round16_float32_sweep_and_overflow():
    # every binary32 exponent that can land in or near binary16's range,
    # with a prime stride through the significands
    e = np.arange(-30, 17)
    m = np.arange(0, 1 << 23, 97, dtype=np.uint32)
    bits = ((e[:, None] + 127).astype(np.uint32) << 23) | m[None, :]
    f = bits.reshape(-1).view(np.float32).astype(np.float64)
    for x in (f, -f):
        assert _same(oracle.round16(x), _np16(x))
    for x, want in ((65504.0, 65504.0), (65519.999, 65504.0), (65520.0, np.inf),
                    (1e6, np.inf), (-65520.0, -np.inf), (2.0 ** -25, 0.0),
                    (np.nextafter(2.0 ** -25, 1), 2.0 ** -24), (-1e-30, -0.0),
                    (np.inf, np.inf), (-np.inf, -np.inf)):
        assert _same(oracle.round16(x), want), x
    assert np.isnan(oracle.round16(np.nan))


def test_round16_random_doubles():
    rng = np.random.default_rng(7)
    x = rng.standard_normal(400_000) * np.exp2(rng.integers(-30, 18, 400_000))
    assert _same(oracle.round16(x), _np16(x))


def test_round32_against_cast():
    rng = np.random.default_rng(8)
    x = rng.standard_normal(400_000) * np.exp2(rng.integers(-160, 130, 400_000))
    assert _same(oracle.round32(x), _np32(x))
    # binary32 midpoints around 1 and in the subnormal range
    f = np.arange(0x3F800000, 0x3F800000 + 20001, dtype=np.uint32).view(np.float32).astype(np.float64)
    mid = 0.5 * (f[:-1] + f[1:])
    assert _same(oracle.round32(mid), _np32(mid))
    s = np.arange(1, 20001, dtype=np.uint32).view(np.float32).astype(np.float64)
    mid = 0.5 * (s[:-1] + s[1:])
    assert _same(oracle.round32(mid), _np32(mid))
    big = np.float64(np.finfo(np.float32).max)
    for v in (big, np.nextafter(big, np.inf), 3.4028235677973366e38, 3.402823567797337e38, 1e39):
        assert _same(oracle.round32(v), _np32(v)), v


@pytest.mark.parametrize("prec", [oracle.FP16, oracle.FP32])
def test_round_is_idempotent_and_monotone(prec):
    rng = np.random.default_rng(9)
    x = np.sort(rng.standard_normal(100_000) * 100)
    y = oracle.round_to(prec, x)
    assert _same(oracle.round_to(prec, y), y)
    assert np.all(np.diff(y) >= 0)
