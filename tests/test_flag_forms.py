"""The integer forms in which the regrid's flag kernels decide FP64
comparisons, checked against the comparisons as defined (CPU, numpy).

- Cell mass: rho 2^(-3 l) > mass is decided as bits(rho) > bits(mass 2^(3 l))
  (signed 64-bit integers; NaN excluded), and for an FP32 state as
  bits32(rho) > bits32(RD32(mass 2^(3 l))), RD32 = rounding down to FP32.
- Jumps: two non-negative doubles compare as the integers of their bits.
- FP32 images of an FP64 state: the bits truncated on the integer pipes.
"""
import math

import numpy as np
import pytest


def _bits64(x):
    return int(np.array([x], np.float64).view(np.int64)[0])


def _bits32(x):
    return int(np.array([x], np.float32).view(np.int32)[0])


def _thresholds(mass, l):
    t = math.ldexp(mass, 3 * l)  # +inf past the range
    f = np.float32(t) if t <= 3.5e38 else np.float32(np.inf)
    if float(f) > t:
        f = np.nextafter(f, np.float32(-np.inf))
    return _bits64(t), _bits32(f)


def _mass_cases(rng):
    for _ in range(400):
        mass = float(np.exp(rng.normal(0.0, 30.0)))
        l = int(rng.integers(0, 16))
        t = math.ldexp(mass, 3 * l)
        near = [t * (1.0 + e) for e in (-1e-15, 0.0, 1e-15, 1e-7, -1e-7)] if math.isfinite(t) else []
        spread = list(np.exp(rng.normal(math.log(t) if 0 < t < 1e300 else 0.0, 3.0, 10)))
        yield mass, l, near + spread + [-1.0, 0.0, -0.0, math.inf, -math.inf, math.nan, 5e-324, 1e308]


def test_mass_criterion_in_bits_fp64_state():
    rng = np.random.default_rng(1)
    n = 0
    for mass, l, rhos in _mass_cases(rng):
        b64, _ = _thresholds(mass, l)
        for r in rhos:
            want = bool(np.ldexp(np.float64(r), -3 * l) > mass)
            b = _bits64(r)
            got = b > b64 and b <= 0x7FF0000000000000
            assert got == want, (mass, l, r)
            n += 1
    assert n > 5000


def test_mass_criterion_in_bits_fp32_state():
    rng = np.random.default_rng(2)
    with np.errstate(over="ignore"):
        for mass, l, rhos in _mass_cases(rng):
            _, b32 = _thresholds(mass, l)
            for r in rhos:
                r32 = np.float32(r)
                want = bool(np.ldexp(np.float64(r32), -3 * l) > mass)
                b = _bits32(r32)
                got = b > b32 and b <= 0x7F800000
                assert got == want, (mass, l, r, r32)


@pytest.mark.parametrize("seed", [0, 1])
def test_non_negative_doubles_order_as_their_bits(seed):
    rng = np.random.default_rng(seed)
    a = np.abs(np.concatenate([rng.standard_normal(2000) * 10.0 ** rng.integers(-300, 300, 2000),
                               [0.0, 5e-324, 2.2250738585072014e-308, 1.7976931348623157e308, math.inf]]))
    b = np.roll(a, 7)
    ia, ib = a.view(np.int64), b.view(np.int64)
    assert np.array_equal(ia > ib, a > b)
    assert np.array_equal(ia == ib, a == b)


def _to_f32_bits(x):
    """The flag kernels' FP32 image of an FP64 value, on the integer pipes:
    sign, exponent rebiased, mantissa truncated; below 2^-126 zero, above the
    FP32 range infinity."""
    b = int(np.array([x], np.float64).view(np.uint64)[0])
    sign = (b >> 32) & 0x80000000
    e = (b >> 52) & 0x7FF
    if e < 1023 - 126:
        bits = sign
    elif e > 1023 + 127:
        bits = sign | 0x7F800000
    else:
        bits = sign | ((e - 896) << 23) | ((b >> 29) & 0x7FFFFF)
    return float(np.array([bits], np.uint32).view(np.float32)[0])


def test_fp32_images_truncate_within_their_bound():
    """Within the normal FP32 range the image is x rounded toward zero to
    FP32 (relative error below 2^-23, the bound the screen assumes), and an
    FP32 value maps to itself."""
    rng = np.random.default_rng(5)
    xs = np.concatenate([np.exp(rng.uniform(-80, 80, 3000)) * rng.choice([-1, 1], 3000),
                         [1.0, -1.0, 1.5, 2.0 ** -126, 3.4e38]])
    for x in xs:
        f = _to_f32_bits(x)
        r = np.float32(x)
        if abs(float(r)) > abs(x):
            r = np.nextafter(r, np.float32(0))
        assert f == float(r), x
        assert abs(f - x) <= 2.0 ** -23 * abs(x), x
        assert _to_f32_bits(float(np.float32(x))) == float(np.float32(x))
    assert _to_f32_bits(1e-300) == 0.0 and _to_f32_bits(1e300) == np.inf and _to_f32_bits(-1e300) == -np.inf
