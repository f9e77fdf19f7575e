"""The bit-pattern forms in which the FP64 level-step kernels take compares,
minima, maxima and the minmod limiter on the integer pipes, checked against
the operations as defined (CPU, numpy; the kernels' results themselves are
checked against the oracle by the GPU parity tests).

- minmod(a, b): 0 for opposite signs or a zero argument, else the argument of
  smaller magnitude; decided on the bits shifted left by one (sign dropped).
- ord(x) = bits ^ ((bits >> 63) & 0x7FF...F) orders every non-NaN double
  (-0 just below +0): vmax / vmin pick by it.
- pos(x) = bits > 0 is x > 0 for every non-NaN x.
- gt_nonneg(a, b) = bits(a) > bits(b) is a > b for a, b >= 0.
"""
import numpy as np
import pytest


def _values(rng, n=4000):
    mags = 10.0 ** rng.uniform(-310, 308, n)
    v = np.where(rng.random(n) < 0.5, -mags, mags)
    special = np.array([0.0, -0.0, 5e-324, -5e-324, 1.0, -1.0, np.inf, -np.inf,
                        2.2250738585072014e-308, -1.7976931348623157e308])
    return np.concatenate([v, special, v[:50]])  # repeats give equal pairs


def _pairs(seed):
    rng = np.random.default_rng(seed)
    a = _values(rng)
    b = np.concatenate([np.roll(a, 3)[:-50], a[-50:]])
    return a, b


def _minmod_bits(a, b):
    ia, ib = a.view(np.int64), b.view(np.int64)
    ma, mb = ia.view(np.uint64) << np.uint64(1), ib.view(np.uint64) << np.uint64(1)
    zero = ((ia ^ ib) < 0) | (ma == 0) | (mb == 0)
    return np.where(zero, 0.0, np.where(ma < mb, a, b))


def _ord(x):
    i = x.view(np.int64)
    return i ^ ((i >> np.int64(63)) & np.int64(0x7FFFFFFFFFFFFFFF))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_minmod_on_bits(seed):
    a, b = _pairs(seed)
    # a b > 0 written on the signs (the product itself can underflow to 0 or
    # overflow for these magnitudes)
    same = (np.signbit(a) == np.signbit(b)) & (a != 0) & (b != 0)
    want = np.where(same, np.where(np.abs(a) < np.abs(b), a, b), 0.0)
    assert np.array_equal(_minmod_bits(a, b), want)


@pytest.mark.parametrize("seed", [3, 4])
def test_order_bits_min_max_pos(seed):
    a, b = _pairs(seed)
    oa, ob = _ord(a), _ord(b)
    nz = (a != 0) | (b != 0)  # the order of -0 and +0 is a choice (-0 below +0)
    assert np.array_equal((oa < ob)[nz], (a < b)[nz])
    assert np.array_equal((oa == ob)[nz], (a == b)[nz])
    vmax = np.where(oa < ob, b, a)
    vmin = np.where(ob < oa, b, a)
    assert np.array_equal(vmax[nz], np.maximum(a, b)[nz])
    assert np.array_equal(vmin[nz], np.minimum(a, b)[nz])
    assert np.array_equal(a.view(np.int64) > 0, a > 0)
    na, nb = np.abs(a), np.abs(b)
    assert np.array_equal(na.view(np.int64) > nb.view(np.int64), na > nb)
