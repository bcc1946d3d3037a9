"""Pins of the oracle's float32 fused multiply-add (``fma32``) against exact
rational arithmetic: a b + c computed with Fractions and rounded once to
float32 (nearest, ties to even) by comparing it with its float32 neighbours.

Random triples of many magnitudes cover the ordinary cases. The hard cases
are those where rounding a b + c first to float64 and then to float32 gives
the wrong float32: a b is an exact float32 midpoint and c, far below the
float64 resolution of the sum, decides the direction. The test builds such
cases from a = 1 + i 2^-12, b = 1 + j 2^-12 with i, j odd (a b = 1 + (i + j)
2^-12 + i j 2^-24, an odd multiple of 2^-24 above a float32 value) and
checks that the naive double rounding fails on them while fma32 does not.
"""
from fractions import Fraction

import numpy as np

from oracle import kf_oracle as O

F32 = np.float32


def exact_f32(fr: Fraction) -> np.float32:
    """The float32 nearest to the rational fr (ties to the even significand)."""
    f = F32(float(fr))
    cands = {F32(np.nextafter(f, F32(-np.inf))), f, F32(np.nextafter(f, F32(np.inf)))}
    best = None
    for c in cands:
        if not np.isfinite(c):
            continue
        d = abs(Fraction(float(c)) - fr)
        key = (d, int(np.array(c, F32).view(np.int32)) & 1)
        if best is None or key < best[0]:
            best = (key, c)
    return best[1]


def exact_fma(a, b, c) -> np.float32:
    return exact_f32(Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c)))


def bits(x):
    return np.asarray(x, F32).view(np.int32)


def test_fma32_matches_exact_rounding_on_random_triples():
    rng = np.random.default_rng(11)
    n = 4000
    a = (rng.uniform(-2, 2, n) * 2.0 ** rng.integers(-20, 20, n)).astype(F32)
    b = (rng.uniform(-2, 2, n) * 2.0 ** rng.integers(-20, 20, n)).astype(F32)
    c = (rng.uniform(-2, 2, n) * 2.0 ** rng.integers(-40, 40, n)).astype(F32)
    got = O.fma32(a, b, c)
    want = np.array([exact_fma(x, y, z) for x, y, z in zip(a, b, c)], F32)
    assert np.array_equal(bits(got), bits(want))


def test_fma32_is_right_where_double_rounding_is_wrong():
    rng = np.random.default_rng(12)
    cases = []
    for _ in range(400):
        i, j = (2 * rng.integers(0, 64, 2) + 1)
        sa, sb = rng.choice([-1.0, 1.0], 2)
        a = F32(sa * (1.0 + i * 2.0 ** -12))
        b = F32(sb * (1.0 + j * 2.0 ** -12))
        # c far below the float64 resolution of a b, either sign
        c = F32(rng.choice([-1.0, 1.0]) * rng.uniform(1, 2) * 2.0 ** -int(rng.integers(58, 90)))
        cases.append((a, b, c))
    a, b, c = (np.array(v, F32) for v in zip(*cases))
    naive = (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(F32)
    got = O.fma32(a, b, c)
    want = np.array([exact_fma(x, y, z) for x, y, z in cases], F32)
    assert np.array_equal(bits(got), bits(want))
    # the construction does reach the double-rounding failures of the naive form
    assert (bits(naive) != bits(want)).sum() > 50


def test_fma32_special_values_and_broadcasting():
    nan = F32(np.nan)
    assert np.isnan(O.fma32(nan, F32(1), F32(1)))
    assert O.fma32(F32(2), F32(3), F32(4)) == F32(10)
    assert O.fma32(F32(0), F32(5), F32(-0.0)) == 0
    # a scalar times an array plus a scalar, as the transform rows use it
    x = np.array([1.0, 2.0, 3.0], F32)
    assert np.array_equal(O.fma32(F32(2), x, F32(1)), np.array([3, 5, 7], F32))
    assert O.fma32(F32(2), x, F32(1)).dtype == F32


def test_transform_rows_are_the_fma_chain():
    rng = np.random.default_rng(13)
    R = rng.normal(size=(3, 3)).astype(F32)
    t = rng.normal(size=3).astype(F32)
    v = rng.normal(size=(50, 3)).astype(F32)
    rows = O._xform32(R, t, v[:, 0], v[:, 1], v[:, 2])
    for i in range(3):
        for k in range(50):
            want = exact_fma(R[i, 2], v[k, 2], exact_fma(R[i, 1], v[k, 1], exact_fma(R[i, 0], v[k, 0], t[i])))
            assert bits(rows[i][k]) == bits(want)


def test_fma32_overflow_and_signed_zero():
    big = F32(1e20)
    assert O.fma32(big, big, F32(0)) == F32(np.inf)          # 1e40 is past float32's range
    assert O.fma32(big, big, F32(-np.inf)) == F32(-np.inf)
    assert bits(O.fma32(F32(-1), F32(1), F32(1))) == bits(exact_fma(F32(-1), F32(1), F32(1)))
    # an exact cancellation rounds to +0 (round to nearest), as the hardware does
    assert bits(O.fma32(F32(2), F32(3), F32(-6))) == bits(F32(0))
