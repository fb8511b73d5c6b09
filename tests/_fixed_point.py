"""Weights for the checks of the fixed point round(w 2^61) used by the
weighted sums of Section 5.2, and that rounding in exact rational
arithmetic (test infrastructure)."""
import math

import numpy as np


def crafted_weights():
    """Weights whose fixed point round(w 2^61) exercises the rounding: exact
    ties (k + 1/2 for k = 0..7, to even), one ulp either side of a tie, the
    smallest normal and a subnormal (0), zero, negative zero and negative
    values (0), exact integers, and small random values."""
    t = 2.0 ** -62
    w = [(2 * k + 1) * t for k in range(8)]
    w += [t, math.nextafter(t, 1.0), math.nextafter(t, 0.0), 2.0 ** -1022, 5e-324, 0.0, -0.0, -2.0 ** -50,
          3 * 2.0 ** -61, 2.0 ** -50, math.nextafter(2.0 ** -50, 1.0), 2.0 ** -50 + t, 2.0 ** -50 + 3 * t,
          2.0 ** -49 + 5 * t]
    rng = np.random.default_rng(17)
    w += list(rng.random(64 - len(w)) * 2.0 ** -48)
    return np.array(w)


def fixed_exact(w):
    """round(w 2^61), ties to even, from the exact rational value of w (0 for
    w <= 0)."""
    from fractions import Fraction
    if not w > 0:
        return 0
    v = Fraction(float(w)) * 2 ** 61
    q, r = divmod(v.numerator, v.denominator)
    twice = 2 * r
    return q + (1 if twice > v.denominator or (twice == v.denominator and q % 2 == 1) else 0)
