"""Pin of the oracle's histogram error (the L2 distance of the
piecewise-constant densities, Eq. piecewise_constant_pdf, used by the
experiments of Section 6): adaptive quadrature of the squared difference of
the two step functions, and a hand-computed case."""
import math

import numpy as np
from scipy import integrate


def test_l2_against_quadrature(orc):
    g = orc.Grid(37, -2.0, 5.4)
    rng = np.random.default_rng(3)
    cdfs = []
    for _ in range(2):
        m = rng.random(g.bins) * (rng.random(g.bins) > 0.3)
        cdfs.append(np.concatenate([[0.0], np.cumsum(m) / m.sum()]))
    e = np.linspace(g.lo, g.hi, g.bins + 1)
    dens = [np.diff(c) / g.h for c in cdfs]

    def sq(x):
        i = min(int((x - g.lo) / g.h), g.bins - 1)
        return (dens[0][i] - dens[1][i]) ** 2
    val = sum(integrate.quad(sq, a + 1e-12, b - 1e-12)[0] for a, b in zip(e[:-1], e[1:]))
    assert abs(orc.l2_density(g, cdfs[0], cdfs[1]) - math.sqrt(val)) < 1e-9 * math.sqrt(val)


def test_l2_hand_case(orc):
    # all mass in bin 0 against all mass in bin 2 of four bins of width 1/2:
    # densities 2 on [0, 1/2) and 2 on [1, 3/2): integral of the square 2 * 4 * 1/2 = 4
    g = orc.Grid(4, 0.0, 2.0)
    a = np.array([0.0, 1.0, 1.0, 1.0, 1.0])
    b = np.array([0.0, 0.0, 0.0, 1.0, 1.0])
    assert orc.l2_density(g, a, b) == 2.0
    assert orc.l2_density(g, a, a) == 0.0
