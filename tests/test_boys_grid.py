"""The Boys-function grid the J/K kernels expand around (built by the library's host code: a long
double series for F_15 and downward recursion), checked against the oracle's independent
evaluation (compensated double series / erf + upward recursion) at every grid point.  No GPU."""
import math

import numpy as np


def test_grid_matches_oracle(mess, oracle_mod):
    tab, dT = mess.boys_grid()
    assert tab.shape == (362, 17) and dT == 0.1
    worst = 0.0
    for k in range(tab.shape[0]):
        T = k * dT
        ref = oracle_mod.boys(15, T)
        rel = np.abs(tab[k, :16] - ref) / np.abs(ref)
        worst = max(worst, float(rel.max()))
        # the grid point k * 0.1 is formed in extended precision there, in double here: the two
        # differ by up to half an ulp of T, which moves exp(-T) by that much relatively
        assert abs(tab[k, 16] - math.exp(-T)) <= (T * 2.0 ** -53 + 4.5e-16) * math.exp(-T)
    assert worst <= 1e-14, worst


def test_grid_closed_forms(mess):
    tab, _ = mess.boys_grid()
    n = np.arange(16)
    np.testing.assert_allclose(tab[0, :16], 1.0 / (2 * n + 1), rtol=1e-15)          # F_n(0)
    T = 361 * 0.1
    assert tab[361, 0] == __import__("pytest").approx(0.5 * math.sqrt(math.pi / T) * math.erf(math.sqrt(T)),
                                                        rel=1e-14)
