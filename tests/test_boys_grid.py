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


def _boys_fp32_scheme(T, L, tab16):
    """The FP32 kernels' Boys evaluation below T = 30, restated in numpy float32 arithmetic: nearest
    point T_k = k/16 of the grid, whose row holds F_L, F_L+1, F_L+2 and exp(-T_k) rounded to FP32;
    F_L+3 and F_L+4 at T_k by the upward recursion F_m+1 = ((2m+1) F_m - exp(-T_k)) / (2 T_k)
    (1/(2m+3) at k = 0); the Taylor expansion sum_j F_L+j(T_k) x^j / j!, x = T_k - T, to fourth
    order; exp(-T) = exp(-T_k) exp(x) with exp(x) to fourth order.  Returns (F_L, exp(-T))."""
    f = np.float32
    T = f(T)
    k = int(np.rint(np.float64(T) * 16.0))
    kf = f(k)
    x = f(kf * f(0.0625) - T)
    a = [f(tab16[k, L]), f(tab16[k, L + 1]), f(tab16[k, L + 2]), f(math.exp(-k / 16.0))]
    ek = a[3]
    if k > 0:
        h = f(8.0 / kf)
        f3 = f((f(2 * L + 5) * a[2] - ek) * h)
        f4 = f((f(2 * L + 7) * f3 - ek) * h)
    else:
        f3, f4 = f(1.0 / (2 * L + 7)), f(1.0 / (2 * L + 9))
    s = f4
    for c, fj in ((0.25, f3), (1.0 / 3, a[2]), (0.5, a[1])):
        s = f(fj + s * x * f(c))
    FL = f(a[0] + s * x)
    ex = f(1 + x * f(1 + x * f(0.5 + x * f(1.0 / 6 + x * f(1.0 / 24)))))
    return float(FL), float(f(ek * ex))


def test_fp32_boys_scheme_is_unbiased(oracle_mod):
    """The FP32 scheme against the oracle at the FP32 argument: relative error within a few FP32
    ulps and no one-signed drift (the mean error stays two orders below one ulp).  Every FP32
    integral inherits the Boys function's bias with one sign, so a drift adds up over a whole J/K
    build (a grid step that FP32 cannot hold, such as 0.1, drifts by up to 9e-8 at T = 30; an
    approximate exponential in the recursion shifted the (H2O)_32 energy error by 1e-7 Ha)."""
    tab16 = np.array([oracle_mod.boys(12, k / 16.0) for k in range(482)])
    rng = np.random.default_rng(5)
    Ts = np.concatenate([rng.uniform(0.0, 30.0, 1500), rng.uniform(0.0, 1.0, 300)])
    T32 = [float(np.float32(T)) for T in Ts]
    refs = [oracle_mod.boys(8, T) for T in T32]
    for L in (0, 1, 2, 4, 8):
        rel = np.array([(_boys_fp32_scheme(T, L, tab16)[0] - r[L]) / r[L] for T, r in zip(T32, refs)])
        assert np.abs(rel).max() < 2.5e-7, (L, np.abs(rel).max())
        assert abs(rel.mean()) < 6e-9, (L, rel.mean())
    # exp(-T) of the downward recursion to the other F_m: same bar
    rel = np.array([(_boys_fp32_scheme(T, 0, tab16)[1] - math.exp(-T)) / math.exp(-T) for T in T32])
    assert np.abs(rel).max() < 2.5e-7 and abs(rel.mean()) < 6e-9, (np.abs(rel).max(), rel.mean())
