"""Pins for the oracle's Boys function F_n(T) = int_0^1 t^{2n} exp(-T t^2) dt."""
import math

import numpy as np
import pytest


def _dfact(k):
    r = 1
    while k > 1:
        r *= k
        k -= 2
    return r


def test_boys_at_zero(oracle_mod):
    F = oracle_mod.boys(16, 0.0)
    for n in range(17):
        assert F[n] == pytest.approx(1.0 / (2 * n + 1), rel=1e-15)


@pytest.mark.parametrize("T", [1e-8, 1e-3, 0.3, 1.0, 4.5, 12.0, 29.9, 49.99, 50.0, 75.0, 300.0])
def test_boys_f0_erf_closed_form(oracle_mod, T):
    F0 = oracle_mod.boys(0, T)[0]
    ref = 0.5 * math.sqrt(math.pi / T) * math.erf(math.sqrt(T))
    assert F0 == pytest.approx(ref, rel=2e-15)


@pytest.mark.parametrize("T", [40.0, 60.0, 120.0, 500.0])
def test_boys_large_T_asymptote(oracle_mod, T):
    F = oracle_mod.boys(8, T)
    for n in range(9):
        asym = _dfact(2 * n - 1) / 2 ** (n + 1) * math.sqrt(math.pi / T ** (2 * n + 1))
        # exact up to terms of order exp(-T)
        assert F[n] == pytest.approx(asym, rel=1e-12)


@pytest.mark.parametrize("T", [1e-4, 0.05, 0.7, 3.3, 11.0, 26.0, 49.5, 50.5, 90.0])
def test_boys_downward_identity(oracle_mod, T):
    F = oracle_mod.boys(12, T)
    for n in range(12, 0, -1):
        lhs = F[n - 1]
        rhs = (2 * T * F[n] + math.exp(-T)) / (2 * n - 1)
        assert lhs == pytest.approx(rhs, rel=2e-14)


@pytest.mark.parametrize("T", [0.0, 0.2, 2.0, 9.0, 25.0, 49.0, 51.0, 70.0])
def test_boys_gauss_legendre(oracle_mod, T):
    x, w = np.polynomial.legendre.leggauss(200)
    t = 0.5 * (x + 1.0)
    F = oracle_mod.boys(10, T)
    for n in range(11):
        ref = 0.5 * float(np.sum(w * t ** (2 * n) * np.exp(-T * t * t)))
        assert F[n] == pytest.approx(ref, rel=1e-13)


def test_boys_continuous_across_branch(oracle_mod):
    a = oracle_mod.boys(8, 50.0 - 1e-9)
    b = oracle_mod.boys(8, 50.0 + 1e-9)
    # the 2e-9 step in T moves F_n by about 2e-9 * F_{n+1}
    assert np.allclose(a, b, rtol=1e-9, atol=0)
