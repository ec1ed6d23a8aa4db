"""Pins for the oracle's Boys function F_m(T) = int_0^1 t^{2m} exp(-T t^2) dt.

Closed forms: F_m(0) = 1/(2m+1); F_0(T) = 1/2 sqrt(pi/T) erf(sqrt T); the
large-T asymptote (2m-1)!!/2^{m+1} sqrt(pi/T^{2m+1}); the downward recursion
F_m = (2T F_{m+1} + e^{-T})/(2m+1); and direct numerical quadrature of the
defining integral.
"""
import math

import numpy as np
import pytest
from scipy.integrate import quad

from oracle import integrals as I


@pytest.mark.parametrize("m", range(0, 16))
def test_boys_at_zero(m):
    assert I.boys(m, 0.0) == pytest.approx(1.0 / (2 * m + 1), rel=1e-15)


@pytest.mark.parametrize("T", [1e-8, 1e-3, 0.3, 1.0, 7.5, 25.0, 39.9, 40.1, 60.0, 300.0])
def test_boys_f0_erf(T):
    ref = 0.5 * math.sqrt(math.pi / T) * math.erf(math.sqrt(T))
    assert I.boys(0, T) == pytest.approx(ref, rel=2e-15)


@pytest.mark.parametrize("m", [0, 3, 7, 12])
@pytest.mark.parametrize("T", [0.05, 2.0, 11.0, 35.0, 45.0])
def test_boys_quadrature(m, T):
    ref, err = quad(lambda t: t ** (2 * m) * math.exp(-T * t * t), 0.0, 1.0, epsabs=0, epsrel=2e-14, limit=200)
    assert I.boys(m, T) == pytest.approx(ref, rel=1e-12)


@pytest.mark.parametrize("m", [0, 2, 5, 9])
def test_boys_asymptote(m):
    T = 120.0
    df = 1
    for k in range(2 * m - 1, 0, -2):
        df *= k
    ref = df / 2 ** (m + 1) * math.sqrt(math.pi / T ** (2 * m + 1))
    assert I.boys(m, T) == pytest.approx(ref, rel=1e-14)


@pytest.mark.parametrize("T", [0.01, 0.9, 5.0, 20.0, 39.0, 41.0, 80.0])
def test_boys_recursion_both_ways(T):
    F = np.array([I.boys(m, T) for m in range(14)])
    for m in range(13):
        down = (2 * T * F[m + 1] + math.exp(-T)) / (2 * m + 1)
        assert F[m] == pytest.approx(down, rel=1e-13)
