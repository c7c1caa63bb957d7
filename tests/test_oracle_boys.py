"""Pins of the oracle's Boys function F_m(T) = int_0^1 t^{2m} exp(-T t^2) dt.

The Boys function supplies the moments of the Rys weight function (Sec. II-C:
sum_mu w_mu t_mu^{2k} = F_k(T)).  It is pinned against closed forms and special
functions that share nothing with the oracle's series/recursion code.
"""
import math

import numpy as np
import pytest

import oracle

scipy_special = pytest.importorskip("scipy.special")


def boys_gamma(m, T):
    """F_m(T) = gamma(m+1/2, T) / (2 T^{m+1/2}) through the regularised incomplete gamma."""
    a = m + 0.5
    return scipy_special.gammainc(a, T) * scipy_special.gamma(a) / (2.0 * T ** a)


@pytest.mark.parametrize("T", [1e-6, 1e-3, 0.1, 0.7, 2.0, 7.5, 15.0, 29.0, 39.99, 40.01, 55.0, 200.0, 3000.0])
def test_boys_vs_incomplete_gamma(T):
    F = oracle.boys(16, T)
    for m in range(17):
        ref = boys_gamma(m, T)
        assert abs(F[m] - ref) <= 2e-14 * abs(ref) + 1e-300, (m, T, F[m], ref)


def test_boys_at_zero():
    F = oracle.boys(20, 0.0)
    np.testing.assert_allclose(F, [1.0 / (2 * m + 1) for m in range(21)], rtol=1e-15)


@pytest.mark.parametrize("T", [0.01, 1.0, 10.0, 39.0, 41.0, 90.0])
def test_boys_f0_erf_closed_form(T):
    ref = 0.5 * math.sqrt(math.pi / T) * math.erf(math.sqrt(T))
    assert abs(oracle.boys(0, T)[0] - ref) <= 1e-15 * ref


def test_boys_numerical_quadrature():
    """Direct adaptive quadrature of the defining integral."""
    from scipy.integrate import quad

    for m in (0, 3, 7, 12):
        for T in (0.25, 4.0, 22.0, 45.0):
            ref, _ = quad(lambda t: t ** (2 * m) * math.exp(-T * t * t), 0.0, 1.0,
                          epsabs=0.0, epsrel=2e-14, limit=200)
            assert abs(oracle.boys(m, T)[m] - ref) <= 1e-13 * ref


@pytest.mark.parametrize("T", [0.5, 12.0, 39.5, 40.5, 70.0])
def test_boys_recursions_consistent(T):
    """Upward and downward recursions F_{m+1} = ((2m+1) F_m - e^{-T}) / (2T) hold between orders."""
    F = oracle.boys(14, T)
    for m in range(14):
        lhs = (2 * m + 1) * F[m]
        rhs = 2 * T * F[m + 1] + math.exp(-T)
        assert abs(lhs - rhs) <= 1e-14 * lhs


def test_boys_large_T_asymptote():
    """F_m(T) -> (2m-1)!! / 2^{m+1} sqrt(pi / T^{2m+1}) for T -> infinity."""
    T = 400.0
    F = oracle.boys(8, T)
    for m in range(9):
        dfact = 1.0
        for k in range(2 * m - 1, 0, -2):
            dfact *= k
        ref = dfact / 2 ** (m + 1) * math.sqrt(math.pi / T ** (2 * m + 1))
        assert abs(F[m] - ref) <= 1e-14 * ref
