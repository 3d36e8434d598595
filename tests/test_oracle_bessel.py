"""Pins of the oracle's modified Bessel function K_nu (needed by eq. matern).

The oracle computes K_nu by Temme's series (x <= 2) and a trapezoid rule on
the integral representation (x > 2).  These tests pin it to things other than
itself: scipy.special.kv/kve (an independent library routine), elementary
closed forms of half-integer orders, the order recurrence and the Wronskian
with scipy's I_nu.
"""
import mpmath
import numpy as np
import pytest
import scipy.special as sp

import oracle

NUS = np.geomspace(0.1, 8.0, 15).tolist() + [0.0, 0.5, 1.0, 1.5, 2.0, 2.5, 3.0, 4.0]
XS = np.concatenate([np.geomspace(1e-8, 2.0, 25), [1.999999, 2.0, 2.000001],
                     np.geomspace(2.0, 700.0, 25)])


@pytest.mark.parametrize("nu", NUS)
def test_scaled_k_matches_scipy(nu):
    got = oracle.bessel_k_scaled(nu, XS)
    ref = sp.kve(nu, XS)
    np.testing.assert_allclose(got, ref, rtol=2e-13, atol=0)


@pytest.mark.parametrize("nu", [0.1, 0.13675, 0.5, 0.9, 1.0, 2.3, 4.75, 8.0, 12.0, 16.5, 20.0])
def test_scaled_k_matches_mpmath(nu):
    # 30-digit reference from mpmath's besselk (an independent library routine)
    mpmath.mp.dps = 30
    x = XS[::3]
    ref = np.array([float(mpmath.besselk(nu, v) * mpmath.exp(v)) for v in x])
    np.testing.assert_allclose(oracle.bessel_k_scaled(nu, x), ref, rtol=3e-15 * 10, atol=0)


@pytest.mark.parametrize("nu", NUS)
def test_unscaled_k_matches_scipy(nu):
    x = XS[XS < 600]
    np.testing.assert_allclose(oracle.bessel_k(nu, x), sp.kv(nu, x), rtol=2e-13, atol=0)


def test_half_integer_closed_forms():
    x = np.geomspace(1e-3, 300, 60)
    base = np.sqrt(np.pi / (2 * x))
    np.testing.assert_allclose(oracle.bessel_k_scaled(0.5, x), base, rtol=2e-14)
    np.testing.assert_allclose(oracle.bessel_k_scaled(1.5, x), base * (1 + 1 / x), rtol=2e-14)
    np.testing.assert_allclose(oracle.bessel_k_scaled(2.5, x), base * (1 + 3 / x + 3 / x**2), rtol=2e-14)


@pytest.mark.parametrize("nu", [0.1, 0.37, 1.0, 2.2, 5.5])
def test_order_recurrence(nu):
    # K_{nu+1}(x) = K_{nu-1}(x) + (2 nu / x) K_nu(x)   (DLMF 10.29.1)
    x = np.geomspace(1e-2, 100, 40)
    lhs = oracle.bessel_k_scaled(nu + 1, x)
    rhs = oracle.bessel_k_scaled(abs(nu - 1), x) + 2 * nu / x * oracle.bessel_k_scaled(nu, x)
    np.testing.assert_allclose(lhs, rhs, rtol=5e-14)


@pytest.mark.parametrize("nu", [0.0, 0.3, 1.0, 2.7, 7.9])
def test_wronskian(nu):
    # I_nu K_{nu+1} + I_{nu+1} K_nu = 1/x   (DLMF 10.28.2)
    x = np.geomspace(1e-2, 50, 30)
    w = sp.ive(nu, x) * oracle.bessel_k_scaled(nu + 1, x) + sp.ive(nu + 1, x) * oracle.bessel_k_scaled(nu, x)
    np.testing.assert_allclose(w * x, 1.0, rtol=1e-13)


def test_small_argument_limit():
    # K_nu(x) ~ Gamma(nu) 2^(nu-1) x^-nu as x -> 0 (nu > 0); K_0(x) ~ -log(x/2) - gamma
    x = 1e-8
    for nu in (0.5, 1.0, 3.0):
        lead = sp.gamma(nu) * 2 ** (nu - 1) * x ** (-nu)
        assert abs(oracle.bessel_k(nu, x) / lead - 1) < 1e-6
    assert abs(oracle.bessel_k(0.0, x) - (-np.log(x / 2) - np.euler_gamma)) < 1e-12
