"""Pins of the oracle's Matern correlation and anisotropic distance (eq. matern).

Readings under test: normaliser 2^(1-kappa)/Gamma(kappa) (so rho(0+) = 1),
argument u = sqrt(8 kappa) d, rotation matrix exactly as printed, phi_Y = phi_X/phi_R.
"""
import math

import numpy as np
import pytest

import oracle

D = np.concatenate([np.geomspace(1e-7, 1.0, 30), np.linspace(1.0, 20.0, 30)])


def test_kappa_half_is_exponential():
    # u = sqrt(4) d = 2d and rho = exp(-u) = exp(-2d)
    np.testing.assert_allclose(oracle.matern(D, 0.5), np.exp(-2 * D), rtol=2e-14, atol=1e-300)


def test_kappa_three_halves_closed_form():
    u = math.sqrt(12.0) * D
    np.testing.assert_allclose(oracle.matern(D, 1.5), (1 + u) * np.exp(-u), rtol=2e-14, atol=1e-300)


def test_kappa_five_halves_closed_form():
    u = math.sqrt(20.0) * D
    np.testing.assert_allclose(oracle.matern(D, 2.5), (1 + u + u * u / 3) * np.exp(-u), rtol=3e-14, atol=1e-300)


@pytest.mark.parametrize("kappa", [0.1, 0.5, 1.0, 1.7, 4.0, 8.0])
def test_zero_distance_limit_and_monotone(kappa):
    assert oracle.matern(0.0, kappa) == 1.0
    small = oracle.matern(1e-9, kappa)
    assert abs(small - 1.0) < 1e-1 if kappa < 0.5 else abs(small - 1.0) < 1e-6
    r = oracle.matern(np.linspace(0, 5, 200), kappa)
    assert np.all(np.diff(r) <= 0)


def test_kappa_to_infinity_is_gaussian():
    # rho -> exp(-2 d^2) with an O(1/kappa) error
    d = np.linspace(0.05, 1.5, 30)
    g = np.exp(-2 * d * d)
    e50 = np.max(np.abs(oracle.matern(d, 50.0) - g))
    e100 = np.max(np.abs(oracle.matern(d, 100.0) - g))
    assert e100 < e50 < 0.02
    assert 1.6 < e50 / e100 < 2.4


def test_distance_literal_rotation():
    # h = (1, 0), phi_A = pi/2: Rot h = (cos, sin) = (0, 1) -> d = 1/phi_Y = phi_R/phi_X
    assert abs(oracle.aniso_distance(1.0, 0.0, 2.0, 3.0, math.pi / 2) - 1.5) < 1e-15
    # h = (0, 1), phi_A = pi/2: Rot h = (-1, 0) -> d = 1/phi_X
    assert abs(oracle.aniso_distance(0.0, 1.0, 2.0, 3.0, math.pi / 2) - 0.5) < 1e-15
    # phi_A = 0: d = sqrt((h1/phi_X)^2 + (h2 phi_R/phi_X)^2)
    assert abs(oracle.aniso_distance(3.0, 4.0, 2.0, 2.0, 0.0) - math.hypot(1.5, 4.0)) < 1e-15


def test_distance_invariants():
    rng = np.random.default_rng(0)
    for _ in range(50):
        h1, h2 = rng.normal(size=2)
        phx, ratio, ang = rng.uniform(0.1, 3), rng.uniform(1, 4), rng.uniform(0, math.pi)
        d = oracle.aniso_distance(h1, h2, phx, ratio, ang)
        # period pi in the angle, sign of h irrelevant
        assert abs(oracle.aniso_distance(h1, h2, phx, ratio, ang + math.pi) - d) < 1e-13
        assert abs(oracle.aniso_distance(-h1, -h2, phx, ratio, ang) - d) < 1e-13
        # isotropy: ratio 1 makes the angle irrelevant
        assert abs(oracle.aniso_distance(h1, h2, phx, 1.0, ang) - math.hypot(h1, h2) / phx) < 1e-13
        # rotating h by -theta and the angle by +theta leaves d unchanged
        th = rng.uniform(0, 2 * math.pi)
        r1 = math.cos(th) * h1 + math.sin(th) * h2
        r2 = -math.sin(th) * h1 + math.cos(th) * h2
        assert abs(oracle.aniso_distance(r1, r2, phx, ratio, ang + th) - d) < 1e-12
        # scaling h and phi_X together leaves d unchanged
        assert abs(oracle.aniso_distance(3 * h1, 3 * h2, 3 * phx, ratio, ang) - d) < 1e-13


def test_build_v_structure():
    rng = np.random.default_rng(1)
    coords = rng.uniform(0, 1, (12, 2))
    V = oracle.build_v(coords, [0.3, 1.3, 0.2, 2.0, 0.4])
    assert np.allclose(V, V.T, rtol=0, atol=0)
    assert np.allclose(np.diag(V), 1.2)
    assert np.linalg.eigvalsh(V).min() > 0.2 - 1e-12   # R is PSD, so V >= nu^2 I
    i, j = 7, 3
    d = oracle.aniso_distance(*(coords[i] - coords[j]), 0.3, 2.0, 0.4)
    assert V[i, j] == oracle.matern(d, 1.3)
