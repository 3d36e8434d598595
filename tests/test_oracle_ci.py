"""Pins of the profile reduction and likelihood-based CI (eq. likelihood).

Reading under test: {theta : l_p(theta) >= max l_p - chi2_1(level)/2}, with
linear interpolation between bracketing grid points and censoring at the grid
edge.
"""
import math

import numpy as np
import pytest
import scipy.stats as st

import oracle


@pytest.mark.parametrize("level", [0.5, 0.8, 0.9, 0.95, 0.99])
def test_chi2_quantile(level):
    assert abs(oracle.chi2_1_quantile(level) - st.chi2.ppf(level, 1)) < 1e-12


@pytest.mark.parametrize("level", [0.9, 0.95])
def test_quadratic_profile_exact_endpoints(level):
    theta0, s = 1.3, 0.4
    half = s * math.sqrt(st.chi2.ppf(level, 1))
    # grid that contains the exact endpoints as grid points: interpolation exact there
    grid = np.sort(np.r_[np.linspace(-1, 3.5, 41), theta0 - half, theta0 + half, theta0])
    prof = -(grid - theta0) ** 2 / (2 * s * s)
    ci = oracle.profile_ci(grid, prof, level)
    assert ci["censored"] == 0 and ci["argmax"] == theta0
    assert abs(ci["lo"] - (theta0 - half)) < 1e-12
    assert abs(ci["hi"] - (theta0 + half)) < 1e-12


def test_linear_profile_interpolation_exact():
    # a tent profile is piecewise linear, so interpolation is exact anywhere
    grid = np.linspace(0, 10, 11)
    prof = -np.abs(grid - 4.0)
    c = 0.5 * oracle.chi2_1_quantile(0.95)
    ci = oracle.profile_ci(grid, prof, 0.95)
    assert abs(ci["lo"] - (4 - c)) < 1e-13 and abs(ci["hi"] - (4 + c)) < 1e-13


def test_censoring_ties_and_nans():
    grid = np.linspace(0, 1, 6)
    prof = np.array([-0.1, 0.0, 0.0, -0.2, -0.3, -0.4])   # never crosses on either side
    ci = oracle.profile_ci(grid, prof, 0.95)
    assert ci["censored"] == 3 and ci["lo"] == 0.0 and ci["hi"] == 1.0 and ci["argmax"] == 0.2
    prof = np.array([-9.0, np.nan, 0.0, np.nan, -9.0, -9.0])
    ci = oracle.profile_ci(grid, prof, 0.95)
    c = 0.5 * oracle.chi2_1_quantile(0.95)
    # lower crossing between grid[0] and grid[2] (grid[1] is NaN and skipped)
    assert ci["censored"] == 0
    assert abs(ci["lo"] - (0.0 + (-c + 9.0) / 9.0 * 0.4)) < 1e-13
    assert abs(ci["hi"] - (0.8 - (-c + 9.0) / 9.0 * 0.4)) < 1e-13
    assert oracle.profile_ci(grid, np.full(6, np.nan), 0.95)["status"] == oracle.OR_INVALID


def test_profile_max_skips_nan():
    vals = np.array([[1.0, np.nan, 3.0], [np.nan, np.nan, np.nan], [-1.0, -2.0, -0.5]])
    prof = oracle.profile_max(vals)
    assert prof[0] == 3.0 and math.isnan(prof[1]) and prof[2] == -0.5
