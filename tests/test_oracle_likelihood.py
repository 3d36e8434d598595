"""Pins of the oracle's profile log-likelihood (eqs. 2, betahat, 4, profile, remlpro).

Each test compares the oracle with something independent of it: a dense
eigen-decomposition of the full likelihood (numpy), a direct GLS solve, a
generic numerical optimiser, the OLS special case, an exact rescaling identity
of the Box-Cox Jacobian, the A-matrix definition of REML, and invariances of
the model.
"""
import math

import numpy as np
import pytest
import scipy.optimize as so

import oracle
from paper_2305_04318_b300 import synth


def small_problem(seed, n=9, p=2):
    rng = np.random.default_rng(seed)
    coords = rng.uniform(0, 1, (n, 2))
    X = np.column_stack([np.ones(n)] + [rng.standard_normal(n) for _ in range(p - 1)])
    y = np.exp(0.3 * rng.standard_normal(n) + 1.0)
    return coords, y, X


OMEGAS = [
    [0.3, 1.0, 0.1, 1.0, 0.0],
    [0.5, 0.4, 0.05, 2.5, 0.7],
    [0.2, 2.5, 0.3, 1.5, 2.0],
    [1.0, 4.0, 0.01, 3.0, 1.1],
]
LAMS = np.array([-0.5, 0.0, 0.5, 1.0, 1.5])


def full_m2loglik(beta, s2, V, yprime, X, y, lam):
    """-2 log-likelihood of eq. 2 by eigen-decomposition of sigma^2 V."""
    n = len(y)
    ev, Q = np.linalg.eigh(s2 * V)
    r = yprime - X @ beta
    z = Q.T @ r
    return (z * z / ev).sum() + np.log(ev).sum() - 2 * (lam - 1) * np.log(y).sum() + n * math.log(2 * math.pi)


def boxcox_np(y, lam):
    return np.log(y) if lam == 0 else (y ** lam - 1) / lam


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("om", OMEGAS)
def test_profile_equals_dense_density_at_gls(seed, om):
    coords, y, X = small_problem(seed)
    V = oracle.build_v(coords, om)
    out = oracle.profile_point(coords, y, X, om, LAMS)
    assert out["status"] == 0
    n = len(y)
    for m, lam in enumerate(LAMS):
        yp = boxcox_np(y, lam)
        Vi = np.linalg.inv(V)
        beta = np.linalg.solve(X.T @ Vi @ X, X.T @ Vi @ yp)          # eq. betahat
        r = yp - X @ beta
        s2 = r @ np.linalg.solve(V, r) / n                            # eq. 4
        np.testing.assert_allclose(out["beta"][m], beta, rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(out["sigma2"][m], s2, rtol=1e-11)
        ll = -0.5 * full_m2loglik(beta, s2, V, yp, X, y, lam)
        np.testing.assert_allclose(out["logL"][m], ll, rtol=1e-12, atol=1e-11)
    # Table 1 statistics
    np.testing.assert_allclose(out["logdet"][0], np.log(np.linalg.eigvalsh(V)).sum(), rtol=1e-12, atol=1e-12)
    Xv = X.T @ np.linalg.solve(V, X)
    np.testing.assert_allclose(out["logdet"][1], np.linalg.slogdet(Xv)[1], rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("om", OMEGAS[:2])
def test_profile_max_is_joint_mle(om):
    """Maximising eq. 2 over (beta, sigma) with a generic optimiser reaches l_p."""
    coords, y, X = small_problem(5, n=10, p=2)
    V = oracle.build_v(coords, om)
    lam = 0.5
    out = oracle.profile_point(coords, y, X, om, [lam])
    yp = boxcox_np(y, lam)
    f = lambda th: full_m2loglik(th[:2], math.exp(th[2]), V, yp, X, y, lam)
    best = so.minimize(f, x0=np.array([0.0, 0.0, 0.0]), method="BFGS", options=dict(gtol=1e-10))
    assert abs(-0.5 * best.fun - out["logL"][0]) < 1e-8
    # and no perturbation of (beta, sigma) beats the profile value
    rng = np.random.default_rng(0)
    th0 = np.r_[out["beta"][0], math.log(out["sigma2"][0])]
    for _ in range(20):
        assert -0.5 * f(th0 + 0.05 * rng.standard_normal(3)) <= out["logL"][0] + 1e-12


def test_ols_limit():
    """phi_X -> 0 makes R = I, V = (1 + nu^2) I and l_p the OLS profile, free of nu^2."""
    rng = np.random.default_rng(3)
    n = 30
    coords = rng.uniform(0, 1, (n, 2))
    X = np.column_stack([np.ones(n), rng.standard_normal(n), rng.standard_normal(n)])
    y = np.exp(rng.standard_normal(n))
    lams = np.array([0.0, 0.5, 1.0])
    vals = []
    for nug in (0.0, 0.3, 2.0):
        out = oracle.profile_point(coords, y, X, [1e-7, 1.5, nug, 1.0, 0.0], lams)
        vals.append(out["logL"])
    for m, lam in enumerate(lams):
        yp = boxcox_np(y, lam)
        res = yp - X @ np.linalg.lstsq(X, yp, rcond=None)[0]
        rss = res @ res
        ref = -0.5 * (n * math.log(rss / n) + n * math.log(2 * math.pi) + n - 2 * (lam - 1) * np.log(y).sum())
        for v in vals:
            np.testing.assert_allclose(v[m], ref, rtol=1e-12)


@pytest.mark.parametrize("lam", [-0.5, 0.0, 0.7, 1.0, 1.5])
def test_boxcox_rescaling(lam):
    """y -> a y shifts l_p by exactly -n log a when X has an intercept."""
    coords, y, X = small_problem(7, n=10, p=2)
    om = OMEGAS[1]
    a = 3.7
    l1 = oracle.profile_point(coords, y, X, om, [lam])["logL"][0]
    l2 = oracle.profile_point(coords, a * y, X, om, [lam])["logL"][0]
    assert abs((l2 - l1) - (-len(y) * math.log(a))) < 1e-10


def test_lambda_one_is_shifted_identity():
    coords, y, X = small_problem(8)
    yp = oracle.boxcox(y, 1.0)
    np.testing.assert_allclose(yp, y - 1, rtol=1e-15)
    np.testing.assert_allclose(oracle.boxcox(y, 0.0), np.log(y), rtol=1e-15)
    np.testing.assert_allclose(oracle.boxcox(y, 1e-12), np.log(y), rtol=1e-9)


def test_isotropy_rotation_scaling_invariance():
    coords, y, X = small_problem(9, n=10, p=2)
    base = oracle.profile_point(coords, y, X, [0.4, 1.2, 0.1, 1.0, 0.0], LAMS)["logL"]
    for ang in (0.3, 1.1, 2.9):   # phi_R = 1: the angle has no effect
        np.testing.assert_allclose(oracle.profile_point(coords, y, X, [0.4, 1.2, 0.1, 1.0, ang], LAMS)["logL"],
                                   base, rtol=1e-13)
    om = [0.4, 1.2, 0.1, 2.5, 0.8]
    ref = oracle.profile_point(coords, y, X, om, LAMS)["logL"]
    # angle period pi
    np.testing.assert_allclose(oracle.profile_point(coords, y, X, [0.4, 1.2, 0.1, 2.5, 0.8 + math.pi], LAMS)["logL"],
                               ref, rtol=1e-12)
    # rotating all sites by -theta and the angle by +theta
    th = 0.6
    Rm = np.array([[math.cos(th), math.sin(th)], [-math.sin(th), math.cos(th)]])
    np.testing.assert_allclose(oracle.profile_point(coords @ Rm.T, y, X, [0.4, 1.2, 0.1, 2.5, 0.8 + th], LAMS)["logL"],
                               ref, rtol=1e-12)
    # scaling sites and range together
    np.testing.assert_allclose(oracle.profile_point(5 * coords, y, X, [2.0, 1.2, 0.1, 2.5, 0.8], LAMS)["logL"],
                               ref, rtol=1e-12)


@pytest.mark.parametrize("om", OMEGAS[:3])
def test_reml_against_a_matrix_definition(om):
    """eq. remlpro equals the likelihood of y* = A y' (A A^T = I, A X = 0, eq. 6)
    profiled over sigma^2, plus the constant p log(2 pi) + log|X^T X| that the
    printed form carries (the identity |A V A^T| = |V||X^T V^-1 X| / |X^T X|)."""
    coords, y, X = small_problem(11, n=10, p=3)
    n, p = X.shape
    V = oracle.build_v(coords, om)
    Qf, _ = np.linalg.qr(X, mode="complete")
    A = Qf[:, p:].T
    out = oracle.profile_point(coords, y, X, om, LAMS, reml=True)
    const = p * math.log(2 * math.pi) + np.linalg.slogdet(X.T @ X)[1]
    for m, lam in enumerate(LAMS):
        ys = A @ boxcox_np(y, lam)
        AVA = A @ V @ A.T
        s2 = ys @ np.linalg.solve(AVA, ys) / (n - p)
        m2 = (n - p) * math.log(s2) + np.linalg.slogdet(AVA)[1] + (n - p) + (n - p) * math.log(2 * math.pi) \
            - 2 * (lam - 1) * np.log(y).sum()
        np.testing.assert_allclose(-2 * out["logL"][m], m2 + const, rtol=1e-12)
        np.testing.assert_allclose(out["sigma2"][m], s2, rtol=1e-11)


def test_not_pd_status_and_nan():
    coords, y, X = small_problem(12, n=8)
    coords[3] = coords[2]              # duplicate site and no nugget: V singular
    out = oracle.profile_point(coords, y, X, [0.3, 1.0, 0.0, 1.0, 0.0], LAMS)
    assert out["status"] == oracle.OR_NOT_PD
    assert np.all(np.isnan(out["logL"]))
    out = oracle.profile_point(coords, y, X, [0.3, 1.0, 0.05, 1.0, 0.0], LAMS)
    assert out["status"] == 0 and np.all(np.isfinite(out["logL"]))


def test_batch_equals_points():
    w = synth.iso100()
    ds = w.datasets[0]
    P = w.params[0][::7]
    b = oracle.profile_batch(ds.coords, ds.y, ds.X, P, w.lambdas, nthreads=2)
    for k in range(len(P)):
        o = oracle.profile_point(ds.coords, ds.y, ds.X, P[k], w.lambdas)
        assert b["status"][k] == o["status"]
        np.testing.assert_array_equal(b["logL"][k], o["logL"])


def test_near_singular_criterion_of_the_mixed_parity_tests():
    """The criterion the mixed-precision parity tests use to accept a status
    disagreement: a V with a duplicated site and no nugget is singular (FP64
    Cholesky fails or leaves a pivot at rounding level), the same V with
    nu^2 = 0.1 is far from singular, and a smooth long-range V (kappa = 8) with
    no nugget is near singular while a small nugget moves it away."""
    from gpu_util import min_pivot, singular_threshold
    rng = np.random.default_rng(3)
    c = rng.uniform(0, 1, size=(40, 2))
    c[7] = c[3]
    w0 = np.array([0.3, 1.0, 0.0, 1.0, 0.0])
    assert min_pivot(c, w0) <= singular_threshold(40, 0.0)
    w1 = w0.copy()
    w1[2] = 0.1
    assert min_pivot(c, w1) > 1e3 * singular_threshold(40, 0.1)
    c2 = rng.uniform(0, 4, size=(200, 2))
    smooth = np.array([40.0, 8.0, 0.0, 1.0, 0.0])
    assert min_pivot(c2, smooth) <= singular_threshold(200, 0.0)
    smooth[2] = 1e-2
    assert min_pivot(c2, smooth) > 1e3 * singular_threshold(200, 1e-2)
