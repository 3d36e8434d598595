"""Pins of the oracle's post-processing of the Table-1 statistics (Sections 3.4-3.6).

Each test compares the oracle with something independent of it:
  - beta_j profile: a direct GLS fit of the offset model y' - X_j b on X_-j and
    the dense eigen-decomposed density of eq. 2; a generic numerical optimiser
    over (beta_-j, sigma); the joint maximum at b = beta-hat_j;
  - sigma profile: the dense density of eq. 2 at (beta-hat, s); the joint
    maximum at s^2 = sigma-hat^2;
  - convex-hull profile: the brute-force upper concave envelope (largest
    interpolation over every bracketing pair of points), scipy's ConvexHull,
    and concave/collinear/degenerate special cases;
  - internal parameters: closed forms and the axis-exchange identity of the
    anisotropic distance.
"""
import math

import numpy as np
import pytest
import scipy.optimize as so
from scipy.spatial import ConvexHull

import oracle


def small_problem(seed, n=12, p=3):
    rng = np.random.default_rng(seed)
    coords = rng.uniform(0, 1, (n, 2))
    X = np.column_stack([np.ones(n)] + [rng.standard_normal(n) for _ in range(p - 1)])
    y = np.exp(0.3 * rng.standard_normal(n) + 1.0 + 0.2 * X[:, -1])
    return coords, y, X


OMEGAS = [
    [0.3, 1.0, 0.1, 1.0, 0.0],
    [0.5, 0.4, 0.05, 2.5, 0.7],
    [0.2, 2.5, 0.3, 1.5, 2.0],
]
LAMS = np.array([-0.5, 0.0, 0.5, 1.0])


def boxcox_np(y, lam):
    return np.log(y) if lam == 0 else (y ** lam - 1) / lam


def dense_m2loglik(beta, s2, V, yp, X, y, lam):
    """-2 log-likelihood of eq. 2 by eigen-decomposition of sigma^2 V."""
    n = len(y)
    ev, Q = np.linalg.eigh(s2 * V)
    z = Q.T @ (yp - X @ beta)
    return (z * z / ev).sum() + np.log(ev).sum() - 2 * (lam - 1) * np.log(y).sum() + n * math.log(2 * math.pi)


def dense_beta_profile_point(coords, y, X, om, lam, j, b):
    """l at beta_j = b with beta_-j and sigma at their maximisers: direct GLS of
    the offset response on X_-j, then the dense density."""
    n, p = X.shape
    V = oracle.build_v(coords, om)
    Vi = np.linalg.inv(V)
    yp = boxcox_np(y, lam)
    r = yp - X[:, j] * b
    Xm = np.delete(X, j, axis=1)
    bm = np.linalg.solve(Xm.T @ Vi @ Xm, Xm.T @ Vi @ r) if p > 1 else np.zeros(0)
    e = r - Xm @ bm
    s2 = float(e @ Vi @ e) / n
    beta = np.insert(bm, j, b)
    return -0.5 * dense_m2loglik(beta, s2, V, yp, X, y, lam)


def stats(coords, y, X, omegas, lams):
    ssq, ld, st, logL, beta, s2 = [], [], [], [], [], []
    for om in omegas:
        o = oracle.profile_point(coords, y, X, om, lams)
        ssq.append(o["ssq"]); ld.append(o["logdet"]); st.append(o["status"])
        logL.append(o["logL"]); beta.append(o["beta"]); s2.append(o["sigma2"])
    return (np.array(ssq), np.array(ld), np.array(st, dtype=np.int32), np.array(logL),
            np.array(beta), np.array(s2))


@pytest.mark.parametrize("seed", [0, 1])
@pytest.mark.parametrize("j", [0, 1, 2])
def test_beta_profile_equals_dense_gls(seed, j):
    coords, y, X = small_problem(seed)
    ssq, ld, st, logL, beta, _ = stats(coords, y, X, OMEGAS, LAMS)
    grid = np.linspace(-1.5, 2.5, 9)
    prof = oracle.profile_beta(len(y), ssq, ld, LAMS, oracle.sum_log(y), j, grid, st)
    for g, b in enumerate(grid):
        dense = max(dense_beta_profile_point(coords, y, X, om, lam, j, b)
                    for om in OMEGAS for lam in LAMS)
        assert abs(prof[g] - dense) <= 1e-9 * max(1.0, abs(dense)), (g, prof[g], dense)


def test_beta_profile_intercept_only():
    # p = 1: no other coefficient to profile out; RSS(b) = (y' - b 1)^T V^-1 (y' - b 1)
    coords, y, X = small_problem(3, p=1)
    ssq, ld, st, *_ = stats(coords, y, X, OMEGAS[:2], LAMS)
    grid = np.linspace(0.0, 3.0, 7)
    prof = oracle.profile_beta(len(y), ssq, ld, LAMS, oracle.sum_log(y), 0, grid, st)
    for g, b in enumerate(grid):
        dense = max(dense_beta_profile_point(coords, y, X, om, lam, 0, b)
                    for om in OMEGAS[:2] for lam in LAMS)
        assert abs(prof[g] - dense) <= 1e-9 * max(1.0, abs(dense))


def test_beta_profile_is_maximum_over_nuisance():
    # a generic optimiser over (beta_-j, log sigma^2) at fixed beta_j reaches the same value
    coords, y, X = small_problem(5)
    om, lam, j, b = OMEGAS[1], 0.5, 1, 0.7
    ssq, ld, st, *_ = stats(coords, y, X, [om], np.array([lam]))
    prof = oracle.profile_beta(len(y), ssq, ld, [lam], oracle.sum_log(y), j, [b], st)[0]
    V = oracle.build_v(coords, om)
    yp = boxcox_np(y, lam)

    def negll(t):
        beta = np.insert(t[:-1], j, b)
        return 0.5 * dense_m2loglik(beta, math.exp(t[-1]), V, yp, X, y, lam)

    res = so.minimize(negll, np.zeros(X.shape[1]), method="Nelder-Mead",
                      options=dict(xatol=1e-10, fatol=1e-12, maxiter=20000, maxfev=40000))
    assert abs(-res.fun - prof) < 1e-6
    assert -res.fun <= prof + 1e-9


def test_beta_profile_touches_joint_maximum():
    # at b = beta-hat_j the profile over beta_j equals l_p(omega, lambda) (eq. profile); elsewhere below
    coords, y, X = small_problem(7)
    om = OMEGAS[2]
    ssq, ld, st, logL, beta, _ = stats(coords, y, X, [om], LAMS)
    sl = oracle.sum_log(y)
    for m, lam in enumerate(LAMS):
        for j in range(X.shape[1]):
            bh = beta[0, m, j]
            # single-lambda stats: restrict ssq to lambda m and the covariates
            sub = np.r_[m, np.arange(len(LAMS), len(LAMS) + X.shape[1])]
            one = oracle.profile_beta(len(y), ssq[:, sub][:, :, sub], ld, [lam], sl, j,
                                      [bh, bh + 0.3, bh - 0.3], st)
            assert abs(one[0] - logL[0, m]) < 1e-9 * abs(logL[0, m])
            assert one[1] < logL[0, m] and one[2] < logL[0, m]


def test_beta_profile_skips_failed_points_and_bad_index():
    coords, y, X = small_problem(2)
    ssq, ld, st, *_ = stats(coords, y, X, OMEGAS[:2], LAMS)
    sl = oracle.sum_log(y)
    st_bad = np.array([1, 3], dtype=np.int32)
    prof = oracle.profile_beta(len(y), ssq, ld, LAMS, sl, 0, [0.5], st_bad)
    assert np.isnan(prof[0])
    # the RETRIED flag bit (16) does not exclude a point
    st_flag = np.array([16, 1], dtype=np.int32)
    a = oracle.profile_beta(len(y), ssq, ld, LAMS, sl, 0, [0.5], st_flag)
    b = oracle.profile_beta(len(y), ssq[:1], ld[:1], LAMS, sl, 0, [0.5], None)
    assert a[0] == b[0]
    with pytest.raises(ValueError):
        oracle.profile_beta(len(y), ssq, ld, LAMS, sl, X.shape[1], [0.5], st)


@pytest.mark.parametrize("seed", [0, 1])
def test_sigma_profile_equals_dense(seed):
    coords, y, X = small_problem(seed)
    ssq, ld, st, logL, beta, _ = stats(coords, y, X, OMEGAS, LAMS)
    sgrid = np.linspace(0.05, 1.5, 11)
    prof = oracle.profile_sigma(len(y), ssq, ld, LAMS, oracle.sum_log(y), sgrid, st)
    for g, s in enumerate(sgrid):
        dense = -np.inf
        for om in OMEGAS:
            V = oracle.build_v(coords, om)
            Vi = np.linalg.inv(V)
            for lam in LAMS:
                yp = boxcox_np(y, lam)
                bh = np.linalg.solve(X.T @ Vi @ X, X.T @ Vi @ yp)
                dense = max(dense, -0.5 * dense_m2loglik(bh, s * s, V, yp, X, y, lam))
        assert abs(prof[g] - dense) <= 1e-9 * max(1.0, abs(dense)), (g, prof[g], dense)


def test_sigma_profile_touches_joint_maximum():
    coords, y, X = small_problem(4)
    ssq, ld, st, logL, beta, s2 = stats(coords, y, X, [OMEGAS[0]], LAMS)
    sl = oracle.sum_log(y)
    q = len(LAMS) + X.shape[1]
    for m, lam in enumerate(LAMS):
        sub = np.r_[m, np.arange(len(LAMS), q)]
        s = math.sqrt(s2[0, m])
        v = oracle.profile_sigma(len(y), ssq[:, sub][:, :, sub], ld, [lam], sl,
                                 [s, 0.8 * s, 1.25 * s], st)
        assert abs(v[0] - logL[0, m]) < 1e-9 * abs(logL[0, m])
        assert v[1] < logL[0, m] and v[2] < logL[0, m]


def test_lambda_profile_is_column_max():
    logL = np.array([[1.0, np.nan, -3.0], [2.0, np.nan, -4.0], [0.5, np.nan, np.nan]])
    prof = oracle.profile_lambda(logL)
    assert prof[0] == 2.0 and np.isnan(prof[1]) and prof[2] == -3.0


def brute_envelope(x, v, xq):
    """Upper concave envelope by definition: in 1-D every point of the hull is a
    convex combination of at most two cloud points (Caratheodory), so the
    envelope at t is the largest interpolation over pairs bracketing t."""
    ok = np.isfinite(v)
    x, v = x[ok], v[ok]
    out = np.full(len(xq), np.nan)
    for t, q in enumerate(xq):
        best = -np.inf
        for a in range(len(x)):
            if x[a] == q:
                best = max(best, v[a])
            for b in range(len(x)):
                if x[a] < q < x[b]:
                    best = max(best, v[a] + (v[b] - v[a]) * (q - x[a]) / (x[b] - x[a]))
        if best > -np.inf:
            out[t] = best
    return out


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_hull_equals_brute_envelope(seed):
    rng = np.random.default_rng(seed)
    K = 40
    x = np.round(rng.uniform(-1, 2, K), 1)           # coarse: repeated x values
    v = -(x - 0.4) ** 2 + 0.3 * rng.standard_normal(K)
    v[rng.choice(K, 4, replace=False)] = np.nan
    xq = np.r_[np.linspace(-1.2, 2.2, 57), x[:10]]
    out, on, nh = oracle.profile_hull(x, v, xq)
    ref = brute_envelope(x, v, xq)
    assert np.array_equal(np.isnan(out), np.isnan(ref))
    f = ~np.isnan(ref)
    assert np.max(np.abs(out[f] - ref[f])) < 1e-12
    assert nh == on.sum() and nh >= 2


@pytest.mark.parametrize("seed", [0, 1])
def test_hull_vertices_match_scipy(seed):
    rng = np.random.default_rng(10 + seed)
    K = 200
    x = rng.uniform(0, 1, K)
    v = rng.standard_normal(K)
    _, on, nh = oracle.profile_hull(x, v, np.array([0.5]))
    hull = ConvexHull(np.column_stack([x, v]))
    il, ir = np.argmin(x), np.argmax(x)
    upper = set()
    for i in hull.vertices:
        # on or above the chord from the leftmost to the rightmost point: upper chain
        chord = v[il] + (v[ir] - v[il]) * (x[i] - x[il]) / (x[ir] - x[il])
        if i in (il, ir) or v[i] > chord:
            upper.add(int(i))
    assert set(np.nonzero(on)[0].tolist()) == upper


def test_hull_concave_and_collinear():
    rng = np.random.default_rng(7)
    xs = np.sort(rng.uniform(0, 1, 25))
    f = -(xs - 0.3) ** 2
    # other points strictly below the chords between the samples, inside their range
    xo = rng.uniform(xs[0], xs[-1], 50)
    x = np.r_[xs, xo]
    v = np.r_[f, np.interp(xo, xs, f) - rng.uniform(0.01, 1, 50)]
    out, on, nh = oracle.profile_hull(x, v, xs)
    assert nh == 25 and on[:25].all() and not on[25:].any()
    assert np.max(np.abs(out - f)) < 1e-15
    # collinear: the middle point lies on the edge and is not a vertex
    out, on, nh = oracle.profile_hull(np.array([0.0, 1.0, 2.0]), np.array([0.0, 1.0, 2.0]),
                                      np.array([0.5, 1.0, 2.0]))
    assert nh == 2 and list(on) == [1, 0, 1]
    assert np.allclose(out, [0.5, 1.0, 2.0], rtol=0, atol=1e-15)


def test_hull_degenerate():
    out, on, nh = oracle.profile_hull(np.array([1.0, 2.0]), np.array([np.nan, np.nan]),
                                      np.array([1.0, 1.5]))
    assert nh == 0 and np.isnan(out).all() and not on.any()
    out, on, nh = oracle.profile_hull(np.array([1.0, 1.0, 1.0]), np.array([3.0, 5.0, 5.0]),
                                      np.array([1.0, 0.9, 1.1]))
    # one distinct x: one vertex, the lowest index among the equal largest values
    assert nh == 1 and list(on) == [0, 1, 0]
    assert out[0] == 5.0 and np.isnan(out[1]) and np.isnan(out[2])
    out, on, nh = oracle.profile_hull(np.zeros(0), np.zeros(0), np.array([0.0]))
    assert nh == 0 and np.isnan(out[0])


def test_internal_params_closed_forms():
    w = oracle.internal_params([[2.0, 1.0, 0.25, 2.0, 0.0]])[0]
    assert np.allclose(w, [math.log(2.0), 0.0, 0.5, 1.0, 0.0], rtol=0, atol=1e-15)
    w = oracle.internal_params([[3.0, 9.0, 0.0, 1.0, 1.234]], kappa_hat_large=True)[0]
    assert np.allclose(w, [2 * math.log(3.0), 1 / 3, 0.0, 0.0, 0.0], rtol=0, atol=1e-15)
    # exp(gamma_1 / 2) is the geometric mean of phi_X and phi_Y
    phx, rat = 1.7, 3.2
    w = oracle.internal_params([[phx, 1.5, 0.1, rat, 0.4]])[0]
    assert abs(math.exp(w[0] / 2) - math.sqrt(phx * phx / rat)) < 1e-14
    assert abs(math.hypot(w[3], w[4]) - math.sqrt(rat - 1)) < 1e-14
    assert abs(math.atan2(w[4], w[3]) - 0.8) < 1e-14


@pytest.mark.parametrize("rat,ang", [(0.5, 0.3), (0.25, 2.0), (0.8, -0.7)])
def test_internal_params_axis_exchange(rat, ang):
    # a ratio below one maps to the same correlation with the axes exchanged
    phx = 1.3
    phy = phx / rat
    swapped = [phy, 1.0, 0.1, phy / phx, ang + math.pi / 2]
    rng = np.random.default_rng(1)
    for h in rng.standard_normal((5, 2)):
        d1 = oracle.aniso_distance(h[0], h[1], phx, rat, ang)
        d2 = oracle.aniso_distance(h[0], h[1], swapped[0], swapped[3], swapped[4])
        assert abs(d1 - d2) < 1e-13 * max(1.0, d1)
    w1 = oracle.internal_params([[phx, 1.0, 0.1, rat, ang]])[0]
    w2 = oracle.internal_params([swapped])[0]
    assert np.allclose(w1, w2, rtol=0, atol=1e-13)


def dense_beta_profile_reml_point(coords, y, X, om, lam, j, b):
    """REML criterion of the Appendix (eq. remlprofileytilde) at beta_j = b:
    (n-p) log(RSS(b)/(n-p)) + log|V| + log|X^T V^-1 X| - 2(lambda-1) sum log y
    + n log(2 pi) + n - p, with RSS(b) from a direct GLS fit of the offset
    response on X_-j and the log-determinants by numpy.linalg.slogdet."""
    n, p = X.shape
    V = oracle.build_v(coords, om)
    Vi = np.linalg.inv(V)
    yp = boxcox_np(y, lam)
    r = yp - X[:, j] * b
    Xm = np.delete(X, j, axis=1)
    bm = np.linalg.solve(Xm.T @ Vi @ Xm, Xm.T @ Vi @ r) if p > 1 else np.zeros(0)
    e = r - Xm @ bm
    rss = float(e @ Vi @ e)
    m2 = ((n - p) * math.log(rss / (n - p)) + np.linalg.slogdet(V)[1] + np.linalg.slogdet(X.T @ Vi @ X)[1]
          - 2 * (lam - 1) * np.log(y).sum() + n * math.log(2 * math.pi) + n - p)
    return -0.5 * m2


@pytest.mark.parametrize("j", [0, 2])
def test_beta_profile_reml_equals_dense(j):
    coords, y, X = small_problem(3)
    ssq, ld, st, logL, beta, _ = stats(coords, y, X, OMEGAS, LAMS)
    grid = np.linspace(-1.5, 2.5, 9)
    prof = oracle.profile_beta(len(y), ssq, ld, LAMS, oracle.sum_log(y), j, grid, st, reml=True)
    for g, b in enumerate(grid):
        dense = max(dense_beta_profile_reml_point(coords, y, X, om, lam, j, b) for om in OMEGAS for lam in LAMS)
        assert abs(prof[g] - dense) <= 1e-9 * max(1.0, abs(dense)), (g, prof[g], dense)


def test_beta_profile_reml_at_gls_estimate_is_remlpro():
    # at b = beta-hat_j the offset fit leaves RSS(b) = RSS: the REML beta profile
    # of one point and lambda equals its REML profile likelihood (eq. remlpro)
    coords, y, X = small_problem(4)
    om, lam = OMEGAS[1], np.array([0.5])
    o = oracle.profile_point(coords, y, X, om, lam, reml=True)
    bj = o["beta"][0][1]
    prof = oracle.profile_beta(len(y), o["ssq"][None], o["logdet"][None], lam, oracle.sum_log(y), 1,
                               np.array([bj]), reml=True)
    assert prof[0] == pytest.approx(o["logL"][0], rel=1e-12)
    ml = oracle.profile_beta(len(y), o["ssq"][None], o["logdet"][None], lam, oracle.sum_log(y), 1, np.array([bj]))
    assert ml[0] != pytest.approx(prof[0], abs=1e-6)
