"""The fused small-n path (one thread block per point, whole bordered matrix
in shared memory, FP64) against the oracle at the FP64 tolerance, for ragged
sizes up to the largest that fits (n + M + p = 224), nu^2 = 0 points,
duplicate sites (not positive definite), REML, the Table-1 statistics, and
against the tiled path (PLK_FLAG_NO_FUSED) on the same points."""
import math

import numpy as np
import pytest

from paper_2305_04318_b300 import native as nv, synth
from gpu_util import RTOL_LOGL, compare, gpu_eval, oracle_eval

pytestmark = pytest.mark.gpu


def _points(seed, K, nug0=2):
    P = synth.omega_from_unit(np.random.default_rng(seed).uniform(size=(K, 5)))
    P[:nug0, 2] = 0.0            # no nugget
    return P


@pytest.mark.parametrize("n,p,M", [(3, 2, 1), (17, 1, 1), (64, 3, 9), (100, 2, 1), (129, 5, 9), (160, 3, 9),
                                   (212, 3, 9), (200, 16, 8)])
def test_fused_matches_oracle(n, p, M):
    assert n + p + M <= 224
    ds = synth.aniso_dataset(300 + n, n, math.sqrt(max(n, 10) / 10), p)
    P = _points(n, 11)
    lams = np.linspace(-0.5, 1.5, M)
    o = oracle_eval(ds, P, lams)
    g = gpu_eval(ds, P, lams, batch=5)
    compare(g, o, rtol=RTOL_LOGL, what=f"fused n={n}")
    assert np.all(g["err_bound"] == 0.0)
    # against the tiled path on the points with a nugget (see test_fused_size_boundary)
    t = gpu_eval(ds, P, lams, batch=5, flags=nv.FLAG_NO_FUSED)
    ok = (o["status"] == 0) & (P[:, 2] > 0)
    np.testing.assert_allclose(g["logL"][ok], t["logL"][ok], rtol=1e-10)
    np.testing.assert_array_equal(g["status"][P[:, 2] > 0], t["status"][P[:, 2] > 0])


def test_fused_size_boundary():
    """n + q = 224 takes the fused kernel, 225 the tiled path: both match the
    oracle (on points with a nugget: with nu^2 = 0 and smooth long-range
    correlations the tiled path's products with explicit diagonal-block
    inverses lose more than 1e-8 of l_p, while the fused kernel's column
    Cholesky, like the oracle's, does not)."""
    lams = synth.LAMBDA_GRID_9
    for n in (212, 213):
        ds = synth.aniso_dataset(400 + n, n, math.sqrt(n / 10), 3)
        P = _points(n, 6, nug0=0)
        compare(gpu_eval(ds, P, lams), oracle_eval(ds, P, lams), rtol=RTOL_LOGL, what=f"n={n}")


def test_fused_reml_and_ssq():
    ds = synth.aniso_dataset(500, 150, math.sqrt(15.0), 3)
    P = _points(500, 20)
    lams = synth.LAMBDA_GRID_9
    f = gpu_eval(ds, P, lams, with_ssq=True)
    compare(gpu_eval(ds, P, lams, reml=True), oracle_eval(ds, P, lams, reml=True), rtol=RTOL_LOGL, what="reml")
    t = gpu_eval(ds, P, lams, with_ssq=True, flags=nv.FLAG_NO_FUSED)
    ok = (f["status"] == 0) & (P[:, 2] > 0)
    np.testing.assert_allclose(f["ssq_yx"][ok], t["ssq_yx"][ok], rtol=1e-9, atol=1e-9)


@pytest.mark.parametrize("n,p,M", [(3, 2, 1), (64, 3, 9), (100, 2, 1), (160, 3, 9), (212, 3, 9)])
def test_fused_mixed_double_float(n, p, M):
    """PLK_MIXED on small datasets: the fused kernel in double-float FP32
    within 1e-3 of the oracle (statuses equal but on near-singular points);
    its bound 2^-36 (1 + nu^2) sum 1/d_j stays above twice the measured error;
    the points it sends to FP64 (bound above the mixed tolerance, or a failed
    factorisation)
    carry the FP64 fused kernel's results exactly."""
    from test_gpu_mixed import mixed_compare
    ds = synth.aniso_dataset(600 + n, n, math.sqrt(max(n, 10) / 10), p)
    P = _points(600 + n, 14, nug0=3)
    P[3:6] = synth.ill_conditioned_points()[[6, 30, 62]]   # kappa = 8, long ranges, small nuggets
    lams = np.linspace(-0.5, 1.5, M)
    o = oracle_eval(ds, P, lams)
    m = gpu_eval(ds, P, lams, precision=nv.MIXED, batch=5)
    mixed_compare(m, o, f"fused df n={n}", coords=ds.coords, params=P)
    g5 = gpu_eval(ds, P, lams, precision=nv.MIXED, flags=nv.FLAG_NO_RETRY)
    ok = (g5["status"] == 0) & (o["status"] == 0)
    err = np.max(np.abs(g5["logL"] - o["logL"]), axis=1)[ok]
    assert np.all((err <= 0.5 * g5["err_bound"][ok]) | (err <= 1e-9)), (err, g5["err_bound"][ok])
    f = gpu_eval(ds, P, lams)
    r = (m["status"] & nv.POINT_FP64) != 0
    assert np.all(m["err_bound"][r] == 0.0) and np.all(m["err_bound"][~r & (m["status"] & 15 == 0)] > 0)
    for k in ("logL", "sigma2", "beta", "logdet"):
        np.testing.assert_array_equal(m[k][r], f[k][r], err_msg=k)
    np.testing.assert_array_equal(m["status"][r] & 15, f["status"][r])


def test_fused_duplicate_sites_and_bad_params():
    """Duplicate sites with no nugget make V exactly singular: whether an FP64
    factorisation fails or survives on a pivot of rounding size is decided by
    rounding, so a status that differs from the oracle's is allowed on such a
    point only (the oracle shows its V singular to FP64 precision); the other
    points match.  An invalid parameter row gives BAD_PARAM and NaN."""
    from gpu_util import compare_fp64_singular
    ds = synth.aniso_dataset(501, 90, 3.0, 2)
    ds.coords[10] = ds.coords[4]
    P = _points(501, 8, nug0=4)
    lams = np.array([0.0, 0.5])
    o = oracle_eval(ds, P, lams)
    g = gpu_eval(ds, P, lams)
    assert ((g["status"] == nv.POINT_NOT_PD) | (o["status"] == nv.POINT_NOT_PD)).sum() >= 1
    assert np.all(g["status"][P[:, 2] > 0] == o["status"][P[:, 2] > 0])   # the points with a nugget
    compare_fp64_singular(g, o, ds.coords, P, what="duplicate sites")
    Q = P.copy()
    Q[5, 0] = -1.0               # invalid range
    g2 = gpu_eval(ds, Q, lams)
    assert g2["status"][5] == nv.POINT_BAD_PARAM and np.all(np.isnan(g2["logL"][5]))
    keep = np.arange(8) != 5
    for k in ("logL", "status"):
        np.testing.assert_array_equal(g2[k][keep], g[k][keep])


def test_fused_batches_and_graph_identical():
    ds = synth.aniso_dataset(502, 120, math.sqrt(12.0), 3)
    P = _points(502, 37)
    lams = synth.LAMBDA_GRID_9
    a = gpu_eval(ds, P, lams, batch=37)
    b = gpu_eval(ds, P, lams, batch=5)
    c = gpu_eval(ds, P, lams, batch=16, flags=nv.FLAG_GRAPH)
    for k in ("logL", "sigma2", "beta", "logdet", "status"):
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)
        np.testing.assert_array_equal(a[k], c[k], err_msg=k)
