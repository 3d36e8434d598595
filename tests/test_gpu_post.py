"""GPU parity of the post-processing kernels (Sections 3.2, 3.4-3.6) and of the
Table-1 cross-products output against the oracle, through the C ABI.

The post-processing inputs are the oracle's own statistics (uploaded to the
device), so the kernels are compared with the oracle on identical inputs; the
end-to-end cases then chain the GPU evaluation into the GPU post-processing
and compare with the oracle's chain."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2305_04318_b300 import native as nv, synth
from gpu_util import gpu_eval, to_dev

pytestmark = pytest.mark.gpu

RTOL = 1e-9   # FP64 closed forms on identical statistics: rounding order only


def oracle_stats(ds, P, lams):
    o = oracle.profile_batch(ds.coords, ds.y, ds.X, P, lams, with_ssq=True)
    return o


def dev_stats(ds, lams, o, status=None):
    st = o["status"] if status is None else status
    return (to_dev(ds.y), to_dev(lams), to_dev(o["ssq"]), to_dev(o["logdet"]),
            torch.as_tensor(np.ascontiguousarray(st, dtype=np.int32), device="cuda"))


def assert_prof_close(g, o, rtol=RTOL, what=""):
    np.testing.assert_array_equal(np.isnan(g), np.isnan(o), err_msg=f"{what} NaN pattern")
    f = ~np.isnan(o)
    if f.any():
        err = np.abs(g[f] - o[f]) / np.maximum(1.0, np.abs(o[f]))
        assert err.max() <= rtol, f"{what} max rel err {err.max():.3e}"


def workload(seed=11, n=200, p=3, K=64, M=9):
    ds = synth.aniso_dataset(seed, n, math.sqrt(n / 10), p)
    P = synth.omega_from_unit(synth.halton(K, start=seed))
    lams = np.linspace(-0.5, 1.5, M)
    return ds, P, lams


def test_ssq_yx_fp64_matches_oracle():
    ds, P, lams = workload(K=40)
    o = oracle_stats(ds, P, lams)
    P[3] = [-0.5, 1.0, 0.1, 1.0, 0.0]   # invalid range: BAD_PARAM on the device
    g = gpu_eval(ds, P, lams, with_ssq=True, batch=16)
    assert g["status"][3] == nv.POINT_BAD_PARAM
    ok = o["status"] == 0
    ok[3] = False
    np.testing.assert_array_equal(g["status"][ok], o["status"][ok])
    d = np.sqrt(np.abs(np.einsum("kaa->ka", o["ssq"][ok])))
    scale = d[:, :, None] * d[:, None, :]
    err = np.abs(g["ssq_yx"][ok] - o["ssq"][ok]) / scale
    assert err.max() <= 1e-9, err.max()
    assert np.isnan(g["ssq_yx"][3]).all()
    # symmetric as written
    np.testing.assert_array_equal(g["ssq_yx"][ok], np.swapaxes(g["ssq_yx"][ok], 1, 2))


def test_ssq_yx_mixed_matches_oracle():
    w = synth.aniso1000(K=24)
    ds, P = w.datasets[0], w.params[0]
    o = oracle_stats(ds, P, w.lambdas)
    g = gpu_eval(ds, P, w.lambdas, precision=nv.MIXED, with_ssq=True)
    ok = ((g["status"] & 15) == 0) & (o["status"] == 0)
    d = np.sqrt(np.abs(np.einsum("kaa->ka", o["ssq"][ok])))
    err = np.abs(g["ssq_yx"][ok] - o["ssq"][ok]) / (d[:, :, None] * d[:, None, :])
    print("mixed ssq max rel err", err.max())
    # the error bound is on |Delta l_p| <= 1e-4 ~ (n/2) |Delta RSS| / RSS
    assert err.max() <= 1e-6


@pytest.mark.parametrize("p", [1, 3, 5])
def test_profile_beta_matches_oracle(p):
    ds, P, lams = workload(seed=20 + p, p=p)
    o = oracle_stats(ds, P, lams)
    st = o["status"].copy()
    st[[2, 9]] = [nv.POINT_NOT_PD, nv.POINT_RSS_NONPOS]   # excluded
    st[[4, 5]] = [nv.POINT_RETRIED, nv.POINT_FP64]        # flag bits only: used
    y, l, s, ld, sd = dev_stats(ds, lams, o, st)
    sl = oracle.sum_log(ds.y)
    for j in range(p):
        bh = o["beta"][:, :, j][o["status"] == 0]
        grid = np.linspace(bh.min() - 1.0, bh.max() + 1.0, 300)   # > 256: grid loop wraps
        ref = oracle.profile_beta(len(ds.y), o["ssq"], o["logdet"], lams, sl, j, grid, st)
        got = nv.profile_beta_device(y, l, s, ld, sd, j, to_dev(grid)).cpu().numpy()
        assert_prof_close(got, ref, what=f"beta_{j}")


def test_profile_sigma_matches_oracle():
    ds, P, lams = workload(seed=31)
    o = oracle_stats(ds, P, lams)
    y, l, s, ld, sd = dev_stats(ds, lams, o)
    sl = oracle.sum_log(ds.y)
    s2 = o["sigma2"][o["status"] == 0]
    grid = np.r_[np.linspace(0.5 * math.sqrt(s2.min()), 2.0 * math.sqrt(s2.max()), 97), 0.0, -1.0]
    ref = oracle.profile_sigma(len(ds.y), o["ssq"], o["logdet"], lams, sl, grid, o["status"])
    got = nv.profile_sigma_device(y, l, s, ld, sd, to_dev(grid)).cpu().numpy()
    assert np.isnan(got[-2:]).all()
    assert_prof_close(got[:-2], ref[:-2], what="sigma")


def test_profile_closed_forms_empty_and_all_failed():
    ds, P, lams = workload(seed=32, K=5)
    o = oracle_stats(ds, P, lams)
    y, l, s, ld, sd = dev_stats(ds, lams, o, np.full(5, nv.POINT_NOT_PD))
    got = nv.profile_beta_device(y, l, s, ld, sd, 0, to_dev(np.linspace(0, 1, 4))).cpu().numpy()
    assert np.isnan(got).all()
    with pytest.raises(nv.PlkError):
        nv.profile_beta_device(y, l, s, ld, sd, 3, to_dev(np.zeros(2)))


def test_profile_lambda_matches_oracle():
    rng = np.random.default_rng(3)
    logL = rng.standard_normal((1000, 9)) - 100
    logL[rng.random(logL.shape) < 0.2] = np.nan
    logL[:, 4] = np.nan
    got = nv.profile_lambda_device(to_dev(logL)).cpu().numpy()
    ref = oracle.profile_lambda(logL)
    np.testing.assert_array_equal(np.isnan(got), np.isnan(ref))
    np.testing.assert_array_equal(got[~np.isnan(ref)], ref[~np.isnan(ref)])


def hull_cloud(seed, K, ties=True):
    rng = np.random.default_rng(seed)
    x = rng.uniform(-2, 3, K)
    if ties:
        x[: K // 2] = np.round(x[: K // 2], 1)
    v = -0.5 * (x - 0.7) ** 2 - np.abs(rng.standard_normal(K)) * 2
    v[rng.random(K) < 0.05] = np.nan
    return x, v


@pytest.mark.parametrize("K", [1, 37, 1000, 5003])
def test_profile_hull_matches_oracle(K):
    x, v = hull_cloud(K, K)
    xq = np.r_[np.linspace(-2.5, 3.5, 200), x[: min(K, 50)]]
    ref, ron, rnh = oracle.profile_hull(x, v, xq)
    out, on = nv.profile_hull_device(to_dev(x), to_dev(v), to_dev(xq))
    out, on = out.cpu().numpy(), on.cpu().numpy()
    np.testing.assert_array_equal(on, ron)
    np.testing.assert_array_equal(np.isnan(out), np.isnan(ref))
    f = ~np.isnan(ref)
    if f.any():
        assert np.max(np.abs(out[f] - ref[f]) / np.maximum(1.0, np.abs(ref[f]))) <= 1e-12


def test_profile_hull_strided_column_and_degenerate():
    rng = np.random.default_rng(5)
    P = synth.omega_from_unit(rng.uniform(size=(300, 5)))
    v = -np.log(P[:, 1]) ** 2 + 0.1 * rng.standard_normal(300)
    xq = np.linspace(P[:, 1].min(), P[:, 1].max(), 64)
    ref, ron, _ = oracle.profile_hull(P[:, 1], v, xq)
    out, on = nv.profile_hull_device(to_dev(P)[:, 1:], to_dev(v), to_dev(xq), x_stride=5)
    np.testing.assert_array_equal(on.cpu().numpy(), ron)
    assert np.max(np.abs(out.cpu().numpy() - ref)) <= 1e-12
    # all-NaN cloud and an empty cloud
    out, on = nv.profile_hull_device(to_dev(np.zeros(3)), to_dev(np.full(3, np.nan)), to_dev(np.zeros(2)))
    assert np.isnan(out.cpu().numpy()).all() and not on.cpu().numpy().any()
    out, on = nv.profile_hull_device(to_dev(np.zeros(0)), to_dev(np.zeros(0)), to_dev(np.zeros(2)))
    assert np.isnan(out.cpu().numpy()).all()


@pytest.mark.parametrize("large", [False, True])
def test_internal_params_matches_oracle(large):
    P = synth.omega_from_unit(synth.halton(500))
    P[::3, 3] = 1.0 / P[::3, 3]          # ratios below one too
    ref = oracle.internal_params(P, large)
    got = nv.internal_params_device(to_dev(P), large).cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-13


@pytest.mark.parametrize("precision", [nv.FP64, nv.MIXED])
def test_end_to_end_profiles(precision):
    """GPU evaluation -> GPU profiles vs oracle evaluation -> oracle profiles."""
    ds, P, lams = workload(seed=41, n=600, K=48, M=5)
    o = oracle_stats(ds, P, lams)
    dev = [to_dev(a) for a in (ds.coords, ds.y, ds.X, lams, P)]
    g = nv.eval_device(*dev, precision=precision, with_ssq=True)
    st = g["status"]
    sl = oracle.sum_log(ds.y)
    tol = 1e-8 if precision == nv.FP64 else 1e-3
    mask_st = o["status"]
    # beta_1
    bh = o["beta"][:, :, 1][o["status"] == 0]
    grid = np.linspace(bh.min() - 0.5, bh.max() + 0.5, 41)
    ref = oracle.profile_beta(len(ds.y), o["ssq"], o["logdet"], lams, sl, 1, grid, mask_st)
    got = nv.profile_beta_device(dev[1], dev[3], g["ssq_yx"], g["logdet"], st, 1, to_dev(grid)).cpu().numpy()
    near = ref >= np.nanmax(ref) - 10
    err = np.abs(got[near] - ref[near])
    assert err.max() <= (tol * np.abs(ref[near]).max() if precision == nv.FP64 else tol), err.max()
    # sigma
    s2 = o["sigma2"][o["status"] == 0]
    sg = np.linspace(0.7 * math.sqrt(s2.min()), 1.4 * math.sqrt(s2.max()), 33)
    ref = oracle.profile_sigma(len(ds.y), o["ssq"], o["logdet"], lams, sl, sg, mask_st)
    got = nv.profile_sigma_device(dev[1], dev[3], g["ssq_yx"], g["logdet"], st, to_dev(sg)).cpu().numpy()
    near = ref >= np.nanmax(ref) - 10
    err = np.abs(got[near] - ref[near])
    assert err.max() <= (tol * np.abs(ref[near]).max() if precision == nv.FP64 else tol), err.max()
    # lambda, and the kappa profile by the hull of the cloud
    got = nv.profile_lambda_device(g["logL"]).cpu().numpy()
    ref = oracle.profile_lambda(o["logL"])
    assert np.max(np.abs(got - ref)) <= (tol * np.abs(ref).max() if precision == nv.FP64 else tol)
    vmax = nv.profile_max_device(g["logL"])
    xq = np.linspace(P[:, 1].min(), P[:, 1].max(), 25)
    out, _ = nv.profile_hull_device(dev[4][:, 1:], vmax, to_dev(xq), x_stride=5)
    ref, _, _ = oracle.profile_hull(P[:, 1], oracle.profile_max(o["logL"]), xq)
    assert np.max(np.abs(out.cpu().numpy() - ref)) <= (tol * np.abs(ref).max() if precision == nv.FP64 else tol)


def test_profile_ci_host_arrays_match_oracle():
    """plk_profile_ci (host arrays, device kernel) against the oracle's CI:
    an exactly quadratic profile (endpoints theta0 +- s sqrt(chi2_1)), a
    profile censored on both sides, and NaN entries."""
    import oracle
    grid = np.linspace(-3.0, 5.0, 81)
    prof = -(grid - 1.0) ** 2 / (2 * 0.7 ** 2)
    prof[[3, 50]] = np.nan
    for g, v in ((grid, prof), (grid, 0.01 * prof)):
        r = nv.profile_ci(g, v, 0.95)
        o = oracle.profile_ci(g, v, 0.95)
        for k in ("lo", "hi", "argmax"):
            assert r[k] == pytest.approx(o[k], abs=1e-12), k
        assert r["censored"] == o["censored"]
    assert nv.profile_ci(grid, 0.01 * prof, 0.95)["censored"] == 3
    with pytest.raises(nv.PlkError):
        nv.profile_ci(grid, prof, 1.5)


@pytest.mark.parametrize("p", [1, 3])
def test_profile_beta_reml_matches_oracle(p):
    """REML profile of beta_j (the Appendix's criterion) from the statistics on
    the device against the oracle's, status-excluded points included."""
    ds, P, lams = workload(seed=40 + p, p=p)
    o = oracle_stats(ds, P, lams)
    st = o["status"].copy()
    st[[3]] = [nv.POINT_NOT_PD]
    y, l, s, ld, sd = dev_stats(ds, lams, o, st)
    sl = oracle.sum_log(ds.y)
    for j in range(p):
        bh = o["beta"][:, :, j][o["status"] == 0]
        grid = np.linspace(bh.min() - 1.0, bh.max() + 1.0, 120)
        ref = oracle.profile_beta(len(ds.y), o["ssq"], o["logdet"], lams, sl, j, grid, st, reml=True)
        got = nv.profile_beta_device(y, l, s, ld, sd, j, to_dev(grid), reml=True).cpu().numpy()
        assert_prof_close(got, ref, what=f"reml beta_{j}")
        ml = nv.profile_beta_device(y, l, s, ld, sd, j, to_dev(grid)).cpu().numpy()
        assert not np.allclose(ml, got)
