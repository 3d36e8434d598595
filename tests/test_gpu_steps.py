"""Steps 1-2 (Sections 3.1-3.2) on the library's GPU evaluation (context
jobs) against the same host code driven by the oracle's likelihood: the
maximum-likelihood estimate, the Hessian, its fixed eigenvalues and every
representative point."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2305_04318_b300 import native as nv, synth

pytestmark = pytest.mark.gpu


def oracle_evaluator(ds):
    return lambda P, lam: oracle.profile_batch(ds.coords, ds.y, ds.X, P, lam)["logL"]


@pytest.fixture(scope="module")
def problem():
    ds = synth.aniso_dataset(9, 70, math.sqrt(7.0), 2)
    arena = torch.empty(2 << 30, dtype=torch.uint8, device="cuda")
    ctx = nv.Context(arena.numel(), arena=arena, n_streams=2)
    did = ctx.create_dataset(ds.coords, ds.y, ds.X)
    yield ds, ctx, did
    ctx.release_dataset(did)
    ctx.close()


@pytest.mark.parametrize("kappa_fixed", [False, True])
def test_fit_mle_gpu_matches_oracle_driven(problem, kappa_fixed):
    ds, ctx, did = problem
    w0 = np.array([1.0, 1.0, 0.2, 1.5, 0.3])
    kw = dict(kappa_fixed=kappa_fixed, kappa=1.0 if kappa_fixed else None)
    g = nv.fit_mle(ctx, did, w0, 0.8, **kw)
    o = nv.fit_mle_cb(oracle_evaluator(ds), w0, 0.8, **kw)
    # the reported maximum is the oracle's l_p at the reported point
    at = oracle_evaluator(ds)(g["omega"][None], np.array([g["lam"]]))[0, 0]
    assert g["logL"] == pytest.approx(at, rel=1e-8)
    if kappa_fixed:
        # a well-identified maximum: both runs end at the same point
        assert g["logL"] == pytest.approx(o["logL"], abs=1e-6)
        np.testing.assert_allclose(g["omega"], o["omega"], rtol=2e-3, atol=2e-3)
        assert g["lam"] == pytest.approx(o["lam"], abs=2e-3)
    else:
        # kappa runs to its bound (20) along a ridge where l_p changes by < 1e-3:
        # the two runs may stop at different points of it
        assert abs(g["logL"] - o["logL"]) <= 1e-3
    # the mixed-precision evaluation reaches the same maximum within its tolerance
    m = nv.fit_mle(ctx, did, w0, 0.8, precision=nv.MIXED, **kw)
    assert abs(m["logL"] - o["logL"]) <= 1e-3


@pytest.mark.parametrize("kappa_fixed", [False, True])
def test_quadratic_cloud_gpu_matches_oracle_driven(problem, kappa_fixed):
    ds, ctx, did = problem
    ev = oracle_evaluator(ds)
    fit = nv.fit_mle_cb(ev, np.array([1.0, 1.0, 0.2, 1.5, 0.3]), 0.8, kappa_fixed=True, kappa=1.0)
    args = (fit["omega"], fit["lam"])
    kw = dict(kappa_fixed=kappa_fixed, n_sphere=60, level_probs=[0.1, 0.5, 0.95], n_lambda=30, seed=11)
    g = nv.quadratic_cloud(ctx, did, *args, **kw)
    o = nv.quadratic_cloud_cb(ev, *args, **kw)
    np.testing.assert_allclose(g["hessian"], o["hessian"], rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(g["eigenvalues"], o["eigenvalues"], rtol=1e-6)
    np.testing.assert_allclose(g["lambdas"], o["lambdas"], rtol=1e-8, atol=1e-8)
    np.testing.assert_allclose(g["params"], o["params"], rtol=1e-5, atol=1e-6)


def test_fit_mle_reml_gpu_matches_oracle_driven(problem):
    """Step 1 on the REML profile likelihood (eq. remlpro)."""
    ds, ctx, did = problem
    w0 = np.array([1.0, 1.0, 0.2, 1.5, 0.3])
    ev = lambda P, lam: oracle.profile_batch(ds.coords, ds.y, ds.X, P, lam, reml=True)["logL"]
    g = nv.fit_mle(ctx, did, w0, 0.8, kappa_fixed=True, kappa=1.0, reml=True)
    o = nv.fit_mle_cb(ev, w0, 0.8, kappa_fixed=True, kappa=1.0)
    assert g["logL"] == pytest.approx(o["logL"], abs=1e-6)
    np.testing.assert_allclose(g["omega"], o["omega"], rtol=2e-3, atol=2e-3)
    ml = nv.fit_mle(ctx, did, w0, 0.8, kappa_fixed=True, kappa=1.0)
    assert ml["logL"] != pytest.approx(g["logL"], abs=1e-3)     # a different objective
