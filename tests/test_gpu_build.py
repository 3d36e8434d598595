"""GPU parity of the Matern build (V = R + nu^2 I, eq. matern; the first item of
Step 3 in Section 3.3) against the oracle's dense V, element by element, in
the three forms the evaluation builds it: FP64 tiles (FP64 path), double-float
tiles evaluated in FP32 pair arithmetic (first pass of the mixed path) and
double-float tiles evaluated in FP64 (7-slice tier of the mixed path).

Tolerances.  The FP64 build evaluates rho as a degree-9 piecewise polynomial
of w = u^2 whose nodes come from a trapezoid rule on K_kappa's integral; the
oracle uses Temme's series / the integral directly: both are good to ~1e-14
relative, so 1e-12 absolute leaves room for the polynomial's interpolation
error.  The double-float forms keep ~44 bits of each entry; the FP32-pair
evaluation adds ~1e-13 absolute (its c_4..c_9 terms in FP32), below 1e-12.
"""
import math

import numpy as np
import pytest
import torch

from paper_2305_04318_b300 import native as nv, synth
from gpu_util import to_dev

pytestmark = pytest.mark.gpu

ATOL = 1e-12
MODES = [nv.BUILD_FP64, nv.BUILD_DF_FAST, nv.BUILD_DF]


def oracle_v(coords, P):
    import oracle
    return np.stack([oracle.build_v(coords, P[k]) for k in range(P.shape[0])])


def gpu_v(coords, P, mode):
    V = nv.build_covariance_device(to_dev(coords), to_dev(P), mode=mode)
    torch.cuda.synchronize()
    return V.cpu().numpy()


def box_points(K, seed):
    return synth.omega_from_unit(np.random.default_rng(seed).uniform(size=(K, 5)))


@pytest.mark.parametrize("mode", MODES)
def test_build_matches_oracle_box(mode):
    # n = 300: three tile rows with a ragged last tile; omega across the whole box
    # (kappa in [0.1, 8], anisotropy ratio up to 4, any angle)
    ds = synth.aniso_dataset(31, 300, math.sqrt(30.0), 2)
    P = box_points(12, 5)
    o = oracle_v(ds.coords, P)
    g = gpu_v(ds.coords, P, mode)
    err = np.abs(g - o)
    assert err.max() <= ATOL, f"mode {mode}: max |dV| {err.max():.3e}"
    assert np.array_equal(g, np.transpose(g, (0, 2, 1)))


@pytest.mark.parametrize("mode", MODES)
def test_build_ill_conditioned_and_edges(mode):
    # kappa = 8 with long ranges (entries near 1, the regime the retry tiers
    # serve), tiny kappa, a very short range (entries underflow to 0, beyond the
    # table), coincident sites (d = 0 -> rho = 1) and n = 129 (one full tile and
    # a one-site tail)
    ds = synth.aniso_dataset(32, 129, math.sqrt(12.9), 3)
    coords = ds.coords.copy()
    coords[7] = coords[3]
    P = np.vstack([synth.ill_conditioned_points()[::9],
                   [[0.5, 0.1, 0.0, 1.0, 0.0],
                    [40.0, 0.15, 1e-3, 3.0, 2.0],
                    [1e-3, 1.0, 0.1, 1.0, 0.0],
                    [2.0, 8.0, 0.0, 4.0, 3.1]]])
    o = oracle_v(coords, P)
    g = gpu_v(coords, P, mode)
    err = np.abs(g - o)
    assert err.max() <= ATOL, f"mode {mode}: max |dV| {err.max():.3e}"
    assert np.all(g[:, 7, 3] == 1.0)


@pytest.mark.parametrize("mode", MODES)
def test_build_large_shapes(mode):
    # kappa up to 20, the largest shape the fitting step explores
    ds = synth.aniso_dataset(34, 200, math.sqrt(20.0), 2)
    P = np.array([[0.3, k, 0.05, 1.5, 0.4] for k in (8.0, 12.0, 16.0, 20.0)] +
                 [[3.0, k, 0.0, 2.0, 1.0] for k in (8.0, 12.0, 16.0, 20.0)])
    o = oracle_v(ds.coords, P)
    g = gpu_v(ds.coords, P, mode)
    err = np.abs(g - o)
    assert err.max() <= ATOL, f"mode {mode}: max |dV| {err.max():.3e}"


def test_fast_double_float_build_against_fp64_build():
    # the FP32-pair evaluation against the FP64 evaluation of the same
    # polynomial: only the arithmetic differs
    ds = synth.aniso_dataset(33, 520, math.sqrt(52.0), 3)
    P = box_points(6, 6)
    f = gpu_v(ds.coords, P, nv.BUILD_FP64)
    d = gpu_v(ds.coords, P, nv.BUILD_DF_FAST)
    err = np.abs(d - f)
    assert err.max() <= 5e-13, f"max |dV| {err.max():.3e}"


def test_build_rejects_bad_arguments():
    c = to_dev(np.zeros((4, 2)))
    P = to_dev(np.ones((1, 5)))
    with pytest.raises(nv.PlkError):
        nv.build_covariance_device(c, P, mode=3)
    with pytest.raises(nv.PlkError):
        nv.build_covariance_device(c, P, workspace=torch.empty((16,), dtype=torch.uint8, device="cuda"))
