"""The counts the paper prints for Step 2 (tests/golden/paper_step2_counts.json,
each entry with its section) against the library's Step-2 code: the Hessian
stencil sizes, the default points per contour level, the number of contour
levels, and the soil example's configuration matrix size."""
import json
import os

import numpy as np

from paper_2305_04318_b300 import native as nv

G = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_step2_counts.json")))


def test_hessian_stencil_sizes():
    c = np.array([0.1, 0.2, 0.3, 0.4, 0.5])
    assert 3 * nv.hessian_stencil(c, kappa_fixed=False).shape[0] == G["hessian_likelihoods_5d"]["value"]
    assert 3 * nv.hessian_stencil(c, kappa_fixed=True).shape[0] == G["hessian_likelihoods_4d"]["value"]


def _cloud_size(kappa_fixed, levels, n_sphere=0):
    # size query only (no evaluation is made): params_out NULL
    import ctypes as C
    o = nv.CloudOptions(0, 0, int(kappa_fixed), int(n_sphere), len(levels) if levels is not None else 0,
                        None if levels is None else nv._np_ptr(levels), 0, 0.0, 0.0, 1, 0)
    K = C.c_int64()
    cb = nv._eval_callback(lambda P, lam: np.zeros((len(P), len(lam))))
    w = np.array([1.0, 1.0, 0.1, 1.0, 0.0])
    nv._check(nv.lib().plk_quadratic_cloud_cb(cb, None, nv._np_ptr(w), 0.0, C.byref(o), None, 0, C.byref(K),
                                              None, None, None))
    return K.value


def test_default_points_per_level_and_levels():
    lo, hi = G["contour_levels_range"]["value"]
    n5 = _cloud_size(False, None)
    n4 = _cloud_size(True, None)
    assert n5 % G["points_per_level_5d"]["value"] == 0
    assert n4 % G["points_per_level_4d"]["value"] == 0
    assert lo <= n5 // G["points_per_level_5d"]["value"] <= hi
    assert lo <= n4 // G["points_per_level_4d"]["value"] <= hi


def test_soil_configuration_matrix_size():
    s = G["soil_configuration_rows"]
    k5 = _cloud_size(False, np.linspace(0.05, 0.95, s["levels_5d"]))
    k4 = _cloud_size(True, np.linspace(0.05, 0.95, s["levels_4d"]))
    assert s["mles"] + k5 + s["fits_4d"] * k4 == s["value"]


def test_python_defaults_match_paper():
    import inspect
    assert inspect.signature(nv.quadratic_cloud).parameters["n_lambda"].default == G["lambda_grid_size"]["value"]
