"""The seeded input generator: determinism, shapes and the workloads' recipes."""
import math

import numpy as np

from paper_2305_04318_b300 import synth


def test_deterministic_and_positive():
    a = synth.aniso1000(K=32)
    b = synth.aniso1000(K=32)
    np.testing.assert_array_equal(a.datasets[0].y, b.datasets[0].y)
    np.testing.assert_array_equal(a.params[0], b.params[0])
    assert np.all(a.datasets[0].y > 0)
    assert a.datasets[0].X.shape == (1000, 3) and np.all(a.datasets[0].X[:, 0] == 1)


def test_halton_first_points():
    h = synth.halton(3)
    np.testing.assert_allclose(h[:, 0], [0.5, 0.25, 0.75])
    np.testing.assert_allclose(h[:, 1], [1 / 3, 2 / 3, 1 / 9])


def test_workload_shapes():
    w = synth.iso100()
    assert w.params[0].shape == (100, 5) and w.lambdas.tolist() == [0.0]
    m = synth.mixed4000(K_halton=8, n=400)
    assert m.params[0].shape == (72, 5) and len(m.lambdas) == 9
    ill = synth.ill_conditioned_points()
    assert ill.shape == (64, 5) and np.all(ill[:, 1] == 8.0)
    P = synth.omega_from_unit(synth.halton(500))
    assert P[:, 0].min() >= 0.5 and P[:, 0].max() <= 8 and P[:, 1].min() >= 0.1 and P[:, 1].max() <= 8
    g, params = synth.profile_job_grid(1, G=8, sub=2)
    assert params.shape == (8 * 16, 5) and np.all(params[:16, 1] == g[0])


def test_field_has_unit_variance():
    rng = np.random.default_rng(0)
    coords = rng.uniform(0, 50, (4000, 2))
    U = synth.gaussian_field(rng, coords, 1.5, 1.0, 2.0, math.pi / 6, J=2048)
    assert abs(U.var() - 1) < 0.1
