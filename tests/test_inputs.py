"""The seeded input recipe (hpcg_inputs.py): the same arrays on every call,
the stated distributions and ranges, and the stated draw order (CPU only)."""
import numpy as np

import hpcg_inputs as hi


def test_deterministic_and_in_range():
    a, b = hi.normal(1000, 7), hi.normal(1000, 7)
    np.testing.assert_array_equal(a, b)
    assert not np.array_equal(a, hi.normal(1000, 8))
    assert abs(a.mean()) < 0.15 and 0.85 < a.std() < 1.15
    u = hi.uniform(1000, 0.0, 1.0, 9)
    assert u.min() >= 0.0 and u.max() < 1.0
    x = hi.mixed_precision_xtrue(1000)
    assert x.min() >= -1.0 and x.max() < 1.0
    np.testing.assert_array_equal(x, np.random.default_rng(1).uniform(-1.0, 1.0, 1000))


def test_multi_rhs_is_rhs_major():
    B = hi.multi_rhs(50, nrhs=4, seed=2)
    assert B.shape == (4, 50)
    np.testing.assert_array_equal(B.ravel(), np.random.default_rng(2).standard_normal(200))


def test_uneven_batch_draw_order():
    d = hi.uneven_batch_dims()
    assert d.shape == (64, 3) and set(np.unique(d)) <= {32, 48, 64, 80, 96}
    flat = np.random.default_rng(3).choice(np.array([32, 48, 64, 80, 96]), size=192)
    np.testing.assert_array_equal(d.ravel(), flat)  # instance-major, then x, y, z


def test_differentiable_inputs_draw_order():
    k, b, xt = hi.differentiable_inputs(100, seed=4)
    rng = np.random.default_rng(4)
    np.testing.assert_array_equal(k, rng.uniform(0.0, 1.0, 100))
    np.testing.assert_array_equal(b, rng.standard_normal(100))
    np.testing.assert_array_equal(xt, rng.standard_normal(100))
    assert k.min() >= 0.0 and k.max() < 1.0
