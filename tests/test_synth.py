"""The seeded input generator (CPU): the trig target function's angle addition
against direct cosines and sines, and determinism of the data sets per seed."""

import numpy as np

from paper_1304_0597_gb300 import synth


def _hidden_direct(rng, X, degree):
    """The trig hidden function written with np.cos(k x) / np.sin(k x) per term, drawing
    the same coefficients in the same order as synth._hidden."""
    n, F = X.shape
    v = np.full(n, rng.uniform(-1.0, 1.0), dtype=np.float64)
    for f in range(F):
        x = X[:, f].astype(np.float64)
        a = rng.uniform(-1.0, 1.0, size=degree)
        b = rng.uniform(-1.0, 1.0, size=degree)
        for k in range(1, degree + 1):
            v += a[k - 1] * np.cos(k * x) + b[k - 1] * np.sin(k * x)
    return v


def test_trig_target_by_angle_addition_matches_direct_terms():
    X = np.random.default_rng(5).uniform(-1.0, 1.0, size=(5000, 6)).astype(np.float32)
    for degree in (1, 3, 10):
        got = synth._hidden(np.random.default_rng(11), X, "trig", degree)
        want = _hidden_direct(np.random.default_rng(11), X, degree)
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)


def test_data_sets_are_deterministic_per_seed():
    for basis in ("chebyshev", "trig"):
        a = synth.make_dataset(3000, 5, 4, basis, seed=7, correlated=True)
        b = synth.make_dataset(3000, 5, 4, basis, seed=7, correlated=True)
        c = synth.make_dataset(3000, 5, 4, basis, seed=8, correlated=True)
        assert np.array_equal(a.X, b.X) and np.array_equal(a.t, b.t)
        assert not np.array_equal(a.X, c.X)
        assert set(np.unique(a.t)) <= {-1.0, 1.0}
        assert a.n_train == round(0.7 * 3000)
