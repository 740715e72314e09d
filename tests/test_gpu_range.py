"""Inputs outside [-1, 1] in the FP32 form.

Eq.1 puts no bound on a feature, and Chebyshev values grow like (2|x|)^d / 2 beyond
[-1, 1]: at d = 8, |x| = 3 gives T_8 = 6.7e5, past fp16's 65504.  The FP32 planes then
hold P / s_g with a power-of-two column scale s_g (folded into the genes), and genes
whose scaled value passes 2^15 get a per-chromosome power of two applied in the
epilogue.  These tests hold every FP32 engine to the float64 oracle (whose Chebyshev
values beyond [-1, 1] come from its cosh branch) and check that values beyond what
float32 can hold are refused instead of turning into NaN.

Tolerance: 1e-5 relative on the fitness where the outputs are of order one (features
mostly inside [-1, 1] with outliers to +-3, small genes).  With unit genes on uniform
[-3, 3] features the outputs reach 1e5 and float32 accumulation leaves an absolute
error of order 2^-24 x 1e5 x sqrt(K) on them; tanh saturates almost everywhere, and
the fitness is held to 1e-4.
"""

import numpy as np
import pytest

from oracle import game_oracle as o
from tests.gpu_helpers import lib, make_game

pytestmark = pytest.mark.gpu

D = 8


def _outlier_data(n=20011, F=12, seed=51):
    rng = np.random.default_rng(seed)
    X = np.clip(rng.normal(0.0, 0.7, size=(n, F)), -3.0, 3.0).astype(np.float32)
    X[0, 0], X[1, 1] = 3.0, -3.0            # the extremes are present
    t = np.where(rng.random(n) < 0.5, 1.0, -1.0).astype(np.float32)
    return X, t, int(0.7 * n)


def _small_genes(g, scale):
    G = g.population()
    G[:, 1:] *= scale
    g.set_population(G)
    return G


@pytest.mark.parametrize("engine,pop", [("tcgen05", 256), ("tcgen05", 24), ("simt", 100)])
def test_chebyshev_beyond_unit_interval_matches_oracle(engine, pop):
    game = lib()
    X, t, ntr = _outlier_data()
    assert np.abs(X).max() == 3.0
    ocfg = o.Config(degree=D, pop=pop, seed=3)
    eng = game.ENGINE_TCGEN05 if engine == "tcgen05" else game.ENGINE_SIMT
    g = make_game(ocfg, X, t, ntr, engine=eng)
    G = _small_genes(g, 1e-3)
    fit, _ = g.evaluate()
    assert np.all(np.isfinite(fit))
    P = o.expand(X[:ntr], "chebyshev", D)
    np.testing.assert_allclose(fit, o.fitness(P, t[:ntr], G, ocfg), rtol=1e-5)


def test_expansion_and_report_beyond_unit_interval():
    """The stored planes reconstruct P (scale included) to the planes' ~22 bits, and the
    float64 report of a chromosome matches the oracle's."""
    X, t, ntr = _outlier_data(n=5003, F=6, seed=52)
    ocfg = o.Config(degree=D, pop=20, seed=1)
    g = make_game(ocfg, X, t, ntr)
    P = o.expand(X, "chebyshev", D)[:, 1:]
    got = g.expansion(0, X.shape[0]).astype(np.float64)
    assert np.all(np.isfinite(got)) and np.abs(P).max() > 65504
    # ~22 bits relative, and the lo plane's subnormal floor scaled by the column's scale
    tol = 2.0 ** -20 * np.abs(P) + 2.0 ** -24 * np.abs(P).max(axis=0)[None, :]
    assert np.all(np.abs(got - P) <= tol), np.max(np.abs(got - P) / tol)
    genes = g.population()[3] * np.r_[1.0, np.full(P.shape[1], 1e-3)].astype(np.float32)
    rep = g.score(genes, 1)
    want = o.report(o.expand(X[ntr:], "chebyshev", D), t[ntr:], genes, ocfg)
    assert rep["rmse"] == pytest.approx(want["rmse"], rel=1e-6)
    assert rep["accuracy"] == pytest.approx(want["accuracy"], abs=1.0 / (X.shape[0] - ntr))


def test_uniform_three_with_unit_genes_is_finite_and_close():
    game = lib()
    rng = np.random.default_rng(53)
    X = rng.uniform(-3, 3, size=(12000, 10)).astype(np.float32)
    t = np.where(rng.random(12000) < 0.5, 1.0, -1.0).astype(np.float32)
    ocfg = o.Config(degree=D, pop=128, seed=2)
    g = make_game(ocfg, X, t, 9000, engine=game.ENGINE_TCGEN05)
    fit, _ = g.evaluate()
    assert np.all(np.isfinite(fit))
    P = o.expand(X[:9000], "chebyshev", D)
    np.testing.assert_allclose(fit, o.fitness(P, t[:9000], g.population(), ocfg), rtol=1e-4)


def test_large_genes_use_the_chromosome_scale():
    """Genes far outside fp16 (the GA without clamping can grow them): the planes take a
    per-chromosome power of two, applied again in the epilogue."""
    game = lib()
    X, t, ntr = _outlier_data(n=8009, F=8, seed=54)
    X = np.clip(X, -1, 1)
    ocfg = o.Config(degree=4, pop=160, seed=6, clamp_genes=False)
    g = make_game(ocfg, X, t, ntr, engine=game.ENGINE_TCGEN05)
    G = g.population()
    G[:40, 1:] *= 3e5                       # |g| up to 3e5 > 65504
    G[40:80, 1:] *= 1e-4
    g.set_population(G)
    fit, _ = g.evaluate()
    assert np.all(np.isfinite(fit))
    P = o.expand(X[:ntr], "chebyshev", 4)
    np.testing.assert_allclose(fit, o.fitness(P, t[:ntr], G, ocfg), rtol=1e-5)


def test_precision_form_rescore_beyond_unit_interval():
    """BF16 P with the FP32 re-score of the top elites: the re-score reads the scaled
    FP32 planes, so the re-scored fitness is the exact one to 1e-5."""
    game = lib()
    X, t, ntr = _outlier_data(n=6007, F=6, seed=55)
    ocfg = o.Config(degree=D, pop=64, seed=7)
    g = make_game(ocfg, X, t, ntr, precision=game.BF16, elite_rescore=16)
    G = _small_genes(g, 1e-3)
    fit, rank = g.evaluate()
    exact = o.fitness(o.expand(X[:ntr], "chebyshev", D), t[:ntr], G, ocfg)
    close = np.isclose(fit, exact, rtol=1e-5, atol=0)
    assert close.sum() >= 16 and close[rank[0]]


@pytest.mark.parametrize("shared", [False, True])
def test_values_beyond_float32_are_refused(shared):
    game = lib()
    rng = np.random.default_rng(56)
    X = rng.uniform(-1, 1, size=(1000, 5)).astype(np.float32)
    X[17, 2] = 1e20                         # T_8(1e20) ~ 1e162
    t = np.where(rng.random(1000) < 0.5, 1.0, -1.0).astype(np.float32)
    ocfg = o.Config(degree=D, pop=20, coefficients="shared" if shared else "per_feature")
    with pytest.raises(game.GameError) as e:
        make_game(ocfg, X, t, 700)
    assert e.value.status == -8
    assert "feature 2" in str(e.value)
