"""The on-the-fly engine: the expansion formed per slab in shared memory from the
features, never stored (the paper's future work of forming the population matrix in
place, Section 6).  Fitness (eq.2 -> eq.3 -> eq.4 / eq.5 / eq.10) against the float64
oracle at 1e-5 relative; its P is float32 from the same recurrences as the stored
expansion, so the read-back matches the oracle's closed form to float32 rounding."""

import numpy as np
import pytest

from oracle import game_oracle as o
from paper_1304_0597_gb300 import synth
from tests.gpu_helpers import lib, make_game

pytestmark = pytest.mark.gpu

FIT_RTOL = 1e-5


def _otf(ocfg, X, t, n_train, **kw):
    game = lib()
    g = make_game(ocfg, X, t, n_train, engine=game.ENGINE_ON_THE_FLY, **kw)
    assert g.timing()["engine"] == game.ENGINE_ON_THE_FLY
    return g


@pytest.mark.parametrize("basis,F,d,pop,n", [("chebyshev", 7, 4, 20, 2000),
                                             ("chebyshev", 32, 8, 1024, 30011),
                                             ("chebyshev", 3, 10, 100, 5003),
                                             ("trig", 6, 5, 64, 4001),
                                             ("trig", 1, 1, 7, 333)])
def test_otf_fitness_matches_oracle(basis, F, d, pop, n):
    ds = synth.make_dataset(n, F, d, basis, seed=71, correlated=F > 16)
    ocfg = o.Config(basis=basis, degree=d, pop=pop, seed=4)
    g = _otf(ocfg, ds.X, ds.t, ds.n_train)
    fit, rank = g.evaluate()
    P = o.expand(ds.X[:ds.n_train], basis, d)
    np.testing.assert_allclose(fit, o.fitness(P, ds.t[:ds.n_train], g.population(), ocfg),
                               rtol=FIT_RTOL)
    np.testing.assert_array_equal(rank, o.rank(fit))


def test_otf_features_beyond_unit_interval():
    """Chebyshev features to +-3 at d = 8 (T_8 reaches 6.7e5): the FP32 planes' power-of-two
    column scales apply to the tiles formed in shared memory as to the stored planes;
    16 features x 8 = whole 8-column chunks (the tensor-core kernel's Chebyshev path)."""
    ds = synth.make_dataset(20011, 16, 8, seed=73)
    X = (ds.X * 3.0).astype(np.float32)
    ocfg = o.Config(degree=8, pop=256, seed=5)
    g = _otf(ocfg, X, ds.t, ds.n_train)
    fit, _ = g.evaluate()
    P = o.expand(X[:ds.n_train], "chebyshev", 8)
    np.testing.assert_allclose(fit, o.fitness(P, ds.t[:ds.n_train], g.population(), ocfg),
                               rtol=FIT_RTOL)


@pytest.mark.parametrize("err,act", [("mse", "tanh"), ("tmse", "linear"), ("rmse", "linear")])
def test_otf_error_forms_and_shared_coefficients(err, act):
    """The paper's own form: shared polytrigo coefficients (eq.9), 0/1 targets."""
    ds = synth.make_dataset(3001, 11, 4, "trig", seed=72)
    t = ds.t if act == "tanh" else ((ds.t + 1) / 2).astype(np.float32)
    ocfg = o.Config(basis="trig", degree=4, pop=23, error=err, activation=act, tmse_R=0.49,
                    coefficients="shared", seed=6)
    g = _otf(ocfg, ds.X, t, ds.n_train)
    fit, _ = g.evaluate()
    P = o.expand(ds.X[:ds.n_train], "trig", 4, shared=True)
    want = o.fitness(P, t[:ds.n_train], g.population(), ocfg)
    tol = dict(rtol=1e-4, atol=1e-6) if err.startswith("tmse") else dict(rtol=FIT_RTOL)
    np.testing.assert_allclose(fit, want, **tol)


@pytest.mark.parametrize("basis,shared", [("chebyshev", False), ("trig", False), ("trig", True)])
def test_otf_expansion_readback_and_report(basis, shared):
    ds = synth.make_dataset(1537, 5, 3, basis, seed=73)
    ocfg = o.Config(basis=basis, degree=3, pop=20, seed=2,
                    coefficients="shared" if shared else "per_feature")
    g = _otf(ocfg, ds.X, ds.t, ds.n_train)
    got = g.expansion(0, ds.n_patterns)
    want = o.expand(ds.X, basis, 3, shared=shared)[:, 1:]
    np.testing.assert_allclose(got, want, rtol=0, atol=6e-7 * (5 if shared else 1))
    genes = g.population()[4]
    rep = g.score(genes, 1)
    ref = o.report(o.expand(ds.X[ds.n_train:], basis, 3, shared=shared), ds.t[ds.n_train:],
                   genes, ocfg)
    assert rep["rmse"] == pytest.approx(ref["rmse"], rel=1e-6)
    assert rep["accuracy"] == pytest.approx(ref["accuracy"], abs=1.0 / (ds.n_patterns - ds.n_train))


def test_otf_evolution_and_operators():
    """Generations run on the engine; the operators applied to its fitness are the
    oracle's bit for bit, and the stop test fires on a planted solution."""
    ds = synth.make_dataset(4003, 6, 4, seed=74)
    ocfg = o.Config(degree=4, pop=96, seed=8)
    g = _otf(ocfg, ds.X, ds.t, ds.n_train)
    G = g.population()
    fit, _ = g.evaluate()
    g.breed(None)
    np.testing.assert_array_equal(g.population(), o.breed(G, fit, ocfg, 0))
    assert g.evolve(5) == 5
    genes, fbest, _, _ = g.best()
    P = o.expand(ds.X[:ds.n_train], "chebyshev", 4)
    np.testing.assert_allclose(fbest, o.fitness(P, ds.t[:ds.n_train], genes[None, :], ocfg)[0],
                               rtol=FIT_RTOL)


def test_otf_holds_no_expansion():
    """Device memory of a data set: the stored FP32 form holds two fp16 planes of
    NP x K_pad, the on-the-fly engine only X."""
    import torch
    game = lib()
    ds = synth.make_dataset(2_000_000, 32, 8, seed=75, correlated=True)
    ocfg = o.Config(degree=8, pop=256, seed=1)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    g = _otf(ocfg, ds.X, ds.t, ds.n_train)
    used = free0 - torch.cuda.mem_get_info()[0]
    planes = 2 * 2 * ds.n_patterns * 256
    assert used < 0.5 * planes, (used, planes)
    fit, _ = g.evaluate()
    assert np.all(np.isfinite(fit))
    g.close()


def test_otf_refusals():
    game = lib()
    ds = synth.make_dataset(1000, 4, 3, seed=76)
    with pytest.raises(game.GameError) as e:
        make_game(o.Config(degree=3, pop=20), ds.X, ds.t, 700, engine=game.ENGINE_ON_THE_FLY,
                  precision=game.BF16)
    assert e.value.status == -8
    g = _otf(o.Config(degree=3, pop=20), ds.X, ds.t, 700)
    with pytest.raises(game.GameError) as e:
        g.autotune(reps=1)
    assert e.value.status == -8
