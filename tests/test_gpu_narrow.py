"""The narrow fitness kernels against the oracle: at most 32 chromosomes, the paper's
own Section 5 settings (population 2N + 1).  The tensor-core form swaps the operands
(patterns on the MMA's M side, FP32 only, any gene count up to 12 k-blocks); the SIMT
form takes 16 or 32 stored basis columns in every precision.

Bars: FP32 fitness within 1e-5 relative (the stated FP32 tolerance); BF16 / FP8
within 1e-5 of the oracle on the dequantised expansion (the kernel rounds only in
float32); the threshold errors (eq.10) allow a pattern within float32 rounding of R
to fall on either side.
"""

import numpy as np
import pytest

from oracle import game_oracle as o
from paper_1304_0597_gb300 import synth
from tests.gpu_helpers import lib, make_game, oracle_fitness_chunked

pytestmark = pytest.mark.gpu

FIT_RTOL = 1e-5


def _cfg(**kw):
    base = dict(basis="chebyshev", degree=4, pop=23, tournament_k=3, p_crossover=0.9,
                p_mutation=0.05, sigma_mutation=0.1, elitism=2, seed=3)
    base.update(kw)
    return o.Config(**base)


@pytest.mark.parametrize("shape", [
    dict(n=5003, F=5, d=3, pop=23, basis="chebyshev"),   # 15 columns -> 16 stored, ragged rows
    dict(n=6007, F=4, d=4, pop=29, basis="chebyshev"),   # 16 columns, 25-32 chromosomes
    dict(n=4099, F=8, d=4, pop=32, basis="chebyshev"),   # 32 columns, a full warp of chromosomes
    dict(n=3001, F=7, d=4, pop=2, basis="chebyshev"),    # the smallest population
    dict(n=777, F=3, d=5, pop=9, basis="trig"),          # 30 columns, fewer rows than one CTA
    dict(n=40, F=2, d=8, pop=5, basis="chebyshev"),      # fewer rows than one warp
])
@pytest.mark.parametrize("engine", ["auto", "simt", "tcgen05"])
def test_narrow_fitness_matches_oracle(shape, engine):
    game = lib()
    ds = synth.make_dataset(shape["n"], shape["F"], shape["d"], shape["basis"], seed=17)
    ocfg = _cfg(basis=shape["basis"], degree=shape["d"], pop=shape["pop"],
                elitism=min(2, shape["pop"]))
    eng = {"auto": game.ENGINE_AUTO, "simt": game.ENGINE_SIMT,
           "tcgen05": game.ENGINE_TCGEN05}[engine]
    g = make_game(ocfg, ds.X, ds.t, ds.n_train, engine=eng)
    # 16 / 32 stored columns: the automatic choice is the narrow kernels (fitness_narrow.cu)
    assert g.timing()["engine"] == (game.ENGINE_TCGEN05 if engine == "tcgen05" else game.ENGINE_SIMT)
    G = g.population()
    fit, rank = g.evaluate()
    P = o.expand(ds.X[:ds.n_train], shape["basis"], shape["d"])
    want = o.fitness(P, ds.t[:ds.n_train], G, ocfg)
    np.testing.assert_allclose(fit, want, rtol=FIT_RTOL)
    assert list(rank) == list(o.rank(fit))


@pytest.mark.parametrize("err,act", [("mse", "tanh"), ("tmse", "tanh"), ("tmse_sq", "tanh"),
                                     ("rmse", "linear"), ("tmse", "linear")])
@pytest.mark.parametrize("engine", ["simt", "tcgen05"])
def test_narrow_error_kinds(err, act, engine):
    """Section 5 form: shared polytrigo coefficients (eq.9), 11 features, d = 8 (16
    stored columns), 23 chromosomes; linear Out with 0/1 labels or tanh with +-1."""
    game = lib()
    ds = synth.make_dataset(6007, 11, 8, "trig", seed=19)
    t = ds.t if act == "tanh" else (ds.t > 0).astype(np.float32)
    ocfg = _cfg(basis="trig", degree=8, coefficients="shared", error=err, activation=act,
                tmse_R=0.49)
    eng = game.ENGINE_SIMT if engine == "simt" else game.ENGINE_TCGEN05
    g = make_game(ocfg, ds.X, t, ds.n_train, engine=eng)
    assert g.timing()["engine"] == eng
    fit, _ = g.evaluate()
    P = o.expand(ds.X[:ds.n_train], "trig", 8, shared=True)
    want = o.fitness(P, t[:ds.n_train], g.population(), ocfg)
    if err.startswith("tmse"):
        np.testing.assert_allclose(fit, want, rtol=1e-4, atol=1e-6)
    else:
        np.testing.assert_allclose(fit, want, rtol=FIT_RTOL)


@pytest.mark.parametrize("fmt,F,d", [("bf16", 5, 3), ("bf16", 8, 4), ("fp8", 7, 4)])
def test_narrow_low_precision(fmt, F, d):
    game = lib()
    ds = synth.make_dataset(4001, F, d, seed=23)
    ocfg = _cfg(degree=d, pop=19)
    g = make_game(ocfg, ds.X, ds.t, ds.n_train, precision=game.BF16 if fmt == "bf16" else game.FP8,
                  elite_rescore=0)
    assert g.timing()["engine"] == game.ENGINE_SIMT
    fit, _ = g.evaluate()
    Q, sc = o.quantize_columns(o.expand(ds.X[:ds.n_train], "chebyshev", d)[:, 1:], fmt)
    Pq = np.concatenate([np.ones((ds.n_train, 1)), o.dequantize_columns(Q, sc)], axis=1)
    np.testing.assert_allclose(fit, o.fitness(Pq, ds.t[:ds.n_train], g.population(), ocfg),
                               rtol=FIT_RTOL)


@pytest.mark.parametrize("pop", [5, 29])
def test_narrow_bf16_chromosome_blocks(pop):
    """BF16 on the warp-MMA narrow kernel with one and with four 8-chromosome blocks
    (16 stored columns), against the oracle on the quantised P with exact genes."""
    game = lib()
    ds = synth.make_dataset(5003, 4, 4, seed=29)
    ocfg = _cfg(degree=4, pop=pop)
    g = make_game(ocfg, ds.X, ds.t, ds.n_train, precision=game.BF16, elite_rescore=0)
    assert g.timing()["engine"] == game.ENGINE_SIMT
    fit, _ = g.evaluate()
    Q, sc = o.quantize_columns(o.expand(ds.X[:ds.n_train], "chebyshev", 4)[:, 1:], "bf16")
    Pq = np.concatenate([np.ones((ds.n_train, 1)), o.dequantize_columns(Q, sc)], axis=1)
    np.testing.assert_allclose(fit, o.fitness(Pq, ds.t[:ds.n_train], g.population(), ocfg),
                               rtol=FIT_RTOL)


@pytest.mark.parametrize("engine", ["simt", "tcgen05"])
def test_narrow_many_blocks_per_thread(engine):
    """Enough rows that every thread folds several 32-pattern blocks into its float64
    sum (SIMT: 2 x 152 CTAs x 256 threads x 32 patterns = 2.49M rows per round;
    tensor cores: 152 CTAs x 2 epilogue sets x 32 tiles of 128 = 1.25M rows)."""
    game = lib()
    ds = synth.make_dataset(4_000_000, 3, 4, seed=29)
    ocfg = _cfg(degree=4, pop=7)
    eng = game.ENGINE_SIMT if engine == "simt" else game.ENGINE_TCGEN05
    g = make_game(ocfg, ds.X, ds.t, ds.n_train, engine=eng)
    assert g.timing()["engine"] == eng
    fit, _ = g.evaluate()
    want = oracle_fitness_chunked(ds.X[:ds.n_train], ds.t[:ds.n_train], g.population(), ocfg,
                                  chunk=1 << 19)
    np.testing.assert_allclose(fit, want, rtol=FIT_RTOL)


def test_narrow_engines_agree():
    """The swapped tensor-core kernel and the narrow kernel give the same fitness
    to 2e-5 (each within 1e-5 of the oracle)."""
    game = lib()
    ds = synth.make_dataset(9000, 6, 4, seed=31)
    ocfg = _cfg(degree=4, pop=24)
    a = make_game(ocfg, ds.X, ds.t, ds.n_train, engine=game.ENGINE_SIMT)
    b = make_game(ocfg, ds.X, ds.t, ds.n_train, engine=game.ENGINE_TCGEN05)
    fa, _ = a.evaluate()
    fb, _ = b.evaluate()
    np.testing.assert_allclose(fa, fb, rtol=2e-5)


@pytest.mark.parametrize("F,d", [(24, 12), (22, 25)])
def test_tensor_core_narrow_many_kblocks(F, d):
    """The swapped kernel over several k-blocks (289 and 551 genes: 5 and 9 k-blocks, the
    ring wraps within a tile; 551 genes exceed the resident planes of the 128-chromosome
    kernel) and the evolve loop on it."""
    game = lib()
    ds = synth.make_dataset(7001, F, d, seed=37, correlated=True)
    ocfg = _cfg(degree=d, pop=17)
    g = make_game(ocfg, ds.X, ds.t, ds.n_train, engine=game.ENGINE_TCGEN05)
    assert g.timing()["engine"] == game.ENGINE_TCGEN05
    fit, _ = g.evaluate()
    P = o.expand(ds.X[:ds.n_train], "chebyshev", d)
    np.testing.assert_allclose(fit, o.fitness(P, ds.t[:ds.n_train], g.population(), ocfg),
                               rtol=FIT_RTOL)
    assert g.evolve(4) == 4
    fit2, _ = g.fitness()
    np.testing.assert_allclose(fit2, o.fitness(P, ds.t[:ds.n_train], g.population(), ocfg),
                               rtol=FIT_RTOL)
