"""GPU path (through the C ABI) against the CPU oracle on identical seeded inputs.

Bars: expansion within 6e-7 absolute (float32 rounding of a float64 value plus
the two-plane fp16 split, both < 2^-22 relative); FP32 fitness within 1e-5
relative (the stated tolerance for FP32 fitness); initial population and
genetic operators bit-for-bit.
"""

import numpy as np
import pytest

from oracle import game_oracle as o
from paper_1304_0597_gb300 import synth
from tests.gpu_helpers import game_config, lib, make_game, oracle_fitness_chunked

pytestmark = pytest.mark.gpu

FIT_RTOL = 1e-5


def _cfg(**kw):
    base = dict(basis="chebyshev", degree=4, pop=20, tournament_k=3, p_crossover=0.9,
                p_mutation=0.05, sigma_mutation=0.1, elitism=2, seed=7)
    base.update(kw)
    return o.Config(**base)


# ------------------------------------------------------------------ expansion

@pytest.mark.parametrize("basis,F,d", [("chebyshev", 7, 4), ("trig", 6, 5), ("chebyshev", 3, 10),
                                       ("trig", 1, 1)])
def test_expansion_matches_closed_form(basis, F, d):
    ds = synth.make_dataset(1537, F, d, basis, seed=3)
    ocfg = _cfg(basis=basis, degree=d)
    g = make_game(ocfg, ds.X, ds.t, ds.n_train)
    got = g.expansion(0, ds.n_patterns)
    want = o.expand(ds.X, basis, d)[:, 1:]
    assert got.shape == want.shape
    np.testing.assert_allclose(got, want, rtol=0, atol=6e-7)


@pytest.mark.parametrize("n", [700, 200_003])
def test_expansion_of_device_inputs_equals_host_inputs(n):
    """From host memory the FP32 expansion runs chunk by chunk as X arrives (200,003 rows:
    four chunks and a ragged last one); from device memory in one launch."""
    import torch
    ds = synth.make_dataset(n, 5, 3, seed=4)
    ocfg = _cfg(degree=3)
    a = make_game(ocfg, ds.X, ds.t, ds.n_train)
    b = make_game(ocfg, torch.from_numpy(ds.X).cuda(), torch.from_numpy(ds.t).cuda(), ds.n_train)
    np.testing.assert_array_equal(a.expansion(0, n), b.expansion(0, n))
    fa, _ = a.evaluate()
    fb, _ = b.evaluate()
    np.testing.assert_array_equal(fa, fb)
    # a second data set of the same shape reuses the device blocks of the first
    a.set_data(ds.X[::-1].copy(), ds.t[::-1].copy(), ds.n_train)
    b.set_data(torch.from_numpy(ds.X[::-1].copy()).cuda(), torch.from_numpy(ds.t[::-1].copy()).cuda(),
               ds.n_train)
    np.testing.assert_array_equal(a.expansion(0, n), b.expansion(0, n))
    m = min(n, 1000)
    P = o.expand(ds.X[::-1][:m], "chebyshev", 3)[:, 1:]
    np.testing.assert_allclose(a.expansion(0, m), P, rtol=0, atol=6e-7)


# ------------------------------------------------------------------- fitness

@pytest.mark.parametrize("engine", ["tcgen05", "simt"])
@pytest.mark.parametrize("shape", [
    dict(n=2000, F=7, d=4, pop=20, basis="chebyshev"),          # the small plain workload
    dict(n=5003, F=9, d=5, pop=300, basis="chebyshev"),         # several tiles, ragged tails
    dict(n=3001, F=6, d=4, pop=129, basis="trig"),              # polytrigo, pop just over a tile
    dict(n=40013, F=32, d=8, pop=1024, basis="chebyshev"),      # the at-scale gene count
    dict(n=9000, F=24, d=12, pop=200, basis="chebyshev"),       # 288 basis columns (5 k-blocks)
])
def test_fitness_matches_oracle(shape, engine):
    game = lib()
    ds = synth.make_dataset(shape["n"], shape["F"], shape["d"], shape["basis"], seed=5,
                            correlated=shape["F"] >= 24)
    ocfg = _cfg(basis=shape["basis"], degree=shape["d"], pop=shape["pop"])
    eng = game.ENGINE_TCGEN05 if engine == "tcgen05" else game.ENGINE_SIMT
    g = make_game(ocfg, ds.X, ds.t, ds.n_train, engine=eng)
    assert g.timing()["engine"] == eng
    G = g.population()
    fit, rank = g.evaluate()
    P = o.expand(ds.X[:ds.n_train], shape["basis"], shape["d"])
    want = o.fitness(P, ds.t[:ds.n_train], G, ocfg)
    np.testing.assert_allclose(fit, want, rtol=FIT_RTOL)
    assert list(rank) == list(o.rank(fit))


@pytest.mark.parametrize("err,act", [("mse", "tanh"), ("tmse", "tanh"), ("tmse_sq", "tanh"),
                                     ("rmse", "linear"), ("tmse", "linear")])
def test_error_kinds_and_activations(err, act):
    ds = synth.make_dataset(2500, 5, 3, seed=6)
    t = ds.t if act == "tanh" else (ds.t > 0).astype(np.float32)   # 0/1 labels with linear Out
    ocfg = _cfg(degree=3, pop=40, error=err, activation=act, tmse_R=0.49)
    g = make_game(ocfg, ds.X, t, ds.n_train)
    G = g.population()
    fit, _ = g.evaluate()
    P = o.expand(ds.X[:ds.n_train], "chebyshev", 3)
    want = o.fitness(P, t[:ds.n_train], G, ocfg)
    if err.startswith("tmse"):
        # a pattern whose error sits within float32 rounding of R may fall on either side
        np.testing.assert_allclose(fit, want, rtol=1e-4, atol=1e-6)
    else:
        np.testing.assert_allclose(fit, want, rtol=FIT_RTOL)


def test_planted_chromosome_fits_exactly():
    rng = np.random.default_rng(9)
    X = rng.uniform(-1, 1, size=(4000, 6)).astype(np.float32)
    ocfg = _cfg(degree=3, pop=33, stop_error=1e-5)
    h = o.init_population(o.Config(pop=1, seed=99), o.n_genes("chebyshev", 6, 3))[0]
    t = synth.planted_targets(X, h, "chebyshev", 3).astype(np.float32)
    g = make_game(ocfg, X, t, 3000)
    G = g.population()
    G[5] = h
    g.set_population(G)
    fit, rank = g.evaluate()
    assert rank[0] == 5
    assert fit[5] < 2e-6
    # the stop test ends evolution on the first generation
    g.set_population(G)
    assert g.evolve(20) == 1
    assert g.state()[1] == 1


# ----------------------------------------------------------------- operators

@pytest.mark.parametrize("init", ["uniform_pm1", "normal_pm1", "uniform_01"])
def test_initial_population_bit_exact(init):
    ds = synth.make_dataset(300, 4, 3, seed=1)
    ocfg = _cfg(degree=3, pop=57, init=init, seed=123, run=4)
    g = make_game(ocfg, ds.X, ds.t, ds.n_train)
    np.testing.assert_array_equal(g.population(), o.init_population(ocfg, g.n_genes))


@pytest.mark.parametrize("kw", [
    dict(),
    dict(pop=31, elitism=3),                                  # odd slots: last child dropped
    dict(pop=64, elite_mode="copies", tournament_k=4, p_mutation=0.2),
    dict(pop=2, elitism=0, p_crossover=1.0),
    dict(pop=10, elitism=10),                                 # everything elite
    dict(pop=45, tournament_k=32, clamp_genes=False, sigma_mutation=0.7, p_mutation=0.5),
    dict(pop=1000, degree=6),
    dict(pop=600, degree=3, elitism=5),                       # counting rank, ragged blocks
    dict(pop=64, immigrants=20),                              # random immigrants
    dict(pop=50, immigrants=48, init="normal_pm1"),           # all non-elite slots immigrate
    dict(pop=80, selection="roulette"),                       # Section 2 selection criteria
    dict(pop=600, degree=3, selection="ranking"),             # ranking on the counting path
])
def test_operators_bit_exact_given_fitness(kw):
    ds = synth.make_dataset(500, 5, kw.get("degree", 4), seed=2)
    ocfg = _cfg(**kw)
    g = make_game(ocfg, ds.X, ds.t, ds.n_train)
    G = g.population()
    np.testing.assert_array_equal(G, o.init_population(ocfg, g.n_genes))
    rng = np.random.default_rng(0)
    for gen in range(4):
        fit = rng.random(ocfg.pop)
        if gen == 2:
            fit[: ocfg.pop // 2] = 0.25                       # ties broken by index
            fit[-1] = np.nan                                  # NaN ranks last
        g.breed(fit)
        want = o.breed(G, fit, ocfg, gen)
        G = g.population()
        np.testing.assert_array_equal(G, want)
        assert g.state()[0] == gen + 1


@pytest.mark.parametrize("pop", [100, 600, 1030])
def test_rank_after_evaluate_is_the_oracle_order(pop):
    """The ranking returned with the fitness is the order (fitness, index) of that
    fitness vector, for one-CTA sorting (pop < 512) and counting over many CTAs."""
    ds = synth.make_dataset(900, 6, 3, seed=12)
    ocfg = _cfg(degree=3, pop=pop, seed=3)
    g = make_game(ocfg, ds.X, ds.t, ds.n_train)
    fit, rank = g.evaluate()
    np.testing.assert_array_equal(rank, o.rank(fit))
    G = g.population()
    G[pop // 3] = G[pop // 5]                                 # a tie in fitness: index decides
    g.set_population(G)
    fit, rank = g.evaluate()
    assert fit[pop // 3] == fit[pop // 5]
    np.testing.assert_array_equal(rank, o.rank(fit))


def test_trajectory_bit_exact_with_gpu_fitness():
    """GPU evaluate + breed for 12 generations equals the oracle's operators fed the
    GPU's fitness vectors; game_evolve reproduces the same trajectory."""
    ds = synth.plain_small()
    ocfg = _cfg(pop=20, degree=4, seed=0)
    g = make_game(ocfg, ds.X, ds.t, ds.n_train)
    G = g.population()
    hist = []
    for gen in range(12):
        fit, _ = g.evaluate()
        hist.append(fit.min())
        if gen == 11:
            break
        g.breed(None)
        want = o.breed(G, fit, ocfg, gen)
        G = g.population()
        np.testing.assert_array_equal(G, want)
    assert all(b <= a for a, b in zip(hist, hist[1:]))       # elitism: best never worsens
    h = make_game(ocfg, ds.X, ds.t, ds.n_train)
    assert h.evolve(12) == 12
    np.testing.assert_array_equal(h.population(), G)
    _, fit_best, _, _ = h.best()
    assert fit_best == pytest.approx(hist[-1], rel=1e-12)


def test_evolve_is_resumable():
    ds = synth.make_dataset(1500, 5, 3, seed=8)
    ocfg = _cfg(degree=3, pop=50)
    a = make_game(ocfg, ds.X, ds.t, ds.n_train)
    b = make_game(ocfg, ds.X, ds.t, ds.n_train)
    assert a.evolve(9) == 9
    assert b.evolve(4) == 4 and b.evolve(5) == 5
    np.testing.assert_array_equal(a.population(), b.population())
    assert a.state() == b.state() == (8, 0)


@pytest.mark.parametrize("pop,per_gen", [(50, 4), (1024, 5)])
def test_launch_count_of_evolve(pop, per_gen):
    # breed, prepare, one fitness launch, then one fused reduce+rank kernel below 512
    # chromosomes or reduce / rank-count (whose last block makes the state transition)
    # from 512 up; plus the state reset
    ds = synth.make_dataset(3000, 5, 3, seed=8)
    g = make_game(_cfg(degree=3, pop=pop), ds.X, ds.t, ds.n_train, engine=lib().ENGINE_TCGEN05)
    assert g.evolve(7) == 7
    assert g.timing()["launches"] == 1 + 7 * per_gen


# ------------------------------------------------ shared coefficients (eq.9)

@pytest.mark.parametrize("basis", ["trig", "chebyshev"])
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("engine", ["tcgen05", "simt"])
def test_shared_coefficients_fitness(basis, prec, engine):
    """The paper's eq.2 / eq.9 form: B*d + 1 genes shared by all features; the stored
    expansion sums every basis member over the features."""
    game = lib()
    ds = synth.make_dataset(4001, 11, 4, basis, seed=63)
    ocfg = _cfg(basis=basis, degree=4, pop=160, coefficients="shared", seed=2)
    g = make_game(ocfg, ds.X, ds.t, ds.n_train, precision=prec, elite_rescore=0,
                  engine=game.ENGINE_TCGEN05 if engine == "tcgen05" else game.ENGINE_SIMT)
    K = o.n_genes(basis, 11, 4, shared=True)
    assert g.n_genes == K
    P = o.expand(ds.X, basis, 4, shared=True)
    got = g.expansion(0, ds.n_patterns)
    if prec == 0:
        np.testing.assert_allclose(got, P[:, 1:], rtol=0, atol=11 * 6e-7)
        fit, _ = g.evaluate()
        np.testing.assert_allclose(fit, o.fitness(P[:ds.n_train], ds.t[:ds.n_train],
                                                  g.population(), ocfg), rtol=FIT_RTOL)
    else:
        Q, sc = o.quantize_columns(P[:, 1:], "bf16")
        np.testing.assert_allclose(got, o.dequantize_columns(Q, sc), rtol=0,
                                   atol=np.abs(P[:, 1:]).max() * 2.0 ** -8)
        fit, _ = g.evaluate()
        Pq = np.concatenate([np.ones((ds.n_train, 1)),
                             o.dequantize_columns(Q[:ds.n_train], sc)], axis=1)
        Gq = o.quantize_genes(g.population(), sc, "bf16", 2) if engine == "tcgen05" \
            else g.population()
        np.testing.assert_allclose(fit, o.fitness(Pq, ds.t[:ds.n_train], Gq, ocfg), rtol=1e-5)
    genes = g.population()[0]
    np.testing.assert_allclose(g.predict(genes, ds.X[:500]),
                               o.activate(o.outputs(P[:500], genes[None, :]), "tanh")[0],
                               rtol=1e-6, atol=1e-6)


def test_paper_configuration_trajectory():
    """Section 5's setting on a KB-shaped set (11 features, 0/1 targets): polytrigo with
    shared coefficients, linear Out, TMSE with R = 0.49, roulette selection, normal init,
    p_c 0.9, p_m 0.2, elitism 2, random immigrants: fitness against the oracle, and the
    oracle's operators fed the GPU's fitness reproduce the GPU population bit for bit."""
    ds = synth.make_dataset(2100, 11, 4, "trig", seed=64)
    t01 = ((ds.t + 1) / 2).astype(np.float32)
    ocfg = _cfg(basis="trig", degree=4, pop=23, coefficients="shared", activation="linear",
                error="tmse", tmse_R=0.49, selection="roulette", init="normal_pm1",
                p_mutation=0.2, tournament_k=4, immigrants=3, seed=11)
    g = make_game(ocfg, ds.X, t01, ds.n_train)
    P = o.expand(ds.X[:ds.n_train], "trig", 4, shared=True)
    G = g.population()
    np.testing.assert_array_equal(G, o.init_population(ocfg, g.n_genes))
    for gen in range(8):
        fit, _ = g.evaluate()
        want_fit = o.fitness(P, t01[:ds.n_train], G, ocfg)
        # TMSE drops patterns with |t - Out| <= R: a pattern within float32 rounding of R
        # can fall on either side (one flip moves the fitness by ~1.6e-4 here)
        rel = np.abs(fit - want_fit) / np.maximum(want_fit, 1e-300)
        assert np.mean(rel <= FIT_RTOL) >= 0.95 and rel.max() <= 2e-3
        g.breed(None)
        want = o.breed(G, fit, ocfg, gen)
        G = g.population()
        np.testing.assert_array_equal(G, want)


# ------------------------------------------------------- predict / checkpoint

@pytest.mark.parametrize("basis,F,d", [("chebyshev", 7, 4), ("trig", 5, 3), ("chebyshev", 3, 10)])
@pytest.mark.parametrize("act", ["tanh", "linear"])
def test_predict_matches_oracle(basis, F, d, act):
    """A chromosome applied to new patterns (no data set on the context)."""
    import torch
    game = lib()
    ds = synth.make_dataset(2501, F, d, basis, seed=61)
    ocfg = _cfg(basis=basis, degree=d, activation=act)
    g = game.Game(game_config(ocfg))
    K = o.n_genes(basis, F, d)
    genes = np.random.default_rng(3).uniform(-1, 1, size=K).astype(np.float32)
    y = g.predict(genes, ds.X)
    want = o.activate(o.outputs(o.expand(ds.X, basis, d), genes[None, :].astype(np.float64)),
                      act)[0]
    np.testing.assert_allclose(y, want, rtol=1e-6, atol=1e-6)
    yd = g.predict(genes, torch.from_numpy(ds.X).cuda())
    np.testing.assert_array_equal(yd.cpu().numpy(), y)
    assert g.predict(genes, ds.X[:0]).shape == (0,)
    with pytest.raises(game.GameError):
        g.predict(genes[:-1], ds.X)


@pytest.mark.parametrize("kw", [dict(), dict(precision=1, gene_planes=1), dict(engine=2)])
def test_checkpoint_resumes_exactly(kw):
    """evolve 6, save, evolve 5 on one context == load into a fresh context, evolve 5:
    same population, fitness and generation (random immigrants on)."""
    game = lib()
    ds = synth.make_dataset(3000, 6, 4, seed=62)
    ocfg = _cfg(pop=64, degree=4, seed=5, immigrants=4)
    a = make_game(ocfg, ds.X, ds.t, ds.n_train, **kw)
    assert a.evolve(6) == 6
    buf = a.save()
    assert a.evolve(5) == 5
    b = make_game(ocfg, ds.X, ds.t, ds.n_train, **kw)
    b.load(buf)
    assert b.evolve(5) == 5
    np.testing.assert_array_equal(b.population(), a.population())
    np.testing.assert_array_equal(b.fitness()[0], a.fitness()[0])
    assert b.state() == a.state()
    other = make_game(_cfg(pop=64, degree=4, seed=6, immigrants=4), ds.X, ds.t, ds.n_train, **kw)
    with pytest.raises(game.GameError) as e:
        other.load(buf)
    assert e.value.status == -1
    sur = make_game(ocfg, ds.X, ds.t, ds.n_train, surrogate_pool=2)
    with pytest.raises(game.GameError) as e:
        sur.save()
    assert e.value.status == -8


# -------------------------------------------------------------------- report

def test_score_matches_oracle_report():
    ds = synth.plain_small()
    ocfg = _cfg()
    g = make_game(ocfg, ds.X, ds.t, ds.n_train)
    g.evolve(15)
    genes, fit, test_rmse, test_acc = g.best()
    P_te = o.expand(ds.X[ds.n_train:], "chebyshev", 4)
    rep = o.report(P_te, ds.t[ds.n_train:], genes, ocfg)
    assert test_rmse == pytest.approx(rep["rmse"], rel=1e-6)
    assert test_acc == pytest.approx(rep["accuracy"], abs=1.0 / 600 + 1e-12)
    s = g.score(genes, 1)
    assert s["completeness"] == pytest.approx(rep["completeness"], abs=2.0 / 600)
    assert s["contamination"] == pytest.approx(rep["contamination"], abs=2.0 / 600)
    P_tr = o.expand(ds.X[:ds.n_train], "chebyshev", 4)
    assert fit == pytest.approx(o.fitness(P_tr, ds.t[:ds.n_train], genes[None, :], ocfg)[0],
                                rel=FIT_RTOL)


# ---------------------------------------------------------------- edge cases

def test_edge_shapes():
    game = lib()
    # one training row, one feature, degree 1: K = 2
    X = np.array([[0.5], [-0.25], [1.0]], dtype=np.float32)
    t = np.array([1, -1, 1], dtype=np.float32)
    ocfg = _cfg(degree=1, pop=2, elitism=1)
    g = make_game(ocfg, X, t, 1)
    G = g.population()
    fit, _ = g.evaluate()
    want = o.fitness(o.expand(X[:1], "chebyshev", 1), t[:1], G, ocfg)
    np.testing.assert_allclose(fit, want, rtol=FIT_RTOL)
    with pytest.raises(game.GameError):
        g.set_data(X, t, 0)
    with pytest.raises(game.GameError):
        g.set_data(X, t, 4)
    Xn = X.copy()
    Xn[1, 0] = np.nan
    with pytest.raises(game.GameError) as e:
        g.set_data(Xn, t, 2)
    assert e.value.status == -7


def test_calls_out_of_order_are_state_errors():
    game = lib()
    g = game.Game(game_config(_cfg()))
    with pytest.raises(game.GameError) as e:
        g.evolve(1)
    assert e.value.status == -2


# ------------------------------------------------------------ tile shapes

# (degree, (patterns per tile, ring depth, cluster, slices per CTA, k-blocks per stage));
# 32 features: degree 8 stores 256 columns (4 k-blocks, both FP32 gene planes 128 KB of
# shared memory per slice), degree 4 stores 128 (two slices per CTA fit).
@pytest.mark.parametrize("degree,tile", [
    (8, (256, 3, 1, 1, 1)), (8, (256, 2, 1, 1, 1)), (8, (128, 5, 1, 1, 1)),
    (8, (128, 4, 1, 1, 1)), (4, (128, 2, 1, 2, 1)), (4, (128, 6, 0, 2, 0)),
    (8, (256, 6, 2, 1, 1)), (8, (256, 4, 2, 1, 1)), (8, (256, 2, 2, 1, 1)),
    (8, (128, 3, 1, 1, 2)), (8, (128, 2, 1, 1, 2)), (4, (256, 2, 1, 1, 2)),
    (4, (128, 3, 1, 2, 2)), (8, (256, 3, 2, 1, 2)), (8, (256, 2, 2, 1, 2))])
def test_tcgen05_tile_shapes_agree(degree, tile):
    """Every tile shape (patterns per tile, ring depth, cluster, slices per CTA, k-blocks
    per TMA request) gives the oracle's fitness, and is the shape that runs; population
    1024 = 8 slices of 128 chromosomes, fed one or two per CTA, or (cluster 2) by CTA
    pairs whose MMAs of 256 chromosomes read both CTAs' halves of each pattern tile."""
    game = lib()
    ds = synth.make_dataset(20011, 32, degree, seed=41, correlated=True)
    ocfg = _cfg(degree=degree, pop=1024, seed=3)
    n, stages, cluster, slices, kgroup = tile
    g = make_game(ocfg, ds.X, ds.t, ds.n_train, engine=game.ENGINE_TCGEN05, tile_n=n,
                  tile_stages=stages, tile_cluster=cluster, tile_slices=slices,
                  tile_kgroup=kgroup)
    got = g.tile()
    assert (got["n"], got["stages"], got["cluster"], got["slices"], got["kgroup"]) == \
        (n, stages, max(cluster, 1), slices, max(kgroup, 1)), got
    fit, _ = g.evaluate()
    P = o.expand(ds.X[:ds.n_train], "chebyshev", degree)
    np.testing.assert_allclose(fit, o.fitness(P, ds.t[:ds.n_train], g.population(), ocfg),
                               rtol=FIT_RTOL)


def test_fp32_pairs_odd_k_blocks():
    """The FP32 form's default plan (CTA pairs, two k-blocks per TMA request) on 40
    features x degree 8 = 320 stored columns: five k-blocks, so the last request is half
    zero fill; training rows 14,008 (a ragged last tile)."""
    game = lib()
    ds = synth.make_dataset(20011, 40, 8, seed=45, correlated=True)
    ocfg = _cfg(degree=8, pop=512, seed=5)
    g = make_game(ocfg, ds.X, ds.t, ds.n_train, engine=game.ENGINE_TCGEN05)
    got = g.tile()
    assert (got["cluster"], got["kgroup"]) == (2, 2), got
    fit, _ = g.evaluate()
    P = o.expand(ds.X[:ds.n_train], "chebyshev", 8)
    np.testing.assert_allclose(fit, o.fitness(P, ds.t[:ds.n_train], g.population(), ocfg),
                               rtol=FIT_RTOL)


def test_unplannable_tile_request_runs_the_default_shape():
    """Two FP32 slices per CTA at 256 stored columns need 256 KB of gene planes: the
    request cannot be planned, the default shape runs (and says so), and the fitness is
    the oracle's."""
    game = lib()
    ds = synth.make_dataset(6007, 32, 8, seed=43, correlated=True)
    ocfg = _cfg(degree=8, pop=512, seed=3)
    g = make_game(ocfg, ds.X, ds.t, ds.n_train, engine=game.ENGINE_TCGEN05, tile_n=128,
                  tile_slices=2)
    assert g.tile()["slices"] == 1
    fit, _ = g.evaluate()
    P = o.expand(ds.X[:ds.n_train], "chebyshev", 8)
    np.testing.assert_allclose(fit, o.fitness(P, ds.t[:ds.n_train], g.population(), ocfg),
                               rtol=FIT_RTOL)


def test_tile_cluster_above_two_is_rejected():
    """Clusters are single CTAs or CTA pairs: a cluster request above 2 is INVALID_ARG."""
    game = lib()
    ds = synth.make_dataset(3001, 8, 4, seed=5)
    with pytest.raises(game.GameError) as e:
        make_game(_cfg(degree=4, pop=256, seed=1), ds.X, ds.t, ds.n_train,
                  engine=game.ENGINE_TCGEN05, tile_cluster=4)
    assert e.value.status == -1


@pytest.mark.parametrize("pop,n", [(256, 5003), (1280, 40013), (384, 2000)])
def test_cta_pairs_ragged_and_odd_slices(pop, n):
    """CTA pairs on a ragged last tile (n_train not a multiple of 256) and few tiles;
    pop 384 has an odd number of slices, where a pair request falls back to single CTAs."""
    game = lib()
    ds = synth.make_dataset(n, 16, 6, seed=44, correlated=True)
    ocfg = _cfg(degree=6, pop=pop, seed=8)
    g = make_game(ocfg, ds.X, ds.t, ds.n_train, engine=game.ENGINE_TCGEN05, tile_cluster=2)
    assert g.tile()["cluster"] == (2 if (pop // 128) % 2 == 0 else 1)
    fit, _ = g.evaluate()
    P = o.expand(ds.X[:ds.n_train], "chebyshev", 6)
    np.testing.assert_allclose(fit, o.fitness(P, ds.t[:ds.n_train], g.population(), ocfg),
                               rtol=FIT_RTOL)
    assert g.evolve(2) == 2


def test_autotune_picks_a_valid_shape(tmp_path, monkeypatch):
    game = lib()
    monkeypatch.setenv("GAME_TUNE_CACHE", str(tmp_path / "tiles.txt"))
    ds = synth.make_dataset(30000, 16, 8, seed=42, correlated=True)
    ocfg = _cfg(degree=8, pop=512, seed=1)
    g = make_game(ocfg, ds.X, ds.t, ds.n_train)
    before, _ = g.evaluate()
    best, cands = g.autotune(reps=2)
    assert len(cands) >= 4 and best["ms"] == min(c["ms"] for c in cands)
    after, _ = g.evaluate()
    np.testing.assert_allclose(after, before, rtol=1e-6)
    assert (tmp_path / "tiles.txt").read_text().strip()
    # a new context with the same shape bucket picks the cached shape up
    h = make_game(ocfg, ds.X, ds.t, ds.n_train)
    np.testing.assert_allclose(h.evaluate()[0], before, rtol=1e-6)


def test_bounded_wait_times_out_without_fault():
    """A wait that nothing satisfies gives up after its limit and reports TIMEOUT; the
    context keeps working afterwards."""
    import ctypes
    game = lib()
    ds = synth.make_dataset(500, 4, 3, seed=61)
    ocfg = _cfg(degree=3, pop=30)
    g = make_game(ocfg, ds.X, ds.t, ds.n_train)
    waited = ctypes.c_int32()
    st = game.lib.game_selftest_timeout(g.h, 2000, ctypes.byref(waited))
    assert st == -6
    assert 1500 <= waited.value < 500000
    fit, _ = g.evaluate()
    P = o.expand(ds.X[:ds.n_train], "chebyshev", 3)
    np.testing.assert_allclose(fit, o.fitness(P, ds.t[:ds.n_train], g.population(), ocfg),
                               rtol=FIT_RTOL)
    assert g.evolve(3) == 3
