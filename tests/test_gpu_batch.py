"""Batched form: independent runs of uneven sizes evolved together through one
grouped persistent fitness launch per generation.  Each run must give what it
gives alone: the same fitness (float64 sums in another order, so 1e-12) and the
same operator trajectory, bit for bit."""

import numpy as np
import pytest

from oracle import game_oracle as o
from paper_1304_0597_gb300 import synth
from tests.gpu_helpers import game_config, lib, make_game

pytestmark = pytest.mark.gpu


def _specs():
    game = lib()
    specs = [  # (patterns, features, degree, pop, basis, precision, planes)
        (3001, 5, 3, 64, "chebyshev", game.FP32, 2),
        (12007, 9, 6, 200, "trig", game.FP32, 2),
        (5003, 20, 10, 96, "chebyshev", game.BF16, 2),
        (8009, 16, 9, 300, "trig", game.BF16, 1),      # 289 genes: beyond the resident limit
        (2000, 7, 4, 20, "chebyshev", game.FP8, 2),
        (20011, 40, 10, 130, "trig", game.FP32, 2),    # 801 genes
    ]
    out = []
    for i, (n, F, d, pop, basis, prec, planes) in enumerate(specs):
        ds = synth.make_dataset(n, F, d, basis, seed=100 + i, correlated=F > 8)
        ocfg = o.Config(basis=basis, degree=d, pop=pop, seed=i)
        cfg = game_config(ocfg, precision=prec, gene_planes=planes, elite_rescore=0)
        out.append((ds, ocfg, cfg))
    return out


def test_batch_matches_single_runs():
    """Runs whose single-context engine is also tcgen05 follow the same trajectory bit
    for bit; every run's grouped-launch fitness matches its single-context fitness."""
    game = lib()
    specs = _specs()
    b = game.Batch([c for _, _, c in specs])
    for i, (ds, _, _) in enumerate(specs):
        b.set_data(i, ds.X, ds.t, ds.n_train)
    assert list(b.evolve(1)) == [1] * len(specs)
    gen0 = [b.runs[i].fitness()[0] for i in range(len(specs))]
    gens = b.evolve(5)
    assert list(gens) == [5] * len(specs)
    for i, (ds, ocfg, cfg) in enumerate(specs):
        # the 20-chromosome run alone would take the narrow kernels: ask for the
        # tensor cores, as in the grouped launch (801 genes stay on SIMT either way)
        eng = game.ENGINE_TCGEN05 if ocfg.pop <= 32 else game.ENGINE_AUTO
        single = game.Game(game_config(ocfg, precision=cfg.precision,
                                       gene_planes=cfg.gene_planes, elite_rescore=0, engine=eng))
        single.set_data(ds.X, ds.t, ds.n_train)
        fs0, _ = single.evaluate()
        same_engine = single.timing()["engine"] == game.ENGINE_TCGEN05
        np.testing.assert_allclose(gen0[i], fs0, rtol=1e-12 if same_engine else 1e-5)
        if same_engine:
            single.breed(None)
            assert single.evolve(5) == 5
            np.testing.assert_array_equal(b.runs[i].population(), single.population())
            np.testing.assert_allclose(b.runs[i].fitness()[0], single.fitness()[0], rtol=1e-12)
        single.close()


def test_batch_fitness_against_oracle_and_autotune():
    game = lib()
    specs = _specs()
    b = game.Batch([c for _, _, c in specs])
    for i, (ds, _, _) in enumerate(specs):
        b.set_data(i, ds.X, ds.t, ds.n_train)
    g, ms = b.autotune(reps=2)
    assert g in (1, 2, 4, 8, 16) and ms > 0
    b.evolve(1)      # generation 0 of every run goes through the grouped launch
    for i, (ds, ocfg, cfg) in enumerate(specs):
        run = b.runs[i]
        G = run.population()
        fit, _ = run.fitness()    # computed by the grouped launch
        if cfg.precision == game.FP32:
            P = o.expand(ds.X[:ds.n_train], ocfg.basis, ocfg.degree)
            want = o.fitness(P, ds.t[:ds.n_train], G, ocfg)
        else:
            # BF16 / FP8 runs: the oracle on the same quantised operands (column scales over
            # every stored row, genes in the run's planes), oracle.quantize_columns and
            # oracle.quantize_genes
            fmt = "bf16" if cfg.precision == game.BF16 else "fp8"
            Q, s = o.quantize_columns(o.expand(ds.X, ocfg.basis, ocfg.degree)[:, 1:], fmt)
            Pq = np.concatenate([np.ones((ds.n_train, 1)),
                                 o.dequantize_columns(Q[:ds.n_train], s)], axis=1)
            want = o.fitness(Pq, ds.t[:ds.n_train], o.quantize_genes(G, s, fmt, cfg.gene_planes),
                             ocfg)
        np.testing.assert_allclose(fit, want, rtol=1e-5)
        _, fbest, _, _ = run.best()
        assert fbest == pytest.approx(fit.min(), rel=1e-12)
