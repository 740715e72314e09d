"""Parity at the benchmark's own size: 1,000,000 patterns x 32 correlated features,
Chebyshev degree 8 (257 genes), population 1024, 700,000 training rows -- every CTA
walks ~150 pattern tiles with wrapping ring phases, the shape the bench times.

The fitness (eq.2 -> eq.3 -> eq.5) of every chromosome is compared with the float64
oracle, which walks the training rows in blocks of 65,536 so that P is never held
whole.  The launch configuration is the bench's: the library autotuner's tile.

Tolerances: FP32 form 1e-5 relative (the stated bar for FP32 fitness); BF16 / FP8
(one gene plane) 1e-5 against the oracle fed the same quantised operands
(``quantize_columns`` with the whole matrix's column scales, ``quantize_genes``),
since products of the format are exact in float32 and only the float32 accumulation
and the 2^-11 tanh.approx per element (which averages out over 700k rows) remain.
"""

import numpy as np
import pytest

from oracle import game_oracle as o
from paper_1304_0597_gb300 import synth
from tests.gpu_helpers import lib, make_game

pytestmark = pytest.mark.gpu

BLOCK = 65536
D = 8


def _blocks(n):
    return [(i, min(i + BLOCK, n)) for i in range(0, n, BLOCK)]


@pytest.fixture(scope="module")
def data():
    ds = synth.plain_at_scale()
    # the oracle's expansion of the training rows, block by block (float64, ~1.4 GB)
    ds.P_blocks = [o.expand(ds.X[a:b], "chebyshev", D) for a, b in _blocks(ds.n_train)]
    return ds


def _fitness_blocks(ds, G, ocfg, transform=None):
    """Oracle RMSE over the training rows in blocks: P of each block from ``o.expand``
    (optionally replaced by its quantised copy), then eq.2 / activation / eq.3 summed."""
    G = np.asarray(G, dtype=np.float64)
    sse = np.zeros(G.shape[0])
    for (a, b), P in zip(_blocks(ds.n_train), ds.P_blocks):
        if transform is not None:
            P = transform(P)
        Y = o.activate(o.outputs(P, G), ocfg.activation)
        sse += o.pattern_errors(ds.t[a:b], Y, ocfg.error, ocfg.tmse_R).sum(axis=1)
    return np.sqrt(sse / ds.n_train)


def _column_scales(ds, fmt):
    """Column scales of the stored expansion over every stored row (training and test),
    from the oracle's own definition applied to the stacked per-block column maxima."""
    M = [np.abs(P[:, 1:]).max(axis=0) for P in ds.P_blocks]
    M += [np.abs(o.expand(ds.X[a:b], "chebyshev", D)[:, 1:]).max(axis=0)
          for a, b in _blocks(ds.n_patterns - ds.n_train)
          for a, b in [(ds.n_train + a, ds.n_train + b)]]
    M = np.stack(M)
    return o.quantize_columns(M, fmt)[1]


def _tuned_game(ds, ocfg, tmp_path, monkeypatch, **kw):
    game = lib()
    monkeypatch.setenv("GAME_TUNE_CACHE", str(tmp_path / "tiles.txt"))
    g = make_game(ocfg, ds.X, ds.t, ds.n_train, engine=game.ENGINE_TCGEN05, **kw)
    tile, _ = g.autotune(reps=2)
    return g, tile


def test_fp32_fitness_at_bench_size(data, tmp_path, monkeypatch):
    ds = data
    ocfg = o.Config(degree=D, pop=1024, seed=0)
    g, tile = _tuned_game(ds, ocfg, tmp_path, monkeypatch)
    assert ds.n_train == 700_000
    G = g.population()
    fit, rank = g.evaluate()
    want = _fitness_blocks(ds, G, ocfg)
    rel = np.abs(fit - want) / want
    assert rel.max() <= 1e-5, (rel.max(), tile)
    np.testing.assert_array_equal(rank, o.rank(fit))
    # the generation graph (breed -> fitness -> rank) on the tuned tile: two bred
    # generations, the last evaluated population against the oracle
    assert g.evolve(3) == 3
    fit3, _ = g.fitness()
    G3 = g.population()
    rows = np.concatenate([np.arange(8), np.random.default_rng(1).choice(1024, 120, replace=False)])
    want3 = _fitness_blocks(ds, G3[rows], ocfg)
    np.testing.assert_allclose(fit3[rows], want3, rtol=1e-5)
    print(f"FP32 at 700k rows, tile {tile}: max rel err {rel.max():.2e}")


@pytest.mark.parametrize("fmt", ["bf16", "fp8"])
def test_low_precision_fitness_at_bench_size(data, fmt, tmp_path, monkeypatch):
    game = lib()
    ds = data
    ocfg = o.Config(degree=D, pop=1024, seed=0)
    prec = game.BF16 if fmt == "bf16" else game.FP8
    g, tile = _tuned_game(ds, ocfg, tmp_path, monkeypatch, precision=prec, gene_planes=1,
                          elite_rescore=0)
    G = g.population()
    fit, _ = g.evaluate()
    s = _column_scales(ds, fmt)
    rows = np.concatenate([np.arange(8), np.random.default_rng(2).choice(1024, 248, replace=False)])
    Gq = o.quantize_genes(G[rows], s, fmt, 1)

    def stored(P):
        Q, _ = o.quantize_columns(P[:, 1:], fmt, s)
        return np.concatenate([P[:, :1], o.dequantize_columns(Q, s)], axis=1)

    want = _fitness_blocks(ds, Gq, ocfg, transform=stored)
    rel = np.abs(fit[rows] - want) / want
    assert rel.max() <= 1e-5, (rel.max(), tile)
    print(f"{fmt} (1 gene plane) at 700k rows, tile {tile}: max rel err {rel.max():.2e}")
