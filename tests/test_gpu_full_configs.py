"""Parity at the full sizes of the batched and learned-surrogate workloads, in the launch
configuration bench.py times, on sampled chromosomes the float64 oracle computes one by one
(eq.2 -> eq.3 -> eq.5; the oracle walks the rows in blocks so that P is never held whole).

* Batched form: the 64 uneven runs (patterns 1e4..5e5 log-uniform, features 5..40, degree
  3..10, population 64..2048, Chebyshev / trig and FP32 / BF16 alternating) through one
  autotuned grouped launch per generation; every run's sampled fitness against the oracle
  (FP32 runs on the exact operands, BF16 runs on the quantised ones).
* Learned-surrogate form: 2,000,000 patterns x 48 features, Chebyshev d = 6 (289 genes),
  population 4096, 8x pool screened by the network, FP8 P with one gene plane and the top-16
  elites re-scored in FP32 -- the elites against the exact oracle, the rest against the
  oracle on the quantised operands; and the plain FP32 run of the same data.

Tolerance 1e-5 relative throughout (the FP32 bar; for quantised operands the products of the
format are exact in float32, only accumulation and the per-element tanh.approx remain).
"""

import numpy as np
import pytest

from oracle import game_oracle as o
from paper_1304_0597_gb300 import synth
from tests.gpu_helpers import lib

pytestmark = pytest.mark.gpu

BLOCK = 65536
RTOL = 1e-5


def _blocks(a, b):
    return [(i, min(i + BLOCK, b)) for i in range(a, b, BLOCK)]


def _column_scales(X, basis, degree, fmt):
    """Column scales over every stored row, from the oracle's definition applied to the
    stacked per-block column maxima."""
    M = np.stack([np.abs(o.expand(X[a:b], basis, degree)[:, 1:]).max(axis=0)
                  for a, b in _blocks(0, X.shape[0])])
    return o.quantize_columns(M, fmt)[1]


def _rmse(X, t, n_train, basis, degree, sets, ocfg):
    """Oracle RMSE of several chromosome sets over the training rows in one pass.
    sets: list of (G [rows x K] float64, scales or None, fmt or None)."""
    sse = [np.zeros(G.shape[0]) for G, _, _ in sets]
    for a, b in _blocks(0, n_train):
        P = o.expand(X[a:b], basis, degree)
        for i, (G, s, fmt) in enumerate(sets):
            Pi = P
            if s is not None:
                Q, _ = o.quantize_columns(P[:, 1:], fmt, s)
                Pi = np.concatenate([P[:, :1], o.dequantize_columns(Q, s)], axis=1)
            Y = o.activate(o.outputs(Pi, G), ocfg.activation)
            sse[i] += o.pattern_errors(t[a:b], Y, ocfg.error, ocfg.tmse_R).sum(axis=1)
    return [np.sqrt(v / n_train) for v in sse]


def test_batched_form_full_size():
    game = lib()
    specs = synth.batched_specs()
    assert len(specs) == 64
    data, cfgs = [], []
    for sp in specs:
        ds = synth.make_dataset(sp.n_patterns, sp.n_features, sp.degree, sp.basis, seed=sp.seed,
                                correlated=True)
        data.append(ds)
        cfgs.append(game.default_config(
            basis=game.CHEBYSHEV if sp.basis == "chebyshev" else game.TRIG, degree=sp.degree,
            pop=sp.pop, seed=sp.seed, precision=game.FP32 if sp.precision == "fp32" else game.BF16,
            elite_rescore=0))
    b = game.Batch(cfgs)
    for i, ds in enumerate(data):
        b.set_data(i, ds.X, ds.t, ds.n_train)
    b.autotune(reps=1)
    assert list(b.evolve(2)) == [2] * 64      # generation 1 bred, both through the grouped launch
    rng = np.random.default_rng(5)
    worst = 0.0
    for i, (sp, ds) in enumerate(zip(specs, data)):
        run = b.runs[i]
        G = run.population().astype(np.float64)
        fit, rank = run.fitness()
        rows = np.unique(np.concatenate([[rank[0]], rng.choice(sp.pop, 5, replace=False)]))
        ocfg = o.Config(basis=sp.basis, degree=sp.degree, pop=len(rows), seed=sp.seed)
        if sp.precision == "fp32":
            sets = [(G[rows], None, None)]
        else:
            s = _column_scales(ds.X, sp.basis, sp.degree, "bf16")
            sets = [(o.quantize_genes(G[rows].astype(np.float32), s, "bf16", 2), s, "bf16")]
        want = _rmse(ds.X, ds.t, ds.n_train, sp.basis, sp.degree, sets, ocfg)[0]
        rel = np.abs(fit[rows] - want) / want
        worst = max(worst, rel.max())
        assert rel.max() <= RTOL, (i, sp, rel.max())
    b.close()
    print(f"batched form, 64 runs: max rel err {worst:.2e}")


def test_surrogate_form_full_size():
    game = lib()
    ds = synth.surrogate_scale()
    assert ds.n_train == 1_400_000
    ocfg = o.Config(degree=6, pop=4096, seed=0)
    # plain FP32 run (the time-to-target baseline)
    plain = game.Game(game.default_config(degree=6, pop=4096, seed=0))
    plain.set_data(ds.X, ds.t, ds.n_train)
    plain.autotune(reps=1)
    Gp = plain.population().astype(np.float64)
    fp, _ = plain.evaluate()
    plain.close()
    # surrogate + FP8 P, one gene plane, top-16 re-scored in FP32
    g = game.Game(game.default_config(degree=6, pop=4096, seed=0, surrogate_pool=8,
                                      precision=game.FP8, gene_planes=1, elite_rescore=16))
    g.set_data(ds.X, ds.t, ds.n_train)
    g.autotune(reps=1)
    assert g.evolve(2) == 2
    G = g.population().astype(np.float64)
    fit, rank = g.fitness()
    # The 16 re-scored rows were the top of the FP8 ranking; after the merge and re-sort
    # they sit near the top but need not be exactly rank[:16].  Every sampled row must
    # match the exact oracle (re-scored) or the oracle on the quantised operands (FP8),
    # at least 16 of the top 32 the exact one, and the best row the exact one.
    rng = np.random.default_rng(6)
    top = rank[:32]
    rest = rng.choice(rank[32:], 48, replace=False)
    rows = np.concatenate([top, rest])
    plain_rows = rng.choice(4096, 64, replace=False)
    s = _column_scales(ds.X, "chebyshev", 6, "fp8")
    want_plain, want_exact, want_q = _rmse(
        ds.X, ds.t, ds.n_train, "chebyshev", 6,
        [(Gp[plain_rows], None, None), (G[rows], None, None),
         (o.quantize_genes(G[rows].astype(np.float32), s, "fp8", 1), s, "fp8")], ocfg)
    rel_plain = np.abs(fp[plain_rows] - want_plain) / want_plain
    assert rel_plain.max() <= RTOL, rel_plain.max()
    rel_exact = np.abs(fit[rows] - want_exact) / want_exact
    rel_q = np.abs(fit[rows] - want_q) / want_q
    assert np.all(np.minimum(rel_exact, rel_q) <= RTOL), np.minimum(rel_exact, rel_q).max()
    assert (rel_exact[:32] <= RTOL).sum() >= 16 and rel_exact[0] <= RTOL
    assert (rel_q[32:] <= RTOL).sum() >= 40
    print(f"surrogate form at 2M x 48: plain FP32 max rel err {rel_plain.max():.2e}; "
          f"re-scored rows {(rel_exact <= RTOL).sum()} of {len(rows)}; "
          f"max rel err against the matching oracle {np.minimum(rel_exact, rel_q).max():.2e}")
    g.close()
