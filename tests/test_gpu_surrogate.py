"""Learned surrogate: the network's forward, gradients and Adam step against the
float64 oracle, and the surrogate-driven generation.

Tolerances: with float32 weights (SIMT kernels) the kernels differ from float64
only by float32 rounding of the GEMMs (K <= 289 terms, |terms| ~ 1): 1e-4
relative to the largest output / gradient entry.  The bfloat16 form runs on the
tensor cores with bfloat16 weights and bfloat16 GEMM operands (x, gelu(Z1), dZ2,
dZ1) and float32 accumulation; the oracle is fed the same bfloat16 weights and
rounds the same operands.  What remains is float32 accumulation order, which can
flip a bfloat16 rounding by one unit (2^-8 relative) for a few operands: 3e-3
relative to the largest entry.
"""

import numpy as np
import pytest

from oracle import game_oracle as o
from paper_1304_0597_gb300 import synth
from tests.gpu_helpers import lib, make_game

pytestmark = pytest.mark.gpu


def _unflatten(flat, D, H=256):
    i = 0
    out = {}
    for name, shape in (("W1", (H, D)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("w3", (H,)),
                        ("b3", ())):
        n = int(np.prod(shape)) if shape else 1
        out[name] = np.asarray(flat[i:i + n], dtype=np.float64).reshape(shape)
        i += n
    return out


def _flatten(p):
    return np.concatenate([np.asarray(p[k], dtype=np.float64).reshape(-1)
                           for k in ("W1", "b1", "W2", "b2", "w3", "b3")])


def _ctx(fp32: bool, **kw):
    ds = synth.make_dataset(1500, 12, 4, seed=51)
    ocfg = o.Config(degree=4, pop=64, seed=5)
    g = make_game(ocfg, ds.X, ds.t, ds.n_train, surrogate_fp32=int(fp32), surrogate_batch=256,
                  **kw)
    return g, ds


@pytest.mark.parametrize("fp32", [True, False])
def test_surrogate_forward_matches_oracle(fp32):
    g, _ = _ctx(fp32)
    D = g.n_genes
    flat = g.surrogate_params()
    p = _unflatten(flat, D)
    if not fp32:
        for k in ("W1", "W2", "w3"):
            p[k] = o.round_bf16(p[k].astype(np.float32)).astype(np.float64)
    X = np.random.default_rng(1).uniform(-1, 1, size=(200, D)).astype(np.float32)
    y = g.surrogate_forward(X)
    want = o.mlp_forward(p, X, None if fp32 else o.bf16_operands)["y"]
    tol = 1e-4 if fp32 else 3e-3
    np.testing.assert_allclose(y, want, rtol=0, atol=tol * max(1.0, np.abs(want).max()))


@pytest.mark.parametrize("fp32", [True, False])
def test_surrogate_gradient_matches_oracle(fp32):
    g, _ = _ctx(fp32)
    D = g.n_genes
    rng = np.random.default_rng(2)
    flat = g.surrogate_params()
    p = _unflatten(flat, D)
    if not fp32:
        for k in ("W1", "W2", "w3"):
            p[k] = o.round_bf16(p[k].astype(np.float32)).astype(np.float64)
    X = rng.uniform(-1, 1, size=(256, D)).astype(np.float32)
    t = rng.standard_normal(256).astype(np.float32)
    loss, grad = g.surrogate_grad(X, t)
    want_loss, gw = o.mlp_loss_grad(p, X, t, None if fp32 else o.bf16_operands)
    tol = 1e-4 if fp32 else 3e-3
    assert loss == pytest.approx(want_loss, rel=tol)
    for name, got in _unflatten(grad, D).items():
        ref = np.asarray(gw[name])
        np.testing.assert_allclose(got, ref, rtol=0, atol=tol * max(1e-6, np.abs(ref).max()),
                                   err_msg=name)


def test_surrogate_tc_shapes_against_oracle():
    """bfloat16 form at a shape with several k-blocks and a ragged one (145 genes),
    three row tiles in the batch (384 rows: weight-gradient K = 384), a ragged
    forward (300 rows) and the bias column of [gW1 | gb1] in a second tile."""
    ds = synth.make_dataset(1500, 24, 6, seed=54)
    ocfg = o.Config(degree=6, pop=64, seed=8)
    g = make_game(ocfg, ds.X, ds.t, ds.n_train, surrogate_batch=384)
    D = g.n_genes
    assert D == 145
    p = _unflatten(g.surrogate_params(), D)
    for k in ("W1", "W2", "w3"):
        p[k] = o.round_bf16(p[k].astype(np.float32)).astype(np.float64)
    rng = np.random.default_rng(9)
    X = rng.uniform(-1, 1, size=(384, D)).astype(np.float32)
    t = rng.standard_normal(384).astype(np.float32)
    y = g.surrogate_forward(X[:300])
    want = o.mlp_forward(p, X[:300], o.bf16_operands)["y"]
    np.testing.assert_allclose(y, want, rtol=0, atol=3e-3 * max(1.0, np.abs(want).max()))
    loss, grad = g.surrogate_grad(X, t)
    want_loss, gw = o.mlp_loss_grad(p, X, t, o.bf16_operands)
    assert loss == pytest.approx(want_loss, rel=3e-3)
    for name, got in _unflatten(grad, D).items():
        ref = np.asarray(gw[name])
        np.testing.assert_allclose(got, ref, rtol=0, atol=3e-3 * max(1e-6, np.abs(ref).max()),
                                   err_msg=name)


def test_surrogate_adam_step_matches_textbook():
    g, _ = _ctx(True)
    D = g.n_genes
    rng = np.random.default_rng(3)
    p0 = g.surrogate_params().astype(np.float64)
    X = rng.uniform(-1, 1, size=(128, D)).astype(np.float32)
    t = rng.standard_normal(128).astype(np.float32)
    _, grad = o.mlp_loss_grad(_unflatten(p0, D), X, t)
    gflat = _flatten(grad)
    g.surrogate_train_step(X, t, 1e-3)
    want, m, v = o.adam_update(p0, gflat, np.zeros_like(p0), np.zeros_like(p0), 1, lr=1e-3)
    got = g.surrogate_params()
    # first Adam step moves each parameter by ~lr along -sign(grad); compare the moves
    np.testing.assert_allclose(got - p0, want - p0, rtol=0, atol=2e-5)


def test_surrogate_learns_on_fixed_data():
    """Training on a fixed batch drives the loss down."""
    g, _ = _ctx(False)
    D = g.n_genes
    rng = np.random.default_rng(4)
    X = rng.uniform(-1, 1, size=(256, D)).astype(np.float32)
    t = (np.sin(X[:, 1] * 2) + X[:, 2] * X[:, 3]).astype(np.float32)
    l0, _ = g.surrogate_grad(X, t)
    for _ in range(200):
        g.surrogate_train_step(X, t, 1e-3)
    l1, _ = g.surrogate_grad(X, t)
    assert l1 < 0.2 * l0


def test_surrogate_ablation_is_the_plain_ga():
    """Keeping the first plain children of the pool (surrogate_select = 1) reproduces the
    GA without a surrogate bit for bit: pair j of the pool is pair j of plain breeding."""
    game = lib()
    ds = synth.make_dataset(3000, 8, 4, seed=52)
    ocfg = o.Config(degree=4, pop=100, seed=6)
    plain = make_game(ocfg, ds.X, ds.t, ds.n_train)
    abl = make_game(ocfg, ds.X, ds.t, ds.n_train, surrogate_pool=4, surrogate_select=1,
                    surrogate_batch=256, surrogate_steps=2)
    assert plain.evolve(8) == 8 and abl.evolve(8) == 8
    np.testing.assert_array_equal(abl.population(), plain.population())
    np.testing.assert_array_equal(abl.fitness()[0], plain.fitness()[0])


def test_surrogate_driven_evolution():
    """Pool of 8x, surrogate selection: elitism keeps the best, the monitor records a
    correlation per bred generation, and the surrogate's children are better than plain
    children drawn from the same pools (mean fitness of the evaluated children)."""
    ds = synth.make_dataset(6000, 10, 4, seed=53)
    ocfg = o.Config(degree=4, pop=256, seed=7)
    sur = make_game(ocfg, ds.X, ds.t, ds.n_train, surrogate_pool=8, surrogate_batch=512,
                    surrogate_steps=16)
    abl = make_game(ocfg, ds.X, ds.t, ds.n_train, surrogate_pool=8, surrogate_select=1,
                    surrogate_batch=512, surrogate_steps=16)
    hist_s, hist_a = [], []
    for gen in range(20):
        sur.evolve(1)
        abl.evolve(1)
        hist_s.append(sur.fitness()[0].min())
        hist_a.append(abl.fitness()[0].min())
    assert all(b <= a for a, b in zip(hist_s, hist_s[1:]))
    mon = sur.surrogate_monitor()
    rho = mon["history"]
    assert len(rho) == 20 and np.isnan(rho[0])
    assert np.nanmean(rho[5:]) > 0.2
    assert hist_s[-1] <= hist_a[-1]


@pytest.mark.parametrize("pop,pool", [(256, 8), (1000, 4)])
def test_surrogate_selection_assembly_and_monitor_match_oracle(pop, pool):
    """The last bred generation, checked row by row against the oracle: the kept pool
    rows are oracle.surrogate_select of the pool's scores; the population after the
    elites is those pool rows (genes bit for bit) with the scores they were kept with;
    the monitor's correlation is oracle.spearman of those scores and the exact fitness
    (both ranked in float32, ties to the lower row, as the kernel ranks them)."""
    ds = synth.make_dataset(5000, 10, 4, seed=54)
    ocfg = o.Config(degree=4, pop=pop, seed=9)
    g = make_game(ocfg, ds.X, ds.t, ds.n_train, surrogate_pool=pool, surrogate_batch=512,
                  surrogate_steps=8)
    assert g.evolve(6) == 6
    e = ocfg.elitism
    p = g.surrogate_pool()
    sel = o.surrogate_select(p["scores"], pop - e)
    np.testing.assert_array_equal(p["selected"], sel)
    G = g.population()
    np.testing.assert_array_equal(G[e:], p["genes"][sel])
    pred = p["predictions"]
    assert np.all(np.isnan(pred[:e]))
    np.testing.assert_array_equal(pred[e:], p["scores"][sel])
    fit, _ = g.fitness()
    rho = g.surrogate_monitor()["rho"]
    want = o.spearman(pred[e:].astype(np.float32), fit[e:].astype(np.float32))
    assert rho == pytest.approx(want, abs=1e-12)
