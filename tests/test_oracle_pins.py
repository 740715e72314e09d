"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

None of these re-types an oracle formula: each checks the oracle against a value
the paper prints, an identity, exact rational arithmetic, a library routine or a
statistical law, so that a dropped term, a wrong sign, an index slip or a
transposed operand in the oracle fails at least one of them.
"""

import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest
from numpy.polynomial import chebyshev as npcheb

from oracle import game_oracle as o

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- expansion

def _cheb_exact(k: int, x: Fraction) -> Fraction:
    """T_k(x) by the three-term recurrence in exact rationals."""
    a, b = Fraction(1), x
    if k == 0:
        return a
    for _ in range(k - 1):
        a, b = b, 2 * x * b - a
    return b


@pytest.mark.parametrize("k", range(1, 11))
def test_chebyshev_special_values(k):
    x = np.array([1.0, -1.0, 0.0])
    v = o.chebyshev_T(k, x)
    assert v[0] == pytest.approx(1.0, abs=1e-14)
    assert v[1] == pytest.approx((-1.0) ** k, abs=1e-14)
    assert v[2] == pytest.approx(0.0 if k % 2 else (-1.0) ** (k // 2), abs=1e-14)


def test_chebyshev_against_exact_recurrence():
    pts = [Fraction(p, q) for p, q in [(0, 1), (1, 2), (-1, 2), (1, 3), (-2, 3), (3, 4), (-7, 8),
                                      (1, 1), (-1, 1), (5, 4), (-3, 2)]]
    for k in range(1, 11):
        got = o.chebyshev_T(k, np.array([float(p) for p in pts]))
        want = np.array([float(_cheb_exact(k, p)) for p in pts])
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)


def test_chebyshev_against_numpy_chebval():
    x = np.linspace(-1, 1, 1001)
    for k in range(1, 11):
        c = np.zeros(k + 1)
        c[k] = 1.0
        np.testing.assert_allclose(o.chebyshev_T(k, x), npcheb.chebval(x, c), atol=1e-12)


def test_chebyshev_discrete_orthogonality():
    N = 16
    xj = np.cos(np.pi * (np.arange(N) + 0.5) / N)
    for m in range(1, 9):
        for n in range(1, 9):
            s = np.sum(o.chebyshev_T(m, xj) * o.chebyshev_T(n, xj))
            assert s == pytest.approx(N / 2 if m == n else 0.0, abs=1e-11)


def test_trig_basis_identities():
    x = np.linspace(-1, 1, 257)
    d = 6
    for k in range(1, d + 1):
        c = o.basis_value("trig", d, k - 1, x)
        s = o.basis_value("trig", d, d + k - 1, x)
        np.testing.assert_allclose(c * c + s * s, 1.0, atol=1e-14)
        # cos(kx) = T_k(cos x): ties the two bases together
        np.testing.assert_allclose(c, o.chebyshev_T(k, np.cos(x)), atol=1e-12)
    # sin(2x) = 2 sin x cos x
    np.testing.assert_allclose(o.basis_value("trig", d, d + 1, x), 2 * np.sin(x) * np.cos(x),
                               atol=1e-14)


@pytest.mark.parametrize("basis", ["chebyshev", "trig"])
def test_gene_layout_one_hot(basis):
    """A chromosome with one non-zero gene (f, b) outputs exactly that basis member of f."""
    rng = np.random.default_rng(1)
    F, d = 3, 4
    X = rng.uniform(-1, 1, size=(9, F))
    K = o.n_genes(basis, F, d)
    Bd = K // F
    for f in range(F):
        for b in range(Bd):
            g = np.zeros(K)
            g[1 + f * Bd + b] = 1.0
            if basis == "chebyshev":
                want = np.cos((b + 1) * np.arccos(X[:, f]))
            elif b < d:
                want = np.cos((b + 1) * X[:, f])
            else:
                want = np.sin((b - d + 1) * X[:, f])
            got = o.outputs(o.expand(X, basis, d), g[None, :])[0]
            np.testing.assert_allclose(got, want, atol=1e-13)


def test_bias_only_chromosome():
    X = np.random.default_rng(2).uniform(-1, 1, size=(11, 5))
    K = o.n_genes("chebyshev", 5, 3)
    g = np.zeros((1, K))
    g[0, 0] = -0.375
    np.testing.assert_array_equal(o.outputs(o.expand(X, "chebyshev", 3), g)[0], -0.375)


def test_tiny_brute_force_exact():
    """Out over 4 patterns, F=2, d=2, x in {0, +-1/2, +-1}, rational genes: exact arithmetic."""
    xs = [[Fraction(0), Fraction(1, 2)], [Fraction(-1, 2), Fraction(1)],
          [Fraction(-1), Fraction(0)], [Fraction(1, 2), Fraction(-1, 2)]]
    genes = [[Fraction(1, 4), Fraction(-1, 2), Fraction(3, 4), Fraction(1, 8), Fraction(-1)],
             [Fraction(-1), Fraction(1), Fraction(0), Fraction(1, 2), Fraction(1, 2)]]
    want = []
    for g in genes:
        row = []
        for x in xs:
            v = g[0]
            for f in range(2):
                for b in range(2):
                    v += g[1 + f * 2 + b] * _cheb_exact(b + 1, x[f])
            row.append(float(v))
        want.append(row)
    X = np.array([[float(v) for v in x] for x in xs])
    G = np.array([[float(v) for v in g] for g in genes])
    np.testing.assert_allclose(o.outputs(o.expand(X, "chebyshev", 2), G), want, atol=1e-15)


@pytest.mark.parametrize("basis", ["chebyshev", "trig"])
def test_expand_matmul_equals_eq2_double_loop(basis):
    rng = np.random.default_rng(3)
    X = rng.uniform(-1, 1, size=(50, 4))
    K = o.n_genes(basis, 4, 3)
    G = rng.uniform(-1, 1, size=(7, K))
    np.testing.assert_allclose(o.outputs(o.expand(X, basis, 3), G),
                               o.outputs_eq2(X, G, basis, 3), atol=1e-12)


def test_tied_genes_equal_paper_shared_polytrigo():
    """Per-feature genes tied across features reproduce the paper's shared-coefficient
    polytrigo (eq.9): Out = a0 + sum_i sum_j a_j cos(j f_i) + b_j sin(j f_i)."""
    rng = np.random.default_rng(4)
    F, d = 5, 3
    X = rng.uniform(-1, 1, size=(13, F))
    v = rng.uniform(-1, 1, size=2 * d + 1)              # [a0, a1..ad, b1..bd]
    want = np.empty(13)
    for k in range(13):                                  # serial loop of the paper's Section 4.1
        ret = v[0]
        for i in range(F):
            for j in range(1, d + 1):
                ret += v[j] * math.cos(j * X[k, i]) + v[j + d] * math.sin(j * X[k, i])
        want[k] = ret
    tied = np.concatenate([[v[0]], np.tile(v[1:], F)])
    np.testing.assert_allclose(o.outputs(o.expand(X, "trig", d), tied[None, :])[0], want,
                               atol=1e-13)
    # the shared-coefficient expansion carries the paper's form with 2d + 1 genes
    assert o.n_genes("trig", F, d, shared=True) == 2 * d + 1
    np.testing.assert_allclose(o.outputs(o.expand(X, "trig", d, shared=True), v[None, :])[0],
                               want, atol=1e-13)
    cheb = rng.uniform(-1, 1, size=d + 1)
    tied_c = np.concatenate([[cheb[0]], np.tile(cheb[1:], F)])
    np.testing.assert_allclose(
        o.outputs(o.expand(X, "chebyshev", d, shared=True), cheb[None, :])[0],
        o.outputs(o.expand(X, "chebyshev", d), tied_c[None, :])[0], atol=1e-13)


# ------------------------------------------------------------------ errors

def test_paper_worked_example_mse_tmse():
    ex = json.load(open(os.path.join(GOLDEN, "paper_tmse_example.json")))
    t = np.array(ex["targets"])
    cfg_lin = o.Config(activation="linear")
    for sol, mse_p, tmse_p, eff_p in zip(ex["solutions"], ex["printed_mse"], ex["printed_tmse"],
                                        ex["printed_efficiency"]):
        Y = np.array([sol])
        mse = o.reduce_errors(o.pattern_errors(t, Y, "mse", 0.0), "mse")[0]
        tmse = o.reduce_errors(o.pattern_errors(t, Y, "tmse", ex["R"]), "tmse")[0]
        assert round(mse, ex["printed_decimals"]) == pytest.approx(mse_p)
        assert round(tmse, ex["printed_decimals"]) == pytest.approx(tmse_p)
        eff = np.mean(o.classify(Y[0], cfg_lin.activation) == t)
        assert eff == pytest.approx(eff_p)
    # the exact values behind the printed two-decimal figures
    assert o.reduce_errors(o.pattern_errors(t, np.array([[0.49, 0.51]]), "mse", 0), "mse")[0] \
        == pytest.approx(0.2401, abs=1e-15)
    assert o.reduce_errors(o.pattern_errors(t, np.array([[0.0, 0.49]]), "mse", 0), "mse")[0] \
        == pytest.approx(0.13005, abs=1e-15)
    # eq.10 as printed (squared error against R) would zero 0.2601 as well
    assert o.reduce_errors(o.pattern_errors(t, np.array([[0.0, 0.49]]), "tmse_sq", 0.5),
                           "tmse_sq")[0] == 0.0


def test_rmse_squared_is_mse_and_permutation_invariance():
    rng = np.random.default_rng(5)
    X = rng.uniform(-1, 1, size=(64, 3))
    t = np.where(rng.random(64) < 0.5, 1.0, -1.0)
    P = o.expand(X, "chebyshev", 3)
    G = rng.uniform(-1, 1, size=(6, P.shape[1]))
    rm = o.fitness(P, t, G, o.Config(error="rmse"))
    ms = o.fitness(P, t, G, o.Config(error="mse"))
    np.testing.assert_allclose(rm ** 2, ms, rtol=1e-13)
    perm = rng.permutation(64)
    np.testing.assert_allclose(o.fitness(P[perm], t[perm], G, o.Config()), rm, rtol=1e-13)


@pytest.mark.parametrize("basis", ["chebyshev", "trig"])
def test_planted_chromosome_has_zero_error(basis):
    """Targets made by numpy's own Chebyshev series routine (or np.cos / np.sin) from the
    planted genes, not by the oracle's expansion: the oracle's output path (eq.2 through
    expand + outputs, the activation, the error and its reduction) must give the planted
    chromosome zero error, and a perturbed copy a positive one."""
    from paper_1304_0597_gb300 import synth
    rng = np.random.default_rng(6)
    X = rng.uniform(-1, 1, size=(500, 6))
    P = o.expand(X, basis, 4)
    h = rng.uniform(-1, 1, size=P.shape[1])
    t = synth.planted_targets(X, h, basis, 4)
    h2 = h.copy()
    h2[-1] += 1e-3                      # the last basis member of the last feature
    G = np.stack([h, rng.uniform(-1, 1, size=h.shape), h2])
    for err in ("rmse", "mse", "tmse"):
        fit = o.fitness(P, t, G, o.Config(basis=basis, degree=4, error=err))
        assert fit[0] <= 1e-15
        assert fit[1] > 1e-4
        assert err == "tmse" or fit[2] > 0.0


def test_rank_orders_by_fitness_then_index_nan_last():
    fit = np.array([0.5, np.nan, 0.1, 0.5, 0.1, np.inf])
    assert list(o.rank(fit)) == [2, 4, 0, 3, 1, 5]


# -------------------------------------------------------------- randomness

def test_philox_matches_numpy_bit_generator():
    """numpy.random.Philox is Philox4x64-10; it increments the counter before each block."""
    for key, ctr in [((1, 2), (0, 0, 0, 0)), ((123456789, 987654321), (7, 3, 2, 5)),
                     ((2 ** 64 - 1, 0), (2 ** 64 - 1, 5, 0, 0))]:
        bg = np.random.Philox(key=np.array(key, dtype=np.uint64),
                              counter=np.array(ctr, dtype=np.uint64))
        raw = bg.random_raw(12)
        c0 = ctr[0]
        blocks = []
        for b in range(3):
            c = [(c0 + 1 + b) % 2 ** 64, ctr[1] + (1 if c0 + 1 + b >= 2 ** 64 else 0), ctr[2],
                 ctr[3]]
            blocks.append(o.philox4x64(tuple(np.array([v], dtype=np.uint64) for v in c), key)[0])
        np.testing.assert_array_equal(np.concatenate(blocks), raw)


def test_philox_word_layout():
    key = (11, 22)
    words = o.philox_words(key, 3, 4, 1, np.arange(16))
    blk0 = o.philox4x64(([3], [4], [1], [0]), key)[0]
    blk1 = o.philox4x64(([3], [4], [1], [1]), key)[0]
    want = []
    for blk in (blk0, blk1):
        for v in blk:
            want += [int(v) & 0xFFFFFFFF, int(v) >> 32]
    assert [int(w) for w in words] == want


def test_uniform_and_index_draws():
    w = np.array([0, 255, 256, 2 ** 32 - 1], dtype=np.uint64)
    u = o.uniform24(w)
    assert u.dtype == np.float32
    assert list(u) == [0.0, 0.0, 2.0 ** -24, 1.0 - 2.0 ** -24]
    assert list(o.index_draw(w, 7)) == [0, 0, 0, 6]
    words = o.philox_words((9, 0), 0, np.arange(200000), 0, 0)
    counts = np.bincount(o.index_draw(words, 10), minlength=10)
    chi2 = np.sum((counts - 20000.0) ** 2 / 20000.0)
    assert chi2 < 30.0          # 9 dof, p ~ 4e-4


def test_log_and_cos_against_libm():
    u = np.concatenate([np.float32(2.0) ** -np.arange(0, 25, dtype=np.float32),
                        np.random.default_rng(7).uniform(2 ** -24, 1, 100000).astype(np.float32)])
    ref = np.log(u.astype(np.float64))
    err = np.abs(o.ln_f32(u).astype(np.float64) - ref)
    assert np.all(err <= 4e-7 * np.maximum(1.0, np.abs(ref)))
    v = (np.arange(1 << 16) * 2.0 ** -16).astype(np.float32)
    assert np.max(np.abs(o.cos2pi_f32(v) - np.cos(2 * np.pi * v.astype(np.float64)))) < 4e-7


def test_gaussian_distribution():
    from scipy import stats
    n = 200000
    j = np.arange(n)
    z = o.gauss_f32(o.philox_words((5, 1), 2, j, 3, 0), o.philox_words((5, 1), 2, j, 3, 1))
    assert abs(z.mean()) < 0.01
    assert abs(z.std() - 1.0) < 0.01
    assert abs(stats.skew(z)) < 0.03
    assert abs(stats.kurtosis(z)) < 0.06
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # against a float64 Box-Muller of the same words
    w0 = o.philox_words((5, 1), 2, j, 3, 0)
    w1 = o.philox_words((5, 1), 2, j, 3, 1)
    u1 = ((w0 >> np.uint64(8)) + np.uint64(1)).astype(np.float64) * 2.0 ** -24
    u2 = (w1 >> np.uint64(8)).astype(np.float64) * 2.0 ** -24
    ref = np.sqrt(-2 * np.log(u1)) * np.cos(2 * np.pi * u2)
    assert np.max(np.abs(z - ref)) < 2e-6


# ----------------------------------------------------------------- operators

def _cfg(**kw):
    base = dict(pop=40, tournament_k=3, p_crossover=0.9, p_mutation=0.05, sigma_mutation=0.1,
                elitism=2, seed=17)
    base.update(kw)
    return o.Config(**base)


def test_init_modes():
    K = 33
    g = o.init_population(_cfg(pop=3000, init="uniform_pm1"), K)
    assert g.dtype == np.float32 and g.min() >= -1 and g.max() < 1
    assert abs(g.mean()) < 0.01 and abs(g.var() - 1 / 3) < 0.01
    g = o.init_population(_cfg(pop=3000, init="uniform_01"), K)
    assert g.min() >= 0 and g.max() < 1 and abs(g.mean() - 0.5) < 0.01
    g = o.init_population(_cfg(pop=3000, init="normal_pm1"), K)
    assert g.min() >= -1 and g.max() <= 1
    # N(0, 0.5^2) truncated at +-2 sigma: variance 0.25 * (1 - 4 phi(2) / (2 Phi(2) - 1))
    from scipy import stats
    trunc_var = 0.25 * (1 - 2 * 2 * stats.norm.pdf(2) / (2 * stats.norm.cdf(2) - 1))
    assert abs(g.var() - trunc_var) < 0.005


def test_tournament_rank_frequencies():
    """P(winner has rank r) = ((n-r+1)^k - (n-r)^k) / n^k for k draws with replacement."""
    n, k = 12, 3
    fit = np.random.default_rng(8).permutation(n).astype(np.float64) + 0.5
    order = o.rank(fit)
    rank_of = np.empty(n, dtype=np.int64)
    rank_of[order] = np.arange(n)
    pairs = np.arange(60000, dtype=np.uint64)
    win = o.tournament((3, 0), 5, pairs, 0, k, fit)
    counts = np.bincount(rank_of[win], minlength=n).astype(np.float64)
    r = np.arange(1, n + 1, dtype=np.float64)
    p = ((n - r + 1) ** k - (n - r) ** k) / n ** k
    chi2 = np.sum((counts - p * len(pairs)) ** 2 / (p * len(pairs)))
    assert abs(p.sum() - 1) < 1e-12
    assert chi2 < 35.0          # 11 dof


def test_crossover_is_a_per_position_swap_and_cut_is_uniform():
    pop, K = 64, 21
    G = o.init_population(_cfg(pop=pop), K)
    cfg = _cfg(pop=pop, elitism=0, p_mutation=0.0, p_crossover=1.0)
    cuts = []
    for gen in range(60):
        fit = np.arange(pop, dtype=np.float64)
        child = o.breed(G, fit, cfg, gen)
        for j in range(pop // 2):
            a, b = child[2 * j], child[2 * j + 1]
            # each position of (a, b) holds two genes drawn from one parent pair
            same = [(a[g] == G[:, g]).any() and (b[g] == G[:, g]).any() for g in range(K)]
            assert all(same)
            # the cut: a switches from one parent to the other exactly once
            src = [int(np.nonzero(G[:, g] == a[g])[0][0]) for g in range(K)]
            sw = [g for g in range(1, K) if src[g] != src[g - 1]]
            if len(sw) == 1:
                cuts.append(sw[0])
    counts = np.bincount(cuts, minlength=K)[1:]
    assert counts.min() > 0.5 * counts.mean()


def test_mutation_count_is_binomial():
    pop, K = 200, 50
    G = np.zeros((pop, K), dtype=np.float32)
    cfg = _cfg(pop=pop, elitism=0, p_crossover=0.0, p_mutation=0.05, clamp_genes=False)
    child = o.breed(G, np.zeros(pop), cfg, 0)
    n = pop * K
    m = np.count_nonzero(child)
    assert abs(m - 0.05 * n) < 4 * math.sqrt(n * 0.05 * 0.95)
    z = child[child != 0] / np.float32(0.1)
    assert abs(z.mean()) < 0.1 and abs(z.std() - 1) < 0.1


def test_clones_without_variation_are_a_fixed_point():
    K = 15
    g = o.init_population(_cfg(pop=1), K)[0]
    G = np.tile(g, (30, 1))
    cfg = _cfg(pop=30, p_crossover=0.0, p_mutation=0.0)
    np.testing.assert_array_equal(o.breed(G, np.arange(30.0), cfg, 4), G)


def test_elitism_keeps_top_and_best_never_worsens():
    from paper_1304_0597_gb300 import synth
    ds = synth.make_dataset(600, 4, 3, seed=11)
    P = o.expand(ds.X[:ds.n_train], "chebyshev", 3)
    t = ds.t[:ds.n_train]
    for mode in ("top", "copies"):
        cfg = _cfg(pop=24, elitism=2, elite_mode=mode, sigma_mutation=0.3, p_mutation=0.2)
        res = o.evolve(P, t, cfg, 25)
        assert all(b <= a + 0.0 for a, b in zip(res.history, res.history[1:]))
        G = o.init_population(cfg, P.shape[1])
        fit = o.fitness(P, t, G, cfg)
        child = o.breed(G, fit, cfg, 0)
        order = o.rank(fit)
        if mode == "top":
            np.testing.assert_array_equal(child[:2], G[order[:2]])
        else:
            np.testing.assert_array_equal(child[:2], G[[order[0], order[0]]])


def test_immigrants_replace_the_last_children_with_fresh_draws():
    """Immigrants: rows pop-I..pop-1 are replaced, every other row is the plain breed;
    the new rows follow the init distribution (moments), differ between generations
    and from generation 0, and elites survive (I <= pop - elitism)."""
    rng = np.random.default_rng(31)
    K, pop, I = 40, 300, 120
    G = rng.uniform(-1, 1, size=(pop, K)).astype(np.float32)
    fit = rng.random(pop)
    base = o.Config(pop=pop, elitism=3, seed=9)
    plain = o.breed(G, fit, base, 5)
    imm = o.breed(G, fit, o.Config(pop=pop, elitism=3, seed=9, immigrants=I), 5)
    np.testing.assert_array_equal(imm[:pop - I], plain[:pop - I])
    new = imm[pop - I:]
    assert not np.any(new == plain[pop - I:])
    assert new.min() >= -1 and new.max() <= 1
    assert abs(new.mean()) < 0.03 and abs(new.var() - 1 / 3) < 0.02          # U[-1, 1]
    imm6 = o.breed(G, fit, o.Config(pop=pop, elitism=3, seed=9, immigrants=I), 6)
    assert not np.any(imm6[pop - I:] == new)
    g0 = o.init_population(o.Config(pop=pop, seed=9), K)
    assert not np.any(g0[pop - I:] == new)
    order = o.rank(fit)
    np.testing.assert_array_equal(imm[:3], G[order[:3]])
    u01 = o.breed(G, fit, o.Config(pop=pop, elitism=3, seed=9, immigrants=I, init="uniform_01"), 5)
    assert u01[pop - I:].min() >= 0 and abs(u01[pop - I:].mean() - 0.5) < 0.02
    nrm = o.breed(G, fit, o.Config(pop=pop, elitism=3, seed=9, immigrants=I, init="normal_pm1"), 5)
    v = nrm[pop - I:]
    # N(0, 0.5^2) truncated to [-1, 1] = +-2 sigma: std = 0.5 sqrt(1 - 4 phi(2) / (2 Phi(2) - 1))
    from scipy import stats
    sd = 0.5 * np.sqrt(1 - 4 * stats.norm.pdf(2) / (2 * stats.norm.cdf(2) - 1))
    assert np.abs(v).max() <= 1 and abs(v.mean()) < 0.02 and abs(v.std() - sd) < 0.01


def test_wheel_draw_exact_boundaries_and_frequencies():
    """Roulette / ranking draw on integer weights: weights 1 and 3 give index 0 exactly
    for the top 24 bits u with (4 u) >> 24 == 0, i.e. u < 2^22; frequencies of a
    roulette on 1 / (1e-12 + f) match w / sum(w) (chi^2); NaN never drawn; a zero total
    draws uniformly."""
    from scipy import stats
    cum = np.cumsum(np.array([1, 3], dtype=np.uint64), dtype=np.uint64)
    words = np.array([0, (1 << 30) - 1, 1 << 30, (1 << 32) - 1], dtype=np.uint64)
    np.testing.assert_array_equal(o.wheel_draw(cum, words), [0, 0, 1, 1])
    fit = np.array([0.5, 0.25, 1.0, np.nan, 0.125])
    cfg = o.Config(pop=5, selection="roulette")
    q = o.selection_weights(fit, cfg)
    assert q[3] == 0 and q[4] == 1 << 24 and q[1] == 1 << 23
    w = np.where(np.isnan(fit), 0, 1 / fit)
    words = o.philox_words((3, 0), 0, np.arange(200000, dtype=np.uint64), 0, 0)
    idx = o.wheel_draw(np.cumsum(q, dtype=np.uint64), words)
    assert not np.any(idx == 3)
    counts = np.bincount(idx, minlength=5)[[0, 1, 2, 4]]
    expect = (w / w.sum())[[0, 1, 2, 4]] * len(idx)
    assert stats.chisquare(counts, expect).pvalue > 1e-3
    z = o.wheel_draw(np.zeros(5, dtype=np.uint64), words[:10])
    np.testing.assert_array_equal(z, o.index_draw(words[:10], 5))


def test_ranking_weights_are_linear_in_rank():
    """Linear ranking: expected values 1.1 (best) to 0.9 (worst), ties by index."""
    fit = np.array([0.3, 0.1, 0.3, 0.2])
    q = o.selection_weights(fit, o.Config(pop=4, selection="ranking"))
    # order: 1 (0.1), 3 (0.2), 0 (0.3, lower index), 2 (0.3)
    np.testing.assert_array_equal(q[[1, 3, 0, 2]], [33, 31, 29, 27])
    assert q[1] / q[2] == pytest.approx(1.1 / 0.9)


def test_clamp_keeps_genes_in_range():
    G = np.full((50, 10), 0.99, dtype=np.float32)
    cfg = _cfg(pop=50, elitism=0, p_mutation=1.0, sigma_mutation=1.0)
    child = o.breed(G, np.zeros(50), cfg, 0)
    assert child.max() <= 1.0 and child.min() >= -1.0 and (child == 1.0).any()


def test_odd_slots_drop_last_second_child():
    G = o.init_population(_cfg(pop=7), 9)
    cfg = _cfg(pop=7, elitism=2, p_mutation=0.0, p_crossover=0.0)
    child = o.breed(G, np.arange(7.0), cfg, 0)
    assert child.shape == (7, 9)


def test_report_figures_of_merit():
    P = np.ones((6, 1))
    t = np.array([1, 1, 1, -1, -1, -1], dtype=np.float64)
    # outputs tanh(g) with g chosen per pattern through a diagonal trick: use K=6 one-hot P
    P = np.eye(6)
    g = np.array([2.0, 2.0, -2.0, 2.0, -2.0, -2.0])
    r = o.report(P, t, g, o.Config())
    # predictions: + + - + - -  -> TP=2, FN=1, FP=1, TN=2
    assert r["accuracy"] == pytest.approx(4 / 6)
    assert r["completeness"] == pytest.approx(2 / 3)
    assert r["contamination"] == pytest.approx(1 / 3)
    assert r["rmse"] == pytest.approx(math.sqrt(np.mean((t - np.tanh(g)) ** 2)))


def test_stop_criterion_on_planted_solution():
    from paper_1304_0597_gb300 import synth
    rng = np.random.default_rng(12)
    X = rng.uniform(-1, 1, size=(300, 3))
    P = o.expand(X, "chebyshev", 2)
    h = o.init_population(_cfg(pop=1), P.shape[1])[0].astype(np.float64)
    t = synth.planted_targets(X, h, "chebyshev", 2)
    cfg = _cfg(pop=10, stop_error=1e-9)
    G0 = o.init_population(cfg, P.shape[1])
    G0[3] = h
    res = o.evolve(P, t, cfg, 50, G0=G0)
    assert res.generations == 1 and res.best_fitness <= 1e-12


# ------------------------------------------------------------ low precision

def test_bf16_rounding_matches_torch():
    import torch
    x = np.concatenate([np.random.default_rng(13).standard_normal(100000).astype(np.float32),
                        np.array([1.0, -1.0, 0.0, 1.00390625, 1.01171875, 3.3895314e38],
                                 dtype=np.float32)])
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    np.testing.assert_array_equal(o.round_bf16(x), want)


def test_e4m3_rounding_matches_torch_in_range():
    import torch
    rng = np.random.default_rng(14)
    x = np.concatenate([rng.uniform(-448, 448, 50000), rng.uniform(-1, 1, 50000),
                        rng.uniform(-0.02, 0.02, 50000)]).astype(np.float32)
    want = torch.from_numpy(x).to(torch.float8_e4m3fn).to(torch.float32).numpy()
    np.testing.assert_array_equal(o.round_e4m3(x), want)
    # saturation of the format's largest finite value
    assert o.round_e4m3(np.array([500.0, -1e6], dtype=np.float32)).tolist() == [448.0, -448.0]
    # every representable magnitude is a fixed point
    reps = np.unique(np.abs(o.round_e4m3(rng.uniform(-448, 448, 200000).astype(np.float32))))
    np.testing.assert_array_equal(o.round_e4m3(reps), reps)
    assert len(reps) <= 127


def test_quantize_columns_bounds():
    rng = np.random.default_rng(15)
    P = o.expand(rng.uniform(-1, 1, size=(3000, 4)), "chebyshev", 5)[:, 1:]
    for fmt, rel in (("bf16", 2.0 ** -8), ("fp8", 2.0 ** -4)):   # unit roundoff: 7 and 3 mantissa bits
        Q, s = o.quantize_columns(P, fmt)
        assert np.max(np.abs(Q)) <= o.QMAX[fmt]
        D = o.dequantize_columns(Q, s)
        # relative rounding bound of the format for normal values, plus the subnormal floor
        floor = s[None, :] * (2.0 ** -9 if fmt == "fp8" else 0.0)
        assert np.all(np.abs(D - P) <= rel * np.abs(P) + floor + 1e-7)


def _gene_case(seed=16, pop=40, K=33):
    """Genes in [-1, 1] (a few chromosomes with one dominant gene) and column scales spread
    over six decades, so that a scale applied on the wrong side or over the wrong axis
    moves genes by orders of magnitude."""
    rng = np.random.default_rng(seed)
    G = rng.uniform(-1, 1, size=(pop, K)).astype(np.float32)
    G[3, 1:] *= 1e-3
    G[3, 7] = 0.9
    G[5, 1:] = 0.0                                           # an all-zero chromosome
    s = (10.0 ** rng.uniform(-3, 3, size=K - 1)).astype(np.float32)
    return G, s


@pytest.mark.parametrize("fmt", ["bf16", "fp8"])
def test_quantize_genes_one_plane_error_bound(fmt):
    """One term: gene g meets the stored Q through w = g s_g / r_c rounded to the format, so
    |Gq - G| <= u |G| + (subnormal half-step) r_c / s_g, with u the format's unit roundoff
    (2^-8 bf16, 2^-4 e4m3; e4m3 half-step below its smallest normal 2^-10) and a float32
    allowance; r_c = max_g |G s_g| / qmax."""
    G, s = _gene_case()
    Gq = o.quantize_genes(G, s, fmt, 1)
    u = 2.0 ** -8 if fmt == "bf16" else 2.0 ** -4
    half_sub = 0.0 if fmt == "bf16" else 2.0 ** -10
    r = np.abs(G[:, 1:].astype(np.float64) * s).max(axis=1) / o.QMAX[fmt]
    r = np.where(r > 0, r, 1.0)
    bound = (u + 2.0 ** -21) * np.abs(G[:, 1:]) + half_sub * r[:, None] / s[None, :]
    assert np.all(np.abs(Gq[:, 1:] - G[:, 1:]) <= bound)
    # the bound is not loose: typical genes do move by a sizeable share of it
    assert np.median(np.abs(Gq[:, 1:] - G[:, 1:]) / np.maximum(bound, 1e-300)) > 0.05


@pytest.mark.parametrize("fmt", ["bf16", "fp8"])
def test_quantize_genes_two_planes_error_bound(fmt):
    """Two terms hi + lo with lo = q(w - hi): the error is the rounding of the remainder,
    |Gq - G| <= (u^2 + 2^-21) |G| + (subnormal half-step) r_c / s_g -- second order in u."""
    G, s = _gene_case()
    Gq = o.quantize_genes(G, s, fmt, 2)
    u = 2.0 ** -8 if fmt == "bf16" else 2.0 ** -4
    half_sub = 0.0 if fmt == "bf16" else 2.0 ** -10
    r = np.abs(G[:, 1:].astype(np.float64) * s).max(axis=1) / o.QMAX[fmt]
    r = np.where(r > 0, r, 1.0)
    bound = (u * u + 2.0 ** -21) * np.abs(G[:, 1:]) + half_sub * r[:, None] / s[None, :]
    assert np.all(np.abs(Gq[:, 1:] - G[:, 1:]) <= bound)
    # where the format's normal range holds the remainder, the second term helps
    normal = half_sub * r[:, None] / s[None, :] <= 0.1 * u * u * np.abs(G[:, 1:])
    assert normal.sum() > 100
    one = np.abs(o.quantize_genes(G, s, fmt, 1)[:, 1:] - G[:, 1:])[normal].sum()
    assert np.abs(Gq[:, 1:] - G[:, 1:])[normal].sum() < 0.25 * one


@pytest.mark.parametrize("fmt", ["bf16", "fp8"])
def test_quantize_genes_largest_scaled_gene_is_exact_and_bias_untouched(fmt):
    """The largest |g s_g| of a chromosome maps to +-qmax, a value of both formats, so that
    gene comes back unchanged (to float32 rounding); gene 0 (the bias, which meets the
    implicit column of ones) is never quantised; a zero chromosome stays zero."""
    G, s = _gene_case()
    for planes in (1, 2):
        Gq = o.quantize_genes(G, s, fmt, planes)
        np.testing.assert_array_equal(Gq[:, 0], G[:, 0].astype(np.float64))
        j = np.argmax(np.abs(G[:, 1:].astype(np.float64) * s), axis=1)
        rows = np.arange(G.shape[0])
        keep = np.abs(G[rows, 1 + j]) > 0
        np.testing.assert_allclose(Gq[rows, 1 + j][keep], G[rows, 1 + j][keep], rtol=3e-7)
        assert np.all(Gq[5, 1:] == 0.0)


@pytest.mark.parametrize("fmt", ["bf16", "fp8"])
def test_quantize_genes_matches_torch_cast_construction(fmt):
    """The same operand built with torch's own format casts (float32 arithmetic, torch
    bfloat16 / float8_e4m3fn conversion)."""
    import torch
    G, s = _gene_case(seed=17)
    dt = torch.bfloat16 if fmt == "bf16" else torch.float8_e4m3fn
    g = torch.from_numpy(G[:, 1:]) * torch.from_numpy(s)[None, :]
    r = g.abs().amax(dim=1) / o.QMAX[fmt]
    r = torch.where(r > 0, r, torch.ones_like(r))
    w = g / r[:, None]
    for planes in (1, 2):
        hi = w.to(dt).to(torch.float32)
        val = hi.double()
        if planes == 2:
            val = val + (w - hi).to(dt).to(torch.float32).double()
        want = val * r.double()[:, None] / torch.from_numpy(s).double()[None, :]
        np.testing.assert_array_equal(o.quantize_genes(G, s, fmt, planes)[:, 1:], want.numpy())


# --------------------------------------------------------------- surrogate

def _mlp(rng, d=7, h=5):
    return {"W1": rng.standard_normal((h, d)) * 0.4, "b1": rng.standard_normal(h) * 0.1,
            "W2": rng.standard_normal((h, h)) * 0.4, "b2": rng.standard_normal(h) * 0.1,
            "w3": rng.standard_normal(h) * 0.4, "b3": np.array(0.05)}


def test_gelu_against_its_definition_and_scipy():
    from scipy import stats
    z = np.linspace(-6, 6, 1001)
    np.testing.assert_allclose(o.gelu(z), z * stats.norm.cdf(z), atol=1e-15)
    # derivative by central differences
    h = 1e-6
    np.testing.assert_allclose(o.gelu_grad(z), (o.gelu(z + h) - o.gelu(z - h)) / (2 * h), atol=1e-8)


def test_mlp_gradient_by_finite_differences():
    rng = np.random.default_rng(21)
    p = _mlp(rng)
    X = rng.uniform(-1, 1, size=(9, 7))
    t = rng.standard_normal(9)
    _, g = o.mlp_loss_grad(p, X, t)
    h = 1e-6
    for name in ("W1", "b1", "W2", "b2", "w3", "b3"):
        flat = p[name].reshape(-1)
        num = np.empty(flat.size)
        for i in range(flat.size):
            old = flat[i]
            flat[i] = old + h
            lp, _ = o.mlp_loss_grad(p, X, t)
            flat[i] = old - h
            lm, _ = o.mlp_loss_grad(p, X, t)
            flat[i] = old
            num[i] = (lp - lm) / (2 * h)
        np.testing.assert_allclose(np.asarray(g[name]).reshape(-1), num, rtol=1e-5, atol=1e-9)


def test_mlp_bf16_operands_bounded_and_applied():
    """The bfloat16-operand network: identity rounding is the exact network; bf16
    rounding of x, gelu(Z1), dZ2 and dZ1 moves every result by no more than the
    rounding bound (relative 2^-8 per operand, propagated through two layers) and
    by more than float64 noise (the rounding is really applied)."""
    rng = np.random.default_rng(23)
    p = _mlp(rng)
    X = rng.uniform(-1, 1, size=(16, 7))
    t = rng.standard_normal(16)
    l0, g0 = o.mlp_loss_grad(p, X, t)
    li, gi = o.mlp_loss_grad(p, X, t, operand_round=lambda a: a)
    assert li == l0
    for k in g0:
        np.testing.assert_array_equal(gi[k], g0[k])
    y0 = o.mlp_forward(p, X)["y"]
    yr = o.mlp_forward(p, X, o.bf16_operands)["y"]
    # |dy| <= 2 u (sum |w3| |gelu'| |W2| |H1| + ...) : bound by the magnitudes of the terms
    f = o.mlp_forward(p, X)
    u = 2.0 ** -8
    bound = u * (np.abs(f["H1"]) @ np.abs(p["W2"]).T @ np.abs(p["w3"]) * 1.2 +
                 np.abs(X) @ np.abs(p["W1"]).T @ np.abs(p["W2"]).T @ np.abs(p["w3"]) * 1.2 * 1.2)
    assert np.all(np.abs(yr - y0) <= bound)
    assert np.max(np.abs(yr - y0)) > 1e-9
    _, gr = o.mlp_loss_grad(p, X, t, operand_round=o.bf16_operands)
    for k in ("W1", "W2", "b1", "b2"):
        rel = np.max(np.abs(gr[k] - g0[k])) / np.max(np.abs(g0[k]))
        assert 1e-9 < rel < 0.05, (k, rel)


def test_adam_first_step_moves_each_parameter_by_lr():
    """At step 1 the bias-corrected update is lr * g/(|g| + eps): size lr, against the gradient."""
    g = np.array([0.3, -2.0, 1e-3])
    p, m, v = o.adam_update(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.01, eps=0.0)
    np.testing.assert_allclose(p, -0.01 * np.sign(g), rtol=1e-12)
    # a constant gradient keeps the step size lr (bias correction exact for a constant)
    for step in range(2, 6):
        p, m, v = o.adam_update(p, g, m, v, step, lr=0.01, eps=0.0)
    np.testing.assert_allclose(p, -0.05 * np.sign(g), rtol=1e-10)


def test_surrogate_select_against_brute_force():
    """The kept set is the n_sel smallest (score, index) pairs, found here by trying every
    row against every other; ties at the cut go to lower indices; the order is the rows
    below the cut, then those at it, each in pool order."""
    rng = np.random.default_rng(21)
    for trial in range(200):
        n = int(rng.integers(1, 40))
        k = int(rng.integers(1, n + 1))
        s = rng.integers(0, 6, size=n).astype(np.float32) * 0.5      # many ties
        if trial % 7 == 0:
            s[rng.integers(0, n)] = np.nan
        got = o.surrogate_select(s, k)
        key = [(np.inf if np.isnan(v) else float(v), i) for i, v in enumerate(s)]
        below = [i for i in range(n) if sum(key[j] < key[i] for j in range(n)) < k]
        assert sorted(got.tolist()) == sorted(below)
        cut = max(key[i][0] for i in below)
        assert got.tolist() == sorted(i for i in below if key[i][0] < cut) + \
            sorted(i for i in below if key[i][0] == cut)
    assert o.surrogate_select(np.zeros(5, np.float32), 3).tolist() == [0, 1, 2]
    assert o.surrogate_select(np.array([3, 1, 2, 1], np.float32), 2).tolist() == [1, 3]
    assert o.surrogate_select(np.array([0.5, 0.1, 0.5, 0.2], np.float32), 3).tolist() == [1, 3, 0]


def test_spearman_known_values():
    a = np.arange(10.0)
    assert o.spearman(a, a) == pytest.approx(1.0)
    assert o.spearman(a, -a) == pytest.approx(-1.0)
    from scipy import stats
    rng = np.random.default_rng(3)
    x, y = rng.standard_normal(200), rng.standard_normal(200)
    assert o.spearman(x, y) == pytest.approx(stats.spearmanr(x, y)[0], abs=1e-12)
