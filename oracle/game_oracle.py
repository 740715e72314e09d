"""GAME oracle: a plain, slow, obviously correct CPU statement of the method.

TEST INFRASTRUCTURE ONLY.  This module is the yardstick the CUDA path is held
against; it is imported by ``tests/``, by ``__graft_entry__.smoke()`` and by the
CPU-baseline legs of ``bench.py`` and by nothing else.  The product library
(``paper_1304_0597_gb300``) never imports it and shares no code with it.

Everything here follows Cavuoti et al., "Astrophysical data mining with GPU.
A case study: genetic classification of globular clusters" (GAME):

* Section 2, eq.1 / eq.2 / eq.9 -- the polynomial expansion of every feature
  and the pattern output as the sum over features and degrees;
* Section 2, eq.3 / eq.4 / eq.5 -- per-pattern squared error, MSE and RMSE;
* Section 2, eq.10 -- the threshold MSE ("convergence tube");
* Section 2 (the list of chromosome properties, eq.6 / eq.7) -- genes are the
  expansion coefficients, random in [-1, +1] at start;
* Section 2 (training options) and Section 4.1 (parallelisation steps 1-4) --
  random initialisation, fitness + sort, stop test, genetic operators;
* Section 5 (experiment parameters) -- crossover / mutation / tournament /
  elitism knobs; classification accuracy, completeness and contamination.

Floating point is float64 unless noted.  Three places deliberately use float32:
the uniform / Gaussian draws and the gene update of mutation, because the genes
of a chromosome are stored as float32 and the operator output is compared
bit-for-bit with the GPU's.  Those float32 steps use only correctly rounded
IEEE operations (+, -, *, /, sqrt, floor, frexp) in a fixed order.

Readings of the paper where it is silent or ambiguous:

* coefficients are per feature (gene = 1 + f*B*d + b); the paper's shared
  coefficients of eq.2 / eq.9 are the special case of tied genes;
* ``g^j`` in eq.1 is the j-th member of the basis (eq.9 writes cos(j f_i));
* TMSE default compares the absolute error |t - Out| with R (the only reading
  that reproduces the worked example of Section 2); eq.10 as printed (squared
  error against R) is available as ``"tmse_sq"``;
* tournament draws are with replacement, ties go to the lower index;
* elitism keeps the top-e distinct chromosomes (``elite_mode="top"``) or e
  copies of the winner (``elite_mode="copies"``);
* "normal distribution in [-1, +1]" initialisation is N(0, 0.5^2) truncated to
  [-1, 1] by resampling.

Random numbers come from a counter-based Philox4x64-10 generator (Salmon,
Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11),
written here from its published definition; Gaussian draws use the Box-Muller
transform (Box & Muller, 1958) with a logarithm (atanh series) and a cosine
(Taylor series) written out in float32 below.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# ---------------------------------------------------------------------------
# Configuration (Section 2 training options; Section 5 experiment parameters)
# ---------------------------------------------------------------------------

CHEBYSHEV, TRIG = "chebyshev", "trig"


@dataclass
class Config:
    basis: str = CHEBYSHEV
    degree: int = 4
    pop: int = 20
    tournament_k: int = 3
    p_crossover: float = 0.9
    p_mutation: float = 0.05
    sigma_mutation: float = 0.1
    elitism: int = 2
    elite_mode: str = "top"          # "top" | "copies"
    error: str = "rmse"              # "rmse" | "mse" | "tmse" | "tmse_sq"
    tmse_R: float = 0.49
    activation: str = "tanh"         # "tanh" | "linear"
    init: str = "uniform_pm1"        # "uniform_pm1" | "normal_pm1" | "uniform_01"
    clamp_genes: bool = True
    stop_error: float = 0.001
    seed: int = 0
    run: int = 0                     # second Philox key word (independent runs)
    immigrants: int = 0              # random chromosomes replacing the last children
    coefficients: str = "per_feature"  # "per_feature" | "shared" (eq.2 / eq.9)
    selection: str = "tournament"    # "tournament" | "roulette" | "ranking"


def basis_multiplier(basis: str) -> int:
    """B of eq.6 / eq.7: 1 for a single-family basis, 2 for polytrigo (eq.8)."""
    return 2 if basis == TRIG else 1


def n_genes(basis: str, n_features: int, degree: int, shared: bool = False) -> int:
    """Genes per chromosome: B*F*d + 1 with per-feature coefficients, B*d + 1 when the
    coefficients are shared by all features (eq.7 / eq.9: 2d + 1 for polytrigo)."""
    return basis_multiplier(basis) * (1 if shared else n_features) * degree + 1


# ---------------------------------------------------------------------------
# Expansion (Section 2, eq.1, eq.8, eq.9)
# ---------------------------------------------------------------------------

def chebyshev_T(k: int, x: np.ndarray) -> np.ndarray:
    """T_k(x) by its closed form: cos(k*acos x) on [-1,1], cosh(k*acosh|x|)*sign^k outside."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    inside = np.abs(x) <= 1.0
    out[inside] = np.cos(k * np.arccos(x[inside]))
    xo = x[~inside]
    out[~inside] = np.cosh(k * np.arccosh(np.abs(xo))) * np.where(xo < 0, (-1.0) ** k, 1.0)
    return out


def basis_value(basis: str, degree: int, b: int, x: np.ndarray) -> np.ndarray:
    """The b-th basis member (0-based) of one feature column.

    Chebyshev: b = 0..d-1 -> T_{b+1}(x).  Polytrigo (eq.8 / eq.9): b = 0..d-1 ->
    cos((b+1) x), b = d..2d-1 -> sin((b-d+1) x), i.e. the per-feature order
    [cos 1x .. cos dx, sin 1x .. sin dx] of the gene vector [a_1..a_d, b_1..b_d].
    """
    x = np.asarray(x, dtype=np.float64)
    if basis == CHEBYSHEV:
        return chebyshev_T(b + 1, x)
    if b < degree:
        return np.cos((b + 1) * x)
    return np.sin((b - degree + 1) * x)


def expand(X: np.ndarray, basis: str, degree: int, shared: bool = False) -> np.ndarray:
    """Expansion matrix P [NP x K] (eq.1 written out per feature, eq.9 for polytrigo).

    Column 0 is the bias (a_0 multiplies 1); column 1 + f*B*d + b holds the
    b-th basis member of feature f.  With shared coefficients (eq.2 / eq.9, one
    a_j for every feature) column 1 + b is the sum over the features of the b-th
    basis member.
    """
    X = np.asarray(X, dtype=np.float64)
    n, F = X.shape
    Bd = basis_multiplier(basis) * degree
    P = np.empty((n, 1 + F * Bd), dtype=np.float64)
    P[:, 0] = 1.0
    for f in range(F):
        for b in range(Bd):
            P[:, 1 + f * Bd + b] = basis_value(basis, degree, b, X[:, f])
    if shared:
        return np.concatenate([P[:, :1], P[:, 1:].reshape(n, F, Bd).sum(axis=1)], axis=1)
    return P


def outputs(P: np.ndarray, G: np.ndarray) -> np.ndarray:
    """Out(pat_k) for every chromosome and pattern (eq.2): S[c, k] = sum_g G[c,g] P[k,g].

    A plain float64 matrix product (library primitive) over the expansion.
    """
    return np.asarray(G, dtype=np.float64) @ np.asarray(P, dtype=np.float64).T


def outputs_eq2(X: np.ndarray, G: np.ndarray, basis: str, degree: int) -> np.ndarray:
    """Out(pat_k) straight from eq.2 without forming P: a0 + sum_i sum_j a_ij g^j(f_i).

    The double loop over features and degrees of eq.2 / eq.9, accumulated in
    float64; used to check ``expand`` + ``outputs`` on small cases.
    """
    X = np.asarray(X, dtype=np.float64)
    G = np.asarray(G, dtype=np.float64)
    F = X.shape[1]
    Bd = basis_multiplier(basis) * degree
    S = np.repeat(G[:, :1], X.shape[0], axis=1)
    for i in range(F):
        for b in range(Bd):
            S += np.outer(G[:, 1 + i * Bd + b], basis_value(basis, degree, b, X[:, i]))
    return S


def activate(S: np.ndarray, activation: str) -> np.ndarray:
    """Output activation: tanh (targets +-1) or the paper's linear Out (eq.2)."""
    return np.tanh(S) if activation == "tanh" else np.asarray(S, dtype=np.float64)


def pattern_errors(t: np.ndarray, Y: np.ndarray, error: str, R: float) -> np.ndarray:
    """E_k per chromosome and pattern.

    Squared error of eq.3 for MSE / RMSE; the threshold form of eq.10 for TMSE:
    ``"tmse"`` zeroes E_k when |t_k - Out| <= R (the reading that reproduces the
    paper's worked example), ``"tmse_sq"`` when (t_k - Out)^2 <= R (eq.10 as
    printed).
    """
    d = np.asarray(t, dtype=np.float64)[None, :] - Y
    E = d * d
    if error == "tmse":
        E = np.where(np.abs(d) > R, E, 0.0)
    elif error == "tmse_sq":
        E = np.where(E > R, E, 0.0)
    return E


def reduce_errors(E: np.ndarray, error: str) -> np.ndarray:
    """Per-chromosome fitness: MSE (eq.4), RMSE (eq.5) or TMSE (eq.10 averaged over NP)."""
    mse = E.mean(axis=1)
    return np.sqrt(mse) if error == "rmse" else mse


def fitness(P: np.ndarray, t: np.ndarray, G: np.ndarray, cfg: Config) -> np.ndarray:
    """Fitness of every chromosome over the patterns of P (eq.2 -> eq.3 -> eq.4/5/10)."""
    S = outputs(P, G)
    return reduce_errors(pattern_errors(t, activate(S, cfg.activation), cfg.error, cfg.tmse_R),
                         cfg.error)


def rank(fit: np.ndarray) -> np.ndarray:
    """Chromosome indices sorted by ascending (fitness, index); NaN counts as +inf.

    Section 4.1 step 2: "find and sort the best chromosomes".
    """
    f = np.where(np.isnan(fit), np.inf, np.asarray(fit, dtype=np.float64))
    return np.argsort(f, kind="stable")


# ---------------------------------------------------------------------------
# Philox4x64-10 (Salmon et al., SC'11), counter = (generation, pair, stream, block)
# ---------------------------------------------------------------------------

_U64 = np.uint64
_M32 = _U64(0xFFFFFFFF)
_PHILOX_M0 = 0xD2E7470EE14C6C93
_PHILOX_M1 = 0xCA5A826395121157
_PHILOX_W0 = 0x9E3779B97F4A7C15   # golden ratio
_PHILOX_W1 = 0xBB67AE8584CAA73B   # sqrt(3) - 1

STREAM_TOURNAMENT, STREAM_CROSSOVER, STREAM_MUT_MASK, STREAM_MUT_NORMAL = 0, 1, 2, 3
STREAM_INIT, STREAM_INIT_NORMAL = 4, 5
STREAM_IMMIGRANT, STREAM_IMMIGRANT_NORMAL = 8, 9   # (6, 7 belong to the surrogate)


def _mulhilo64(a: int, b: np.ndarray):
    """High and low 64-bit halves of the 128-bit product a*b (schoolbook on 32-bit limbs)."""
    a_lo, a_hi = _U64(a & 0xFFFFFFFF), _U64(a >> 32)
    b_lo, b_hi = b & _M32, b >> _U64(32)
    ll, lh, hl, hh = a_lo * b_lo, a_lo * b_hi, a_hi * b_lo, a_hi * b_hi
    mid = (ll >> _U64(32)) + (lh & _M32) + (hl & _M32)
    lo = (ll & _M32) | ((mid & _M32) << _U64(32))
    hi = hh + (lh >> _U64(32)) + (hl >> _U64(32)) + (mid >> _U64(32))
    return hi, lo


def philox4x64(ctr, key) -> np.ndarray:
    """Ten Philox4x64 rounds; ``ctr`` is four uint64 arrays (broadcastable), ``key`` two ints.

    Returns an array [..., 4] of uint64.
    """
    with np.errstate(over="ignore"):
        x = [np.asarray(c, dtype=np.uint64) for c in ctr]
        x = list(np.broadcast_arrays(*x))
        k0, k1 = int(key[0]) & 0xFFFFFFFFFFFFFFFF, int(key[1]) & 0xFFFFFFFFFFFFFFFF
        for r in range(10):
            if r:
                k0 = (k0 + _PHILOX_W0) & 0xFFFFFFFFFFFFFFFF
                k1 = (k1 + _PHILOX_W1) & 0xFFFFFFFFFFFFFFFF
            hi0, lo0 = _mulhilo64(_PHILOX_M0, x[0])
            hi1, lo1 = _mulhilo64(_PHILOX_M1, x[2])
            x = [hi1 ^ x[1] ^ _U64(k0), lo1, hi0 ^ x[3] ^ _U64(k1), lo0]
        return np.stack(x, axis=-1)


def philox_words(key, gen, pair, stream, word) -> np.ndarray:
    """32-bit word ``word`` of the Philox stream (gen, pair, stream): uint64 array holding u32.

    Block b = word // 8 is the fourth counter word; inside a block word w = word % 8
    is the low (w even) or high (w odd) half of output lane w // 2.
    """
    word = np.asarray(word, dtype=np.uint64)
    gen, pair, stream = (np.asarray(v, dtype=np.uint64) for v in (gen, pair, stream))
    out = philox4x64((gen, pair, stream, word >> _U64(3)), key)       # [..., 4]
    word = np.broadcast_to(word, out.shape[:-1])
    lane = ((word & _U64(7)) >> _U64(1)).astype(np.int64)
    v = np.take_along_axis(out, lane[..., None], axis=-1)[..., 0]
    odd = (word & _U64(1)).astype(bool)
    return np.where(odd, v >> _U64(32), v & _M32)


def uniform24(w: np.ndarray) -> np.ndarray:
    """u = (w >> 8) * 2^-24 in float32 (exact; in [0, 1))."""
    return ((np.asarray(w, dtype=np.uint64) >> _U64(8)).astype(np.float32)
            * np.float32(2.0 ** -24))


def index_draw(w: np.ndarray, n: int) -> np.ndarray:
    """Uniform integer in [0, n) from a 32-bit word: (w * n) >> 32."""
    return ((np.asarray(w, dtype=np.uint64) * _U64(n)) >> _U64(32)).astype(np.int64)


# --- float32 logarithm and cosine used by Box-Muller (correctly rounded ops only) ---

_F = np.float32
_LN2 = _F(float.fromhex("0x1.62e430p-1"))
_SQRT_HALF = _F(float.fromhex("0x1.6a09e6p-1"))
_HALF_PI = _F(float.fromhex("0x1.921fb6p+0"))
# 1/(2n+1), n = 5..1: coefficients of atanh(s)/s = 1 + s^2/3 + s^4/5 + ...
_ATANH = [_F(float.fromhex(h)) for h in
          ("0x1.745d18p-4", "0x1.c71c72p-4", "0x1.24924ap-3", "0x1.99999ap-3", "0x1.555556p-2")]
# (-1)^n/(2n)!, n = 8..1: Taylor series of cos
_COS = [_F(float.fromhex(h)) for h in
        ("0x1.ae7f3ep-45", "-0x1.93974ap-37", "0x1.1eed8ep-29", "-0x1.27e4fcp-22",
         "0x1.a01a02p-16", "-0x1.6c16c2p-10", "0x1.555556p-5", "-0x1.000000p-1")]
# (-1)^n/(2n+1)!, n = 7..1: Taylor series of sin(a)/a
_SIN = [_F(float.fromhex(h)) for h in
        ("-0x1.ae7f3ep-41", "0x1.612462p-33", "-0x1.ae6456p-26", "0x1.71de3ap-19",
         "-0x1.a01a02p-13", "0x1.111112p-7", "-0x1.555556p-3")]


def ln_f32(u: np.ndarray) -> np.ndarray:
    """Natural log of positive normal float32 values.

    u = m * 2^e with m in [sqrt(1/2), sqrt(2)); ln m = 2 atanh(s), s = (m-1)/(m+1),
    summed as 2 s (1 + s^2/3 + ... + s^10/11) (|s| <= 0.1716, truncation < 1e-10).
    """
    u = np.asarray(u, dtype=np.float32)
    m, e = np.frexp(u)                       # m in [0.5, 1), exact
    m = m.astype(np.float32)
    low = m < _SQRT_HALF
    m = np.where(low, m * _F(2.0), m)
    e = np.where(low, e - 1, e)
    f = m - _F(1.0)                          # exact (Sterbenz)
    s = f / (f + _F(2.0))
    z = s * s
    p = _ATANH[0]
    for c in _ATANH[1:]:
        p = p * z
        p = p + c
    p = p * z
    p = p + _F(1.0)
    a = s * p
    a = a + a
    return e.astype(np.float32) * _LN2 + a


def cos2pi_f32(v: np.ndarray) -> np.ndarray:
    """cos(2 pi v) for float32 v in [0, 1): quadrant split, then Taylor series on [0, pi/2)."""
    v = np.asarray(v, dtype=np.float32)
    v4 = v * _F(4.0)                         # exact
    q = np.floor(v4)
    a = (v4 - q) * _HALF_PI
    a2 = a * a
    c = _COS[0]
    for k in _COS[1:]:
        c = c * a2
        c = c + k
    c = c * a2
    c = c + _F(1.0)
    s = _SIN[0]
    for k in _SIN[1:]:
        s = s * a2
        s = s + k
    s = s * a2
    s = s + _F(1.0)
    s = a * s
    qi = q.astype(np.int64)
    return np.select([qi == 0, qi == 1, qi == 2], [c, -s, -c], s).astype(np.float32)


def gauss_f32(w0: np.ndarray, w1: np.ndarray) -> np.ndarray:
    """Standard normal from two 32-bit words by Box-Muller: sqrt(-2 ln u1) cos(2 pi u2).

    u1 = ((w0 >> 8) + 1) 2^-24 in (0, 1], u2 = (w1 >> 8) 2^-24 in [0, 1).
    """
    u1 = (((np.asarray(w0, dtype=np.uint64) >> _U64(8)) + _U64(1)).astype(np.float32)
          * _F(2.0 ** -24))
    u2 = uniform24(w1)
    r = np.sqrt(ln_f32(u1) * _F(-2.0))
    return (r * cos2pi_f32(u2)).astype(np.float32)


# ---------------------------------------------------------------------------
# Population initialisation (Section 2: three random generation criteria)
# ---------------------------------------------------------------------------

def draw_chromosomes(key, gen: int, rows: np.ndarray, K: int, init: str, stream_u: int,
                     stream_n: int) -> np.ndarray:
    """Random chromosomes [len(rows) x K] float32 of the init distribution, row r drawn
    with the Philox counter (gen, r, stream, word): U[-1,1], N(0,0.5^2) truncated to
    [-1,1] by resampling (64 rounds, then clamp), or U[0,1]."""
    c = np.asarray(rows, dtype=np.uint64)[:, None]
    g = np.arange(K, dtype=np.uint64)[None, :]
    if init == "normal_pm1":
        out = np.zeros((c.shape[0], K), dtype=np.float32)
        done = np.zeros((c.shape[0], K), dtype=bool)
        for r in range(64):
            w = _U64(2) * (_U64(r) * _U64(K) + g)
            z = gauss_f32(philox_words(key, gen, c, stream_n, w),
                          philox_words(key, gen, c, stream_n, w + _U64(1)))
            v = z * _F(0.5)
            ok = (~done) & (np.abs(v) <= _F(1.0))
            out = np.where(ok, v, out)
            if r == 63:
                out = np.where(done | ok, out, np.clip(v, _F(-1.0), _F(1.0)))
            done |= ok
        return out
    u = uniform24(philox_words(key, gen, c, stream_u, g))
    if init == "uniform_01":
        return u
    return (u * _F(2.0) - _F(1.0)).astype(np.float32)


def init_population(cfg: Config, K: int) -> np.ndarray:
    """Generation-0 genes [pop x K] float32 (Section 2: the first population is random)."""
    return draw_chromosomes((cfg.seed, cfg.run), 0, np.arange(cfg.pop), K, cfg.init,
                            STREAM_INIT, STREAM_INIT_NORMAL)


# ---------------------------------------------------------------------------
# Genetic operators (Section 2 options; Section 5 experiment parameters)
# ---------------------------------------------------------------------------

def tournament(key, gen: int, pairs: np.ndarray, first_word: int, k: int,
               fit: np.ndarray) -> np.ndarray:
    """Tournament of k draws with replacement; winner = smallest (fitness, index)."""
    pop = fit.shape[0]
    f = np.where(np.isnan(fit), np.inf, fit)
    best = None
    for i in range(k):
        idx = index_draw(philox_words(key, gen, pairs, STREAM_TOURNAMENT, first_word + i), pop)
        if best is None:
            best = idx
        else:
            better = (f[idx] < f[best]) | ((f[idx] == f[best]) & (idx < best))
            best = np.where(better, idx, best)
    return best


ROULETTE_EPS = 1e-12


def selection_weights(fit: np.ndarray, cfg: Config) -> np.ndarray:
    """Integer selection weights (Section 2: ranking and roulette selection).

    roulette: w_c = 1 / (1e-12 + f_c) in float64, quantised q_c = floor(2^24 w_c / max w)
    (fitness-proportionate selection for an error to minimise; NaN weighs 0);
    ranking: linear ranking with expected values from 1.1 (best) to 0.9 (worst),
    q = 9 (N - 1) + 2 (N - 1 - r) for rank position r.
    Integers make the cumulative sums exact in any order of addition."""
    fit = np.asarray(fit, dtype=np.float64)
    pop = fit.shape[0]
    if cfg.selection == "ranking":
        q = np.empty(pop, dtype=np.uint64)
        q[rank(fit)] = (_U64(9 * (pop - 1)) +
                        _U64(2) * (_U64(pop - 1) - np.arange(pop, dtype=np.uint64)))
        return q
    w = np.where(np.isnan(fit), 0.0, 1.0 / (ROULETTE_EPS + np.where(np.isnan(fit), 0.0, fit)))
    wmax = w.max() if pop else 0.0
    if not wmax > 0:
        return np.zeros(pop, dtype=np.uint64)
    return np.floor(w / wmax * float(1 << 24)).astype(np.uint64)


def wheel_draw(cum: np.ndarray, words: np.ndarray) -> np.ndarray:
    """Parent of each 32-bit word: t = (u24 Q) >> 24 with u24 the top 24 bits and Q
    the total weight; the first index whose inclusive cumulative weight exceeds t.
    A zero total falls back to a uniform index draw."""
    pop = cum.shape[0]
    total = cum[-1]
    if total == 0:
        return index_draw(words, pop)
    t = ((np.asarray(words, dtype=np.uint64) >> _U64(8)) * total) >> _U64(24)
    return np.searchsorted(cum, t, side="right").astype(np.int64)


def breed(G: np.ndarray, fit: np.ndarray, cfg: Config, gen: int) -> np.ndarray:
    """One application of the genetic operators: population ``gen`` -> ``gen + 1``.

    * elitism: children 0..e-1 are the top-e chromosomes by (fitness, index), or
      e copies of the winner;
    * remaining children come in pairs j = 0, 1, ...: two tournaments pick the
      parents, single-point crossover with probability p_c swaps the tails after
      a cut in [1, K-1], then every gene of both children mutates with
      probability p_m by sigma * N(0,1) and is clamped to [-1, 1];
    * an odd number of non-elite slots drops the last pair's second child.

    ``fit`` is the float64 fitness vector the selection compares.
    """
    G = np.asarray(G, dtype=np.float32)
    fit = np.asarray(fit, dtype=np.float64)
    pop, K = G.shape
    key = (cfg.seed, cfg.run)
    order = rank(fit)
    e = min(cfg.elitism, pop)
    out = np.empty_like(G)
    if e:
        out[:e] = G[order[:e]] if cfg.elite_mode == "top" else G[order[0]][None, :]
    n_child = pop - e
    n_pairs = (n_child + 1) // 2
    if n_pairs == 0:
        return immigrate(out, cfg, gen)
    j = np.arange(n_pairs, dtype=np.uint64)
    if cfg.selection == "tournament":
        p1 = tournament(key, gen, j, 0, cfg.tournament_k, fit)
        p2 = tournament(key, gen, j, cfg.tournament_k, cfg.tournament_k, fit)
    else:
        cum = np.cumsum(selection_weights(fit, cfg), dtype=np.uint64)
        p1 = wheel_draw(cum, philox_words(key, gen, j, STREAM_TOURNAMENT, 0))
        p2 = wheel_draw(cum, philox_words(key, gen, j, STREAM_TOURNAMENT, 1))
    u_c = uniform24(philox_words(key, gen, j, STREAM_CROSSOVER, 0))
    cut = 1 + index_draw(philox_words(key, gen, j, STREAM_CROSSOVER, 1), max(K - 1, 1))
    do_x = (u_c < _F(cfg.p_crossover)) & (K >= 2)
    cut = np.where(do_x, cut, K)                      # no crossover == cut after last gene
    gidx = np.arange(K)[None, :]
    head = gidx < cut[:, None]
    ca = np.where(head, G[p1], G[p2])
    cb = np.where(head, G[p2], G[p1])
    pm, sg = _F(cfg.p_mutation), _F(cfg.sigma_mutation)
    for s, child in ((0, ca), (1, cb)):
        w = _U64(s) * _U64(K) + np.arange(K, dtype=np.uint64)[None, :]
        mask = uniform24(philox_words(key, gen, j[:, None], STREAM_MUT_MASK, w)) < pm
        z = gauss_f32(philox_words(key, gen, j[:, None], STREAM_MUT_NORMAL, _U64(2) * w),
                      philox_words(key, gen, j[:, None], STREAM_MUT_NORMAL, _U64(2) * w + _U64(1)))
        mutated = child + sg * z
        if cfg.clamp_genes:
            mutated = np.minimum(np.maximum(mutated, _F(-1.0)), _F(1.0))
        child[...] = np.where(mask, mutated, child)
    slots = np.empty((2 * n_pairs, K), dtype=np.float32)
    slots[0::2], slots[1::2] = ca, cb
    out[e:] = slots[:n_child]
    return immigrate(out, cfg, gen)


def immigrate(G: np.ndarray, cfg: Config, gen: int) -> np.ndarray:
    """Random immigrants (Section 4.1: a number of chromosomes are generated at random
    to replace older individuals): the last cfg.immigrants rows of the population bred
    at step gen are replaced by chromosomes of the init distribution, drawn with the
    counter of the new generation gen + 1 on streams of their own."""
    n = min(cfg.immigrants, G.shape[0])
    if n <= 0:
        return G
    pop, K = G.shape
    rows = np.arange(pop - n, pop)
    G = G.copy()
    G[rows] = draw_chromosomes((cfg.seed, cfg.run), gen + 1, rows, K, cfg.init,
                               STREAM_IMMIGRANT, STREAM_IMMIGRANT_NORMAL)
    return G


# ---------------------------------------------------------------------------
# Training loop and report (Section 4.1 steps 1-4; Section 5 figures of merit)
# ---------------------------------------------------------------------------

@dataclass
class RunResult:
    best_genes: np.ndarray
    best_fitness: float
    generations: int
    history: list = field(default_factory=list)   # best fitness per evaluated generation
    population: np.ndarray | None = None
    fitness: np.ndarray | None = None


def evolve(P_train: np.ndarray, t_train: np.ndarray, cfg: Config, max_generations: int,
           G0: np.ndarray | None = None, fitness_fn=None) -> RunResult:
    """GA training (Section 4.1): init, then per generation fitness + sort, stop test, operators.

    Generation 0 is the initial population; every later generation is bred from
    the previous one.  The loop stops after ``max_generations`` evaluated
    populations or as soon as the best fitness is <= ``cfg.stop_error``.
    ``fitness_fn(G) -> fit`` may replace the float64 fitness (trajectory tests
    feed the GPU's fitness vectors through it).
    """
    K = P_train.shape[1]
    G = init_population(cfg, K) if G0 is None else np.asarray(G0, dtype=np.float32)
    fitfn = fitness_fn or (lambda g: fitness(P_train, t_train, g, cfg))
    hist = []
    gen = 0
    fit = None
    for i in range(max_generations):
        if fit is not None:
            G = breed(G, fit, cfg, gen)
            gen += 1
        fit = fitfn(G)
        best = rank(fit)[0]
        hist.append(float(fit[best]))
        if fit[best] <= cfg.stop_error:
            break
    best = rank(fit)[0]
    return RunResult(best_genes=G[best].copy(), best_fitness=float(fit[best]),
                     generations=len(hist), history=hist, population=G, fitness=fit)


def classify(y: np.ndarray, activation: str) -> np.ndarray:
    """Class decision: sign with sign(0) = +1 for tanh (+-1 targets); y >= 0.5 -> 1 for linear 0/1."""
    if activation == "tanh":
        return np.where(y >= 0.0, 1.0, -1.0)
    return np.where(y >= 0.5, 1.0, 0.0)


def report(P: np.ndarray, t: np.ndarray, genes: np.ndarray, cfg: Config) -> dict:
    """Figures of merit of one chromosome on a pattern set (Section 5).

    rmse: eq.5 in float64.  accuracy: fraction classified correctly.
    completeness: fraction of the positive class (GC) classified as positive.
    contamination: fraction of the patterns classified positive that are
    negative (FP / (TP + FP)).
    """
    y = activate(outputs(P, np.asarray(genes, dtype=np.float64)[None, :])[0], cfg.activation)
    t = np.asarray(t, dtype=np.float64)
    pos = 1.0
    cls = classify(y, cfg.activation)
    tp = np.sum((cls == pos) & (t == pos))
    fp = np.sum((cls == pos) & (t != pos))
    fn = np.sum((cls != pos) & (t == pos))
    return {
        "rmse": float(np.sqrt(np.mean((t - y) ** 2))) if len(t) else 0.0,
        "accuracy": float(np.mean(cls == t)) if len(t) else 0.0,
        "completeness": float(tp / (tp + fn)) if tp + fn else 0.0,
        "contamination": float(fp / (tp + fp)) if tp + fp else 0.0,
    }


# ---------------------------------------------------------------------------
# Low-precision storage of P (precision form): per-column scale, then rounding
# to the storage format.  The paper computes in double; these functions state
# what a reduced-precision copy of P holds, so that a fitness computed from it
# can be compared with the exact one.
# ---------------------------------------------------------------------------

def round_bf16(x: np.ndarray) -> np.ndarray:
    """Round float32 values to bfloat16 (round to nearest, ties to even); returned as float32."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + np.uint64(0x7FFF) + ((b >> np.uint64(16)) & np.uint64(1))) & np.uint64(0xFFFF0000)
    return b.astype(np.uint32).view(np.float32)


def round_e4m3(x: np.ndarray) -> np.ndarray:
    """Round float32 values to FP8 E4M3 (OCP: 3 mantissa bits, exponent bias 7, largest
    finite 448, subnormal step 2^-9), ties to even, saturating to +-448; returned as float32."""
    x = np.asarray(x, dtype=np.float64)
    a = np.abs(x)
    _, e = np.frexp(a)                     # a = m 2^e, m in [0.5, 1)
    expo = np.maximum(e - 1, -6)           # unbiased exponent, clamped to the subnormal range
    step = np.ldexp(1.0, expo - 3)
    q = np.round(a / step) * step          # numpy rounds halves to even
    q = np.minimum(q, 448.0)
    return (np.sign(x) * q).astype(np.float32)


QMAX = {"bf16": 1.0, "fp8": 448.0}


def quantize_columns(P: np.ndarray, fmt: str, s: np.ndarray | None = None):
    """P held in a low-precision format with a per-column scale: P ~ Q * s.

    P is first rounded to float32 (the working precision of the expansion);
    s_g = max_k |P[k,g]| / qmax (1 where the column is zero); Q = round(P / s)
    in the format.  Returns (Q, s) as float32 arrays.  A caller that walks a
    large P in row blocks passes the scales of the whole matrix as ``s`` (for
    instance those this function returns for the stacked per-block column
    maxima of |P|).
    """
    P32 = np.asarray(P, dtype=np.float32)
    if s is None:
        m = np.max(np.abs(P32), axis=0) if P32.shape[0] else np.zeros(P32.shape[1], np.float32)
        s = np.where(m > 0, m / np.float32(QMAX[fmt]), np.float32(1.0)).astype(np.float32)
    s = np.asarray(s, dtype=np.float32)
    R = (P32 / s[None, :]).astype(np.float32)
    Q = round_bf16(R) if fmt == "bf16" else round_e4m3(R)
    return Q, s


def dequantize_columns(Q: np.ndarray, s: np.ndarray) -> np.ndarray:
    return np.asarray(Q, dtype=np.float64) * np.asarray(s, dtype=np.float64)[None, :]


def quantize_genes(G: np.ndarray, s: np.ndarray, fmt: str, planes: int) -> np.ndarray:
    """Genes as a low-precision contraction meets them.

    With P stored as Q * s (``quantize_columns``), gene g of chromosome c meets Q
    through g' = g s_g (float32 product); per chromosome r_c = max_g |g'| / qmax;
    the operand holds one term hi = q(g'/r_c) or two, hi + q(g'/r_c - hi), in the
    format.  Returns the genes the contraction effectively multiplies with the
    dequantised P: (hi [+ lo]) r_c / s_g, with the bias (gene 0) unchanged.
    """
    G = np.asarray(G, dtype=np.float32)
    s = np.asarray(s, dtype=np.float32)
    q = round_bf16 if fmt == "bf16" else round_e4m3
    gp = (G[:, 1:] * s[None, :]).astype(np.float32)
    m = np.max(np.abs(gp), axis=1)
    r = np.where(m > 0, m / np.float32(QMAX[fmt]), np.float32(1.0)).astype(np.float32)
    w = (gp / r[:, None]).astype(np.float32)
    hi = q(w)
    val = hi.astype(np.float64)
    if planes == 2:
        val = val + q((w - hi).astype(np.float32)).astype(np.float64)
    out = np.empty(G.shape, dtype=np.float64)
    out[:, 0] = G[:, 0]
    out[:, 1:] = val * r.astype(np.float64)[:, None] / s.astype(np.float64)[None, :]
    return out


# ---------------------------------------------------------------------------
# Learned surrogate of the fitness (no paper counterpart): a small MLP that
# maps a chromosome's genes to its standardised log fitness.  Float64 forward,
# backward (chain rule written out) and the Adam update of Kingma & Ba (2015).
# ---------------------------------------------------------------------------

def gelu(z: np.ndarray) -> np.ndarray:
    """GELU, erf form: z * Phi(z) = z/2 (1 + erf(z / sqrt 2))."""
    from scipy.special import erf
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z: np.ndarray) -> np.ndarray:
    """d/dz of z Phi(z) = Phi(z) + z phi(z)."""
    from scipy.special import erf
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def bf16_operands(a: np.ndarray) -> np.ndarray:
    """A GEMM operand as the tensor cores see it in the bfloat16 form: the float32
    value rounded to bfloat16."""
    return round_bf16(np.asarray(a, dtype=np.float32)).astype(np.float64)


def mlp_forward(params: dict, X: np.ndarray, operand_round=None) -> dict:
    """y = w3 . gelu(W2 gelu(W1 x + b1) + b2) + b3 for every row x of X; keeps the
    intermediate values the backward pass needs.

    operand_round, if given, is applied to the activations where they enter a
    matrix product (x and gelu(Z1)): the bfloat16 form rounds its GEMM operands
    and accumulates in float32; None is the exact network."""
    r = operand_round if operand_round is not None else (lambda a: a)
    X = r(np.asarray(X, dtype=np.float64))
    Z1 = X @ params["W1"].T + params["b1"]
    H1 = r(gelu(Z1))
    Z2 = H1 @ params["W2"].T + params["b2"]
    H2 = gelu(Z2)
    y = H2 @ params["w3"] + params["b3"]
    return {"X": X, "Z1": Z1, "H1": H1, "Z2": Z2, "H2": H2, "y": y}


def mlp_loss_grad(params: dict, X: np.ndarray, target: np.ndarray, operand_round=None):
    """Mean squared error L = mean((y - target)^2) and its gradient for every parameter
    (backpropagation).  operand_round as in mlp_forward; it also applies to the
    back-propagated dZ2 and dZ1 where they enter a matrix product."""
    r = operand_round if operand_round is not None else (lambda a: a)
    f = mlp_forward(params, X, operand_round)
    B = X.shape[0]
    dy = 2.0 * (f["y"] - np.asarray(target, dtype=np.float64)) / B
    g = {"w3": f["H2"].T @ dy, "b3": np.array(dy.sum())}
    dZ2 = r(np.outer(dy, params["w3"]) * gelu_grad(f["Z2"]))
    g["W2"] = dZ2.T @ f["H1"]
    g["b2"] = dZ2.sum(axis=0)
    dZ1 = r((dZ2 @ params["W2"]) * gelu_grad(f["Z1"]))
    g["W1"] = dZ1.T @ f["X"]
    g["b1"] = dZ1.sum(axis=0)
    loss = float(np.mean((f["y"] - target) ** 2))
    return loss, g


def adam_update(param: np.ndarray, grad: np.ndarray, m: np.ndarray, v: np.ndarray, step: int,
                lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    """One Adam step (Kingma & Ba 2015, Algorithm 1), step counted from 1."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mh = m / (1 - beta1 ** step)
    vh = v / (1 - beta2 ** step)
    return param - lr * mh / (np.sqrt(vh) + eps), m, v


def surrogate_select(scores: np.ndarray, n_sel: int) -> np.ndarray:
    """Pool rows kept by the learned-surrogate form (no paper counterpart): the n_sel
    rows of lowest predicted fitness, ties at the cut going to lower pool indices
    (NaN counts as +inf).  Listed as the kept rows strictly below the cut value in
    pool order, then the kept rows equal to it in pool order."""
    s = np.where(np.isnan(scores), np.inf, np.asarray(scores, dtype=np.float64))
    idx = np.arange(len(s))
    order = np.lexsort((idx, s))            # by value, then by index
    kept = order[:n_sel]
    cut = s[order[n_sel - 1]]
    return np.concatenate([np.sort(kept[s[kept] < cut]), np.sort(kept[s[kept] == cut])])


def spearman(a: np.ndarray, b: np.ndarray) -> float:
    """Spearman rank correlation (no ties expected): 1 - 6 sum d^2 / (n (n^2 - 1))."""
    n = len(a)
    ra = np.empty(n)
    rb = np.empty(n)
    ra[np.argsort(a, kind="stable")] = np.arange(n)
    rb[np.argsort(b, kind="stable")] = np.arange(n)
    return float(1.0 - 6.0 * np.sum((ra - rb) ** 2) / (n * (n * n - 1.0)))
