"""Seeded synthetic inputs shaped like the paper's globular-cluster knowledge base.

The paper's data (Section 3) are ~2,100 patterns of 11 continuous photometric and
morphological features with a binary GC / not-GC label.  That catalogue is not
available, so every workload here is synthetic and seeded:

* features: uniform in [-1, 1], or Gaussian with a seeded random correlation
  matrix, scaled by 0.5 and clipped to [-1, 1];
* labels: +-1 from the sign of a seeded hidden polynomial in the same basis
  (median-centred for class balance), then 5% of the labels flipped;
* a seeded 70/30 train/test split, returned with the training rows first.

This module only produces inputs.  It holds none of the method's arithmetic:
the hidden labelling function is evaluated with numpy's own Chebyshev routine
(``numpy.polynomial.chebyshev.chebval``) or with ``np.cos`` / ``np.sin``, and
both the CUDA path and the oracle receive the arrays it returns.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np
from numpy.polynomial import chebyshev as _cheb

DATA_SEED = 1304


@dataclass
class Dataset:
    X: np.ndarray          # [NP, F] float32, training rows first
    t: np.ndarray          # [NP] float32 targets (+-1)
    n_train: int
    basis: str
    degree: int

    @property
    def n_patterns(self) -> int:
        return self.X.shape[0]

    @property
    def n_features(self) -> int:
        return self.X.shape[1]


def _features(rng: np.random.Generator, n: int, F: int, correlated: bool) -> np.ndarray:
    if not correlated:
        return rng.uniform(-1.0, 1.0, size=(n, F)).astype(np.float32)
    A = rng.standard_normal((F, F))
    S0 = A @ A.T
    d = np.sqrt(np.diag(S0))
    L = np.linalg.cholesky(S0 / np.outer(d, d))
    out = np.empty((n, F), dtype=np.float32)
    step = 1 << 18
    for i in range(0, n, step):
        m = min(step, n - i)
        z = rng.standard_normal((m, F))
        out[i:i + m] = np.clip(0.5 * (z @ L.T), -1.0, 1.0)
    return out


def _hidden(rng: np.random.Generator, X: np.ndarray, basis: str, degree: int) -> np.ndarray:
    """Value of a seeded random function of the features (coefficients uniform in [-1, 1])."""
    n, F = X.shape
    v = np.full(n, rng.uniform(-1.0, 1.0), dtype=np.float64)
    for f in range(F):
        x = X[:, f].astype(np.float64)
        if basis == "chebyshev":
            c = np.concatenate([[0.0], rng.uniform(-1.0, 1.0, size=degree)])
            v += _cheb.chebval(x, c)
        else:
            a = rng.uniform(-1.0, 1.0, size=degree)
            b = rng.uniform(-1.0, 1.0, size=degree)
            # cos(kx), sin(kx) by angle addition from cos x, sin x (float64; the
            # values agree with np.cos(k x) / np.sin(k x) to ~1e-15)
            c1, s1 = np.cos(x), np.sin(x)
            ck, sk = c1, s1
            for k in range(1, degree + 1):
                if k > 1:
                    ck, sk = ck * c1 - sk * s1, sk * c1 + ck * s1
                v += a[k - 1] * ck + b[k - 1] * sk
    return v


def make_dataset(n_patterns: int, n_features: int, degree: int, basis: str = "chebyshev",
                 seed: int = DATA_SEED, correlated: bool = False, flip: float = 0.05,
                 train_frac: float = 0.7) -> Dataset:
    rng = np.random.default_rng(seed)
    X = _features(rng, n_patterns, n_features, correlated)
    v = _hidden(rng, X, basis, degree)
    t = np.where(v - np.median(v) >= 0.0, 1.0, -1.0)
    t = np.where(rng.random(n_patterns) < flip, -t, t).astype(np.float32)
    perm = rng.permutation(n_patterns)
    n_train = int(round(train_frac * n_patterns))
    return Dataset(X=np.ascontiguousarray(X[perm]), t=np.ascontiguousarray(t[perm]),
                   n_train=n_train, basis=basis, degree=degree)


def planted_targets(X: np.ndarray, h: np.ndarray, basis: str, degree: int) -> np.ndarray:
    """Regression targets tanh(f_h(x)) of a planted chromosome h, float64.

    f_h is the function whose coefficients h holds in the gene layout (h[0] the
    constant; h[1 + f*B*d + b] the b-th basis member of feature f: Chebyshev T_{b+1},
    or for the trig basis cos((b+1)x) for b < d and sin((b-d+1)x) after), evaluated
    feature by feature with numpy's Chebyshev series routine or with np.cos / np.sin,
    never through an expansion matrix.
    """
    X = np.asarray(X, dtype=np.float64)
    h = np.asarray(h, dtype=np.float64)
    n, F = X.shape
    Bd = (2 if basis == "trig" else 1) * degree
    assert h.shape == (1 + F * Bd,)
    v = np.full(n, h[0])
    for f in range(F):
        c = h[1 + f * Bd: 1 + (f + 1) * Bd]
        if basis == "chebyshev":
            v += _cheb.chebval(X[:, f], np.concatenate([[0.0], c]))
        else:
            for k in range(1, degree + 1):
                v += c[k - 1] * np.cos(k * X[:, f]) + c[degree + k - 1] * np.sin(k * X[:, f])
    return np.tanh(v)


# --- the workloads -------------------------------------------------------------------

def paper_kb(replicas: int = 1, seed: int = DATA_SEED) -> Dataset:
    """Stand-in for the paper's knowledge base (Section 3 / Section 5: 2,100 patterns,
    11 input features, 0/1 class target), replicated `replicas` times the way the
    paper grows it to 16 / 128 / 512 MB.  Features uniform in [-1, 1]; labels from a
    seeded hidden degree-4 polytrigo function with 5% flips, mapped to 0/1.  The
    first 70% of the base rows train; every replica keeps that split (train rows of
    all replicas first)."""
    base = make_dataset(2100, 11, 4, "trig", seed=seed)
    t01 = ((base.t + 1.0) / 2.0).astype(np.float32)
    n_tr = base.n_train
    X = np.concatenate([np.tile(base.X[:n_tr], (replicas, 1)),
                        np.tile(base.X[n_tr:], (replicas, 1))])
    t = np.concatenate([np.tile(t01[:n_tr], replicas), np.tile(t01[n_tr:], replicas)])
    return Dataset(X=np.ascontiguousarray(X), t=np.ascontiguousarray(t),
                   n_train=n_tr * replicas, basis="trig", degree=4)


def plain_small(seed: int = DATA_SEED) -> Dataset:
    """2,000 patterns x 7 uniform features, Chebyshev degree 4 (29 genes)."""
    return make_dataset(2000, 7, 4, "chebyshev", seed=seed)


def plain_at_scale(seed: int = DATA_SEED, n_patterns: int = 1_000_000) -> Dataset:
    """1,000,000 patterns x 32 correlated features, Chebyshev degree 8 (257 genes)."""
    return make_dataset(n_patterns, 32, 8, "chebyshev", seed=seed, correlated=True)


def surrogate_scale(seed: int = DATA_SEED, n_patterns: int = 2_000_000) -> Dataset:
    """2,000,000 patterns x 48 correlated features, Chebyshev degree 6 (289 genes)."""
    return make_dataset(n_patterns, 48, 6, "chebyshev", seed=seed, correlated=True)


@dataclass
class RunSpec:
    n_patterns: int
    n_features: int
    degree: int
    pop: int
    basis: str
    precision: str         # "fp32" | "bf16"
    seed: int


def batched_specs(n_runs: int = 64, seed: int = DATA_SEED) -> list[RunSpec]:
    """Uneven run sizes: patterns log-uniform 1e4..5e5, features 5..40, degree 3..10,
    population log-uniform 64..2048 rounded to 32; bases and precisions alternate."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_runs):
        n = int(round(np.exp(rng.uniform(np.log(1e4), np.log(5e5)))))
        F = int(rng.integers(5, 41))
        d = int(rng.integers(3, 11))
        pop = int(round(np.exp(rng.uniform(np.log(64), np.log(2048))) / 32.0)) * 32
        pop = min(max(pop, 64), 2048)
        out.append(RunSpec(n, F, d, pop, "chebyshev" if i % 2 == 0 else "trig",
                           "fp32" if (i // 2) % 2 == 0 else "bf16", seed + 1 + i))
    return out
