"""Shared helpers of the GPU parity tests (marshalling between oracle and library configs)."""

import os

import numpy as np

from oracle import game_oracle as o


def lib():
    from paper_1304_0597_gb300 import build
    if not os.path.exists(build.LIB):
        build.build()
    from paper_1304_0597_gb300 import game
    return game


_ERR = {"rmse": 0, "mse": 1, "tmse": 2, "tmse_sq": 3}
_INIT = {"uniform_pm1": 0, "normal_pm1": 1, "uniform_01": 2}


def game_config(ocfg: o.Config, **kw):
    game = lib()
    cfg = game.default_config(
        basis=game.CHEBYSHEV if ocfg.basis == o.CHEBYSHEV else game.TRIG,
        degree=ocfg.degree, pop=ocfg.pop, tournament_k=ocfg.tournament_k,
        p_crossover=ocfg.p_crossover, p_mutation=ocfg.p_mutation,
        sigma_mutation=ocfg.sigma_mutation, elitism=ocfg.elitism,
        elite_mode=game.ELITE_TOP if ocfg.elite_mode == "top" else game.ELITE_COPIES,
        error=_ERR[ocfg.error], tmse_R=ocfg.tmse_R,
        activation=game.TANH if ocfg.activation == "tanh" else game.LINEAR,
        init=_INIT[ocfg.init], clamp_genes=int(ocfg.clamp_genes), stop_error=ocfg.stop_error,
        seed=ocfg.seed, run=ocfg.run, immigrants=ocfg.immigrants,
        coefficients=game.COEF_SHARED if ocfg.coefficients == "shared" else game.COEF_PER_FEATURE,
        selection={"tournament": game.SEL_TOURNAMENT, "roulette": game.SEL_ROULETTE,
                   "ranking": game.SEL_RANKING}[ocfg.selection])
    for k, v in kw.items():
        setattr(cfg, k, v)
    return cfg


def make_game(ocfg: o.Config, X, t, n_train, **kw):
    game = lib()
    g = game.Game(game_config(ocfg, **kw))
    g.set_data(X, t, n_train)
    return g


def oracle_fitness_chunked(X, t, G, ocfg: o.Config, chunk: int = 65536):
    """Oracle fitness over many patterns without holding the whole P in memory."""
    G = np.asarray(G, dtype=np.float64)
    sse = np.zeros(G.shape[0])
    for i in range(0, X.shape[0], chunk):
        P = o.expand(X[i:i + chunk], ocfg.basis, ocfg.degree)
        Y = o.activate(o.outputs(P, G), ocfg.activation)
        sse += o.pattern_errors(t[i:i + chunk], Y, ocfg.error, ocfg.tmse_R).sum(axis=1)
    mse = sse / X.shape[0]
    return np.sqrt(mse) if ocfg.error == "rmse" else mse
