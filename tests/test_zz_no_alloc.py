"""game_fitness_noalloc: fitness for callers that cannot allocate device memory
(graph-captured work, fixed memory arenas, latency-critical paths).  Checked
through the C ABI against game_evaluate, the context path, on two calls in a
row.  Kept in its own file so that pytest collects it last."""

import numpy as np
import pytest

from oracle import game_oracle as o
from paper_1304_0597_gb300 import synth
from tests.gpu_helpers import lib, make_game

pytestmark = pytest.mark.gpu


def test_noalloc_fitness_matches_context_path_twice():
    import torch
    game = lib()
    ds = synth.make_dataset(6001, 6, 4, seed=21)
    ocfg = o.Config(basis="chebyshev", degree=4, pop=150, seed=3)
    g = make_game(ocfg, ds.X, ds.t, ds.n_train, engine=game.ENGINE_SIMT)
    G = g.population()
    want, _ = g.evaluate()
    P = torch.from_numpy(g.expansion(0, ds.n_train)).cuda()
    t = torch.from_numpy(ds.t[:ds.n_train].copy()).cuda()
    Gd = torch.from_numpy(G).cuda()
    out = torch.empty(ocfg.pop, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        out.fill_(float("nan"))
        st = game.lib.game_fitness_noalloc(P.data_ptr(), t.data_ptr(), Gd.data_ptr(),
                                           ds.n_train, g.n_genes, ocfg.pop, game.RMSE,
                                           game.TANH, 0.49, out.data_ptr(), stream)
        assert st == 0, game.lib.game_last_error(None)
        torch.cuda.synchronize()
        np.testing.assert_allclose(out.cpu().numpy(), want, rtol=1e-5)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    game = lib()
    st = game.lib.game_fitness_noalloc(1, 1, 1, 10, 5, 4097, game.RMSE, game.TANH, 0.49, 1, None)
    assert st == -8
    assert b"4096" in game.lib.game_last_error(None)
