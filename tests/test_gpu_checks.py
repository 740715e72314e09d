"""The bounds-checked debug build (-DGAME_CHECKS, _lib/libgame_checks.so).

Its kernels guard their indexed accesses and record the first failing guard instead
of trapping; the API turns a record into GAME_ERR_CHECK.  A child process loads that
build (GAME_LIB_PATH) and runs the main paths -- FP32 on the tensor cores, the
precision form with the FP32 re-score, the CUDA-core and on-the-fly engines, trig
and shared coefficients, the generation graph -- which must raise no check and still
match the oracle."""

import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import numpy as np
from oracle import game_oracle as o
from paper_1304_0597_gb300 import synth
from tests.gpu_helpers import make_game
from paper_1304_0597_gb300 import game
assert game.LIB_PATH.endswith("libgame_checks.so"), game.LIB_PATH
cases = [
    (dict(basis="chebyshev", degree=8, pop=256), dict(engine=game.ENGINE_TCGEN05), (20011, 32, 8)),
    (dict(basis="chebyshev", degree=8, pop=256), dict(engine=game.ENGINE_TCGEN05, tile_cluster=2), (9001, 16, 8)),
    (dict(basis="chebyshev", degree=4, pop=24), dict(engine=game.ENGINE_TCGEN05), (3001, 7, 4)),
    (dict(basis="trig", degree=5, pop=100), dict(engine=game.ENGINE_SIMT), (4001, 6, 5)),
    (dict(basis="trig", degree=4, pop=23, coefficients="shared"), dict(), (3001, 11, 4)),
    (dict(basis="chebyshev", degree=6, pop=130), dict(engine=game.ENGINE_ON_THE_FLY), (5003, 9, 6)),
]
for ocfg_kw, kw, (n, F, d) in cases:
    ds = synth.make_dataset(n, F, d, ocfg_kw["basis"], seed=91)
    ocfg = o.Config(seed=3, **ocfg_kw)
    g = make_game(ocfg, ds.X, ds.t, ds.n_train, **kw)
    fit, _ = g.evaluate()
    P = o.expand(ds.X[:ds.n_train], ocfg.basis, d, shared=ocfg.coefficients == "shared")
    np.testing.assert_allclose(fit, o.fitness(P, ds.t[:ds.n_train], g.population(), ocfg), rtol=1e-5)
    assert g.evolve(4) == 4
    g.best()
    g.close()
ds = synth.make_dataset(6007, 9, 5, seed=92)
g = make_game(o.Config(degree=5, pop=64, seed=4), ds.X, ds.t, ds.n_train, precision=game.BF16,
              elite_rescore=16)
g.evaluate()
assert g.evolve(4) == 4
print("checked build clean")
'''


def test_checked_build_runs_clean():
    from paper_1304_0597_gb300 import build
    lib = build.build(checks=True)
    env = dict(os.environ, GAME_LIB_PATH=lib, PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "checked build clean" in r.stdout
