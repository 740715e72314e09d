"""Host-side checks of the C ABI: the library builds, loads and exports every
entry point include/game.h declares; argument validation and the no-device
error need no GPU."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lib_path():
    from paper_1304_0597_gb300 import build
    if not os.path.exists(build.LIB):
        build.build()
    return build.LIB


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(game_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("game_create", "game_set_data", "game_evolve", "game_get_best", "game_destroy",
                 "game_last_error", "game_n_genes", "game_evaluate", "game_breed"):
        assert must in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(_lib_path())
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    _lib_path()
    from paper_1304_0597_gb300 import game
    for n in _declared():
        assert getattr(game.lib, n).argtypes is not None or n == "game_config_default", n


def test_defaults_and_validation_without_gpu():
    _lib_path()
    from paper_1304_0597_gb300 import game
    cfg = game.default_config()
    assert (cfg.degree, cfg.pop, cfg.tournament_k, cfg.elitism) == (4, 20, 3, 2)
    assert cfg.p_crossover == pytest.approx(0.9) and cfg.sigma_mutation == pytest.approx(0.1)
    assert cfg.stop_error == pytest.approx(0.001)
    h = ctypes.c_void_p()
    bad = game.default_config(pop=1)
    assert game.lib.game_create(ctypes.byref(bad), ctypes.byref(h)) == -1
    assert b"pop" in game.lib.game_last_error(None)
    bad = game.default_config(tmse_R=1.5, error=game.TMSE)
    assert game.lib.game_create(ctypes.byref(bad), ctypes.byref(h)) == -1
    bad = game.default_config(elitism=30)
    assert game.lib.game_create(ctypes.byref(bad), ctypes.byref(h)) == -1


def test_no_device_is_an_error_not_a_fallback():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    _lib_path()
    from paper_1304_0597_gb300 import game
    h = ctypes.c_void_p()
    cfg = game.default_config()
    assert game.lib.game_create(ctypes.byref(cfg), ctypes.byref(h)) == -5
    # calls on a NULL context fail cleanly
    assert game.lib.game_evolve(None, 1, None) == -1
    assert game.lib.game_n_genes(None) == 0
