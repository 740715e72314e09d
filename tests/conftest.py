import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libgame.so")
    # Contexts without a tile request read the autotuner's cache file; the tests get a
    # private one, so that what runs is the default plan unless a test tunes or asks.
    if "GAME_TUNE_CACHE" not in os.environ:
        import tempfile
        os.environ["GAME_TUNE_CACHE"] = os.path.join(tempfile.mkdtemp(prefix="game_tiles_"),
                                                     "tiles.txt")


def pytest_collection_modifyitems(config, items):
    """Skip GPU tests when no CUDA device is visible (the CPU suite deselects them anyway)."""
    try:
        import torch
        have_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        have_gpu = False
    if have_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for item in items:
        if "gpu" in item.keywords:
            item.add_marker(skip)
