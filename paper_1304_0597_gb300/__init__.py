"""GB300-native GAME population-fitness engine (sm_103a CUDA behind a C ABI).

``paper_1304_0597_gb300.game`` is the ctypes binding of ``libgame.so``; it is
imported lazily so that ``synth`` (seeded input generators) works on machines
without the built library.
"""

import importlib

__all__ = ["game", "synth"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
