"""Per-tile timeline of CTA 0 of the tensor-core fitness kernel (a profiling aid).

The profiling build (``build(timeline=True)``, -DGAME_TC_TIMELINE) stamps ``clock64`` in
CTA 0 of ``fitness_tc_kernel`` for its first 32 tiles:
* the producer issuing each B k-block;
* the MMA warp passing each ring wait, passing the accumulator wait, and committing the tile;
* epilogue warps 2 and 17 starting and ending the tile.

This script builds that variant, loads it through ``GAME_LIB_PATH`` and runs a workload. The
workload is 1,000,000 patterns x 32 features (700,000 training rows), Chebyshev d = 8,
population 1024, in FP32, BF16 and FP8 (one gene plane), each on its autotuned tile. For the
last fitness launch it prints, per tile of CTA 0, the stamps in SM cycles from the MMA
warp's first tile start.

Usage (one GPU): ``python -m paper_1304_0597_gb300.tc_timeline [--tiles 16]``
"""

from __future__ import annotations

import argparse
import ctypes as C
import os

import numpy as np

from . import build as _build

PRECISIONS = ("fp32", "bf16", "fp8")


def main() -> None:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--tiles", type=int, default=16)
    ap.add_argument("--n-patterns", type=int, default=1_000_000)
    args = ap.parse_args()
    os.environ["GAME_LIB_PATH"] = _build.build(timeline=True)
    from . import game, synth   # loads the profiling build

    stamp = game.lib.game_tc_timeline
    stamp.argtypes = [C.c_void_p]
    stamp.restype = C.c_int
    ds = synth.plain_at_scale(seed=synth.DATA_SEED, n_patterns=args.n_patterns)
    buf = np.zeros(2048, dtype=np.int64)
    for name in PRECISIONS:
        prec = {"fp32": game.FP32, "bf16": game.BF16, "fp8": game.FP8}[name]
        kw = {} if prec == game.FP32 else {"gene_planes": 1}
        # no elite re-score: its FP32 launch would overwrite the stamps
        cfg = game.default_config(degree=8, pop=1024, seed=0, engine=game.ENGINE_TCGEN05,
                                  precision=prec, elite_rescore=0, **kw)
        with game.Game(cfg) as g:
            g.set_data(ds.X, ds.t, ds.n_train)
            tile, _ = g.autotune(reps=3)
            g.evolve(4)
            if stamp(buf.ctypes.data) != 0:
                raise RuntimeError("reading the timeline failed")
        T = buf.reshape(8, 32, 8)
        t0 = T[2, 0, 0]
        nkb = {"fp32": 4, "bf16": 4, "fp8": 2}[name]
        print(f"{name}: tile {tile}")
        print("tile | producer issues k-block 0..   | MMA past ring wait k-block 0..  "
              "| MMA start  commit | epi w2 start end | epi w17 start end")
        for it in range(min(args.tiles, 32)):
            rel = lambda e, k=0: int(T[e, it, k] - t0)
            print("%4d | %s | %s | %6d %6d | %6d %6d | %6d %6d" % (
                it, " ".join("%6d" % rel(0, k) for k in range(nkb)),
                " ".join("%6d" % rel(1, k) for k in range(nkb)),
                rel(2), rel(3), rel(4), rel(5), rel(6), rel(7)), flush=True)
        period = np.diff(T[2, 2:args.tiles, 0]).mean()
        gaps = np.diff(T[1, 2:args.tiles, :nkb], axis=1).mean() if nkb > 1 else float("nan")
        epi = (T[5, 2:args.tiles, 0] - T[4, 2:args.tiles, 0]).mean()
        print(f"{name}: tile period {period:.0f} cycles, MMA ring waits {gaps:.0f} cycles apart "
              f"within a tile, epilogue warp 2 busy {epi:.0f} cycles per tile\n", flush=True)


if __name__ == "__main__":
    main()
