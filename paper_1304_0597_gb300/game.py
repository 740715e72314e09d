"""ctypes binding of libgame.so (the C ABI declared in include/game.h).

Argument marshalling only: every computation runs in the library's CUDA
kernels.  Host arrays are numpy; device arrays are torch CUDA tensors (passed by
``data_ptr()`` with ``device_ptrs=1``).  Importing this module loads the
in-tree ``_lib/libgame.so`` and raises if it is missing.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# GAME_LIB_PATH selects another build of the same library (the profiling variant
# _lib/libgame_timeline.so); unset, the in-tree libgame.so.
LIB_PATH = os.environ.get("GAME_LIB_PATH") or os.path.join(_HERE, "_lib", "libgame.so")

GAME_OK = 0
STATUS = {0: "OK", -1: "INVALID_ARG", -2: "STATE", -3: "OOM", -4: "CUDA", -5: "NO_DEVICE",
          -6: "TIMEOUT", -7: "NUMERIC", -8: "UNSUPPORTED", -9: "CHECK"}

CHEBYSHEV, TRIG = 0, 1
RMSE, MSE, TMSE, TMSE_SQ = 0, 1, 2, 3
TANH, LINEAR = 0, 1
INIT_UNIFORM_PM1, INIT_NORMAL_PM1, INIT_UNIFORM_01 = 0, 1, 2
ELITE_TOP, ELITE_COPIES = 0, 1
FP32, BF16, FP8 = 0, 1, 2
COEF_PER_FEATURE, COEF_SHARED = 0, 1
SEL_TOURNAMENT, SEL_ROULETTE, SEL_RANKING = 0, 1, 2
ENGINE_AUTO, ENGINE_TCGEN05, ENGINE_SIMT, ENGINE_ON_THE_FLY = 0, 1, 2, 3


class GameConfig(C.Structure):
    _fields_ = [
        ("basis", C.c_int32), ("degree", C.c_int32), ("coefficients", C.c_int32),
        ("pop", C.c_int32), ("tournament_k", C.c_int32), ("selection", C.c_int32),
        ("p_crossover", C.c_float), ("p_mutation", C.c_float),
        ("sigma_mutation", C.c_float), ("elitism", C.c_int32), ("elite_mode", C.c_int32),
        ("error", C.c_int32), ("tmse_R", C.c_float), ("activation", C.c_int32),
        ("init", C.c_int32), ("clamp_genes", C.c_int32), ("immigrants", C.c_int32),
        ("stop_error", C.c_double),
        ("seed", C.c_uint64), ("run", C.c_uint64), ("precision", C.c_int32),
        ("elite_rescore", C.c_int32), ("gene_planes", C.c_int32), ("surrogate_pool", C.c_int32),
        ("surrogate_steps", C.c_int32), ("surrogate_batch", C.c_int32), ("surrogate_lr", C.c_float),
        ("surrogate_select", C.c_int32), ("surrogate_fp32", C.c_int32), ("engine", C.c_int32),
        ("tile_n", C.c_int32), ("tile_stages", C.c_int32), ("tile_cluster", C.c_int32),
        ("tile_slices", C.c_int32), ("tile_kgroup", C.c_int32), ("device", C.c_int32),
        ("stream", C.c_void_p),
    ]


class GameTiming(C.Structure):
    _fields_ = [("ms_breed", C.c_double), ("ms_fitness", C.c_double), ("ms_rank", C.c_double),
                ("ms_total", C.c_double), ("generations", C.c_int32), ("engine", C.c_int32),
                ("launches", C.c_int32)]


class GameTile(C.Structure):
    _fields_ = [("n", C.c_int32), ("stages", C.c_int32), ("cluster", C.c_int32),
                ("prefetch", C.c_int32), ("slices", C.c_int32), ("kgroup", C.c_int32),
                ("ms", C.c_double)]


def _tile_dict(t: "GameTile") -> dict:
    return {"n": t.n, "stages": t.stages, "cluster": t.cluster, "prefetch": t.prefetch,
            "slices": t.slices, "kgroup": t.kgroup, "ms": t.ms}


class GameError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _load() -> C.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_1304_0597_gb300.build "
                          "(there is no non-CUDA fallback)")
    lib = C.CDLL(LIB_PATH)
    P, I32, I64, D, F = C.c_void_p, C.c_int32, C.c_int64, C.c_double, C.c_float
    sig = {
        "game_config_default": (None, [C.POINTER(GameConfig)]),
        "game_create": (I32, [C.POINTER(GameConfig), C.POINTER(P)]),
        "game_set_data": (I32, [P, P, P, I64, I32, I64, I32]),
        "game_evolve": (I32, [P, I32, C.POINTER(I32)]),
        "game_get_best": (I32, [P, P, I32, C.POINTER(D), C.POINTER(D), C.POINTER(D)]),
        "game_n_genes": (I32, [P]),
        "game_last_error": (C.c_char_p, [P]),
        "game_destroy": (None, [P]),
        "game_set_population": (I32, [P, P, I32, I32, I32]),
        "game_get_population": (I32, [P, P, I32, I32]),
        "game_evaluate": (I32, [P, P, P]),
        "game_breed": (I32, [P, P]),
        "game_get_fitness": (I32, [P, P, P]),
        "game_get_expansion": (I32, [P, P, I64, I64]),
        "game_score": (I32, [P, P, I32, C.POINTER(D), C.POINTER(D), C.POINTER(D), C.POINTER(D)]),
        "game_get_state": (I32, [P, C.POINTER(I64), C.POINTER(I32)]),
        "game_predict": (I32, [P, P, I32, P, I64, I32, P, I32]),
        "game_save": (I32, [P, P, I64, C.POINTER(I64)]),
        "game_load": (I32, [P, P, I64]),
        "game_get_timing": (I32, [P, C.POINTER(GameTiming)]),
        "game_set_timing": (I32, [P, I32]),
        "game_selftest_timeout": (I32, [P, I32, C.POINTER(I32)]),
        "game_get_tile": (I32, [P, C.POINTER(GameTile)]),
        "game_autotune": (I32, [P, I32, C.POINTER(GameTile), C.POINTER(GameTile), I32,
                                C.POINTER(I32)]),
        "game_fitness_noalloc": (I32, [P, P, P, I64, I32, I32, I32, I32, F, P, P]),
        "game_surrogate_n_params": (I64, [P]),
        "game_surrogate_get_params": (I32, [P, P]),
        "game_surrogate_set_params": (I32, [P, P]),
        "game_surrogate_forward": (I32, [P, P, I32, P]),
        "game_surrogate_grad": (I32, [P, P, P, I32, C.POINTER(D), P]),
        "game_surrogate_train_step": (I32, [P, P, P, I32, F]),
        "game_surrogate_monitor": (I32, [P, C.POINTER(D), C.POINTER(D), C.POINTER(I32), P, I32,
                                         C.POINTER(I32)]),
        "game_surrogate_pool": (I32, [P, P, P, P, P, C.POINTER(I32)]),
        "game_batch_create": (I32, [C.POINTER(GameConfig), I32, C.POINTER(P)]),
        "game_batch_set_data": (I32, [P, I32, P, P, I64, I32, I64, I32]),
        "game_batch_run": (P, [P, I32]),
        "game_batch_evolve": (I32, [P, I32, P]),
        "game_batch_set_granularity": (I32, [P, I32]),
        "game_batch_autotune": (I32, [P, I32, C.POINTER(I32), C.POINTER(D)]),
        "game_batch_get_timing": (I32, [P, C.POINTER(GameTiming)]),
        "game_batch_destroy": (None, [P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


def exported_symbols() -> list[str]:
    """Names of the C entry points this binding expects libgame.so to export."""
    return [n for n in dir(lib) if n.startswith("game_")]


def default_config(**overrides) -> GameConfig:
    cfg = GameConfig()
    lib.game_config_default(C.byref(cfg))
    for k, v in overrides.items():
        if k == "stream" and v is not None and not isinstance(v, int):
            v = int(v)
        setattr(cfg, k, v)
    return cfg


def _ptr(a) -> tuple[int, int, object]:
    """(address, device flag, keep-alive) for a numpy array or a torch tensor."""
    if hasattr(a, "data_ptr") and hasattr(a, "is_cuda"):
        if a.is_cuda:
            if not a.is_contiguous():
                raise ValueError("device tensors must be contiguous")
            return a.data_ptr(), 1, a
        a = a.detach().cpu().numpy()
    arr = np.ascontiguousarray(a, dtype=np.float32)
    return arr.ctypes.data, 0, arr


class Game:
    """One GAME training context (``game_ctx``)."""

    def __init__(self, config: GameConfig | None = None, **overrides):
        cfg = config if config is not None else default_config()
        for k, v in overrides.items():
            setattr(cfg, k, v)
        self.cfg = cfg
        h = C.c_void_p()
        self._check(lib.game_create(C.byref(cfg), C.byref(h)), None)
        self.h = h

    def _check(self, status: int, h) -> None:
        if status != GAME_OK:
            raise GameError(status, lib.game_last_error(h).decode())

    def close(self) -> None:
        if getattr(self, "h", None):
            lib.game_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def n_genes(self) -> int:
        return lib.game_n_genes(self.h)

    @property
    def pop(self) -> int:
        return self.cfg.pop

    def set_data(self, X, t, n_train: int) -> None:
        xp, xd, kx = _ptr(X)
        tp, td, kt = _ptr(t)
        if xd != td:
            raise ValueError("X and t must both be host arrays or both device tensors")
        n, F = X.shape
        self._check(lib.game_set_data(self.h, xp, tp, n, F, n_train, xd), self.h)

    def evolve(self, generations: int) -> int:
        run = C.c_int32(0)
        self._check(lib.game_evolve(self.h, generations, C.byref(run)), self.h)
        return run.value

    def best(self):
        g = np.empty(self.n_genes, dtype=np.float32)
        fit, rm, acc = C.c_double(), C.c_double(), C.c_double()
        self._check(lib.game_get_best(self.h, g.ctypes.data, g.size, C.byref(fit), C.byref(rm),
                                      C.byref(acc)), self.h)
        return g, fit.value, rm.value, acc.value

    def set_population(self, G) -> None:
        gp, gd, keep = _ptr(G)
        self._check(lib.game_set_population(self.h, gp, self.pop, self.n_genes, gd), self.h)

    def population(self) -> np.ndarray:
        G = np.empty((self.pop, self.n_genes), dtype=np.float32)
        self._check(lib.game_get_population(self.h, G.ctypes.data, self.pop, self.n_genes),
                    self.h)
        return G

    def evaluate(self):
        fit = np.empty(self.pop, dtype=np.float64)
        rank = np.empty(self.pop, dtype=np.int32)
        self._check(lib.game_evaluate(self.h, fit.ctypes.data, rank.ctypes.data), self.h)
        return fit, rank

    def fitness(self):
        """Fitness and ranking of the last evaluated population (no new evaluation)."""
        fit = np.empty(self.pop, dtype=np.float64)
        rank = np.empty(self.pop, dtype=np.int32)
        self._check(lib.game_get_fitness(self.h, fit.ctypes.data, rank.ctypes.data), self.h)
        return fit, rank

    def breed(self, fitness=None) -> None:
        if fitness is None:
            self._check(lib.game_breed(self.h, None), self.h)
        else:
            f = np.ascontiguousarray(fitness, dtype=np.float64)
            self._check(lib.game_breed(self.h, f.ctypes.data), self.h)

    def expansion(self, row0: int, n_rows: int) -> np.ndarray:
        out = np.empty((n_rows, self.n_genes - 1), dtype=np.float32)
        self._check(lib.game_get_expansion(self.h, out.ctypes.data, row0, n_rows), self.h)
        return out

    def score(self, genes, split: int) -> dict:
        g = np.ascontiguousarray(genes, dtype=np.float32)
        v = [C.c_double() for _ in range(4)]
        self._check(lib.game_score(self.h, g.ctypes.data, split, *[C.byref(x) for x in v]),
                    self.h)
        return dict(zip(("rmse", "accuracy", "completeness", "contamination"),
                        (x.value for x in v)))

    def predict(self, genes, X) -> np.ndarray:
        """Outputs of one chromosome on patterns X [n x F] (host arrays or CUDA tensors;
        a CUDA X gives a CUDA result)."""
        g = np.ascontiguousarray(genes, dtype=np.float32)
        if hasattr(X, "is_cuda") and X.is_cuda:
            import torch
            Xd = X.contiguous()
            out = torch.empty(Xd.shape[0], dtype=torch.float32, device=Xd.device)
            self._check(lib.game_predict(self.h, g.ctypes.data, g.size, Xd.data_ptr(),
                                         Xd.shape[0], Xd.shape[1], out.data_ptr(), 1), self.h)
            return out
        Xh = np.ascontiguousarray(X, dtype=np.float32)
        out = np.empty(Xh.shape[0], dtype=np.float32)
        self._check(lib.game_predict(self.h, g.ctypes.data, g.size, Xh.ctypes.data, Xh.shape[0],
                                     Xh.shape[1], out.ctypes.data, 0), self.h)
        return out

    def save(self) -> bytes:
        """Checkpoint of the GA state (population, fitness, ranking, generation)."""
        n = C.c_int64(0)
        self._check(lib.game_save(self.h, None, 0, C.byref(n)), self.h)
        buf = C.create_string_buffer(n.value)
        self._check(lib.game_save(self.h, buf, n.value, C.byref(n)), self.h)
        return buf.raw

    def load(self, data: bytes) -> None:
        self._check(lib.game_load(self.h, data, len(data)), self.h)

    def state(self) -> tuple[int, int]:
        gen, stopped = C.c_int64(), C.c_int32()
        self._check(lib.game_get_state(self.h, C.byref(gen), C.byref(stopped)), self.h)
        return gen.value, stopped.value

    def autotune(self, reps: int = 5):
        best = GameTile()
        cands = (GameTile * 64)()
        n = C.c_int32(0)
        self._check(lib.game_autotune(self.h, reps, C.byref(best), cands, 64, C.byref(n)), self.h)
        return _tile_dict(best), [_tile_dict(cands[i]) for i in range(n.value)]

    def tile(self) -> dict:
        """The tcgen05 tile shape the fitness launches use (see game_get_tile)."""
        t = GameTile()
        self._check(lib.game_get_tile(self.h, C.byref(t)), self.h)
        return _tile_dict(t)

    # ---- learned surrogate ----
    def surrogate_params(self) -> np.ndarray:
        n = lib.game_surrogate_n_params(self.h)
        if n <= 0:
            raise GameError(-2, lib.game_last_error(self.h).decode())
        out = np.empty(n, dtype=np.float32)
        self._check(lib.game_surrogate_get_params(self.h, out.ctypes.data), self.h)
        return out

    def set_surrogate_params(self, params) -> None:
        p = np.ascontiguousarray(params, dtype=np.float32)
        self._check(lib.game_surrogate_set_params(self.h, p.ctypes.data), self.h)

    def surrogate_forward(self, X) -> np.ndarray:
        X = np.ascontiguousarray(X, dtype=np.float32)
        y = np.empty(X.shape[0], dtype=np.float32)
        self._check(lib.game_surrogate_forward(self.h, X.ctypes.data, X.shape[0], y.ctypes.data),
                    self.h)
        return y

    def surrogate_grad(self, X, target):
        X = np.ascontiguousarray(X, dtype=np.float32)
        t = np.ascontiguousarray(target, dtype=np.float32)
        g = np.empty(lib.game_surrogate_n_params(self.h), dtype=np.float32)
        loss = C.c_double()
        self._check(lib.game_surrogate_grad(self.h, X.ctypes.data, t.ctypes.data, X.shape[0],
                                            C.byref(loss), g.ctypes.data), self.h)
        return loss.value, g

    def surrogate_train_step(self, X, target, lr: float) -> None:
        X = np.ascontiguousarray(X, dtype=np.float32)
        t = np.ascontiguousarray(target, dtype=np.float32)
        self._check(lib.game_surrogate_train_step(self.h, X.ctypes.data, t.ctypes.data,
                                                  X.shape[0], lr), self.h)

    def surrogate_monitor(self, cap: int = 4096) -> dict:
        rho, loss = C.c_double(), C.c_double()
        fb, n = C.c_int32(), C.c_int32()
        hist = np.empty(cap, dtype=np.float64)
        self._check(lib.game_surrogate_monitor(self.h, C.byref(rho), C.byref(loss), C.byref(fb),
                                               hist.ctypes.data, cap, C.byref(n)), self.h)
        return {"rho": rho.value, "loss": loss.value, "fallback": fb.value,
                "history": hist[:n.value].copy()}

    def surrogate_pool(self) -> dict:
        """The last bred generation's offspring pool: scores, selected rows, genes, and the
        score each current row was selected with."""
        n = C.c_int32()
        self._check(lib.game_surrogate_pool(self.h, None, None, None, None, C.byref(n)), self.h)
        e = min(self.cfg.elitism, self.pop)
        scores = np.empty(n.value, dtype=np.float32)
        sel = np.empty(self.pop - e, dtype=np.int32)
        genes = np.empty((n.value, self.n_genes), dtype=np.float32)
        pred = np.empty(self.pop, dtype=np.float32)
        self._check(lib.game_surrogate_pool(self.h, scores.ctypes.data, sel.ctypes.data,
                                            genes.ctypes.data, pred.ctypes.data, None), self.h)
        return {"scores": scores, "selected": sel, "genes": genes, "predictions": pred}

    def set_timing(self, enabled: bool) -> None:
        self._check(lib.game_set_timing(self.h, int(bool(enabled))), self.h)

    def timing(self) -> dict:
        t = GameTiming()
        self._check(lib.game_get_timing(self.h, C.byref(t)), self.h)
        return {f: getattr(t, f) for f, _ in GameTiming._fields_}


class _RunView(Game):
    """A run owned by a Batch: the Game API without ownership of the context."""

    def __init__(self, handle, cfg):
        self.h = C.c_void_p(handle)
        self.cfg = cfg
        self._owned = False

    def close(self) -> None:
        self.h = None


class Batch:
    """Many independent GAME runs evolved together (``game_batch``)."""

    def __init__(self, configs):
        arr = (GameConfig * len(configs))(*configs)
        h = C.c_void_p()
        st = lib.game_batch_create(arr, len(configs), C.byref(h))
        if st != GAME_OK:
            raise GameError(st, lib.game_last_error(None).decode())
        self.h = h
        self.configs = list(configs)
        self.runs = [_RunView(lib.game_batch_run(h, i), configs[i]) for i in range(len(configs))]

    def _check(self, status: int) -> None:
        if status != GAME_OK:
            raise GameError(status, lib.game_last_error(None).decode())

    def set_data(self, run: int, X, t, n_train: int) -> None:
        xp, xd, kx = _ptr(X)
        tp, td, kt = _ptr(t)
        n, F = X.shape
        self._check(lib.game_batch_set_data(self.h, run, xp, tp, n, F, n_train, xd))

    def evolve(self, generations: int):
        out = np.zeros(len(self.runs), dtype=np.int32)
        self._check(lib.game_batch_evolve(self.h, generations, out.ctypes.data))
        return out

    def autotune(self, reps: int = 3):
        g, ms = C.c_int32(), C.c_double()
        self._check(lib.game_batch_autotune(self.h, reps, C.byref(g), C.byref(ms)))
        return g.value, ms.value

    def set_granularity(self, items_per_sm: int) -> None:
        self._check(lib.game_batch_set_granularity(self.h, items_per_sm))

    def timing(self) -> dict:
        t = GameTiming()
        self._check(lib.game_batch_get_timing(self.h, C.byref(t)))
        return {f: getattr(t, f) for f, _ in GameTiming._fields_}

    def close(self) -> None:
        if getattr(self, "h", None):
            for r in self.runs:
                r.h = None
            lib.game_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
