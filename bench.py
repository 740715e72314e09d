#!/usr/bin/env python3
"""Benchmark: chromosome x pattern evaluations per second of GAME training on one GB300.

Workload (default): 1,000,000 patterns x 32 Gaussian-correlated features clipped
to [-1, 1], Chebyshev degree 8 (257 genes), population 1,024, 70/30 split,
tournament 3, single-point crossover 0.9, Gaussian mutation (0.1, 0.05),
elitism 2, tanh output, RMSE fitness, float32 fitness.

A step is one GAME generation (breed -> prepare -> fitness -> reduce + rank) on
the device; ``value`` = population x training patterns x steps / device time of
the K timed steps (inputs resident in HBM).  ``e2e`` times complete training runs
through the public C ABI from pinned host buffers: game_set_data (host -> device
copy + expansion) + game_evolve(50) + game_get_best (device -> host).

``--impl reference`` times the CPU oracle (float64 numpy, the method's plain
statement) on a bounded sample of the same workload.  Under torchrun each rank
runs an independent GA run (its own data seed) with no collective on the data
path (weak scaling); rank 0 prints one JSON line.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "chromosome*pattern evals/s (GAME population fitness, 1 GB300)"
UNIT = "evals/s"
GENS_PER_RUN = 50


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--engine", choices=["auto", "tcgen05", "simt", "on_the_fly"], default="auto")
    ap.add_argument("--n-patterns", type=int, default=1_000_000)
    ap.add_argument("--e2e-runs", type=int, default=2)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the library's default tile (no trial launches before the steps)")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the BF16 / FP8 precision-form record of the default line")
    ap.add_argument("--no-surrogate", action="store_true",
                    help="skip the one-seed learned-surrogate time-to-target record of the "
                         "default line")
    ap.add_argument("--no-batched-form", action="store_true",
                    help="skip the batched-form record (64 uneven runs) of the default line")
    ap.add_argument("--precision", choices=["fp32", "bf16", "fp8"], default="fp32")
    ap.add_argument("--gene-planes", type=int, choices=[1, 2], default=2,
                    help="low precision: genes as one or two terms of P's format")
    ap.add_argument("--batched", action="store_true",
                    help="the batched form: 64 uneven runs in one grouped launch per generation "
                         "against the same runs launched one by one; prints its own JSON line")
    ap.add_argument("--surrogate", action="store_true",
                    help="learned-surrogate form: time to the plain FP32 GA's final train RMSE")
    ap.add_argument("--seeds", type=int, default=5)
    ap.add_argument("--budget", type=int, default=200, help="plain GA generations (target run)")
    ap.add_argument("--paper", action="store_true",
                    help="the paper's experiment shape: Section 5 settings on the knowledge-base "
                         "stand-in replicated to 0.15 / 16 / 128 / 512 MB, degrees 1 / 2 / 4 / 8")
    ap.add_argument("--paper-iterations", type=int, default=4000)
    ap.add_argument("--paper-mb", type=float, nargs="+", default=None,
                    help="subset of the paper's sizes (0.15 16 128 512)")
    ap.add_argument("--paper-degrees", type=int, nargs="+", default=None,
                    help="subset of the paper's degrees (1 2 4 8)")
    ap.add_argument("--precision-table", action="store_true",
                    help="print the per-precision fitness error / accuracy table and exit")
    ap.add_argument("--timeline", action="store_true",
                    help="CTA-0 clock64 timeline of one tensor-core fitness launch per precision "
                         "(builds the -DGAME_TC_TIMELINE variant of the library)")
    ap.add_argument("--timeline-tiles", type=int, default=16)
    ap.add_argument("--engine-table", action="store_true",
                    help="fitness time per engine (stored tcgen05 / stored SIMT / on-the-fly) and "
                         "device bytes of the stored expansion, on a few shapes")
    ap.add_argument("--oracle-sample", action="store_true", help=argparse.SUPPRESS)
    return ap.parse_args()


def max_over_ranks(value: float, world: int) -> float:
    """Largest value over all ranks (the job time of a weak-scaling step); the
    process group's backend does the exchange (NCCL on GPUs, gloo on CPU)."""
    import torch
    import torch.distributed as dist
    if world <= 1:
        return float(value)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_units(pop: int, n_train: int, steps: int, world: int) -> int:
    """Chromosome x pattern evaluations of the whole job: every rank runs its own run."""
    return pop * n_train * steps * world


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def workload_config(n_patterns, precision="fp32"):
    return {"workload": f"plain GAME at scale, {precision.upper()} fitness",
            "n_patterns": n_patterns, "n_features": 32, "basis": "chebyshev", "degree": 8,
            "n_genes": 257, "pop": 1024, "train_frac": 0.7, "tournament_k": 3,
            "p_crossover": 0.9, "p_mutation": 0.05, "sigma_mutation": 0.1, "elitism": 2,
            "activation": "tanh", "error": "rmse"}


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        time.sleep(0.25)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=2)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ helpers

def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d.get("hbm_gbs"), d.get("bf16_tflops"), "measured"
    except OSError:
        return 6800.0, 1900.0, "fallback"


def kernel_traffic(kernel_file: str, variant: str):
    """DRAM bytes per launch from the committed ncu summary, if taken on this exact source.

    A record is keyed by kernel file and variant (precision and gene planes) and carries
    the sha256 of every source file the kernel is compiled from; any edit voids it."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f).get(f"{kernel_file}:{variant}")
        if not rec:
            return None
        for name, want in rec.get("source_sha256", {}).items():
            with open(os.path.join(ROOT, "paper_1304_0597_gb300", "csrc", name), "rb") as f:
                if hashlib.sha256(f.read()).hexdigest() != want:
                    return None
    except (OSError, ValueError, AttributeError):
        return None
    return rec.get("bytes_per_launch")


def host_cores() -> int:
    """Cores this process may run on (nproc)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


_THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS",
                "BLIS_NUM_THREADS", "NUMEXPR_NUM_THREADS")


def oracle_sample_subprocess(threads: int, seconds: float, n_sample: int = 10_000):
    """The oracle's generation rate on a bounded sample, in a fresh interpreter whose BLAS
    is limited to `threads` threads (the environment is read when numpy loads)."""
    env = dict(os.environ, **{v: str(threads) for v in _THREAD_VARS})
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample",
                        "--cpu-seconds", str(seconds)], env=env, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"oracle sample failed: {r.stderr[-400:]}")
    rec = json.loads(r.stdout.strip().splitlines()[-1])
    rec["threads"] = threads
    return rec


def oracle_sample_main(args):
    from paper_1304_0597_gb300 import synth
    n_sample = 10_000
    ds = synth.make_dataset(max(n_sample * 2, 20_000), 32, 8, "chebyshev", correlated=True)
    rate, n, el = oracle_generation_rate(ds, n_sample, 1024, args.cpu_seconds)
    print(json.dumps({"rate": rate, "generations": n, "seconds": el, "n_sample": n_sample}))


def cpu_baseline_record(seconds: float):
    """cpu_baseline of the bench line: the oracle as it stands on all host cores, plus the
    same sample on one thread."""
    cores = host_cores()
    allc = oracle_sample_subprocess(cores, seconds)
    one = oracle_sample_subprocess(1, seconds)
    sample = lambda r: (f"{r['generations']} generations (fitness+rank+breed, float64) of pop "
                        f"1024 on {r['n_sample']:,} training patterns, {r['seconds']:.1f} s")
    return {"value": allc["rate"], "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": sample(allc),
            "single_thread": {"value": one["rate"], "unit": UNIT, "cores": 1,
                              "sample": sample(one)}}


def oracle_generation_rate(ds, n_sample: int, pop: int, seconds: float, min_steps: int = 1,
                           steps: int | None = None, warmup: int = 0):
    """Time oracle generations (fitness + rank + breed, float64 numpy) on a sample of the rows."""
    from oracle import game_oracle as o
    ocfg = o.Config(basis="chebyshev", degree=8, pop=pop, seed=0)
    P = o.expand(ds.X[:n_sample], "chebyshev", 8)
    t = ds.t[:n_sample]
    G = o.init_population(ocfg, P.shape[1])
    gen = 0

    def step():
        nonlocal G, gen
        fit = o.fitness(P, t, G, ocfg)
        o.rank(fit)
        G = o.breed(G, fit, ocfg, gen)
        gen += 1

    for _ in range(warmup):
        step()
    n = 0
    t0 = time.perf_counter()
    while True:
        step()
        n += 1
        el = time.perf_counter() - t0
        if steps is not None:
            if n >= steps:
                break
        elif n >= min_steps and el >= seconds:
            break
    return pop * n_sample * n / el, n, el


# ------------------------------------------------------------------ reference arm

def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    from paper_1304_0597_gb300 import synth
    n_sample = 10_000
    ds = synth.make_dataset(max(n_sample * 2, 20_000), 32, 8, "chebyshev", correlated=True)
    rate, n, el = oracle_generation_rate(ds, n_sample, 1024, 0.0, steps=args.steps,
                                         warmup=args.warmup)
    cores = host_cores()
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * el / n, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(workload_config(args.n_patterns, args.precision), sample_train_patterns=n_sample),
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{n} generations (fitness+rank+breed) of pop 1024 on "
                                   f"{n_sample} training patterns of the workload"},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm

def forms_record(ds, X_pin, t_pin, stream, steps, warmup, bf16_peak):
    """The precision form on the same workload, measured after the headline (outside its
    timed region): P in BF16 and in FP8-E4M3 with one gene plane and the top-16 elites
    re-scored in FP32 each generation.  Per-stage device times over `steps` generations
    (CUDA events) and the fitness contraction's fraction of its dense peak (FP8: the
    measured bf16 peak x 2, the nominal ratio)."""
    from paper_1304_0597_gb300 import game
    out = {}
    flops = 2.0 * ds.n_train * 257 * 1024
    for name, prec, ratio in (("bf16", game.BF16, 1.0), ("fp8", game.FP8, 2.0)):
        cfg = game.default_config(degree=8, pop=1024, seed=0, stream=stream.cuda_stream,
                                  precision=prec, gene_planes=1, elite_rescore=16)
        with game.Game(cfg) as g:
            g.set_data(X_pin, t_pin, ds.n_train)
            tile, _ = g.autotune(reps=3)
            g.evolve(warmup)
            g.set_timing(True)
            ran = g.evolve(steps)
            tm = g.timing()
        fit_ms = tm["ms_fitness"] / steps
        out[name] = {"gene_planes": 1, "elite_rescore": 16, "tile": tile, "generations": ran,
                     "ms_per_generation": tm["ms_total"] / steps,
                     "stage_ms": {"breed_prepare": tm["ms_breed"] / steps, "fitness": fit_ms,
                                  "reduce_rank_rescore": tm["ms_rank"] / steps},
                     "evals_per_s": 1024 * ds.n_train / (tm["ms_total"] / steps / 1e3),
                     "fitness_tflops": flops / (fit_ms / 1e3) / 1e12,
                     "fitness_frac_of_peak": flops / (fit_ms / 1e3) / 1e12 / (bf16_peak * ratio)}
    return out


def run_ours(args):
    import torch
    import torch.distributed as dist

    rank, local_rank, world = dist_env()
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local_rank)
    from paper_1304_0597_gb300 import game, synth

    ds = synth.plain_at_scale(seed=synth.DATA_SEED + rank, n_patterns=args.n_patterns)
    X_pin = torch.from_numpy(ds.X).pin_memory()
    t_pin = torch.from_numpy(ds.t).pin_memory()
    stream = torch.cuda.current_stream()
    engine = {"auto": game.ENGINE_AUTO, "tcgen05": game.ENGINE_TCGEN05,
              "simt": game.ENGINE_SIMT, "on_the_fly": game.ENGINE_ON_THE_FLY}[args.engine]
    prec = {"fp32": game.FP32, "bf16": game.BF16, "fp8": game.FP8}[args.precision]
    cfg = game.default_config(degree=8, pop=1024, seed=rank, stream=stream.cuda_stream,
                              engine=engine, device=local_rank, precision=prec,
                              gene_planes=args.gene_planes)
    g = game.Game(cfg)
    g.set_data(X_pin, t_pin, ds.n_train)
    tile = None
    if g.timing()["engine"] == game.ENGINE_TCGEN05 and not args.no_autotune:
        tile, tile_cands = g.autotune(reps=3)     # library autotuner, outside the timed region
    K, W = args.steps, args.warmup
    g.evolve(W)
    g.set_timing(True)
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            dist.barrier()

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clk:
        barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        ran = g.evolve(K)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
    ms = e0.elapsed_time(e1)
    tm = g.timing()
    assert ran == K, f"evolution stopped after {ran} of {K} generations"
    ms_max = max_over_ranks(ms, world)
    pop, n_train, n_genes = 1024, ds.n_train, g.n_genes
    units = job_units(pop, n_train, K, world)
    value = units / (ms_max / 1e3)

    # End to end through the C ABI from pinned host memory: one training run per step.
    g.set_timing(False)
    e2e_t = []
    genes = np.empty(n_genes, dtype=np.float32)
    for i in range(args.e2e_runs + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.set_data(X_pin, t_pin, ds.n_train)
        ran_e = g.evolve(GENS_PER_RUN)
        genes[:], fit_best, test_rmse, test_acc = g.best()
        el = time.perf_counter() - t0
        if i > 0:
            e2e_t.append(el)
    e2e_value = pop * n_train * GENS_PER_RUN / statistics.median(e2e_t)
    h2d = ds.X.nbytes + ds.t.nbytes
    d2h = n_genes * 4 + 3 * 8 + 4 + 40

    # Roofline of the dominant kernel (fitness), from its CUDA-event time in the timed region.
    hbm, bf16_tf, peak_src = measured_peaks()
    fit_ms = tm["ms_fitness"] / K
    engine_used = tm["engine"]
    flops = 2.0 * n_train * n_genes * pop
    # tensor products issued per algorithmic product: FP32 = fp16 hi/lo split (3),
    # BF16 / FP8 = one per gene plane
    products = 3 if args.precision == "fp32" else args.gene_planes
    variant = "fp32" if args.precision == "fp32" else f"{args.precision}x{args.gene_planes}"
    ratio = 1.0
    if engine_used == game.ENGINE_TCGEN05:
        # e4m3 products run at twice the 16-bit rate (nominal dense 4.5 vs 2.25 PFLOP/s)
        ratio = 2.0 if args.precision == "fp8" else 1.0
        kfile, bound, peak, punit = "fitness_tc.cu", "tensor", bf16_tf * ratio, "TFLOP/s"
        achieved = flops / (fit_ms / 1e3) / 1e12
    else:
        # float32 FFMA: 152 SMs x 128 lanes x 2 flops x max SM clock
        kfile = "fitness_otf.cu" if engine_used == game.ENGINE_ON_THE_FLY else "fitness_simt.cu"
        bound, punit = "alu", "TFLOP/s"
        peak = 152 * 128 * 2 * 2.07e9 / 1e12
        achieved = flops / (fit_ms / 1e3) / 1e12
    traffic = kernel_traffic(kfile, variant)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": ms_max / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp32": "f32", "bf16": "bf16", "fp8": "e4m3"}[args.precision],
        "data": "synthetic",
        "config": dict(workload_config(args.n_patterns, args.precision), n_train=n_train,
                       precision=args.precision,
                       gene_planes=args.gene_planes if args.precision != "fp32" else None,
                       engine={1: "tcgen05", 2: "simt", 3: "on_the_fly"}.get(engine_used, "?"),
                       tile=tile,
                       l2="inputs larger than L2 (expansion planes of the training rows: "
                          f"{2 * 2 * n_train * 256 / 1e6:.0f} MB)",
                       parallelism=f"{world} independent runs (one per GPU)"),
        "stage_ms_per_step": {"breed_prepare": tm["ms_breed"] / K, "fitness": fit_ms,
                              "reduce_rank": tm["ms_rank"] / K},
        "roofline": {"bound": bound, "achieved": achieved, "peak": peak, "unit": punit,
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": kfile, "variant": variant,
                     "peak_source": (f"{peak_src} bf16" + (" x 2 (e4m3 nominal ratio)"
                                                           if ratio != 1.0 else ""))
                     if bound == "tensor" else "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz",
                     "tensor_products_per_term": products if bound == "tensor" else None,
                     "issued_frac": achieved * products / peak if bound == "tensor" else None},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "step": f"one training run: set_data + "
                f"{GENS_PER_RUN} generations + get_best", "runs": len(e2e_t)},
        "gpu_launches": tm["launches"],
        "clocks": clk.summary(),
        "best": {"train_rmse": fit_best, "test_rmse": test_rmse, "test_accuracy": test_acc},
    }
    if rank == 0 and world == 1 and args.precision == "fp32" and not args.no_forms:
        line["forms"] = forms_record(ds, X_pin, t_pin, stream, K, W, bf16_tf)
    if rank == 0 and world == 1 and args.precision == "fp32" and not args.no_surrogate:
        line["surrogate"] = surrogate_record()
    if rank == 0 and world == 1 and args.precision == "fp32" and not args.no_batched_form:
        line["batched"] = {"workload": "batched form: 64 independent runs of uneven sizes in "
                                       "one grouped persistent launch per generation",
                           **batched_measure(10, 3)}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_record(args.cpu_seconds)
    g.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def precision_table(args):
    """Fitness error against the float64 report, and test accuracy, per storage precision
    (the plain small workload: 2,000 x 7, Chebyshev d=4, pop 20, 100 generations; top-16
    elites re-scored in FP32 for BF16 / FP8), on the automatic engine (for this population
    of 20 the narrow kernels, whose BF16 / FP8 form keeps the genes in float32) and on the
    tensor-core engine (genes in 1 or 2 planes of P's format)."""
    from paper_1304_0597_gb300 import game, synth
    ds = synth.plain_small()
    rows = []
    for ename, eng in (("auto", game.ENGINE_AUTO), ("tcgen05", game.ENGINE_TCGEN05)):
        for name, prec in (("fp32", game.FP32), ("bf16", game.BF16), ("fp8", game.FP8)):
            for rescore, planes in (((0, 2),) if prec == game.FP32 else
                                    ((0, 2), (16, 2), (0, 1), (16, 1))):
                g = game.Game(game.default_config(degree=4, pop=20, seed=0, precision=prec,
                                                  elite_rescore=rescore, gene_planes=planes,
                                                  engine=eng))
                g.set_data(ds.X, ds.t, ds.n_train)
                G = g.population()
                fit, _ = g.evaluate()
                exact = np.array([g.score(G[i], 0)["rmse"] for i in range(20)])
                rel = np.abs(fit - exact) / exact
                g.set_timing(True)
                g.evolve(100)
                tm = g.timing()
                genes, fbest, test_rmse, acc = g.best()
                exact_best = g.score(genes, 0)["rmse"]
                rows.append({"engine": ename, "precision": name, "elite_rescore": rescore,
                             "gene_planes": planes,
                             "gen0_fitness_rel_err_vs_fp64": {"max": float(rel.max()),
                                                              "median": float(np.median(rel))},
                             "best_train_rmse_reported": fbest, "best_train_rmse_fp64": exact_best,
                             "test_rmse": test_rmse, "test_accuracy": acc,
                             "ms_per_generation": tm["ms_total"] / 100})
                g.close()
    print(json.dumps({"table": "precision form on the plain small workload", "rows": rows}))


def batched_measure(K: int, W: int) -> dict:
    """64 independent runs of uneven sizes (seeded: patterns 1e4..5e5 log-uniform, features
    5..40, degree 3..10, population 64..2048, Chebyshev / trig and FP32 / BF16 alternating)
    evolved together for K generations after W warm-up ones, against the sum of the same
    runs evolved one at a time (device time from the library's CUDA events)."""
    from paper_1304_0597_gb300 import game, synth
    specs = synth.batched_specs()
    data, cfgs = [], []
    for sp in specs:
        ds = synth.make_dataset(sp.n_patterns, sp.n_features, sp.degree, sp.basis, seed=sp.seed,
                                correlated=True)
        data.append(ds)
        cfgs.append(game.default_config(
            basis=game.CHEBYSHEV if sp.basis == "chebyshev" else game.TRIG, degree=sp.degree,
            pop=sp.pop, seed=sp.seed, precision=game.FP32 if sp.precision == "fp32" else game.BF16,
            elite_rescore=0))
    evals_per_gen = sum(sp.pop * ds.n_train for sp, ds in zip(specs, data))
    flops_per_gen = sum(2.0 * ds.n_train * (c.basis + 1) * sp.n_features * sp.degree * sp.pop
                        for sp, ds, c in zip(specs, data, cfgs))
    b = game.Batch(cfgs)
    for i, ds in enumerate(data):
        b.set_data(i, ds.X, ds.t, ds.n_train)
    gran, gran_ms = b.autotune(reps=2)
    b.evolve(W)
    with ClockSampler(0) as clk:
        gens = b.evolve(K)
    tb = b.timing()["ms_total"]
    assert all(g == K for g in gens)
    b.close()
    single_ms = 0.0
    engines = {"tcgen05": 0, "simt": 0}
    for cfg, ds in zip(cfgs, data):
        g = game.Game(cfg)
        g.set_data(ds.X, ds.t, ds.n_train)
        g.evolve(W)
        g.evolve(K)
        single_ms += g.timing()["ms_total"]
        engines["tcgen05" if g.timing()["engine"] == game.ENGINE_TCGEN05 else "simt"] += 1
        g.close()
    return {"runs": len(specs), "generations": K, "warmup": W,
            "evals_per_generation": evals_per_gen,
            "algorithmic_tflop_per_generation": flops_per_gen / 1e12,
            "schedule_items_per_sm": gran, "grouped_launch_ms": gran_ms,
            "ms_per_generation": tb / K, "evals_per_s": evals_per_gen * K / (tb / 1e3),
            "achieved_tflops": flops_per_gen * K / (tb / 1e3) / 1e12,
            "one_at_a_time": {"ms_per_generation": single_ms / K,
                              "evals_per_s": evals_per_gen * K / (single_ms / 1e3),
                              "engines": engines},
            "speedup_vs_one_at_a_time": single_ms / tb, "clocks": clk.summary()}


def batched(args):
    """The batched form as a bench line of its own (see batched_measure)."""
    r = batched_measure(args.steps, args.warmup)
    line = {"metric": METRIC + ", batched form", "value": r["evals_per_s"],
            "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": r["ms_per_generation"], "higher_is_better": True, "data": "synthetic",
            "config": {"workload": "64 independent runs of uneven sizes", "runs": r["runs"],
                       "evals_per_generation": r["evals_per_generation"],
                       "algorithmic_tflop_per_generation": r["algorithmic_tflop_per_generation"],
                       "schedule_items_per_sm": r["schedule_items_per_sm"],
                       "grouped_launch_ms": r["grouped_launch_ms"]},
            "one_at_a_time": {"value": r["one_at_a_time"]["evals_per_s"],
                              "ms_per_step": r["one_at_a_time"]["ms_per_generation"],
                              "engines": r["one_at_a_time"]["engines"]},
            "speedup_vs_one_at_a_time": r["speedup_vs_one_at_a_time"],
            "achieved_tflops": r["achieved_tflops"], "clocks": r["clocks"]}
    print(json.dumps(line), flush=True)


def ttt_seed(ds, seed, budget, contenders, tuned):
    """One seed of the time-to-target comparison on the learned-surrogate workload: the
    plain FP32 GA runs `budget` generations and sets the target (its final best train
    RMSE); each contender runs in steps of 5 generations until it reaches the target (at
    most 2 x budget).  Device time from the library's CUDA events around each generation."""
    from paper_1304_0597_gb300 import game

    def make(**kw):
        g = game.Game(game.default_config(degree=6, pop=4096, seed=seed, **kw))
        g.set_data(ds.X, ds.t, ds.n_train)
        key = (kw.get("precision", game.FP32), kw.get("gene_planes", 2))
        if key not in tuned and g.timing()["engine"] == game.ENGINE_TCGEN05:
            g.autotune(reps=2)      # the tile cache serves the later contexts
            tuned.add(key)
        g.set_timing(False)
        return g

    plain = make()
    plain.evolve(budget)
    t_plain = plain.timing()["ms_total"]
    _, target, _, acc_plain = plain.best()
    plain.close()
    row = {"seed": seed, "target_rmse": target, "plain_fp32": {"ms": t_plain,
           "generations": budget, "test_accuracy": acc_plain}}
    for name, kw in contenders:
        g = make(**kw)
        ms, gens, hit = 0.0, 0, False
        while gens < 2 * budget:
            g.evolve(5)
            ms += g.timing()["ms_total"]
            gens += 5
            _, best, _, acc = g.best()
            if best <= target:
                hit = True
                break
        rec = {"ms": ms, "generations": gens, "reached": hit, "best_rmse": best,
               "test_accuracy": acc, "speedup_vs_plain": t_plain / ms if hit else None}
        if kw.get("surrogate_pool"):
            rho = g.surrogate_monitor()["history"]
            rec["spearman_mean"] = float(np.nanmean(rho)) if len(rho) else None
        row[name] = rec
        g.close()
    return row


def surrogate_record(budget: int = 200) -> dict:
    """The learned-surrogate form for the default line: one seed (0) of the time-to-target
    comparison, plain FP32 GA against surrogate + FP8 P (8x pool, top-16 elites re-scored in
    FP32), on the 2,000,000 x 48 (Chebyshev d=6, pop 4096) workload."""
    from paper_1304_0597_gb300 import game, synth
    ds = synth.surrogate_scale(n_patterns=2_000_000)
    contenders = (("surrogate_fp8", dict(surrogate_pool=8, precision=game.FP8, gene_planes=1,
                                         elite_rescore=16)),)
    row = ttt_seed(ds, 0, budget, contenders, set())
    sur = row["surrogate_fp8"]
    return {"workload": "learned-surrogate form: 2,000,000 patterns x 48 features, Chebyshev "
                        "d=6, 289 genes, pop 4096, 8x pool, MLP 289-256-256-1",
            "seed": 0, "budget_generations": budget, "target_rmse": row["target_rmse"],
            "plain_fp32": row["plain_fp32"], "surrogate_fp8": sur,
            "time_to_target_speedup": sur["speedup_vs_plain"],
            "test_accuracy_delta": sur["test_accuracy"] - row["plain_fp32"]["test_accuracy"],
            "note": "one seed; bench.py --surrogate gives the median over seeds and the other "
                    "contenders"}


def surrogate_ttt(args):
    """Time to target RMSE on 2,000,000 patterns x 48 features (Chebyshev d=6, 289 genes),
    population 4096.  Target = final best train RMSE of the plain FP32 GA after --budget
    generations (same seed).  Contenders: the surrogate (MLP 289-256-256-1, 8x pool, top
    1/8 evaluated exactly) with FP8 and with BF16 P (one gene plane, top-16 elites
    re-scored in FP32); the same with a 4x pool; FP8 P alone (no surrogate); and the
    ablation (plain children of the same 8x pools) for the gain of the network itself.
    Every contender is timed on the device (CUDA events around each generation)."""
    from paper_1304_0597_gb300 import game, synth
    ds = synth.surrogate_scale(n_patterns=args.n_patterns if args.n_patterns != 1_000_000
                               else 2_000_000)
    lowp = dict(gene_planes=1, elite_rescore=16)
    contenders = (
        ("surrogate_fp8", dict(surrogate_pool=8, precision=game.FP8, **lowp)),
        ("surrogate_bf16", dict(surrogate_pool=8, precision=game.BF16, **lowp)),
        ("surrogate_fp8_pool4", dict(surrogate_pool=4, precision=game.FP8, **lowp)),
        ("fp8_only", dict(precision=game.FP8, **lowp)),
        ("ablation_fp8", dict(surrogate_pool=8, surrogate_select=1, precision=game.FP8, **lowp)),
    )
    tuned = set()
    results = []
    for seed in range(args.seeds):
        row = ttt_seed(ds, seed, args.budget, contenders, tuned)
        results.append(row)
        print(json.dumps(row), flush=True)

    def med(name):
        v = [r[name]["speedup_vs_plain"] for r in results if r[name]["speedup_vs_plain"]]
        return float(np.median(v)) if v else None

    def dacc(name):
        return float(np.mean([r[name]["test_accuracy"] - r["plain_fp32"]["test_accuracy"]
                              for r in results]))

    print(json.dumps({
        "metric": "time-to-target-RMSE speedup vs plain FP32 GA (learned surrogate + FP8 P)",
        "value": med("surrogate_fp8"), "unit": "x", "higher_is_better": True,
        "seeds": args.seeds, "budget_generations": args.budget,
        "median_speedup": {name: med(name) for name, _ in contenders},
        "mean_test_accuracy_delta": {name: dacc(name) for name, _ in contenders},
        "config": {"workload": "2,000,000 patterns x 48 features, Chebyshev d=6, 289 genes, "
                               "pop 4096, 8x pool, surrogate MLP 289-256-256-1 (bf16, tcgen05)",
                   "surrogate_steps_per_generation": 6, "surrogate_batch": 1024,
                   "surrogate_lr": 2e-3, "replay_ring": "latest population (4096 pairs)",
                   "inputs": "genes standardised by running per-gene statistics"}}), flush=True)


# The paper's Table benchgpu (GT540M, float64 Thrust): total training time of 4000
# iterations, polytrigo degree d, the 0.15 MB knowledge base replicated to 16 / 128 /
# 512 MB.  Context for the table below, not a target (another machine, a 2011 GPU).
PAPER_TOT_S = {1: (15.00, 240.00, 1870.50, 7680.00), 2: (16.00, 256.00, 1993.55, 8192.00),
               4: (19.00, 304.00, 2372.11, 9728.00), 8: (24.00, 384.00, 3006.12, 12288.00)}
PAPER_MB = (0.15, 16, 128, 512)


def paper_table(args):
    """The paper's experiment shape (Section 5): shared-coefficient polytrigo (eq.9),
    degrees 1 / 2 / 4 / 8, TMSE with R = 0.49, linear Out, 0/1 targets, roulette
    selection, normal init in [-1, 1], p_c 0.9, p_m 0.2, elitism 2, stop 0.001,
    population 23 (eq.6: 2 N + 1 for N = 11 features), on the knowledge-base
    stand-in replicated to the paper's sizes; 4000 iterations each, wall time of
    set_data (host arrays) + evolve + get_best."""
    import torch
    from paper_1304_0597_gb300 import game, synth
    rows = []
    for mb in (args.paper_mb or PAPER_MB):
        if mb not in PAPER_MB:
            raise SystemExit(f"--paper-mb: {mb} is not one of {PAPER_MB}")
        reps = max(1, int(round(mb / PAPER_MB[0])))
        ds = synth.paper_kb(replicas=reps)
        for d in (args.paper_degrees or (1, 2, 4, 8)):
            if d not in PAPER_TOT_S:
                raise SystemExit(f"--paper-degrees: {d} is not one of {tuple(PAPER_TOT_S)}")
            cfg = game.default_config(basis=game.TRIG, degree=d, coefficients=game.COEF_SHARED,
                                      pop=23, error=game.TMSE, tmse_R=0.49,
                                      activation=game.LINEAR, selection=game.SEL_ROULETTE,
                                      init=game.INIT_NORMAL_PM1, p_crossover=0.9,
                                      p_mutation=0.2, elitism=2, tournament_k=4,
                                      stop_error=0.001, seed=0)
            g = game.Game(cfg)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            g.set_data(ds.X, ds.t, ds.n_train)
            ran = g.evolve(args.paper_iterations)
            _, fit_best, test_err, acc = g.best()
            tot = time.perf_counter() - t0
            tm = g.timing()
            ms_gen = tm["ms_total"] / max(ran, 1)
            engine = {1: "tcgen05", 2: "simt", 3: "on_the_fly"}.get(tm["engine"], "?")
            g.close()
            paper_s = PAPER_TOT_S[d][PAPER_MB.index(mb)] * args.paper_iterations / 4000.0
            rows.append({"mb": mb, "patterns": int(ds.X.shape[0]), "degree": d,
                         "iterations": ran, "tot_s": tot, "ms_per_iteration": ms_gen,
                         "engine": engine,
                         "train_tmse": fit_best, "test_accuracy": acc,
                         "paper_tot_s_gt540m_context": paper_s})
            print(json.dumps(rows[-1]), flush=True)
    print(json.dumps({"table": "paper experiment shape (Section 5, Table benchgpu sizes)",
                      "rows": len(rows), "engines": sorted({r["engine"] for r in rows}),
                      "note": "paper numbers are a GT540M laptop GPU in float64: context only"}))


def timeline(args):
    """Per-tile clock64 timeline of CTA 0 of the tensor-core fitness kernel, one launch per
    precision (FP32; BF16 and FP8 with one gene plane), on the bench workload with the
    autotuned tile and no elite re-score.  Builds the -DGAME_TC_TIMELINE variant of the
    library (stamps: the producer issuing each pattern k-block, the MMA warp passing each
    ring wait and the accumulator wait and committing the tile, epilogue warps 2 and 17
    starting and ending the tile) and prints them in cycles from the first tile start."""
    import ctypes as C
    from paper_1304_0597_gb300 import build as _build
    os.environ["GAME_LIB_PATH"] = _build.build(timeline=True)
    from paper_1304_0597_gb300 import game, synth
    read, clear = game.lib.game_tc_timeline, game.lib.game_tc_timeline_clear
    read.argtypes, read.restype, clear.restype = [C.c_void_p], C.c_int, C.c_int
    ds = synth.plain_at_scale(n_patterns=args.n_patterns)
    buf = np.zeros(2048, dtype=np.int64)
    for name, prec in (("fp32", game.FP32), ("bf16", game.BF16), ("fp8", game.FP8)):
        kw = {} if prec == game.FP32 else {"gene_planes": 1}
        cfg = game.default_config(degree=8, pop=1024, seed=0, engine=game.ENGINE_TCGEN05,
                                  precision=prec, elite_rescore=0, **kw)
        with game.Game(cfg) as g:
            g.set_data(ds.X, ds.t, ds.n_train)
            tile, _ = g.autotune(reps=3)
            g.evolve(3)
            if clear() != 0:
                raise RuntimeError("clearing the timeline failed")
            g.evolve(1)                      # one fitness launch
            if read(buf.ctypes.data) != 0:
                raise RuntimeError("reading the timeline failed")
        T = buf.reshape(8, 32, 8)
        nkb = {"fp32": 4, "bf16": 4, "fp8": 2}[name]
        ks = list(range(0, nkb, max(1, tile.get("kgroup", 1))))   # stamped: one per ring stage
        ran = [it for it in range(32) if T[2, it, 0] != 0]      # tiles CTA 0 ran
        n = min(args.timeline_tiles, len(ran))
        t0 = T[2, 0, 0]
        print(f"{name}: tile {tile}, CTA 0 ran {len(ran)} stamped tiles")
        print("tile | producer issues stage (k-block) .. | MMA past ring wait .. "
              "| MMA start  commit | epi w2 start end | epi w17 start end")
        for it in range(n):
            rel = lambda e, k=0: int(T[e, it, k] - t0)
            print("%4d | %s | %s | %6d %6d | %6d %6d | %6d %6d" % (
                it, " ".join("%6d" % rel(0, k) for k in ks),
                " ".join("%6d" % rel(1, k) for k in ks),
                rel(2), rel(3), rel(4), rel(5), rel(6), rel(7)), flush=True)
        if n > 3:
            period = np.diff(T[2, 2:n, 0]).mean()
            gaps = np.diff(T[1, 2:n][:, ks], axis=1).mean() if len(ks) > 1 else float("nan")
            epi = (T[5, 2:n, 0] - T[4, 2:n, 0]).mean()
            print(f"{name}: tile period {period:.0f} cycles, MMA ring waits (first plane of each "
                  f"stage) {gaps:.0f} cycles apart within a tile, epilogue warp 2 busy "
                  f"{epi:.0f} cycles per tile\n", flush=True)


def engine_table(args):
    """Stored expansion against the on-the-fly engine: median fitness time of 10
    generations per engine (CUDA events) on shapes where P dominates the traffic to
    ones where the contraction does, with the bytes the stored FP32 planes take."""
    from paper_1304_0597_gb300 import game, synth
    shapes = (
        ("c2: 1M x 32, Chebyshev d=8, pop 1024", dict(n=1_000_000, F=32, d=8, basis="chebyshev",
                                                     pop=1024, correlated=True)),
        ("narrow: 1M x 40, trig d=10 (801 genes), pop 32", dict(n=1_000_000, F=40, d=10,
                                                               basis="trig", pop=32)),
        ("paper: 7.17M x 11, shared trig d=8, pop 23", dict(n=7_168_500, F=11, d=8, basis="trig",
                                                           pop=23, shared=True)),
        ("mid: 1M x 16, Chebyshev d=6, pop 128", dict(n=1_000_000, F=16, d=6, basis="chebyshev",
                                                     pop=128)),
    )
    for label, sh in shapes:
        if sh.get("shared"):
            ds = synth.paper_kb(replicas=3413)
        else:
            ds = synth.make_dataset(sh["n"], sh["F"], sh["d"], sh["basis"], seed=synth.DATA_SEED,
                                    correlated=sh.get("correlated", False))
        row = {"shape": label, "n_train": ds.n_train}
        for name, eng in (("tcgen05", game.ENGINE_TCGEN05), ("simt", game.ENGINE_SIMT),
                          ("on_the_fly", game.ENGINE_ON_THE_FLY)):
            cfg = game.default_config(
                basis=game.CHEBYSHEV if sh["basis"] == "chebyshev" else game.TRIG, degree=sh["d"],
                pop=sh["pop"], seed=0, engine=eng, stop_error=-1.0,
                coefficients=game.COEF_SHARED if sh.get("shared") else game.COEF_PER_FEATURE)
            try:
                g = game.Game(cfg)
                g.set_data(ds.X, ds.t, ds.n_train)
            except game.GameError as e:
                row[name] = f"unavailable: {e}"
                continue
            if eng == game.ENGINE_TCGEN05:
                try:
                    g.autotune(reps=2)
                except game.GameError:
                    pass
            g.evolve(3)
            g.set_timing(True)
            g.evolve(10)
            row[name + "_ms"] = g.timing()["ms_fitness"] / 10
            g.close()
        kb = (2 if sh["basis"] == "trig" else 1) * (1 if sh.get("shared") else sh["F"]) * sh["d"]
        kp = (kb + 15) // 16 * 16
        row["stored_fp32_planes_bytes"] = 4 * ds.n_patterns * kp
        row["features_bytes"] = 4 * ds.X.size
        print(json.dumps(row), flush=True)


def main():
    args = parse()
    if args.surrogate:
        surrogate_ttt(args)
        return
    if args.batched:
        batched(args)
        return
    if args.precision_table:
        precision_table(args)
        return
    if args.paper:
        paper_table(args)
        return
    if args.timeline:
        timeline(args)
        return
    if args.oracle_sample:
        oracle_sample_main(args)
        return
    if args.engine_table:
        engine_table(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
