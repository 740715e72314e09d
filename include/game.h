/*
 * game.h -- C ABI of libgame.so, a GB300 (sm_103a) engine for the population
 * fitness evaluation of GAME, the polynomial-expansion genetic algorithm of
 * Cavuoti et al., "Astrophysical data mining with GPU. A case study: genetic
 * classification of globular clusters".
 *
 * Method (paper Section 2): every pattern pat_k = (f_1..f_N, t_k) is expanded
 * feature by feature into a polynomial sequence (eq.1; polytrigo eq.8/eq.9, or
 * Chebyshev T_1..T_d); a chromosome is the vector of expansion coefficients;
 * its output on pattern k is Out(pat_k) = a_0 + sum_i sum_j a_ij g^j(f_i)
 * (eq.2), its fitness the MSE / RMSE / threshold-MSE of the outputs against
 * the targets (eq.3, eq.4, eq.5, eq.10).  Training (Section 4.1, steps 1-4)
 * draws a random population, then repeats: fitness + sort, stop test,
 * genetic operators.
 *
 * Conventions for every call:
 *  - A call returns GAME_OK or a negative game_status; it never aborts the
 *    process.  game_last_error() returns a message for the last failure on a
 *    context (valid until the next call on that context).
 *  - Host buffers passed in are read during the call only; the library copies
 *    what it keeps.  Output buffers are caller-owned and caller-sized.
 *  - "device pointer" arguments are CUDA global-memory addresses on the
 *    context's device; the caller keeps ownership.
 *  - All work is queued on the context's stream (game_config.stream, or the
 *    legacy default stream when NULL); calls that return data to the host
 *    synchronise that stream before returning.
 *  - One context is used by one host thread at a time.
 *  - Gene layout: gene 0 is the bias a_0; gene 1 + f*B*d + b is the b-th basis
 *    member of feature f (B = 1 Chebyshev, b = 0..d-1 -> T_{b+1}; B = 2
 *    polytrigo, b = 0..d-1 -> cos((b+1)x), b = d..2d-1 -> sin((b-d+1)x)),
 *    so n_genes = B*F*d + 1 (eq.7 generalised to per-feature coefficients).
 */
#ifndef GAME_H
#define GAME_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct game_ctx game_ctx;

typedef enum {
  GAME_OK = 0,
  GAME_ERR_INVALID_ARG = -1,  /* a size, pointer or option is out of range        */
  GAME_ERR_STATE = -2,        /* calls made in the wrong order (e.g. no data yet)   */
  GAME_ERR_OOM = -3,          /* device allocation failed                           */
  GAME_ERR_CUDA = -4,         /* a CUDA runtime / driver call failed                */
  GAME_ERR_NO_DEVICE = -5,    /* no usable sm_103a device                           */
  GAME_ERR_TIMEOUT = -6,      /* a bounded device-side wait gave up                 */
  GAME_ERR_NUMERIC = -7,      /* NaN / Inf in the input data                        */
  GAME_ERR_UNSUPPORTED = -8,  /* valid request outside this build's limits          */
  GAME_ERR_CHECK = -9         /* debug build (-DGAME_CHECKS): a device bounds check
                                 failed; the access was skipped (no trap)           */
} game_status;

enum { GAME_CHEBYSHEV = 0, GAME_TRIG = 1 };                       /* basis g(x)     */
enum { GAME_RMSE = 0, GAME_MSE = 1, GAME_TMSE = 2, GAME_TMSE_SQ = 3 };  /* error       */
enum { GAME_TANH = 0, GAME_LINEAR = 1 };                          /* activation     */
enum { GAME_INIT_UNIFORM_PM1 = 0, GAME_INIT_NORMAL_PM1 = 1, GAME_INIT_UNIFORM_01 = 2 };
enum { GAME_ELITE_TOP = 0, GAME_ELITE_COPIES = 1 };               /* elitism reading */
enum { GAME_COEF_PER_FEATURE = 0, GAME_COEF_SHARED = 1 };         /* eq.2 coefficients */
enum { GAME_SEL_TOURNAMENT = 0, GAME_SEL_ROULETTE = 1, GAME_SEL_RANKING = 2 };   /* selection */
enum { GAME_FP32 = 0, GAME_BF16 = 1, GAME_FP8 = 2 };              /* storage of P    */
/* Fitness engine.  TCGEN05: the tensor-core contraction (128-chromosome tiles, or
 * for at most 32 FP32 chromosomes the kernel with patterns on the MMA's M side).
 * SIMT: no tcgen05.  For at most 32 chromosomes on 16 or 32 stored columns, the
 * narrow kernels (FP32 and BF16 on warp-level MMAs, FP8 on CUDA-core FMAs); otherwise
 * CUDA-core FMA tiles.  ON_THE_FLY: the expansion matrix is never stored (device
 * memory of X instead of P; FP32 form only, no surrogate, not in batches): with
 * per-feature coefficients, warps of the tensor-core kernel form each k-block of P in
 * shared memory from the features for the MMAs; with shared coefficients (or genes
 * beyond what that kernel keeps in shared memory), CUDA-core FMAs on slabs formed the
 * same way.
 * AUTO: SIMT for the narrow shapes (the paper's own population of 2N + 1) and where
 * the genes exceed what the tensor-core kernels keep in shared memory, TCGEN05
 * otherwise; ON_THE_FLY only when the stored FP32 planes would not fit in the
 * device's free memory. */
enum { GAME_ENGINE_AUTO = 0, GAME_ENGINE_TCGEN05 = 1, GAME_ENGINE_SIMT = 2,
       GAME_ENGINE_ON_THE_FLY = 3 };

/*
 * Training options.  Paper Section 2 lists the user options (error function,
 * selection, elitism, random initialisation criteria); Section 5 gives the
 * experiment values.  Fill with game_config_default() and override.
 */
typedef struct game_config {
  int32_t basis;          /* GAME_CHEBYSHEV | GAME_TRIG (polytrigo, eq.8)                 */
  int32_t degree;         /* d >= 1 (eq.1)                                                 */
  int32_t coefficients;   /* GAME_COEF_PER_FEATURE: B*F*d+1 genes, one coefficient per feature
                             and basis member; GAME_COEF_SHARED: B*d+1 genes shared by all
                             features, the paper's eq.2 / eq.9 form (expansion summed over f) */
  int32_t pop;            /* chromosomes, 2..8192 (eq.6 gives B*N+1 as one choice)         */
  int32_t tournament_k;   /* tournament size, 1..32, draws with replacement               */
  int32_t selection;      /* GAME_SEL_TOURNAMENT (k draws) | GAME_SEL_ROULETTE (weight
                             1/(1e-12 + fitness)) | GAME_SEL_RANKING (linear ranking) (Sec. 2) */
  float p_crossover;      /* single-point crossover probability per pair                   */
  float p_mutation;       /* per-gene mutation probability                                 */
  float sigma_mutation;   /* std-dev of the Gaussian mutation step                          */
  int32_t elitism;        /* elite chromosomes copied unchanged, 0..pop                    */
  int32_t elite_mode;     /* GAME_ELITE_TOP (top-e distinct) | GAME_ELITE_COPIES (e x best) */
  int32_t error;          /* GAME_RMSE | GAME_MSE | GAME_TMSE (|t-Out|>R) | GAME_TMSE_SQ (eq.10 literal) */
  float tmse_R;           /* threshold R in ]0,1[ (eq.10)                                   */
  int32_t activation;     /* GAME_TANH | GAME_LINEAR (the paper's Out)                      */
  int32_t init;           /* GAME_INIT_* (Section 2, three random generation criteria)     */
  int32_t clamp_genes;    /* 1: genes clamped to [-1,1] after mutation                      */
  int32_t immigrants;     /* random chromosomes replacing the last children of every bred
                             generation (Section 4.1), 0..pop - elitism; default 0          */
  double stop_error;      /* stop when the best fitness <= this (Section 5: 0.001)         */
  uint64_t seed;          /* Philox key word 0                                              */
  uint64_t run;           /* Philox key word 1 (independent runs with one seed)            */
  int32_t precision;      /* GAME_FP32 | GAME_BF16 | GAME_FP8 storage of P                  */
  int32_t elite_rescore;  /* low precision: top-n re-scored with the FP32 path each gen     */
  int32_t gene_planes;    /* low precision: genes as 1 or 2 terms in P's format (0 = 2)     */
  int32_t surrogate_pool; /* 0 off; else offspring pool multiplier screened by the MLP      */
  int32_t surrogate_steps;  /* Adam steps per generation (0 = 6)                            */
  int32_t surrogate_batch;  /* training batch rows (0 = 1024)                               */
  float surrogate_lr;       /* Adam learning rate (0 = 2e-3)                                */
  int32_t surrogate_select; /* 0: surrogate's best of the pool; 1: plain children (ablation)*/
  int32_t surrogate_fp32;   /* 1: float32 weights in the GEMMs (checks); 0: bfloat16        */
  int32_t engine;         /* GAME_ENGINE_* fitness kernel choice (see the enum above)      */
  int32_t tile_n;         /* tcgen05 tile: patterns per tile, 128 | 256 (0 = tuned / auto)  */
  int32_t tile_stages;    /* tcgen05 tile: depth of the pattern-tile ring (0 = auto)        */
  int32_t tile_cluster;   /* tcgen05 tile: 1 = each CTA alone; 2 = CTA pairs sharing every MMA
                             (tcgen05 cta_group::2, M = 256 chromosomes: each CTA stages half of
                             each pattern tile; needs an even number of 128-chromosome slices);
                             0 = tuned, else pairs for the FP32 form where they fit with two
                             k-blocks per stage, else 1.  Other values are INVALID_ARG.  No
                             TMA multicast.  A request that cannot be planned for the
                             problem runs the default shape (game_get_tile says which). */
  int32_t tile_slices;    /* tcgen05 tile: 128-chromosome slices per CTA, 1 | 2 (2 needs tile_n 128; 0 = auto) */
  int32_t tile_kgroup;    /* tcgen05 tile: 128-byte k-blocks per pattern-tile stage, 1 | 2 (2 fetches
                             two k-blocks per TMA request; needs the stored genes to be whole
                             k-blocks, 64 for FP32 / BF16, 128 for FP8; 0 = auto) */
  int32_t device;         /* CUDA device ordinal                                            */
  void* stream;           /* cudaStream_t, or NULL for the legacy default stream           */
} game_config;

/* Fill *cfg with defaults: Chebyshev d=4, pop 20, k=3, pc 0.9, pm 0.05, sigma 0.1,
 * elitism 2 (top), RMSE, tanh, U[-1,1] init, clamp on, stop 0.001, seed 0, FP32. */
void game_config_default(game_config* cfg);

/* Create a context on cfg->device.  *out receives an owned handle (free with
 * game_destroy).  Errors: INVALID_ARG (bad option), NO_DEVICE (no sm_103a GPU),
 * CUDA. */
game_status game_create(const game_config* cfg, game_ctx** out);

/* Load the knowledge base (Section 2: patterns (f_1..f_N, t); train / test
 * subsets) and build the expansion matrix once (Section 4.1: the sums of sines
 * and cosines are computed in advance and kept on the device).
 *   X: n_patterns x n_features float32, row-major; t: n_patterns float32.
 *   The first n_train rows are the training set, the rest the test set.
 *   device_ptrs: 0 = X and t are host pointers, 1 = device pointers.
 * Resets the population to generation 0 (drawn from cfg->init).
 * Errors: INVALID_ARG (sizes, n_train outside 1..n_patterns), NUMERIC (NaN/Inf
 * in X or t), OOM, UNSUPPORTED (shape beyond this build's limits). */
game_status game_set_data(game_ctx* ctx, const float* X, const float* t, int64_t n_patterns,
                          int32_t n_features, int64_t n_train, int32_t device_ptrs);

/* Run up to max_generations generations of Section 4.1 steps 2-4 (fitness +
 * sort, stop test, operators).  Resumable: continues from the current
 * population and Philox counter.  Each generation evaluates one population;
 * every generation after the first evaluated one is bred from its parent.
 * *generations_run (may be NULL) receives the number evaluated by this call;
 * evolution stops early when the best fitness <= cfg->stop_error.
 * Errors: STATE (no data), CUDA, TIMEOUT. */
game_status game_evolve(game_ctx* ctx, int32_t max_generations, int32_t* generations_run);

/* Best chromosome of the last evaluated population (Section 2 "train" use case:
 * build and store the best population).  genes: caller buffer of cap >=
 * game_n_genes floats (may be NULL).  train_fitness: its fitness under
 * cfg->error on the training rows; test_rmse / test_accuracy: float64 report on
 * the test rows (accuracy by sign with sign(0)=+1 for tanh, y>=0.5 for linear).
 * Any output pointer may be NULL.  Errors: STATE (nothing evaluated), INVALID_ARG. */
game_status game_get_best(game_ctx* ctx, float* genes, int32_t cap, double* train_fitness,
                          double* test_rmse, double* test_accuracy);

/* Genes per chromosome (B*F*d + 1); 0 before game_set_data. */
int32_t game_n_genes(const game_ctx* ctx);

/* Message for the last failing call on ctx (or a global message when ctx is NULL). */
const char* game_last_error(const game_ctx* ctx);

/* Release every resource of ctx.  NULL is ignored. */
void game_destroy(game_ctx* ctx);

/* ---- step-level calls (tests, trajectory replay, custom loops) ------------- */

/* Replace the current population: G is pop x n_genes float32 row-major (host
 * or device per device_ptrs).  Marks it not yet evaluated; the generation
 * counter is unchanged.  Errors: STATE, INVALID_ARG. */
game_status game_set_population(game_ctx* ctx, const float* G, int32_t pop, int32_t n_genes,
                                int32_t device_ptrs);

/* Copy the current population (pop x n_genes float32) to the host buffer G. */
game_status game_get_population(game_ctx* ctx, float* G, int32_t pop, int32_t n_genes);

/* Fitness of the current population on the training rows (eq.2 -> eq.3 ->
 * eq.4/eq.5/eq.10), ranked by (fitness, index).  fitness (host, pop doubles)
 * and rank (host, pop int32) may be NULL.  Does not breed. */
game_status game_evaluate(game_ctx* ctx, double* fitness, int32_t* rank);

/* Fitness vector and ranking of the last evaluated population (no new
 * evaluation): host arrays of pop doubles / int32, either may be NULL.
 * Errors: STATE (nothing evaluated yet). */
game_status game_get_fitness(game_ctx* ctx, double* fitness, int32_t* rank);

/* One application of the genetic operators to the current population using
 * the given fitness vector (host, pop doubles; NULL = the last evaluated one),
 * with Philox counter word 0 = the current generation, which then advances by
 * one.  Elitism, tournament selection, single-point crossover, Gaussian
 * mutation and clamping as in Section 2 / Section 5. */
game_status game_breed(game_ctx* ctx, const double* fitness);

/* Copy expansion-matrix rows [row0, row0+n_rows) as float32 into out
 * (n_rows x (n_genes-1), the basis columns; the bias column of ones is
 * implicit), reconstructed from the stored precision. */
game_status game_get_expansion(game_ctx* ctx, float* out, int64_t row0, int64_t n_rows);

/* Float64 figures of merit of one chromosome (host genes, n_genes floats) on
 * the training (split 0) or test (split 1) rows: RMSE (eq.5), accuracy,
 * completeness (TP/(TP+FN)) and contamination (FP/(TP+FP)) with class +1 as
 * the positive (GC) class (Section 5).  Any output may be NULL. */
game_status game_score(game_ctx* ctx, const float* genes, int32_t split, double* rmse,
                       double* accuracy, double* completeness, double* contamination);

/* Current generation counter (number of breeding steps applied) and stop flag. */
game_status game_get_state(game_ctx* ctx, int64_t* generation, int32_t* stopped);

/* Device time of the last game_evolve call split by stage, in milliseconds
 * (CUDA events): breed, fitness (contraction + epilogue), rank (reduce +
 * sort).  Also the engine actually used (GAME_ENGINE_*) and the number of
 * kernels the call launched: the state reset plus, per requested generation,
 * the kernel nodes of the captured generation graph (a generation skipped
 * after a stop still launches them and they return at once). */
typedef struct game_timing {
  double ms_breed, ms_fitness, ms_rank, ms_total;
  int32_t generations;
  int32_t engine;
  int32_t launches;
} game_timing;
game_status game_get_timing(game_ctx* ctx, game_timing* out);

/* Outputs of a chromosome on new patterns, the paper's test and run use cases
 * (Section 2: a trained chromosome applied to data outside the training set):
 * out[k] = activation(g_0 + sum_f sum_b genes[1 + f*B*d + b] g_b(X[k][f])), eq.2
 * with the context's basis (eq.8 / eq.9 family, per-feature coefficients), degree
 * and activation, the expansion computed on the fly in float64.  X: n x n_features
 * float32 row-major, out: n float32; both host memory (device_ptrs = 0) or both
 * device memory (1); genes: host or device, n_genes = B*n_features*d + 1.  Needs
 * no game_set_data.  Errors: INVALID_ARG (sizes), CUDA. */
game_status game_predict(game_ctx* ctx, const float* genes, int32_t n_genes, const float* X,
                         int64_t n, int32_t n_features, float* out, int32_t device_ptrs);

/* Checkpoint of the GA (Section 2: the population is stored and training can
 * resume): the current population, its fitness and ranking and the loop state
 * (the generation that keys the counter-based random numbers), so that
 * game_evolve after game_load continues exactly as without the interruption.
 * game_save writes at most cap bytes to buf (host) and the needed size to *size;
 * buf = NULL only asks the size.  game_load takes a buffer of a context with the
 * same configuration (population, genes, basis, degree, seed, run) and data
 * shape.  Contexts with the learned surrogate return UNSUPPORTED (its network
 * and replay state are not part of the checkpoint).  Errors: STATE (no data),
 * INVALID_ARG (buffer size, foreign checkpoint), UNSUPPORTED, CUDA. */
game_status game_save(game_ctx* ctx, void* buf, int64_t cap, int64_t* size);
game_status game_load(game_ctx* ctx, const void* buf, int64_t size);

/* Failure-detection self-test (no paper counterpart): a device thread waits on
 * an mbarrier that nothing completes, with the bounded-wait code of the
 * tensor-core kernels but a limit of wait_us microseconds; the wait gives up,
 * records GAME_ERR_TIMEOUT in the device state and the call returns it (the
 * state's status is cleared again, so the context stays usable).  *waited_us
 * (may be NULL) receives the time waited.  Nothing faults, traps or hangs. */
game_status game_selftest_timeout(game_ctx* ctx, int32_t wait_us, int32_t* waited_us);

/* Tile shape of the tcgen05 fitness engine, as chosen by the autotuner. */
typedef struct game_tile {
  int32_t n;          /* patterns per tile (MMA N)                            */
  int32_t stages;     /* pattern-tile ring depth                              */
  int32_t cluster;    /* 1: one CTA per work unit; 2: CTA pairs (cta_group::2) */
  int32_t prefetch;   /* 1: L2 prefetch of each CTA's next pattern tile       */
  int32_t slices;     /* 128-chromosome slices per CTA fed by each pattern tile */
  int32_t kgroup;     /* 128-byte k-blocks of the pattern tile per ring stage (one TMA request) */
  double ms;          /* median fitness time of this shape, milliseconds      */
} game_tile;

/* Autotuner (no paper counterpart; the paper has one fixed Thrust code path):
 * times every valid tcgen05 tile shape for this context's problem (pattern
 * count, genes, population, precision) on the current population, reps
 * launches each (CUDA events on the context's stream, median), switches the
 * context to the fastest and records it in a cache file (GAME_TUNE_CACHE, else
 * $HOME/.cache/game_gb300_tiles.txt) that later contexts with the same shape
 * bucket read when their tile fields are 0.  *best (may be NULL) receives the
 * choice; candidates (may be NULL, cap entries) receives every timing and
 * *n_candidates their number.  Errors: STATE (no data), UNSUPPORTED (the shape
 * runs on the SIMT engine). */
game_status game_autotune(game_ctx* ctx, int32_t reps, game_tile* best, game_tile* candidates,
                          int32_t cap, int32_t* n_candidates);

/* The tcgen05 tile shape this context's fitness launches use (ms = 0).  A tile
 * request in the config that cannot be planned for the problem (too little
 * shared memory for the genes, pairs on an odd number of slices, grouped
 * k-blocks on genes that are not whole k-blocks) runs the default shape; this
 * call says which one runs.  Errors: STATE (no data), UNSUPPORTED (the shape
 * runs on a CUDA-core engine). */
game_status game_get_tile(game_ctx* ctx, game_tile* out);

/* enabled = 1: game_evolve records CUDA events around every stage of every
 * generation (on the context's stream) and game_get_timing reports their sums
 * for the last call; enabled = 0 (default): only the total is timed. */
game_status game_set_timing(game_ctx* ctx, int32_t enabled);

/* ---- learned surrogate (no paper counterpart) ------------------------------- */

/* With cfg.surrogate_pool = m > 0, every generation breeds m x (pop - elitism)
 * children with the usual operators, scores them with an MLP (genes -> 256 ->
 * 256 -> 1, GELU, bfloat16 weights and GEMM operands, float32 accumulation; the
 * genes standardised by running per-gene statistics of the evaluated
 * populations) that predicts the standardised log fitness, keeps the
 * pop - elitism best-scored children, and evaluates them exactly.  The exact (chromosome, fitness) pairs go to a replay
 * ring (the latest population, pop rows) on which the MLP takes surrogate_steps Adam steps per
 * generation.  The Spearman correlation of predicted and exact fitness of each
 * generation's children is recorded; below 0.1 the next generation keeps plain
 * children instead (the fallback).  The calls below expose the network for
 * checks and diagnostics; parameters are one flat float32 vector
 * [W1 (256 x n_genes) | b1 | W2 (256 x 256) | b2 | w3 (256) | b3]. */
int64_t game_surrogate_n_params(game_ctx* ctx);
game_status game_surrogate_get_params(game_ctx* ctx, float* params);
game_status game_surrogate_set_params(game_ctx* ctx, const float* params);
/* y[b] for B host rows X (B x n_genes float32). */
game_status game_surrogate_forward(game_ctx* ctx, const float* X, int32_t B, float* y);
/* Mean squared error of the network on (X, target) and its gradient (host,
 * n_params floats); B <= the training batch size. */
game_status game_surrogate_grad(game_ctx* ctx, const float* X, const float* target, int32_t B,
                                double* loss, float* grad);
/* One Adam step (Kingma & Ba 2015; beta 0.9 / 0.999, eps 1e-8) on (X, target). */
game_status game_surrogate_train_step(game_ctx* ctx, const float* X, const float* target,
                                      int32_t B, float lr);
/* Monitor: Spearman correlation of the last generation (NaN before the first
 * prediction), last training loss, fallback flag, and up to cap past values. */
game_status game_surrogate_monitor(game_ctx* ctx, double* rho_last, double* loss_last,
                                   int32_t* fallback, double* history, int32_t cap,
                                   int32_t* n_history);

/* The offspring pool of the last bred generation, for checks: its n_pool surrogate
 * scores (host, n_pool floats), the pool rows selected into the population (host,
 * pop - elitism int32: the pool indices whose scores are below the selection
 * threshold, in index order, then those equal to it, in index order, up to pop -
 * elitism), the pool's genes (host, n_pool x n_genes floats) and the score each row
 * of the current population was selected with (host, pop floats; NaN for elites and
 * rows bred without the network).  Any pointer may be NULL; *n_pool (may be NULL)
 * receives the pool size.  Errors: STATE (no data, or no pool). */
game_status game_surrogate_pool(game_ctx* ctx, float* scores, int32_t* selected, float* pool_genes,
                                float* predictions, int32_t* n_pool);

/* ---- batched form: many independent runs ----------------------------------- */

/* A batch of independent GAME runs (no paper counterpart: the paper trains one
 * model at a time).  Each run has its own configuration, data, population and
 * Philox key; a generation of every run is one CUDA graph whose fitness step is
 * a single persistent grouped launch over all runs (static schedule of (run,
 * slice, pattern-tile range) items balanced over the SMs).  A run's results are
 * those of the same run alone, up to the order of float64 partial sums. */
typedef struct game_batch game_batch;

/* n_runs contexts from cfgs[0..n_runs); all share cfgs[0].device and .stream. */
game_status game_batch_create(const game_config* cfgs, int32_t n_runs, game_batch** out);
/* Data of one run (as game_set_data). */
game_status game_batch_set_data(game_batch* b, int32_t run, const float* X, const float* t,
                                int64_t n_patterns, int32_t n_features, int64_t n_train,
                                int32_t device_ptrs);
/* The context of one run (owned by the batch): game_get_best, game_score,
 * game_get_population ... work on it; NULL for a bad index. */
game_ctx* game_batch_run(game_batch* b, int32_t run);
/* max_generations generations of every run; generations_run (may be NULL) is an
 * n_runs array receiving each run's count (runs stop on their own stop test). */
game_status game_batch_evolve(game_batch* b, int32_t max_generations, int32_t* generations_run);
/* Work items per SM of the grouped launch (schedule granularity, default 4). */
game_status game_batch_set_granularity(game_batch* b, int32_t items_per_sm);
/* Autotuner of the grouped launch: times the schedule granularities 1..16 items
 * per SM on the current populations, keeps the fastest (*items_per_sm, *ms). */
game_status game_batch_autotune(game_batch* b, int32_t reps, int32_t* items_per_sm, double* ms);
/* Total device time of the last game_batch_evolve (ms_total, generations). */
game_status game_batch_get_timing(game_batch* b, game_timing* out);
void game_batch_destroy(game_batch* b);

/* ---- fitness without device allocation ------------------------------------ */

/* Population fitness for callers that cannot allocate device memory.  The
 * paper has no counterpart: this is a packaging of the fitness step (float32
 * CUDA-core tiles, as in the tiled kernel of GAME_ENGINE_SIMT) for code that must
 * not call cudaMalloc -- a service whose device memory is a fixed arena owned by another
 * allocator, a plugin inside a program that owns every device allocation, or a
 * latency-critical path that cannot afford cudaMalloc's device-wide
 * synchronisation.  It calls no cudaMalloc, cudaFree or allocating library
 * routine.
 *   P: device, n_patterns x (n_genes-1) float32 row-major: the basis columns
 *      of the expansion (the bias column of ones is implicit), e.g. as
 *      returned by game_get_expansion.
 *   t: device, n_patterns float32 targets.  G: device, pop x n_genes float32
 *      (gene 0 = bias).  fitness: device, pop float64 output (eq.4 / eq.5 /
 *      eq.10 over the n_patterns rows for the given error and activation).
 *   stream: cudaStream_t (NULL = legacy default); the call only enqueues work.
 * Limits: 1 <= pop <= 4096 (else GAME_ERR_UNSUPPORTED).  Partial sums live in
 * one file-scope device array of 32 x 4096 doubles (1 MiB) that every device
 * loading the library keeps until exit; all calls share it and it keeps the
 * last call's contents (each call overwrites what it reads).  Calls whose work
 * overlaps on the GPU race on that array.  The first call on a device looks up
 * the array's address with that device current: make it before any stream
 * capture.  Errors also set game_last_error(NULL). */
game_status game_fitness_noalloc(const float* P, const float* t, const float* G,
                                 int64_t n_patterns, int32_t n_genes, int32_t pop, int32_t error,
                                 int32_t activation, float tmse_R, double* fitness, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* GAME_H */
