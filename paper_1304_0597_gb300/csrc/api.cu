// C ABI of libgame.so: context, device buffers, the generation loop and the
// step-level calls.  Every compute step runs in this library's kernels; the
// host code only validates arguments, allocates, launches and copies.
//
// Loop (paper Section 4.1): (1) random initial population; (2) fitness of all
// chromosomes and sort; (3) stop test (error threshold or iteration budget);
// (4) genetic operators, back to (2).  One generation on the device is:
//   breed -> prepare operands -> fitness (tensor cores or SIMT) -> reduce+rank
// with the loop state (current buffer, generation, stop flag) kept in device
// memory, so a generation is a fixed sequence of launches that is captured once
// into a CUDA graph and replayed.
#include "game_internal.h"
#include "fitness_tc.h"
#include "surrogate.h"

#include <math_constants.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <math.h>
#include <stdlib.h>
#include <sys/stat.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

using namespace game;

struct game_ctx {
  game_config cfg{};
  std::string err;
  int dev = 0;
  int n_sm = 0;
  cudaStream_t st = nullptr;
  bool have_data = false;
  Shape s{};
  Fitness fit{};
  ExpDev e{};
  PopDev p{};
  double* d_fit = nullptr;
  int* d_rank = nullptr;
  double* d_partial = nullptr;
  int n_part = 0;          // partial rows used by the engine in use
  int part_rows = 0;       // partial rows allocated
  OtfTcPlan otf_tc;        // on-the-fly engine: the tensor-core kernel's plan ...
  bool otf_tc_ok = false;  // ... when it takes the shape (else the CUDA-core kernel)
  DevState* d_state = nullptr;
  float* d_scratch = nullptr;   // expansion column maxima
  double* d_score_blocks = nullptr;
  double* d_score_out = nullptr;
  int score_nb = 0;
  float* d_genes = nullptr;     // one chromosome (report)
  int engine = GAME_ENGINE_SIMT;
  bool otf = false;             // on-the-fly engine: no stored expansion
  const float* d_X = nullptr;   // the device copy of X (read by the on-the-fly engine)
  TcPlan tc{};
  // Precision form: FP32 copy of P and the FP32 re-score of the top elites.
  bool lowp = false;            // P stored in BF16 / FP8
  int n_rescore = 0;            // elites re-scored in FP32 each generation
  int part_rows_r = 0;          // rows of d_partial_r
  Shape s32{};                  // FP32 shape of P (report, re-score)
  ExpDev e32{};                 // FP32 planes of P (== e when precision is FP32)
  std::vector<float> scale32;   // power-of-two column scales of the FP32 planes (host copy)
  Shape sr{};                   // shape of the re-score population (pop = n_rescore)
  PopDev pr{};                  // gene planes of the gathered elites
  int engine_r = GAME_ENGINE_SIMT;
  TcPlan tc_r{};
  int n_part_r = 0;
  double* d_partial_r = nullptr;
  // Learned surrogate (cfg.surrogate_pool > 0 drives the generation; the network
  // also exists on demand for the checking calls).
  bool sg_alloc = false;
  cudaStream_t st_sg = nullptr;        // the surrogate training step's second stream
  cudaEvent_t ev_sg[2] = {};           // its fork / join events
  Surrogate sg{};
  int n_pool = 0;               // children bred per generation
  int sg_steps = 4, sg_batch = 1024;
  float sg_lr = 2e-3f;
  float* d_pool = nullptr;      // [n_pool x kstride]
  float* d_score = nullptr;     // [n_pool]
  int* d_sel = nullptr;         // [pop]
  float* d_pred = nullptr;      // [pop_pad] surrogate score of each evaluated child
  int* d_fallback = nullptr;
  float* d_ring_x = nullptr;    // [ring_cap x kstride]
  float* d_ring_f = nullptr;    // [ring_cap]
  long long* d_dsq = nullptr;   // [pop_pad] squared rank differences of the monitor
  unsigned long long* d_cum = nullptr;   // [pop_pad] roulette / ranking cumulative weights
  int* d_ring_meta = nullptr;   // head, count, evals appended, generations monitored
  int ring_cap = 0;
  float* d_norm = nullptr;      // mean, std of log fitness over the ring
  double* d_monitor = nullptr;  // [4096] Spearman per generation
  float* d_bx = nullptr;        // [batch x kstride] training rows
  float* d_bt = nullptr;        // [batch] standardised targets
  cudaGraphExec_t graph = nullptr;     // one generation
  int gen_kernels = 0;                 // kernel nodes of one captured generation
  cudaGraph_t graph_t_tmpl = nullptr;  // one generation with stage events (template kept alive)
  cudaGraphExec_t graph_t = nullptr;
  cudaGraphNode_t ev_node[4] = {};     // event-record nodes of graph_t, stage order
  std::vector<cudaEvent_t> ev_pool;    // 4 events per generation of a timed call
  bool timing_on = false;
  game_timing timing{};
  // Device blocks of the data set, in allocation order.  A later game_set_data walks
  // the same order and reuses every block whose size matches (same shapes: all of
  // them), so repeated runs on equal shapes pay no cudaMalloc / cudaFree.
  struct Block {
    void* p;
    size_t bytes;
  };
  std::vector<Block> allocs;
  size_t alloc_next = 0;
  cudaStream_t st_copy = nullptr;      // host-to-device copies of set_data, overlapped with the expansion
  std::vector<cudaEvent_t> copy_ev;    // one per copied chunk
};

static std::string g_global_err;

namespace game {
void set_global_error(const char* msg) { g_global_err = msg; }
}  // namespace game

static game_status fail(game_ctx* c, game_status code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  else g_global_err = buf;
  return code;
}

#define CUDA_OK(ctx, call)                                                                  \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? GAME_ERR_OOM : GAME_ERR_CUDA,      \
                  "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__);     \
  } while (0)

// Debug build (-DGAME_CHECKS): a device bounds check that failed since the last read
// turns into GAME_ERR_CHECK, naming the file, the site and the offending index.
static game_status collect_checks(game_ctx* c) {
#ifdef GAME_CHECKS
  const unsigned long long w[3] = {check_word_expand(), check_word_ga(), check_word_tc()};
  static const char* const file[3] = {"expand.cu", "ga.cu", "fitness_tc.cu"};
  for (int i = 0; i < 3; ++i)
    if (w[i])
      return fail(c, GAME_ERR_CHECK, "bounds check failed in %s: site %d, index %llu", file[i],
                  (int)(w[i] >> 48), (unsigned long long)(w[i] & 0xFFFFFFFFFFFFull));
#else
  (void)c;
#endif
  return GAME_OK;
}

// Blocks from position alloc_next on are released (the sequence changed or ended).
static void release_tail(game_ctx* c) {
  for (size_t i = c->alloc_next; i < c->allocs.size(); ++i) cudaFree(c->allocs[i].p);
  c->allocs.resize(c->alloc_next);
}

// The next zero-filled device block of the data set: the block at this position of
// the previous sequence when its size matches, else a new one.
template <typename T>
static game_status dalloc(game_ctx* c, T** ptr, size_t bytes) {
  *ptr = nullptr;
  if (bytes == 0) bytes = 16;
  if (c->alloc_next < c->allocs.size()) {
    if (c->allocs[c->alloc_next].bytes == bytes) {
      *ptr = static_cast<T*>(c->allocs[c->alloc_next++].p);
    } else {
      release_tail(c);
    }
  }
  if (!*ptr) {
    cudaError_t e = cudaMalloc((void**)ptr, bytes);
    if (e != cudaSuccess)
      return fail(c, GAME_ERR_OOM, "cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
    c->allocs.push_back(game_ctx::Block{*ptr, bytes});
    ++c->alloc_next;
  }
  cudaError_t e = cudaMemsetAsync(*ptr, 0, bytes, c->st);
  if (e != cudaSuccess) return fail(c, GAME_ERR_CUDA, "cudaMemset: %s", cudaGetErrorString(e));
  return GAME_OK;
}

static void drop_graphs(game_ctx* c) {
  if (c->graph) cudaGraphExecDestroy(c->graph);
  if (c->graph_t) cudaGraphExecDestroy(c->graph_t);
  if (c->graph_t_tmpl) cudaGraphDestroy(c->graph_t_tmpl);
  c->graph = c->graph_t = nullptr;
  c->graph_t_tmpl = nullptr;
}

static void free_all(game_ctx* c) {
  drop_graphs(c);
  c->alloc_next = 0;
  release_tail(c);
  c->have_data = false;
}

// Start a new data set on the blocks of the last one (see game_ctx::allocs).
static void reuse_blocks(game_ctx* c) {
  cudaStreamSynchronize(c->st);   // nothing of the last data set is still in flight
  drop_graphs(c);
  c->alloc_next = 0;
  c->have_data = false;
}

static int round_up(int v, int m) { return (v + m - 1) / m * m; }

extern "C" void game_config_default(game_config* cfg) {
  if (!cfg) return;
  memset(cfg, 0, sizeof(*cfg));
  cfg->basis = GAME_CHEBYSHEV;
  cfg->degree = 4;
  cfg->pop = 20;
  cfg->tournament_k = 3;
  cfg->p_crossover = 0.9f;
  cfg->p_mutation = 0.05f;
  cfg->sigma_mutation = 0.1f;
  cfg->elitism = 2;
  cfg->elite_mode = GAME_ELITE_TOP;
  cfg->error = GAME_RMSE;
  cfg->tmse_R = 0.49f;
  cfg->activation = GAME_TANH;
  cfg->init = GAME_INIT_UNIFORM_PM1;
  cfg->clamp_genes = 1;
  cfg->stop_error = 0.001;
  cfg->seed = 0;
  cfg->run = 0;
  cfg->precision = GAME_FP32;
  cfg->elite_rescore = 16;
  cfg->surrogate_pool = 0;
  cfg->engine = GAME_ENGINE_AUTO;
  cfg->device = 0;
  cfg->stream = nullptr;
}

static game_status validate(game_ctx* c, const game_config* cfg) {
  if (cfg->basis != GAME_CHEBYSHEV && cfg->basis != GAME_TRIG)
    return fail(c, GAME_ERR_INVALID_ARG, "basis must be GAME_CHEBYSHEV or GAME_TRIG");
  if (cfg->degree < 1 || cfg->degree > 32)
    return fail(c, GAME_ERR_INVALID_ARG, "degree must be in 1..32 (got %d)", cfg->degree);
  if (cfg->pop < 2 || cfg->pop > 8192)
    return fail(c, GAME_ERR_INVALID_ARG, "pop must be in 2..8192 (got %d)", cfg->pop);
  if (cfg->tournament_k < 1 || cfg->tournament_k > 32)
    return fail(c, GAME_ERR_INVALID_ARG, "tournament_k must be in 1..32");
  if (!(cfg->p_crossover >= 0.0f && cfg->p_crossover <= 1.0f) ||
      !(cfg->p_mutation >= 0.0f && cfg->p_mutation <= 1.0f) || !(cfg->sigma_mutation >= 0.0f))
    return fail(c, GAME_ERR_INVALID_ARG, "probabilities must be in [0,1] and sigma >= 0");
  if (cfg->elitism < 0 || cfg->elitism > cfg->pop)
    return fail(c, GAME_ERR_INVALID_ARG, "elitism must be in 0..pop");
  if (cfg->elite_mode != GAME_ELITE_TOP && cfg->elite_mode != GAME_ELITE_COPIES)
    return fail(c, GAME_ERR_INVALID_ARG, "bad elite_mode");
  if (cfg->error < GAME_RMSE || cfg->error > GAME_TMSE_SQ)
    return fail(c, GAME_ERR_INVALID_ARG, "bad error kind");
  if ((cfg->error == GAME_TMSE || cfg->error == GAME_TMSE_SQ) &&
      !(cfg->tmse_R > 0.0f && cfg->tmse_R < 1.0f))
    return fail(c, GAME_ERR_INVALID_ARG, "tmse_R must be in ]0,1[");
  if (cfg->activation != GAME_TANH && cfg->activation != GAME_LINEAR)
    return fail(c, GAME_ERR_INVALID_ARG, "bad activation");
  if (cfg->init < GAME_INIT_UNIFORM_PM1 || cfg->init > GAME_INIT_UNIFORM_01)
    return fail(c, GAME_ERR_INVALID_ARG, "bad init mode");
  if (cfg->precision < GAME_FP32 || cfg->precision > GAME_FP8)
    return fail(c, GAME_ERR_INVALID_ARG, "bad precision");
  if (cfg->engine < GAME_ENGINE_AUTO || cfg->engine > GAME_ENGINE_ON_THE_FLY)
    return fail(c, GAME_ERR_INVALID_ARG, "bad engine");
  if (cfg->coefficients < GAME_COEF_PER_FEATURE || cfg->coefficients > GAME_COEF_SHARED)
    return fail(c, GAME_ERR_INVALID_ARG, "bad coefficients");
  if (cfg->selection < GAME_SEL_TOURNAMENT || cfg->selection > GAME_SEL_RANKING)
    return fail(c, GAME_ERR_INVALID_ARG, "bad selection");
  if (cfg->immigrants < 0 || cfg->immigrants > cfg->pop - (cfg->elitism < cfg->pop ? cfg->elitism : cfg->pop))
    return fail(c, GAME_ERR_INVALID_ARG, "immigrants must be in 0..pop - elitism");
  if ((cfg->tile_n != 0 && cfg->tile_n != 128 && cfg->tile_n != 256) || cfg->tile_stages < 0 ||
      cfg->tile_cluster < 0 || cfg->tile_cluster > 2 || cfg->tile_slices < 0 || cfg->tile_slices > 2 ||
      (cfg->tile_slices == 2 && cfg->tile_n == 256) || cfg->tile_kgroup < 0 || cfg->tile_kgroup > 2)
    return fail(c, GAME_ERR_INVALID_ARG, "bad tile request");
  if (cfg->surrogate_pool < 0) return fail(c, GAME_ERR_INVALID_ARG, "bad surrogate_pool");
  if (cfg->surrogate_steps < 0 || cfg->surrogate_batch < 0 || cfg->surrogate_batch > 65536 ||
      !(cfg->surrogate_lr >= 0.0f) || cfg->surrogate_select < 0 || cfg->surrogate_select > 1)
    return fail(c, GAME_ERR_INVALID_ARG, "bad surrogate settings");
  if (cfg->gene_planes < 0 || cfg->gene_planes > 2)
    return fail(c, GAME_ERR_INVALID_ARG, "gene_planes must be 0, 1 or 2");
  return GAME_OK;
}

extern "C" game_status game_create(const game_config* cfg, game_ctx** out) {
  if (!cfg || !out) return fail(nullptr, GAME_ERR_INVALID_ARG, "cfg and out must be non-NULL");
  *out = nullptr;
  game_ctx* c = new game_ctx();
  game_status s = validate(c, cfg);
  if (s != GAME_OK) {
    g_global_err = c->err;
    delete c;
    return s;
  }
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || n <= 0 || cfg->device < 0 || cfg->device >= n) {
    cudaGetLastError();
    delete c;
    return fail(nullptr, GAME_ERR_NO_DEVICE, "no CUDA device %d", cfg->device);
  }
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, cfg->device) != cudaSuccess) {
    delete c;
    return fail(nullptr, GAME_ERR_NO_DEVICE, "cannot query device %d", cfg->device);
  }
  if (prop.major != 10 || prop.minor != 3) {
    delete c;
    return fail(nullptr, GAME_ERR_NO_DEVICE,
                "device %d is sm_%d%d; this library is built for sm_103a only", cfg->device,
                prop.major, prop.minor);
  }
  c->cfg = *cfg;
  c->dev = cfg->device;
  c->n_sm = prop.multiProcessorCount;
  c->st = (cudaStream_t)cfg->stream;
  cudaSetDevice(c->dev);
  cudaError_t e = ga_init_attributes();
  if (e == cudaSuccess) e = tc_init_attributes();
  if (e == cudaSuccess) e = simt_init_attributes();
  if (e == cudaSuccess) e = otf_tc_init_attributes();
  if (e == cudaSuccess) e = batch_init_attributes();
  if (e == cudaSuccess) e = surrogate_ga_init_attributes();
  if (e == cudaSuccess) e = surrogate_tc_init_attributes();
  if (e != cudaSuccess) {
    delete c;
    return fail(nullptr, GAME_ERR_CUDA, "kernel attributes: %s", cudaGetErrorString(e));
  }
  *out = c;
  return GAME_OK;
}

extern "C" void game_destroy(game_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->dev);
  cudaStreamSynchronize(c->st);
  free_all(c);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  for (cudaEvent_t e : c->copy_ev) cudaEventDestroy(e);
  if (c->st_copy) cudaStreamDestroy(c->st_copy);
  if (c->st_sg) {
    cudaStreamSynchronize(c->st_sg);
    cudaStreamDestroy(c->st_sg);
    cudaEventDestroy(c->ev_sg[0]);
    cudaEventDestroy(c->ev_sg[1]);
  }
  delete c;
}

extern "C" const char* game_last_error(const game_ctx* c) {
  return c ? c->err.c_str() : g_global_err.c_str();
}

extern "C" int32_t game_n_genes(const game_ctx* c) {
  return (c && c->have_data) ? c->s.n_genes : 0;
}

__global__ void check_data_kernel(const float* X, long long nx, const float* t, long long nt,
                                  long long n_train, unsigned int* flags) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  unsigned int bad = 0, notpm1 = 0;
  for (long long k = i; k < nx; k += stride) bad |= !isfinite(X[k]);
  for (long long k = i; k < nt; k += stride) {
    bad |= !isfinite(t[k]);
    if (k < n_train) notpm1 |= !(t[k] == 1.0f || t[k] == -1.0f);
  }
  if (bad) atomicOr(flags, 1u);
  if (notpm1) atomicOr(flags, 2u);
}

// ---- tile cache of the autotuner: one line per shape bucket -------------------
//   <kp> <pop_pad> <precision> <log2 n_train> <n> <stages> <cluster> <prefetch> <slices> <ms>
// (lines of any other form are skipped)
static std::string tune_cache_path() {
  const char* e = getenv("GAME_TUNE_CACHE");
  if (e && *e) return e;
  const char* h = getenv("HOME");
  return std::string(h && *h ? h : "/tmp") + "/.cache/game_gb300_tiles.txt";
}

static int ntrain_bucket(long long n) { return (int)floor(log2((double)(n > 0 ? n : 1))); }

static bool tune_cache_lookup(const Shape& s, TileReq* out) {
  FILE* f = fopen(tune_cache_path().c_str(), "r");
  if (!f) return false;
  int kp, pp, pr, nb, n, st, cl, pf, sp, kg;
  double ms;
  bool found = false;
  char line[256];
  while (fgets(line, sizeof(line), f))
    if (sscanf(line, "%d %d %d %d %d %d %d %d %d %d %lf", &kp, &pp, &pr, &nb, &n, &st, &cl, &pf,
               &sp, &kg, &ms) == 11 &&
        kp == s.kp && pp == s.pop_pad && pr == s.precision && nb == ntrain_bucket(s.n_train)) {
      *out = TileReq{n, st, cl, pf, sp, kg};   // the last record for a bucket wins
      found = true;
    }
  fclose(f);
  return found;
}

static void tune_cache_store(const Shape& s, const game_tile& t) {
  const std::string path = tune_cache_path();
  const size_t slash = path.rfind('/');
  if (slash != std::string::npos && slash > 0) mkdir(path.substr(0, slash).c_str(), 0755);
  FILE* f = fopen(path.c_str(), "a");
  if (!f) return;
  fprintf(f, "%d %d %d %d %d %d %d %d %d %d %.6f\n", s.kp, s.pop_pad, s.precision,
          ntrain_bucket(s.n_train), t.n, t.stages, t.cluster, t.prefetch, t.slices, t.kgroup, t.ms);
  fclose(f);
}

static game_status choose_engine(game_ctx* c, Shape& s, const ExpDev& e, const PopDev& p,
                                 int* engine, TcPlan* plan, int* n_part) {
  if (c->otf) {
    *engine = GAME_ENGINE_ON_THE_FLY;
    // the tensor-core form where it takes the shape (FP32, per-feature coefficients,
    // the gene planes and two ring stages in shared memory), else the CUDA-core one
    c->otf_tc_ok = otf_tc_supported(s) && otf_tc_plan(s, p, c->n_sm, &c->otf_tc) == cudaSuccess;
    if (!c->otf_tc_ok) cudaGetLastError();
    *n_part = c->otf_tc_ok ? c->otf_tc.cps : otf_partials(s, c->n_sm);
    return GAME_OK;
  }
  int want = c->cfg.engine;
  // Automatic: the narrow SIMT kernel for at most 32 chromosomes on 16 or 32 stored
  // columns (the paper's own settings); otherwise the tensor cores where a kernel
  // keeps the genes resident, else SIMT.  Among the tensor-core kernels the swapped
  // one (patterns on M) takes an FP32 population of at most 32 when the tensor cores
  // are asked for by name, or when the 128-chromosome kernel cannot hold the genes;
  // for the automatic choice (the 16-elite re-score) the 128-chromosome kernel
  // measured faster (c2: 0.157 against 0.199 ms for re-score and rank).
  const bool tc_ok = tc_narrow_fits(s) || tc_supported(s);
  if (want == GAME_ENGINE_AUTO)
    want = simt_narrow(s) || !tc_ok ? GAME_ENGINE_SIMT : GAME_ENGINE_TCGEN05;
  s.tc_narrow = want == GAME_ENGINE_TCGEN05 && tc_narrow_fits(s) &&
                (c->cfg.engine == GAME_ENGINE_TCGEN05 || !tc_supported(s));
  if (want == GAME_ENGINE_TCGEN05) {
    if (!tc_ok)
      return fail(c, GAME_ERR_UNSUPPORTED, "tcgen05 engine does not support this shape");
    TileReq req{c->cfg.tile_n,      c->cfg.tile_stages, c->cfg.tile_cluster, -1,
                c->cfg.tile_slices, c->cfg.tile_kgroup};
    if (!req.n && !req.stages && !req.cluster && !req.sp && !req.kg) tune_cache_lookup(s, &req);
    cudaError_t err = tc_plan(s, e, p, c->n_sm, plan, req);
    if (err != cudaSuccess) {
      cudaGetLastError();
      err = tc_plan(s, e, p, c->n_sm, plan);   // a stale cache entry falls back to the default
    }
    if (err != cudaSuccess) return fail(c, GAME_ERR_CUDA, "tcgen05 plan: %s", cudaGetErrorString(err));
    *engine = GAME_ENGINE_TCGEN05;
    *n_part = plan->n_part;
  } else {
    *engine = GAME_ENGINE_SIMT;
    *n_part = simt_partials(s, c->n_sm);
  }
  return GAME_OK;
}

__global__ void fill_f32_kernel(float* p, long long n, float v) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

// Network, pool, replay ring and training buffers of the surrogate.
static game_status alloc_surrogate(game_ctx* c) {
  const Shape& s = c->s;
  c->sg_steps = c->cfg.surrogate_steps > 0 ? c->cfg.surrogate_steps : 6;
  c->sg_batch = c->cfg.surrogate_batch > 0 ? c->cfg.surrogate_batch : 1024;
  c->sg_lr = c->cfg.surrogate_lr > 0.0f ? c->cfg.surrogate_lr : 2e-3f;
  const int e = c->cfg.elitism < s.pop ? c->cfg.elitism : s.pop;
  const int m = c->cfg.surrogate_pool > 0 ? c->cfg.surrogate_pool : 1;
  c->n_pool = m * (s.pop - e);
  if (c->n_pool < 1) c->n_pool = 1;
  // the replay ring holds the latest evaluated population (at least one batch):
  // older generations' pairs describe a landscape the GA has left
  c->ring_cap = std::max(s.pop, c->sg_batch);
  Surrogate& sg = c->sg;
  sg = Surrogate{};
  sg.D = s.n_genes;
  sg.H = 256;
  sg.bf16 = c->cfg.surrogate_fp32 == 0;
  sg.max_rows = std::max(c->n_pool, c->sg_batch);
  const size_t np = sg.n_params();
  game_status r;
  // bfloat16 weights run on the tensor cores and need none of the float32
  // activation planes of the SIMT path
  const bool use_tc = sg.bf16;
  const size_t act = use_tc ? 1 : (size_t)sg.max_rows * sg.H;
  if ((r = dalloc(c, &sg.p, sizeof(float) * np)) != GAME_OK) return r;
  if ((r = dalloc(c, &sg.g, sizeof(float) * np)) != GAME_OK) return r;
  if ((r = dalloc(c, &sg.m, sizeof(float) * np)) != GAME_OK) return r;
  if ((r = dalloc(c, &sg.v, sizeof(float) * np)) != GAME_OK) return r;
  if ((r = dalloc(c, &sg.ph, sizeof(__nv_bfloat16) * np)) != GAME_OK) return r;
  if ((r = dalloc(c, &sg.step, sizeof(int))) != GAME_OK) return r;
  if ((r = dalloc(c, &sg.Z1, sizeof(float) * act)) != GAME_OK) return r;
  if ((r = dalloc(c, &sg.H1, sizeof(float) * act)) != GAME_OK) return r;
  if ((r = dalloc(c, &sg.Z2, sizeof(float) * act)) != GAME_OK) return r;
  if ((r = dalloc(c, &sg.H2, sizeof(float) * act)) != GAME_OK) return r;
  if ((r = dalloc(c, &sg.dZ1, sizeof(float) * act)) != GAME_OK) return r;
  if ((r = dalloc(c, &sg.dZ2, sizeof(float) * act)) != GAME_OK) return r;
  if ((r = dalloc(c, &sg.yb, sizeof(float) * sg.max_rows)) != GAME_OK) return r;
  if ((r = dalloc(c, &sg.dy, sizeof(float) * sg.max_rows)) != GAME_OK) return r;
  if ((r = dalloc(c, &sg.sq, sizeof(float) * sg.max_rows)) != GAME_OK) return r;
  if ((r = dalloc(c, &sg.loss, sizeof(float))) != GAME_OK) return r;
  if ((r = dalloc(c, &sg.ws, sizeof(float) * (use_tc ? 1 : 16 * (size_t)sg.H * std::max(sg.D, sg.H)))) != GAME_OK)
    return r;
  if (use_tc) {
    uint8_t* tcbuf = nullptr;
    if ((r = dalloc(c, &tcbuf, sg.tc_bytes(sg.max_rows, c->sg_batch))) != GAME_OK) return r;
    sg.state = c->d_state;
    sg.tc_carve(tcbuf, c->sg_batch);
    if (!c->st_sg) {
      CUDA_OK(c, cudaStreamCreateWithFlags(&c->st_sg, cudaStreamNonBlocking));
      CUDA_OK(c, cudaEventCreateWithFlags(&c->ev_sg[0], cudaEventDisableTiming));
      CUDA_OK(c, cudaEventCreateWithFlags(&c->ev_sg[1], cudaEventDisableTiming));
    }
    sg.side = c->st_sg;
    sg.ev_fork = c->ev_sg[0];
    sg.ev_join = c->ev_sg[1];
  }
  if ((r = dalloc(c, &c->d_pool, sizeof(float) * (size_t)c->n_pool * s.kstride)) != GAME_OK) return r;
  if ((r = dalloc(c, &c->d_score, sizeof(float) * c->n_pool)) != GAME_OK) return r;
  if ((r = dalloc(c, &c->d_sel, sizeof(int) * s.pop_pad)) != GAME_OK) return r;
  if ((r = dalloc(c, &c->d_pred, sizeof(float) * s.pop_pad)) != GAME_OK) return r;
  if ((r = dalloc(c, &c->d_fallback, sizeof(int))) != GAME_OK) return r;
  if ((r = dalloc(c, &c->d_ring_x, sizeof(float) * (size_t)c->ring_cap * s.kstride)) != GAME_OK) return r;
  if ((r = dalloc(c, &c->d_ring_f, sizeof(float) * c->ring_cap)) != GAME_OK) return r;
  if ((r = dalloc(c, &c->d_ring_meta, sizeof(int) * 8)) != GAME_OK) return r;
  if ((r = dalloc(c, &c->d_norm, sizeof(float) * 2)) != GAME_OK) return r;
  if ((r = dalloc(c, &c->d_dsq, sizeof(long long) * s.pop_pad)) != GAME_OK) return r;
  if ((r = dalloc(c, &c->d_monitor, sizeof(double) * 4096)) != GAME_OK) return r;
  if ((r = dalloc(c, &c->d_bx, sizeof(float) * (size_t)c->sg_batch * s.kstride)) != GAME_OK) return r;
  if ((r = dalloc(c, &c->d_bt, sizeof(float) * c->sg_batch)) != GAME_OK) return r;
  fill_f32_kernel<<<(s.pop_pad + 255) / 256, 256, 0, c->st>>>(c->d_pred, s.pop_pad, NAN);
  const int meta[8] = {0, 0, -1, 0, 0, 0, 0, 0};
  CUDA_OK(c, cudaMemcpyAsync(c->d_ring_meta, meta, sizeof(meta), cudaMemcpyHostToDevice, c->st));
  const float norm[2] = {0.0f, 1.0f};
  CUDA_OK(c, cudaMemcpyAsync(c->d_norm, norm, sizeof(norm), cudaMemcpyHostToDevice, c->st));
  CUDA_OK(c, launch_surrogate_init(sg, c->cfg.seed ^ 0x53ull, c->st));
  if (sg.tc) CUDA_OK(c, sg.tc_prepare(c->st));
  CUDA_OK(c, cudaStreamSynchronize(c->st));
  c->sg_alloc = true;
  return GAME_OK;
}

extern "C" game_status game_set_data(game_ctx* c, const float* X, const float* t,
                                     int64_t n_patterns, int32_t n_features, int64_t n_train,
                                     int32_t device_ptrs) {
  if (!c) return fail(nullptr, GAME_ERR_INVALID_ARG, "ctx is NULL");
  if (!X || !t) return fail(c, GAME_ERR_INVALID_ARG, "X and t must be non-NULL");
  if (n_patterns < 1 || n_features < 1 || n_train < 1 || n_train > n_patterns)
    return fail(c, GAME_ERR_INVALID_ARG,
                "need n_patterns >= 1, n_features >= 1, 1 <= n_train <= n_patterns");
  cudaSetDevice(c->dev);
  const int B = c->cfg.basis == GAME_TRIG ? 2 : 1;
  const int shared = c->cfg.coefficients == GAME_COEF_SHARED;
  const long long kb = (long long)B * (shared ? 1 : n_features) * c->cfg.degree;
  if (kb > 4096)
    return fail(c, GAME_ERR_UNSUPPORTED, "%lld basis columns exceed 4096", kb);
  reuse_blocks(c);
  Shape& s = c->s;
  s.n_patterns = n_patterns;
  s.n_train = n_train;
  s.n_features = n_features;
  s.degree = c->cfg.degree;
  s.basis = c->cfg.basis;
  s.bd = B * c->cfg.degree;
  s.shared = shared;
  s.kb = (int)kb;
  s.kp = round_up(s.kb, c->cfg.precision == GAME_FP8 ? 32 : 16);
  s.n_genes = s.kb + 1;
  s.kstride = round_up(s.n_genes, 4);
  s.pop = c->cfg.pop;
  s.pop_pad = round_up(s.pop, 128);
  s.precision = c->cfg.precision;
  s.gene_planes = (s.precision == GAME_FP32 || c->cfg.gene_planes != 1) ? 2 : 1;
  c->fit.error = c->cfg.error;
  c->fit.activation = c->cfg.activation;
  c->fit.tmse_R = c->cfg.tmse_R;

  game_status r;
  // Knowledge base on the device.
  float* dX = nullptr;
  const size_t xbytes = sizeof(float) * (size_t)n_patterns * n_features;
  if ((r = dalloc(c, &dX, xbytes)) != GAME_OK) return r;
  const long long tpad = (n_patterns + 255) / 256 * 256 + 256;
  if ((r = dalloc(c, &c->e.t, sizeof(float) * tpad)) != GAME_OK) return r;
  unsigned int* dflags = nullptr;
  if ((r = dalloc(c, &dflags, sizeof(unsigned int))) != GAME_OK) return r;
  unsigned int* dfmax = nullptr;   // per-feature max |x| (float bits)
  if ((r = dalloc(c, &dfmax, sizeof(unsigned int) * n_features)) != GAME_OK) return r;
  if ((r = dalloc(c, &c->e.tcoef, sizeof(float) * tpad)) != GAME_OK) return r;
  c->d_X = dX;
  const size_t esz = s.precision == GAME_FP32 ? 2 : (s.precision == GAME_BF16 ? 2 : 1);
  const size_t pbytes = esz * (size_t)n_patterns * s.kp;
  // On-the-fly engine: P is never stored.  Asked for by name, or chosen automatically
  // in the FP32 form when the stored planes would not fit in the device's free memory
  // (measured slower than the stored engines wherever P fits).
  const size_t stored = pbytes * (s.precision == GAME_FP32 ? 2 : 3);   // + the FP32 copy
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    free_b = (size_t)-1;
  }
  c->otf = c->cfg.engine == GAME_ENGINE_ON_THE_FLY ||
           (c->cfg.engine == GAME_ENGINE_AUTO && s.precision == GAME_FP32 &&
            c->cfg.surrogate_pool == 0 && (double)stored > 0.85 * (double)free_b);
  if (c->otf && (s.precision != GAME_FP32 || c->cfg.surrogate_pool > 0)) {
    free_all(c);
    return fail(c, GAME_ERR_UNSUPPORTED,
                "the on-the-fly engine takes the FP32 form without the surrogate");
  }
  if (!c->otf) {
    if ((r = dalloc(c, &c->e.p0, pbytes)) != GAME_OK) return r;
    if (s.precision == GAME_FP32) {
      if ((r = dalloc(c, &c->e.p1, pbytes)) != GAME_OK) return r;
    }
  } else {
    c->e.p0 = c->e.p1 = nullptr;
  }
  if ((r = dalloc(c, &c->e.colscale, sizeof(float) * s.kp)) != GAME_OK) return r;
  if ((r = dalloc(c, &c->d_scratch, sizeof(float) * s.kp)) != GAME_OK) return r;
  // FP32 planes start unscaled; out-of-range Chebyshev columns get scales below.
  c->e.unit_scale32 = 1;
  if (s.precision == GAME_FP32) CUDA_OK(c, launch_fill_ones(c->e.colscale, s.kp, c->st));
  CUDA_OK(c, cudaMemcpyAsync(c->e.t, t, sizeof(float) * n_patterns,
                             device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->st));

  // Expansion matrix (Section 4.1: computed once, reused every generation).  From
  // host memory in the FP32 form, X comes over in chunks on a copy stream and each
  // chunk is expanded as soon as it lands (the rows are independent); the
  // quantised forms need the column maxima of all rows first.
  if (!device_ptrs && s.precision == GAME_FP32 && !c->otf) {
    if (!c->st_copy) CUDA_OK(c, cudaStreamCreateWithFlags(&c->st_copy, cudaStreamNonBlocking));
    const long long chunk = std::max<long long>(65536, ((long long)n_patterns + 7) / 8);
    const int n_chunks = (int)((n_patterns + chunk - 1) / chunk);
    while ((int)c->copy_ev.size() < n_chunks) {
      cudaEvent_t e;
      CUDA_OK(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      c->copy_ev.push_back(e);
    }
    // the copy stream starts after this call's earlier work (the block memsets)
    CUDA_OK(c, cudaEventRecord(c->copy_ev[0], c->st));
    CUDA_OK(c, cudaStreamWaitEvent(c->st_copy, c->copy_ev[0], 0));
    for (int i = 0; i < n_chunks; ++i) {
      const long long r0 = i * chunk;
      const long long nr = std::min<long long>(chunk, (long long)n_patterns - r0);
      CUDA_OK(c, cudaMemcpyAsync(dX + r0 * n_features, X + r0 * n_features,
                                 sizeof(float) * (size_t)nr * n_features, cudaMemcpyHostToDevice,
                                 c->st_copy));
      CUDA_OK(c, cudaEventRecord(c->copy_ev[i], c->st_copy));
      CUDA_OK(c, cudaStreamWaitEvent(c->st, c->copy_ev[i], 0));
      Shape sc = s;
      sc.n_patterns = nr;
      ExpDev ec = c->e;
      ec.p0 = static_cast<__half*>(c->e.p0) + r0 * s.kp;
      ec.p1 = static_cast<__half*>(c->e.p1) + r0 * s.kp;
      CUDA_OK(c, launch_expand(dX + r0 * n_features, sc, ec, c->d_scratch, c->st));
    }
  } else {
    CUDA_OK(c, cudaMemcpyAsync(dX, X, xbytes,
                               device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                               c->st));
  }
  check_data_kernel<<<4 * c->n_sm, 256, 0, c->st>>>(dX, n_patterns * n_features, c->e.t,
                                                      n_patterns, n_train, dflags);
  CUDA_OK(c, cudaGetLastError());
  const bool cheb = s.basis == GAME_CHEBYSHEV;
  std::vector<float> fmax(cheb ? n_features : 0);
  if (cheb) {
    CUDA_OK(c, launch_feature_absmax(dX, n_patterns, n_features, dfmax, c->n_sm, c->st));
    CUDA_OK(c, cudaMemcpyAsync(fmax.data(), dfmax, sizeof(float) * n_features,
                               cudaMemcpyDeviceToHost, c->st));
  }
  unsigned int flags = 0;
  CUDA_OK(c, cudaMemcpyAsync(&flags, dflags, sizeof(flags), cudaMemcpyDeviceToHost, c->st));
  CUDA_OK(c, cudaStreamSynchronize(c->st));
  if (flags & 1u) {
    free_all(c);
    return fail(c, GAME_ERR_NUMERIC, "X or t holds NaN or Inf");
  }
  // Chebyshev values grow without bound outside [-1, 1] (eq.1 bounds no feature):
  // |T_j(x)| <= T_j(max(1, |x|)) = cosh(j acosh max(1, |x|)).  Columns whose bound
  // passes 2^15 get a power-of-two scale in the FP32 planes (fp16 tops out at 65504);
  // values beyond float32 are refused.
  c->scale32.assign(s.kp, 1.0f);
  bool scaled = false;
  if (cheb) {
    std::vector<double> bound(s.kb, 0.0);
    for (int f = 0; f < n_features; ++f) {
      const double a = std::max(1.0, (double)fmax[f]);
      for (int b = 0; b < s.degree; ++b) {
        const double v = a == 1.0 ? 1.0 : std::cosh((b + 1) * std::acosh(a));
        if (!(v < 0x1p100)) {
          free_all(c);
          return fail(c, GAME_ERR_UNSUPPORTED,
                      "feature %d reaches |x| = %g: T_%d there exceeds 2^100 (rescale the feature)",
                      f, (double)fmax[f], b + 1);
        }
        bound[shared ? b : f * s.degree + b] += v;
      }
    }
    for (int col = 0; col < s.kb; ++col) {
      int ex = 0;
      std::frexp(bound[col], &ex);                   // bound < 2^ex
      if (ex > 15) {
        c->scale32[col] = std::ldexp(1.0f, ex - 15);
        scaled = true;
      }
    }
  }
  c->fit.pm1_targets = (flags & 2u) ? 0 : 1;
  CUDA_OK(c, launch_target_coef(c->e.t, c->e.tcoef, n_patterns, c->st));
  if (scaled && s.precision == GAME_FP32) {
    CUDA_OK(c, cudaMemcpyAsync(c->e.colscale, c->scale32.data(), sizeof(float) * s.kp,
                               cudaMemcpyHostToDevice, c->st));
    c->e.unit_scale32 = 0;
  }
  // (the host chunks of the FP32 form were expanded unscaled as they landed)
  if ((device_ptrs || s.precision != GAME_FP32 || scaled) && !c->otf)
    CUDA_OK(c, launch_expand(dX, s, c->e, c->d_scratch, c->st));
  c->lowp = s.precision != GAME_FP32;
  c->s32 = s;
  c->e32 = c->e;
  if (c->lowp) {
    // The FP32 planes serve the elite re-score and the float64 report.
    c->s32.precision = GAME_FP32;
    c->s32.gene_planes = 2;
    c->s32.kp = round_up(s.kb, 16);
    c->e32 = ExpDev{};
    c->e32.t = c->e.t;
    c->e32.tcoef = c->e.tcoef;
    const size_t b32 = sizeof(__half) * (size_t)n_patterns * c->s32.kp;
    if ((r = dalloc(c, &c->e32.p0, b32)) != GAME_OK) return r;
    if ((r = dalloc(c, &c->e32.p1, b32)) != GAME_OK) return r;
    if ((r = dalloc(c, &c->e32.colscale, sizeof(float) * c->s32.kp)) != GAME_OK) return r;
    c->scale32.resize(c->s32.kp, 1.0f);
    c->e32.unit_scale32 = scaled ? 0 : 1;
    CUDA_OK(c, cudaMemcpyAsync(c->e32.colscale, c->scale32.data(), sizeof(float) * c->s32.kp,
                               cudaMemcpyHostToDevice, c->st));
    CUDA_OK(c, launch_expand(dX, c->s32, c->e32, c->d_scratch, c->st));
  }

  // Population buffers.
  const size_t g32b = sizeof(float) * (size_t)s.pop_pad * s.kstride;
  for (int i = 0; i < 2; ++i)
    if ((r = dalloc(c, &c->p.g32[i], g32b)) != GAME_OK) return r;
  c->p.pop_rows = s.pop;
  if ((r = dalloc(c, &c->p.geval, sizeof(float) * (size_t)s.pop_pad * s.kp)) != GAME_OK) return r;
  if ((r = dalloc(c, &c->p.bias, sizeof(float) * s.pop_pad)) != GAME_OK) return r;
  if ((r = dalloc(c, &c->p.rscale, sizeof(float) * s.pop_pad)) != GAME_OK) return r;
  const size_t gpl = esz * (size_t)s.pop_pad * s.kp;
  if ((r = dalloc(c, &c->p.ghi, gpl)) != GAME_OK) return r;
  if ((r = dalloc(c, &c->p.glo, gpl)) != GAME_OK) return r;
  if ((r = dalloc(c, &c->d_fit, sizeof(double) * s.pop_pad)) != GAME_OK) return r;
  if ((r = dalloc(c, &c->d_rank, sizeof(int) * s.pop_pad)) != GAME_OK) return r;
  if ((r = dalloc(c, &c->d_cum, sizeof(unsigned long long) * s.pop_pad)) != GAME_OK) return r;
  if ((r = dalloc(c, &c->d_state, sizeof(DevState))) != GAME_OK) return r;
  if ((r = dalloc(c, &c->d_genes, sizeof(float) * (size_t)s.kstride)) != GAME_OK) return r;
  c->score_nb = score_blocks(n_patterns, c->n_sm);
  if ((r = dalloc(c, &c->d_score_blocks, sizeof(double) * 5 * c->score_nb)) != GAME_OK) return r;
  if ((r = dalloc(c, &c->d_score_out, sizeof(double) * 8)) != GAME_OK) return r;

  if ((r = choose_engine(c, s, c->e, c->p, &c->engine, &c->tc, &c->n_part)) != GAME_OK) {
    free_all(c);
    return r;
  }
  // Any tile shape uses at most one partial row per SM.
  c->part_rows = std::max(std::max(c->n_part, simt_partials(s, c->n_sm)), c->n_sm);
  if (c->otf) c->part_rows = std::max(c->part_rows, otf_partials(s, c->n_sm));
  if ((r = dalloc(c, &c->d_partial, sizeof(double) * (size_t)c->part_rows * s.pop_pad)) != GAME_OK)
    return r;
  c->n_rescore = 0;
  if (c->lowp && c->cfg.elite_rescore > 0) {
    c->n_rescore = c->cfg.elite_rescore < s.pop ? c->cfg.elite_rescore : s.pop;
    if (c->n_rescore > 128) c->n_rescore = 128;
    c->sr = c->s32;
    c->sr.pop = c->n_rescore;
    c->sr.pop_pad = 128;
    c->pr = PopDev{};
    c->pr.g32[0] = c->p.g32[0];
    c->pr.g32[1] = c->p.g32[1];
    c->pr.pop_rows = s.pop;
    if ((r = dalloc(c, &c->pr.geval, sizeof(float) * 128 * (size_t)c->sr.kp)) != GAME_OK) return r;
    if ((r = dalloc(c, &c->pr.bias, sizeof(float) * 128)) != GAME_OK) return r;
    if ((r = dalloc(c, &c->pr.rscale, sizeof(float) * 128)) != GAME_OK) return r;
    if ((r = dalloc(c, &c->pr.ghi, sizeof(__half) * 128 * (size_t)c->sr.kp)) != GAME_OK) return r;
    if ((r = dalloc(c, &c->pr.glo, sizeof(__half) * 128 * (size_t)c->sr.kp)) != GAME_OK) return r;
    if ((r = choose_engine(c, c->sr, c->e32, c->pr, &c->engine_r, &c->tc_r, &c->n_part_r)) != GAME_OK) {
      free_all(c);
      return r;
    }
    // any tile shape of one slice uses at most one partial row per SM
    const int rows = std::max(std::max(c->n_part_r, simt_partials(c->sr, c->n_sm)), c->n_sm);
    c->part_rows_r = rows;
    if ((r = dalloc(c, &c->d_partial_r, sizeof(double) * (size_t)rows * 128)) != GAME_OK) return r;
  }

  c->sg_alloc = false;
  if (c->cfg.surrogate_pool > 0) {
    if ((r = alloc_surrogate(c)) != GAME_OK) {
      free_all(c);
      return r;
    }
  }
  CUDA_OK(c, launch_state_op(c->d_state, kStateReset, c->st));
  CUDA_OK(c, launch_init_population(s, c->cfg.init, c->cfg.seed, c->cfg.run, c->p.g32[0], c->st));
  CUDA_OK(c, cudaStreamSynchronize(c->st));
  // The blocks of a longer earlier sequence are not needed.  X stays allocated (it
  // is no longer read once P exists) for the next data set of the same shape.
  release_tail(c);
  if ((r = collect_checks(c)) != GAME_OK) return r;
  c->have_data = true;
  return GAME_OK;
}

// Launch the fitness of the prepared population into the partial-sum buffer.
static game_status launch_fitness(game_ctx* c, const DevState* state) {
  if (c->engine == GAME_ENGINE_TCGEN05) {
    CUDA_OK(c, tc_launch(c->tc, c->s, c->fit, c->p, c->e, c->d_partial, state, c->st));
  } else if (c->engine == GAME_ENGINE_ON_THE_FLY && c->otf_tc_ok) {
    CUDA_OK(c, otf_tc_launch(c->otf_tc, c->s, c->fit, c->p, c->e, c->d_X, c->d_partial, c->d_state,
                             state != nullptr, c->st));
  } else if (c->engine == GAME_ENGINE_ON_THE_FLY) {
    CUDA_OK(c, launch_fitness_otf(c->s, c->fit, c->p, c->d_X, c->e, c->d_partial, c->n_part, state,
                                  c->st));
  } else {
    CUDA_OK(c, launch_fitness_simt(c->s, c->fit, c->p, c->e, c->d_partial, c->n_part, state,
                                   c->d_state, c->st));
  }
  return GAME_OK;
}

// Precision form: the top n_rescore chromosomes of the ranking just made are
// re-evaluated on the FP32 planes, their fitness replaced, and the population
// re-sorted (with the stop test on the re-scored best).
static game_status enqueue_rescore(game_ctx* c, int in_evolve) {
  const DevState* st = in_evolve ? c->d_state : nullptr;
  CUDA_OK(c, launch_prepare(c->sr, c->pr, c->e32, c->d_state, in_evolve ? 2 : 0, c->st, c->d_rank,
                            &c->p));
  if (c->engine_r == GAME_ENGINE_TCGEN05) {
    CUDA_OK(c, tc_launch(c->tc_r, c->sr, c->fit, c->pr, c->e32, c->d_partial_r, st, c->st));
  } else {
    CUDA_OK(c, launch_fitness_simt(c->sr, c->fit, c->pr, c->e32, c->d_partial_r, c->n_part_r, st,
                                   c->d_state, c->st));
  }
  CUDA_OK(c, launch_rescore_merge(c->sr, c->cfg, c->d_partial_r, c->n_part_r, c->d_rank, c->d_fit,
                                  c->d_state, in_evolve, c->st));
  CUDA_OK(c, launch_reduce_rank(c->s, c->cfg, nullptr, 0, c->d_fit, c->d_rank, c->d_state,
                                kRankResort | (in_evolve ? kRankInEvolve : 0), c->st));
  return GAME_OK;
}

// One generation: breed (if the current population was evaluated), prepare,
// fitness, reduce + rank.  Reads and writes only device state.
// Generation steps before the fitness launch: breed (if the current population
// was evaluated) and the operand planes of the population to evaluate.
static game_status enqueue_pre(game_ctx* c, cudaStream_t st) {
  if (c->cfg.surrogate_pool > 0) {
    // Oversized pool, scored by the surrogate; its best children (or plain ones
    // under the fallback / the ablation) form the next population.
    PoolArgs pa;
    pa.g32_0 = c->p.g32[0];
    pa.g32_1 = c->p.g32[1];
    pa.pool = c->d_pool;
    pa.fit = c->d_fit;
    pa.rank = c->d_rank;
    pa.state = c->d_state;
    pa.k0 = c->cfg.seed;
    pa.k1 = c->cfg.run;
    pa.pop = c->s.pop;
    pa.n_genes = c->s.n_genes;
    pa.kstride = c->s.kstride;
    pa.n_pool = c->n_pool;
    pa.tournament_k = c->cfg.tournament_k;
    pa.clamp = c->cfg.clamp_genes;
    pa.p_c = c->cfg.p_crossover;
    pa.p_m = c->cfg.p_mutation;
    pa.sigma = c->cfg.sigma_mutation;
    const int e = std::min(c->cfg.elitism, c->s.pop);
    pa.cum = c->cfg.selection != GAME_SEL_TOURNAMENT ? c->d_cum : nullptr;
    CUDA_OK(c, launch_selection_weights(c->cfg, c->s, c->d_fit, c->d_rank, c->d_cum, st));
    CUDA_OK(c, launch_pool_breed(pa, st));
    CUDA_OK(c, c->sg.forward(c->d_pool, c->s.kstride, c->n_pool, c->d_score, st));
    CUDA_OK(c, launch_select(c->d_score, c->n_pool, c->s.pop - e, c->d_sel, c->d_state,
                             c->d_fallback, c->cfg.surrogate_select, st));
    CUDA_OK(c, launch_assemble(c->d_pool, c->d_sel, c->d_score, c->p, c->s, e,
                               c->cfg.elite_mode == GAME_ELITE_COPIES, c->d_rank, c->d_state,
                               c->d_pred, st));
    CUDA_OK(c, launch_immigrants(c->s, c->cfg, c->p, c->d_state, st));
  } else {
    CUDA_OK(c, launch_breed(c->s, c->cfg, c->p, c->d_fit, c->d_rank, c->d_state, 1 | 2, st, c->d_cum));
  }
  CUDA_OK(c, launch_prepare(c->s, c->p, c->e, c->d_state, 1 | 2, st));
  return GAME_OK;
}

// After an exact evaluation: replay ring, monitor, and the generation's training.
static game_status enqueue_surrogate_train(game_ctx* c, cudaStream_t st) {
  if (c->sg.tc) CUDA_OK(c, launch_gene_stats(c->p, c->s, c->d_state, c->d_ring_meta, c->sg, st));
  CUDA_OK(c, launch_replay_update(c->p, c->s, std::min(c->cfg.elitism, c->s.pop), c->d_fit,
                                  c->d_pred, c->d_state, c->d_ring_x, c->d_ring_f, c->d_ring_meta,
                                  c->ring_cap, c->d_norm, c->d_monitor, c->d_fallback, 0.1f,
                                  c->d_dsq, st));
  for (int k = 0; k < c->sg_steps; ++k) {
    if (c->sg.tc) {
      // bf16 form: the batch goes straight into the tensor-core operands
      CUDA_OK(c, launch_sample_batch_tc(c->d_ring_x, c->d_ring_f, c->d_ring_meta, c->s.kstride,
                                        c->sg, c->sg_batch, c->cfg.seed, c->cfg.run,
                                        0x51ull << 32, k, c->d_state, c->d_bt, st));
      CUDA_OK(c, c->sg.tc_train_step(c->sg_batch, c->d_bt, c->sg_lr, st));
      continue;
    }
    CUDA_OK(c, launch_sample_batch(c->d_ring_x, c->d_ring_f, c->d_ring_meta, c->s.kstride,
                                   c->s.n_genes, c->d_norm, c->sg_batch, c->cfg.seed, c->cfg.run,
                                   0x51ull << 32, k, c->d_state, c->d_bx, c->d_bt, st));
    CUDA_OK(c, c->sg.backward(c->d_bx, c->s.kstride, c->sg_batch, c->d_bt, st));
    CUDA_OK(c, c->sg.adam(c->sg_lr, st));
  }
  return GAME_OK;
}

// Generation steps after the fitness launch: reduce + rank (+ FP32 re-score).
static game_status enqueue_post(game_ctx* c, int n_part, cudaStream_t st) {
  const cudaStream_t saved = c->st;
  c->st = st;
  game_status r = GAME_OK;
  cudaError_t e = launch_reduce_rank(c->s, c->cfg, c->d_partial, n_part, c->d_fit, c->d_rank,
                                     c->d_state,
                                     kRankEvaluate | kRankInEvolve | (c->n_rescore ? kRankNoStop : 0),
                                     st);
  if (e != cudaSuccess) r = fail(c, GAME_ERR_CUDA, "reduce_rank: %s", cudaGetErrorString(e));
  if (r == GAME_OK && c->n_rescore) r = enqueue_rescore(c, 1);
  if (r == GAME_OK && c->cfg.surrogate_pool > 0) r = enqueue_surrogate_train(c, st);
  c->st = saved;
  return r;
}

static game_status enqueue_generation(game_ctx* c, const cudaEvent_t* ev) {
  if (ev) CUDA_OK(c, cudaEventRecordWithFlags(ev[0], c->st, cudaEventRecordExternal));
  game_status r = enqueue_pre(c, c->st);
  if (r != GAME_OK) return r;
  if (ev) CUDA_OK(c, cudaEventRecordWithFlags(ev[1], c->st, cudaEventRecordExternal));
  r = launch_fitness(c, c->d_state);
  if (r != GAME_OK) return r;
  if (ev) CUDA_OK(c, cudaEventRecordWithFlags(ev[2], c->st, cudaEventRecordExternal));
  r = enqueue_post(c, c->n_part, c->st);
  if (r != GAME_OK) return r;
  if (ev) CUDA_OK(c, cudaEventRecordWithFlags(ev[3], c->st, cudaEventRecordExternal));
  return GAME_OK;
}

// Kernel nodes of a captured generation: the kernels one replay launches.
static int count_kernel_nodes(cudaGraph_t g) {
  size_t n = 0;
  if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess) return -1;
  std::vector<cudaGraphNode_t> nodes(n);
  if (cudaGraphGetNodes(g, nodes.data(), &n) != cudaSuccess) return -1;
  int k = 0;
  for (cudaGraphNode_t nd : nodes) {
    cudaGraphNodeType ty;
    if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++k;
  }
  return k;
}

static game_status ensure_events(game_ctx* c, size_t n) {
  while (c->ev_pool.size() < n) {
    cudaEvent_t e;
    CUDA_OK(c, cudaEventCreate(&e));
    c->ev_pool.push_back(e);
  }
  return GAME_OK;
}

static game_status build_graph(game_ctx* c, bool timed) {
  if (timed ? c->graph_t != nullptr : c->graph != nullptr) return GAME_OK;
  if (timed) {
    game_status r0 = ensure_events(c, 4);
    if (r0 != GAME_OK) return r0;
  }
  cudaStream_t cap = c->st;
  bool own = false;
  if (cap == nullptr) {
    CUDA_OK(c, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    own = true;
  }
  cudaStream_t saved = c->st;
  c->st = cap;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  game_status r = GAME_OK;
  if (e == cudaSuccess) {
    r = enqueue_generation(c, timed ? c->ev_pool.data() : nullptr);
    e = cudaStreamEndCapture(cap, &g);
  }
  c->st = saved;
  if (own) cudaStreamDestroy(cap);
  if (r != GAME_OK) {
    if (g) cudaGraphDestroy(g);
    return r;
  }
  if (e != cudaSuccess) return fail(c, GAME_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
  c->gen_kernels = count_kernel_nodes(g);
  if (!timed) {
    e = cudaGraphInstantiate(&c->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(c, GAME_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
    return GAME_OK;
  }
  // Locate the four event-record nodes so that each replay can record into its own events.
  size_t n = 0;
  CUDA_OK(c, cudaGraphGetNodes(g, nullptr, &n));
  std::vector<cudaGraphNode_t> nodes(n);
  CUDA_OK(c, cudaGraphGetNodes(g, nodes.data(), &n));
  int found = 0;
  for (cudaGraphNode_t nd : nodes) {
    cudaGraphNodeType ty;
    CUDA_OK(c, cudaGraphNodeGetType(nd, &ty));
    if (ty != cudaGraphNodeTypeEventRecord) continue;
    cudaEvent_t ev;
    CUDA_OK(c, cudaGraphEventRecordNodeGetEvent(nd, &ev));
    for (int j = 0; j < 4; ++j)
      if (ev == c->ev_pool[j]) {
        c->ev_node[j] = nd;
        ++found;
      }
  }
  if (found != 4) {
    cudaGraphDestroy(g);
    return fail(c, GAME_ERR_CUDA, "timed graph: found %d of 4 event nodes", found);
  }
  e = cudaGraphInstantiate(&c->graph_t, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return fail(c, GAME_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
  }
  c->graph_t_tmpl = g;
  return GAME_OK;
}

extern "C" game_status game_evolve(game_ctx* c, int32_t max_generations, int32_t* generations_run) {
  if (!c) return fail(nullptr, GAME_ERR_INVALID_ARG, "ctx is NULL");
  if (!c->have_data) return fail(c, GAME_ERR_STATE, "game_set_data must come first");
  if (max_generations < 0) return fail(c, GAME_ERR_INVALID_ARG, "max_generations < 0");
  cudaSetDevice(c->dev);
  const bool timed = c->timing_on;
  game_status r = build_graph(c, timed);
  if (r != GAME_OK) return r;
  if (timed && (r = ensure_events(c, 4 * (size_t)max_generations + 4)) != GAME_OK) return r;
  cudaEvent_t e0, e1;
  CUDA_OK(c, cudaEventCreate(&e0));
  CUDA_OK(c, cudaEventCreate(&e1));
  CUDA_OK(c, launch_state_op(c->d_state, kStateBeginEvolve, c->st));
  CUDA_OK(c, cudaEventRecord(e0, c->st));
  for (int i = 0; i < max_generations; ++i) {
    if (timed) {
      for (int j = 0; j < 4; ++j)
        CUDA_OK(c, cudaGraphExecEventRecordNodeSetEvent(c->graph_t, c->ev_node[j],
                                                        c->ev_pool[4 + 4 * i + j]));
      CUDA_OK(c, cudaGraphLaunch(c->graph_t, c->st));
    } else {
      CUDA_OK(c, cudaGraphLaunch(c->graph, c->st));
    }
  }
  CUDA_OK(c, cudaEventRecord(e1, c->st));
  DevState hs;
  CUDA_OK(c, cudaMemcpyAsync(&hs, c->d_state, sizeof(hs), cudaMemcpyDeviceToHost, c->st));
  CUDA_OK(c, cudaStreamSynchronize(c->st));
  float ms = 0.0f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->timing = game_timing{};
  if (timed) {
    // Generations skipped after a stop still record their (empty) stages.
    for (int i = 0; i < max_generations; ++i) {
      const cudaEvent_t* ev = &c->ev_pool[4 + 4 * i];
      float a = 0.f, b = 0.f, d = 0.f;
      cudaEventElapsedTime(&a, ev[0], ev[1]);
      cudaEventElapsedTime(&b, ev[1], ev[2]);
      cudaEventElapsedTime(&d, ev[2], ev[3]);
      c->timing.ms_breed += a;
      c->timing.ms_fitness += b;
      c->timing.ms_rank += d;
    }
  }
  c->timing.ms_total = ms;
  c->timing.generations = hs.gens_run;
  c->timing.engine = c->engine;
  c->timing.launches = 1 + c->gen_kernels * max_generations;
  if (hs.status != 0) return fail(c, GAME_ERR_TIMEOUT, "device-side wait timed out (status %d)", hs.status);
  if ((r = collect_checks(c)) != GAME_OK) return r;
  if (generations_run) *generations_run = hs.gens_run;
  return GAME_OK;
}

extern "C" game_status game_evaluate(game_ctx* c, double* fitness, int32_t* rank) {
  if (!c) return fail(nullptr, GAME_ERR_INVALID_ARG, "ctx is NULL");
  if (!c->have_data) return fail(c, GAME_ERR_STATE, "game_set_data must come first");
  cudaSetDevice(c->dev);
  // A breed launch with allow = 0 records "not bred" for this evaluation.
  CUDA_OK(c, launch_breed(c->s, c->cfg, c->p, c->d_fit, c->d_rank, c->d_state, 0, c->st, c->d_cum));
  CUDA_OK(c, launch_prepare(c->s, c->p, c->e, c->d_state, 0, c->st));
  game_status r = launch_fitness(c, nullptr);
  if (r != GAME_OK) return r;
  CUDA_OK(c, launch_reduce_rank(c->s, c->cfg, c->d_partial, c->n_part, c->d_fit, c->d_rank,
                                c->d_state, kRankEvaluate, c->st));
  if (c->n_rescore) {
    r = enqueue_rescore(c, 0);
    if (r != GAME_OK) return r;
  }
  if (fitness)
    CUDA_OK(c, cudaMemcpyAsync(fitness, c->d_fit, sizeof(double) * c->s.pop, cudaMemcpyDeviceToHost, c->st));
  if (rank)
    CUDA_OK(c, cudaMemcpyAsync(rank, c->d_rank, sizeof(int) * c->s.pop, cudaMemcpyDeviceToHost, c->st));
  CUDA_OK(c, cudaStreamSynchronize(c->st));
  return collect_checks(c);
}

extern "C" game_status game_get_fitness(game_ctx* c, double* fitness, int32_t* rank) {
  if (!c) return fail(nullptr, GAME_ERR_INVALID_ARG, "ctx is NULL");
  if (!c->have_data) return fail(c, GAME_ERR_STATE, "game_set_data must come first");
  cudaSetDevice(c->dev);
  DevState hs;
  CUDA_OK(c, cudaMemcpyAsync(&hs, c->d_state, sizeof(hs), cudaMemcpyDeviceToHost, c->st));
  CUDA_OK(c, cudaStreamSynchronize(c->st));
  if (!hs.evaluated) return fail(c, GAME_ERR_STATE, "no evaluated population yet");
  if (fitness)
    CUDA_OK(c, cudaMemcpyAsync(fitness, c->d_fit, sizeof(double) * c->s.pop, cudaMemcpyDeviceToHost, c->st));
  if (rank)
    CUDA_OK(c, cudaMemcpyAsync(rank, c->d_rank, sizeof(int) * c->s.pop, cudaMemcpyDeviceToHost, c->st));
  CUDA_OK(c, cudaStreamSynchronize(c->st));
  return GAME_OK;
}

extern "C" game_status game_breed(game_ctx* c, const double* fitness) {
  if (!c) return fail(nullptr, GAME_ERR_INVALID_ARG, "ctx is NULL");
  if (!c->have_data) return fail(c, GAME_ERR_STATE, "game_set_data must come first");
  cudaSetDevice(c->dev);
  if (fitness) {
    CUDA_OK(c, cudaMemcpyAsync(c->d_fit, fitness, sizeof(double) * c->s.pop, cudaMemcpyHostToDevice, c->st));
    CUDA_OK(c, launch_reduce_rank(c->s, c->cfg, nullptr, 0, c->d_fit, c->d_rank, c->d_state,
                                  kRankSortOnly, c->st));
  } else {
    DevState hs;
    CUDA_OK(c, cudaMemcpyAsync(&hs, c->d_state, sizeof(hs), cudaMemcpyDeviceToHost, c->st));
    CUDA_OK(c, cudaStreamSynchronize(c->st));
    if (!hs.evaluated) return fail(c, GAME_ERR_STATE, "population not evaluated; pass a fitness vector");
  }
  CUDA_OK(c, launch_breed(c->s, c->cfg, c->p, c->d_fit, c->d_rank, c->d_state, 1, c->st, c->d_cum));
  CUDA_OK(c, launch_state_op(c->d_state, kStateAfterBreed, c->st));
  CUDA_OK(c, cudaStreamSynchronize(c->st));
  return GAME_OK;
}

extern "C" game_status game_set_population(game_ctx* c, const float* G, int32_t pop,
                                           int32_t n_genes, int32_t device_ptrs) {
  if (!c) return fail(nullptr, GAME_ERR_INVALID_ARG, "ctx is NULL");
  if (!c->have_data) return fail(c, GAME_ERR_STATE, "game_set_data must come first");
  if (!G || pop != c->s.pop || n_genes != c->s.n_genes)
    return fail(c, GAME_ERR_INVALID_ARG, "population must be %d x %d", c->s.pop, c->s.n_genes);
  cudaSetDevice(c->dev);
  DevState hs;
  CUDA_OK(c, cudaMemcpyAsync(&hs, c->d_state, sizeof(hs), cudaMemcpyDeviceToHost, c->st));
  CUDA_OK(c, cudaStreamSynchronize(c->st));
  CUDA_OK(c, cudaMemcpy2DAsync(c->p.g32[hs.cur], sizeof(float) * c->s.kstride, G,
                               sizeof(float) * n_genes, sizeof(float) * n_genes, pop,
                               device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->st));
  CUDA_OK(c, launch_state_op(c->d_state, kStatePopulationSet, c->st));
  CUDA_OK(c, cudaStreamSynchronize(c->st));
  return GAME_OK;
}

extern "C" game_status game_get_population(game_ctx* c, float* G, int32_t pop, int32_t n_genes) {
  if (!c) return fail(nullptr, GAME_ERR_INVALID_ARG, "ctx is NULL");
  if (!c->have_data) return fail(c, GAME_ERR_STATE, "game_set_data must come first");
  if (!G || pop != c->s.pop || n_genes != c->s.n_genes)
    return fail(c, GAME_ERR_INVALID_ARG, "population must be %d x %d", c->s.pop, c->s.n_genes);
  cudaSetDevice(c->dev);
  DevState hs;
  CUDA_OK(c, cudaMemcpyAsync(&hs, c->d_state, sizeof(hs), cudaMemcpyDeviceToHost, c->st));
  CUDA_OK(c, cudaStreamSynchronize(c->st));
  CUDA_OK(c, cudaMemcpy2DAsync(G, sizeof(float) * n_genes, c->p.g32[hs.cur],
                               sizeof(float) * c->s.kstride, sizeof(float) * n_genes, pop,
                               cudaMemcpyDeviceToHost, c->st));
  CUDA_OK(c, cudaStreamSynchronize(c->st));
  return GAME_OK;
}

extern "C" game_status game_get_expansion(game_ctx* c, float* out, int64_t row0, int64_t n_rows) {
  if (!c) return fail(nullptr, GAME_ERR_INVALID_ARG, "ctx is NULL");
  if (!c->have_data) return fail(c, GAME_ERR_STATE, "game_set_data must come first");
  if (!out || row0 < 0 || n_rows < 0 || row0 + n_rows > c->s.n_patterns)
    return fail(c, GAME_ERR_INVALID_ARG, "rows out of range");
  if (n_rows == 0) return GAME_OK;
  cudaSetDevice(c->dev);
  float* tmp = nullptr;
  const size_t bytes = sizeof(float) * (size_t)n_rows * c->s.kb;
  CUDA_OK(c, cudaMalloc(&tmp, bytes));
  cudaError_t e = c->otf ? launch_expand_get_otf(c->s, c->d_X, row0, n_rows, tmp, c->st)
                         : launch_expand_get(c->s, c->e, row0, n_rows, tmp, c->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, tmp, bytes, cudaMemcpyDeviceToHost, c->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  cudaFree(tmp);
  CUDA_OK(c, e);
  return GAME_OK;
}

static game_status score(game_ctx* c, const float* genes_host_or_null, int split, double out[5],
                         long long* rows) {
  const long long r0 = split == 0 ? 0 : c->s.n_train;
  const long long r1 = split == 0 ? c->s.n_train : c->s.n_patterns;
  *rows = r1 - r0;
  if (genes_host_or_null)
    CUDA_OK(c, cudaMemcpyAsync(c->d_genes, genes_host_or_null, sizeof(float) * c->s.n_genes,
                               cudaMemcpyHostToDevice, c->st));
  if (c->otf)
    CUDA_OK(c, launch_score_otf(c->s, c->fit, c->d_X, c->e.t, c->d_genes, r0, r1, c->d_score_blocks,
                                c->score_nb, c->d_score_out, c->st));
  else
    CUDA_OK(c, launch_score(c->s32, c->fit, c->e32, c->d_genes, r0, r1, c->d_score_blocks,
                            c->score_nb, c->d_score_out, c->st));
  CUDA_OK(c, cudaMemcpyAsync(out, c->d_score_out, sizeof(double) * 5, cudaMemcpyDeviceToHost, c->st));
  CUDA_OK(c, cudaStreamSynchronize(c->st));
  return GAME_OK;
}

static void fill_report(const double v[5], long long rows, double* rmse, double* acc,
                        double* compl_, double* contam) {
  const double n = rows > 0 ? (double)rows : 1.0;
  if (rmse) *rmse = rows > 0 ? sqrt(v[0] / n) : 0.0;
  if (acc) *acc = rows > 0 ? v[1] / n : 0.0;
  if (compl_) *compl_ = (v[2] + v[4]) > 0 ? v[2] / (v[2] + v[4]) : 0.0;
  if (contam) *contam = (v[2] + v[3]) > 0 ? v[3] / (v[2] + v[3]) : 0.0;
}

extern "C" game_status game_score(game_ctx* c, const float* genes, int32_t split, double* rmse,
                                  double* accuracy, double* completeness, double* contamination) {
  if (!c) return fail(nullptr, GAME_ERR_INVALID_ARG, "ctx is NULL");
  if (!c->have_data) return fail(c, GAME_ERR_STATE, "game_set_data must come first");
  if (!genes || (split != 0 && split != 1)) return fail(c, GAME_ERR_INVALID_ARG, "bad genes/split");
  cudaSetDevice(c->dev);
  double v[5];
  long long rows = 0;
  game_status r = score(c, genes, split, v, &rows);
  if (r != GAME_OK) return r;
  fill_report(v, rows, rmse, accuracy, completeness, contamination);
  return GAME_OK;
}

extern "C" game_status game_get_best(game_ctx* c, float* genes, int32_t cap, double* train_fitness,
                                     double* test_rmse, double* test_accuracy) {
  if (!c) return fail(nullptr, GAME_ERR_INVALID_ARG, "ctx is NULL");
  if (!c->have_data) return fail(c, GAME_ERR_STATE, "game_set_data must come first");
  if (genes && cap < c->s.n_genes)
    return fail(c, GAME_ERR_INVALID_ARG, "cap %d < n_genes %d", cap, c->s.n_genes);
  cudaSetDevice(c->dev);
  DevState hs;
  CUDA_OK(c, cudaMemcpyAsync(&hs, c->d_state, sizeof(hs), cudaMemcpyDeviceToHost, c->st));
  CUDA_OK(c, cudaStreamSynchronize(c->st));
  if (!hs.evaluated) return fail(c, GAME_ERR_STATE, "no evaluated population yet");
  int best = 0;
  CUDA_OK(c, cudaMemcpyAsync(&best, c->d_rank, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  CUDA_OK(c, cudaStreamSynchronize(c->st));
  const float* row = c->p.g32[hs.cur] + (size_t)best * c->s.kstride;
  CUDA_OK(c, cudaMemcpyAsync(c->d_genes, row, sizeof(float) * c->s.n_genes, cudaMemcpyDeviceToDevice, c->st));
  if (genes)
    CUDA_OK(c, cudaMemcpyAsync(genes, c->d_genes, sizeof(float) * c->s.n_genes, cudaMemcpyDeviceToHost, c->st));
  if (train_fitness) {
    CUDA_OK(c, cudaMemcpyAsync(train_fitness, c->d_fit + best, sizeof(double), cudaMemcpyDeviceToHost, c->st));
  }
  CUDA_OK(c, cudaStreamSynchronize(c->st));
  if (test_rmse || test_accuracy) {
    double v[5];
    long long rows = 0;
    game_status r = score(c, nullptr, 1, v, &rows);
    if (r != GAME_OK) return r;
    fill_report(v, rows, test_rmse, test_accuracy, nullptr, nullptr);
  }
  return GAME_OK;
}

extern "C" game_status game_predict(game_ctx* c, const float* genes, int32_t n_genes,
                                    const float* X, int64_t n, int32_t n_features, float* out,
                                    int32_t device_ptrs) {
  if (!c) return fail(nullptr, GAME_ERR_INVALID_ARG, "ctx is NULL");
  const int B = c->cfg.basis == GAME_TRIG ? 2 : 1;
  const int shared = c->cfg.coefficients == GAME_COEF_SHARED;
  const int want = B * (shared ? 1 : n_features) * c->cfg.degree + 1;
  if (!genes || !X || !out || n < 0 || n_features < 1 || n_genes != want)
    return fail(c, GAME_ERR_INVALID_ARG, "genes must hold %d values for F = %d", want, n_features);
  if (n == 0) return GAME_OK;
  cudaSetDevice(c->dev);
  float *dg = nullptr, *dX = nullptr, *dy = nullptr;
  auto release = [&]() {
    if (dg) cudaFree(dg);
    if (!device_ptrs) {
      if (dX) cudaFree(dX);
      if (dy) cudaFree(dy);
    }
  };
  cudaError_t e = cudaMalloc((void**)&dg, sizeof(float) * n_genes);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dg, genes, sizeof(float) * n_genes, cudaMemcpyDefault, c->st);
  if (e == cudaSuccess && !device_ptrs) {
    e = cudaMalloc((void**)&dX, sizeof(float) * (size_t)n * n_features);
    if (e == cudaSuccess) e = cudaMalloc((void**)&dy, sizeof(float) * (size_t)n);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(dX, X, sizeof(float) * (size_t)n * n_features, cudaMemcpyHostToDevice,
                          c->st);
  } else if (e == cudaSuccess) {
    dX = const_cast<float*>(X);
    dy = out;
  }
  if (e == cudaSuccess)
    e = launch_predict(dX, n, n_features, dg, n_genes, c->cfg.basis, c->cfg.degree, shared,
                       c->cfg.activation, dy, c->st);
  if (e == cudaSuccess && !device_ptrs)
    e = cudaMemcpyAsync(out, dy, sizeof(float) * (size_t)n, cudaMemcpyDeviceToHost, c->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  release();
  if (e != cudaSuccess) return fail(c, GAME_ERR_CUDA, "predict: %s", cudaGetErrorString(e));
  return GAME_OK;
}

// ---- checkpoint of the GA state -------------------------------------------
namespace {
struct SaveHeader {
  uint32_t magic;          // "GAMS"
  uint32_t version;        // 1
  int32_t pop, n_genes, basis, degree;
  uint64_t seed, run;
  int64_t gen;             // Philox counter word 0 of the next breeding
  int32_t evaluated, stopped, gens_run, evals;
  double best;
};
constexpr uint32_t kSaveMagic = 0x534D4147u;   // 'G' 'A' 'M' 'S'
}  // namespace

static int64_t save_bytes(const game_ctx* c) {
  return (int64_t)sizeof(SaveHeader) + (int64_t)c->s.pop * c->s.n_genes * 4 +
         (int64_t)c->s.pop * 8 + (int64_t)c->s.pop * 4;
}

extern "C" game_status game_save(game_ctx* c, void* buf, int64_t cap, int64_t* size) {
  if (!c) return fail(nullptr, GAME_ERR_INVALID_ARG, "ctx is NULL");
  if (!c->have_data) return fail(c, GAME_ERR_STATE, "game_set_data must come first");
  if (c->cfg.surrogate_pool > 0)
    return fail(c, GAME_ERR_UNSUPPORTED, "the surrogate's state is not part of a checkpoint");
  const int64_t need = save_bytes(c);
  if (size) *size = need;
  if (!buf) return GAME_OK;
  if (cap < need) return fail(c, GAME_ERR_INVALID_ARG, "buffer holds %lld of %lld bytes",
                              (long long)cap, (long long)need);
  cudaSetDevice(c->dev);
  DevState hs;
  CUDA_OK(c, cudaMemcpyAsync(&hs, c->d_state, sizeof(hs), cudaMemcpyDeviceToHost, c->st));
  CUDA_OK(c, cudaStreamSynchronize(c->st));
  SaveHeader h{kSaveMagic, 1u, c->s.pop, c->s.n_genes, c->cfg.basis, c->cfg.degree,
               c->cfg.seed, c->cfg.run, hs.gen, hs.evaluated, hs.stopped, hs.gens_run,
               hs.evals, hs.best};
  uint8_t* b = static_cast<uint8_t*>(buf);
  memcpy(b, &h, sizeof(h));
  b += sizeof(h);
  const int pop = c->s.pop, K = c->s.n_genes;
  CUDA_OK(c, cudaMemcpy2DAsync(b, sizeof(float) * K, c->p.g32[hs.cur], sizeof(float) * c->s.kstride,
                               sizeof(float) * K, pop, cudaMemcpyDeviceToHost, c->st));
  b += (size_t)pop * K * 4;
  CUDA_OK(c, cudaMemcpyAsync(b, c->d_fit, sizeof(double) * pop, cudaMemcpyDeviceToHost, c->st));
  b += (size_t)pop * 8;
  CUDA_OK(c, cudaMemcpyAsync(b, c->d_rank, sizeof(int) * pop, cudaMemcpyDeviceToHost, c->st));
  CUDA_OK(c, cudaStreamSynchronize(c->st));
  return GAME_OK;
}

extern "C" game_status game_load(game_ctx* c, const void* buf, int64_t size) {
  if (!c) return fail(nullptr, GAME_ERR_INVALID_ARG, "ctx is NULL");
  if (!c->have_data) return fail(c, GAME_ERR_STATE, "game_set_data must come first");
  if (c->cfg.surrogate_pool > 0)
    return fail(c, GAME_ERR_UNSUPPORTED, "the surrogate's state is not part of a checkpoint");
  if (!buf || size < (int64_t)sizeof(SaveHeader))
    return fail(c, GAME_ERR_INVALID_ARG, "not a checkpoint");
  SaveHeader h;
  memcpy(&h, buf, sizeof(h));
  if (h.magic != kSaveMagic || h.version != 1u || size != save_bytes(c))
    return fail(c, GAME_ERR_INVALID_ARG, "not a checkpoint of this version and size");
  if (h.pop != c->s.pop || h.n_genes != c->s.n_genes || h.basis != c->cfg.basis ||
      h.degree != c->cfg.degree || h.seed != c->cfg.seed || h.run != c->cfg.run)
    return fail(c, GAME_ERR_INVALID_ARG,
                "checkpoint of another configuration (population, genes, basis, seed or run)");
  cudaSetDevice(c->dev);
  const uint8_t* b = static_cast<const uint8_t*>(buf) + sizeof(h);
  const int pop = c->s.pop, K = c->s.n_genes;
  CUDA_OK(c, cudaMemcpy2DAsync(c->p.g32[0], sizeof(float) * c->s.kstride, b, sizeof(float) * K,
                               sizeof(float) * K, pop, cudaMemcpyHostToDevice, c->st));
  b += (size_t)pop * K * 4;
  CUDA_OK(c, cudaMemcpyAsync(c->d_fit, b, sizeof(double) * pop, cudaMemcpyHostToDevice, c->st));
  b += (size_t)pop * 8;
  CUDA_OK(c, cudaMemcpyAsync(c->d_rank, b, sizeof(int) * pop, cudaMemcpyHostToDevice, c->st));
  DevState hs{};
  hs.gen = h.gen;
  hs.cur = 0;
  hs.evaluated = h.evaluated;
  hs.bred = 0;
  hs.stopped = h.stopped;
  hs.gens_run = h.gens_run;
  hs.status = 0;
  hs.evals = h.evals;
  hs.best = h.best;
  CUDA_OK(c, cudaMemcpyAsync(c->d_state, &hs, sizeof(hs), cudaMemcpyHostToDevice, c->st));
  CUDA_OK(c, cudaStreamSynchronize(c->st));
  return GAME_OK;
}

extern "C" game_status game_get_state(game_ctx* c, int64_t* generation, int32_t* stopped) {
  if (!c) return fail(nullptr, GAME_ERR_INVALID_ARG, "ctx is NULL");
  if (!c->have_data) return fail(c, GAME_ERR_STATE, "game_set_data must come first");
  cudaSetDevice(c->dev);
  DevState hs;
  CUDA_OK(c, cudaMemcpyAsync(&hs, c->d_state, sizeof(hs), cudaMemcpyDeviceToHost, c->st));
  CUDA_OK(c, cudaStreamSynchronize(c->st));
  if (generation) *generation = hs.gen;
  if (stopped) *stopped = hs.stopped;
  return GAME_OK;
}

// Times every valid tile shape of one fitness launch (shape s, population planes
// pd, partial rows at most part_rows) and returns the fastest plan.
static game_status tune_shape(game_ctx* c, const Shape& s, const ExpDev& e, const PopDev& pd,
                              double* partial, int part_rows, int reps, TcPlan* best_plan,
                              game_tile* bt, game_tile* candidates, int cap, int* n_done) {
  std::vector<TileReq> cands;
  tc_candidates(s, &cands);
  cudaEvent_t e0, e1;
  CUDA_OK(c, cudaEventCreate(&e0));
  CUDA_OK(c, cudaEventCreate(&e1));
  *bt = game_tile{0, 0, 0, 0, 0, 0, 1e30};
  for (const TileReq& rq : cands) {
    TcPlan plan{};
    if (tc_plan(s, e, pd, c->n_sm, &plan, rq) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    if (plan.n_part > part_rows) continue;
    std::vector<float> t;
    bool ok = true;
    for (int i = 0; i <= reps && ok; ++i) {
      ok = cudaEventRecord(e0, c->st) == cudaSuccess &&
           tc_launch(plan, s, c->fit, pd, e, partial, nullptr, c->st) == cudaSuccess &&
           cudaEventRecord(e1, c->st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess;
      float ms = 0.f;
      if (ok && i > 0 && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) t.push_back(ms);
    }
    if (!ok) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return fail(c, GAME_ERR_CUDA, "autotune launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    }
    std::sort(t.begin(), t.end());
    const game_tile gt{plan.bn, plan.stages, plan.cluster, plan.prefetch, plan.sp, plan.kg,
                       t[t.size() / 2]};
    if (candidates && *n_done < cap) candidates[*n_done] = gt;
    ++*n_done;
    if (gt.ms < bt->ms) {
      *bt = gt;
      *best_plan = plan;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (bt->n == 0) return fail(c, GAME_ERR_UNSUPPORTED, "no tile shape could be planned");
  return GAME_OK;
}

extern "C" game_status game_autotune(game_ctx* c, int32_t reps, game_tile* best,
                                     game_tile* candidates, int32_t cap, int32_t* n_candidates) {
  if (!c) return fail(nullptr, GAME_ERR_INVALID_ARG, "ctx is NULL");
  if (!c->have_data) return fail(c, GAME_ERR_STATE, "game_set_data must come first");
  if (c->engine != GAME_ENGINE_TCGEN05)
    return fail(c, GAME_ERR_UNSUPPORTED, "this shape runs on a CUDA-core engine; nothing to tune");
  if (reps < 1) reps = 1;
  cudaSetDevice(c->dev);
  // Operand planes of the current population.
  CUDA_OK(c, launch_breed(c->s, c->cfg, c->p, c->d_fit, c->d_rank, c->d_state, 0, c->st, c->d_cum));
  CUDA_OK(c, launch_prepare(c->s, c->p, c->e, c->d_state, 0, c->st));
  int n_done = 0;
  game_tile bt;
  TcPlan best_plan{};
  game_status r = tune_shape(c, c->s, c->e, c->p, c->d_partial, c->part_rows, reps, &best_plan,
                             &bt, candidates, cap, &n_done);
  if (r != GAME_OK) return r;
  if (n_candidates) *n_candidates = n_done < cap ? n_done : cap;
  c->tc = best_plan;
  c->n_part = best_plan.n_part;
  tune_cache_store(c->s, bt);
  // The FP32 re-score of the elites (precision form) is a launch of its own
  // shape: one 128-row slice over the FP32 planes.
  if (c->n_rescore && c->engine_r == GAME_ENGINE_TCGEN05) {
    CUDA_OK(c, launch_prepare(c->sr, c->pr, c->e32, c->d_state, 0, c->st, c->d_rank, &c->p));
    int n_r = 0;
    game_tile bt_r;
    TcPlan plan_r{};
    r = tune_shape(c, c->sr, c->e32, c->pr, c->d_partial_r, c->part_rows_r, reps, &plan_r, &bt_r,
                   nullptr, 0, &n_r);
    if (r != GAME_OK) return r;
    c->tc_r = plan_r;
    c->n_part_r = plan_r.n_part;
    tune_cache_store(c->sr, bt_r);
  }
  drop_graphs(c);
  if (best) *best = bt;
  return GAME_OK;
}

extern "C" game_status game_get_tile(game_ctx* c, game_tile* out) {
  if (!c || !out) return fail(c, GAME_ERR_INVALID_ARG, "ctx or out is NULL");
  if (!c->have_data) return fail(c, GAME_ERR_STATE, "game_set_data must come first");
  if (c->engine != GAME_ENGINE_TCGEN05)
    return fail(c, GAME_ERR_UNSUPPORTED, "this shape runs on a CUDA-core engine");
  const TcPlan& t = c->tc;
  *out = game_tile{t.bn, t.stages, t.cluster, t.prefetch, t.sp, t.kg, 0.0};
  return GAME_OK;
}

static game_status need_surrogate(game_ctx* c) {
  if (!c) return fail(nullptr, GAME_ERR_INVALID_ARG, "ctx is NULL");
  if (!c->have_data) return fail(c, GAME_ERR_STATE, "game_set_data must come first");
  cudaSetDevice(c->dev);
  if (!c->sg_alloc) return alloc_surrogate(c);
  return GAME_OK;
}

extern "C" int64_t game_surrogate_n_params(game_ctx* c) {
  if (need_surrogate(c) != GAME_OK) return -1;
  return (int64_t)c->sg.n_params();
}

extern "C" game_status game_surrogate_get_params(game_ctx* c, float* params) {
  game_status r = need_surrogate(c);
  if (r != GAME_OK) return r;
  if (!params) return fail(c, GAME_ERR_INVALID_ARG, "params is NULL");
  CUDA_OK(c, cudaMemcpyAsync(params, c->sg.p, sizeof(float) * c->sg.n_params(), cudaMemcpyDeviceToHost, c->st));
  CUDA_OK(c, cudaStreamSynchronize(c->st));
  return GAME_OK;
}

extern "C" game_status game_surrogate_set_params(game_ctx* c, const float* params) {
  game_status r = need_surrogate(c);
  if (r != GAME_OK) return r;
  if (!params) return fail(c, GAME_ERR_INVALID_ARG, "params is NULL");
  CUDA_OK(c, cudaMemcpyAsync(c->sg.p, params, sizeof(float) * c->sg.n_params(), cudaMemcpyHostToDevice, c->st));
  CUDA_OK(c, c->sg.refresh(c->st));
  CUDA_OK(c, cudaStreamSynchronize(c->st));
  return GAME_OK;
}

static game_status upload_rows(game_ctx* c, const float* X, const float* t, int B) {
  if (B < 1 || B > c->sg_batch) return fail(c, GAME_ERR_INVALID_ARG, "B must be in 1..%d", c->sg_batch);
  CUDA_OK(c, cudaMemcpy2DAsync(c->d_bx, sizeof(float) * c->s.kstride, X, sizeof(float) * c->s.n_genes,
                               sizeof(float) * c->s.n_genes, B, cudaMemcpyHostToDevice, c->st));
  if (t) CUDA_OK(c, cudaMemcpyAsync(c->d_bt, t, sizeof(float) * B, cudaMemcpyHostToDevice, c->st));
  return GAME_OK;
}

extern "C" game_status game_surrogate_forward(game_ctx* c, const float* X, int32_t B, float* y) {
  game_status r = need_surrogate(c);
  if (r != GAME_OK) return r;
  if (!X || !y) return fail(c, GAME_ERR_INVALID_ARG, "X and y must be non-NULL");
  if ((r = upload_rows(c, X, nullptr, B)) != GAME_OK) return r;
  CUDA_OK(c, c->sg.forward(c->d_bx, c->s.kstride, B, c->sg.yb, c->st));
  CUDA_OK(c, cudaMemcpyAsync(y, c->sg.yb, sizeof(float) * B, cudaMemcpyDeviceToHost, c->st));
  CUDA_OK(c, cudaStreamSynchronize(c->st));
  return GAME_OK;
}

extern "C" game_status game_surrogate_grad(game_ctx* c, const float* X, const float* target,
                                           int32_t B, double* loss, float* grad) {
  game_status r = need_surrogate(c);
  if (r != GAME_OK) return r;
  if (!X || !target) return fail(c, GAME_ERR_INVALID_ARG, "X and target must be non-NULL");
  if ((r = upload_rows(c, X, target, B)) != GAME_OK) return r;
  CUDA_OK(c, c->sg.backward(c->d_bx, c->s.kstride, B, c->d_bt, c->st));
  float l = 0.f;
  CUDA_OK(c, cudaMemcpyAsync(&l, c->sg.loss, sizeof(float), cudaMemcpyDeviceToHost, c->st));
  if (grad)
    CUDA_OK(c, cudaMemcpyAsync(grad, c->sg.g, sizeof(float) * c->sg.n_params(), cudaMemcpyDeviceToHost, c->st));
  CUDA_OK(c, cudaStreamSynchronize(c->st));
  if (loss) *loss = l;
  return GAME_OK;
}

extern "C" game_status game_surrogate_train_step(game_ctx* c, const float* X, const float* target,
                                                 int32_t B, float lr) {
  game_status r = need_surrogate(c);
  if (r != GAME_OK) return r;
  if (!X || !target) return fail(c, GAME_ERR_INVALID_ARG, "X and target must be non-NULL");
  if ((r = upload_rows(c, X, target, B)) != GAME_OK) return r;
  CUDA_OK(c, c->sg.backward(c->d_bx, c->s.kstride, B, c->d_bt, c->st));
  CUDA_OK(c, c->sg.adam(lr, c->st));
  CUDA_OK(c, cudaStreamSynchronize(c->st));
  return GAME_OK;
}

extern "C" game_status game_surrogate_monitor(game_ctx* c, double* rho_last, double* loss_last,
                                              int32_t* fallback, double* history, int32_t cap,
                                              int32_t* n_history) {
  game_status r = need_surrogate(c);
  if (r != GAME_OK) return r;
  int meta[8];
  float l = 0.f;
  int fb = 0;
  CUDA_OK(c, cudaMemcpyAsync(meta, c->d_ring_meta, sizeof(meta), cudaMemcpyDeviceToHost, c->st));
  CUDA_OK(c, cudaMemcpyAsync(&l, c->sg.loss, sizeof(float), cudaMemcpyDeviceToHost, c->st));
  CUDA_OK(c, cudaMemcpyAsync(&fb, c->d_fallback, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  std::vector<double> hist(4096);
  CUDA_OK(c, cudaMemcpyAsync(hist.data(), c->d_monitor, sizeof(double) * 4096, cudaMemcpyDeviceToHost, c->st));
  CUDA_OK(c, cudaStreamSynchronize(c->st));
  const int n = std::min(meta[3], 4096);
  if (rho_last) *rho_last = n > 0 ? hist[(meta[3] - 1) % 4096] : NAN;
  if (loss_last) *loss_last = l;
  if (fallback) *fallback = fb;
  int k = 0;
  if (history)
    for (int i = std::max(0, meta[3] - std::min(cap, 4096)); i < meta[3] && k < cap; ++i)
      history[k++] = hist[i % 4096];
  if (n_history) *n_history = k;
  return GAME_OK;
}

extern "C" game_status game_surrogate_pool(game_ctx* c, float* scores, int32_t* selected,
                                           float* pool_genes, float* predictions,
                                           int32_t* n_pool) {
  if (!c) return fail(nullptr, GAME_ERR_INVALID_ARG, "ctx is NULL");
  if (!c->have_data) return fail(c, GAME_ERR_STATE, "game_set_data must come first");
  if (c->cfg.surrogate_pool <= 0 || !c->d_pool)
    return fail(c, GAME_ERR_STATE, "no offspring pool: surrogate_pool is 0");
  cudaSetDevice(c->dev);
  const int e = std::min(c->cfg.elitism, c->s.pop);
  if (n_pool) *n_pool = c->n_pool;
  if (scores)
    CUDA_OK(c, cudaMemcpyAsync(scores, c->d_score, sizeof(float) * c->n_pool,
                               cudaMemcpyDeviceToHost, c->st));
  if (selected)
    CUDA_OK(c, cudaMemcpyAsync(selected, c->d_sel, sizeof(int) * (c->s.pop - e),
                               cudaMemcpyDeviceToHost, c->st));
  if (pool_genes)
    CUDA_OK(c, cudaMemcpy2DAsync(pool_genes, sizeof(float) * c->s.n_genes, c->d_pool,
                                 sizeof(float) * c->s.kstride, sizeof(float) * c->s.n_genes,
                                 c->n_pool, cudaMemcpyDeviceToHost, c->st));
  if (predictions)
    CUDA_OK(c, cudaMemcpyAsync(predictions, c->d_pred, sizeof(float) * c->s.pop,
                               cudaMemcpyDeviceToHost, c->st));
  CUDA_OK(c, cudaStreamSynchronize(c->st));
  return GAME_OK;
}

extern "C" game_status game_selftest_timeout(game_ctx* c, int32_t wait_us, int32_t* waited_us) {
  if (!c) return fail(nullptr, GAME_ERR_INVALID_ARG, "ctx is NULL");
  if (!c->have_data) return fail(c, GAME_ERR_STATE, "game_set_data must come first");
  if (wait_us < 1 || wait_us > 2000000) return fail(c, GAME_ERR_INVALID_ARG, "wait_us in 1..2e6");
  cudaSetDevice(c->dev);
  int* d_out = nullptr;
  CUDA_OK(c, cudaMalloc(&d_out, 2 * sizeof(int)));
  int h[2] = {0, 0};
  cudaError_t e = tc_timeout_selftest(c->d_state, (unsigned long long)wait_us * 1000ull, d_out, c->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, d_out, sizeof(h), cudaMemcpyDeviceToHost, c->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  cudaFree(d_out);
  CUDA_OK(c, e);
  DevState hs;
  CUDA_OK(c, cudaMemcpy(&hs, c->d_state, sizeof(hs), cudaMemcpyDeviceToHost));
  // clear the recorded status so the context stays usable
  CUDA_OK(c, launch_state_op(c->d_state, kStateClearStatus, c->st));
  CUDA_OK(c, cudaStreamSynchronize(c->st));
  if (waited_us) *waited_us = h[1];
  if (h[0] == 1 && hs.status == GAME_ERR_TIMEOUT)
    return fail(c, GAME_ERR_TIMEOUT, "bounded wait gave up after %d us", h[1]);
  return GAME_OK;
}

extern "C" game_status game_set_timing(game_ctx* c, int32_t enabled) {
  if (!c) return fail(nullptr, GAME_ERR_INVALID_ARG, "ctx is NULL");
  c->timing_on = enabled != 0;
  return GAME_OK;
}

extern "C" game_status game_get_timing(game_ctx* c, game_timing* out) {
  if (!c || !out) return fail(c, GAME_ERR_INVALID_ARG, "ctx and out must be non-NULL");
  *out = c->timing;
  out->engine = c->engine;
  return GAME_OK;
}


// ===========================================================================
// Batched form: many independent runs, one persistent grouped fitness launch
// per generation, the whole generation of every run in one CUDA graph.
// ===========================================================================

extern "C" void game_batch_destroy(game_batch* b);

struct game_batch {
  std::vector<game_ctx*> runs;
  cudaStream_t st = nullptr;
  int dev = 0, n_sm = 0;
  std::string err;
  bool planned = false;
  int items_per_sm = 4;
  int grid = 0;
  std::vector<int> parts;          // partial rows per run (chunks * 4)
  BatchRunDev* d_runs = nullptr;
  WorkItem* d_items = nullptr;
  int* d_item_off = nullptr;
  int n_items = 0;
  cudaGraphExec_t graph = nullptr;
  int gen_kernels = 0;  // kernel nodes of one captured generation (all runs)
  game_timing timing{};
  std::vector<cudaStream_t> side;      // capture-time branches for the per-run kernels
  std::vector<cudaEvent_t> ev;         // fork / join events of those branches
};

static game_status bfail(game_batch* b, game_status code, const char* msg) {
  if (b) b->err = msg;
  g_global_err = msg;
  return code;
}

static void batch_free_plan(game_batch* b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
  cudaFree(b->d_runs);
  cudaFree(b->d_items);
  cudaFree(b->d_item_off);
  b->d_runs = nullptr;
  b->d_items = nullptr;
  b->d_item_off = nullptr;
  b->planned = false;
}

extern "C" game_status game_batch_create(const game_config* cfgs, int32_t n_runs,
                                         game_batch** out) {
  if (!cfgs || !out || n_runs < 1 || n_runs > 4096)
    return bfail(nullptr, GAME_ERR_INVALID_ARG, "need cfgs, out and 1 <= n_runs <= 4096");
  *out = nullptr;
  game_batch* b = new game_batch();
  for (int i = 0; i < n_runs; ++i) {
    if (cfgs[i].device != cfgs[0].device || cfgs[i].stream != cfgs[0].stream) {
      for (game_ctx* c : b->runs) game_destroy(c);
      delete b;
      return bfail(nullptr, GAME_ERR_INVALID_ARG, "every run of a batch shares one device and stream");
    }
    game_ctx* c = nullptr;
    game_status s = game_create(&cfgs[i], &c);
    if (s != GAME_OK) {
      for (game_ctx* x : b->runs) game_destroy(x);
      delete b;
      return s;
    }
    b->runs.push_back(c);
  }
  b->st = (cudaStream_t)cfgs[0].stream;
  b->dev = cfgs[0].device;
  b->n_sm = b->runs[0]->n_sm;
  const int ns = n_runs < 16 ? n_runs : 16;
  for (int k = 0; k < ns; ++k) {
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) break;
    b->side.push_back(s);
  }
  for (int k = 0; k <= (int)b->side.size(); ++k) {
    cudaEvent_t e;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) break;
    b->ev.push_back(e);
  }
  if (b->side.empty() || b->ev.size() != b->side.size() + 1) {
    game_batch_destroy(b);
    return bfail(nullptr, GAME_ERR_CUDA, "streams / events of the batch");
  }
  *out = b;
  return GAME_OK;
}

extern "C" game_ctx* game_batch_run(game_batch* b, int32_t run) {
  if (!b || run < 0 || run >= (int)b->runs.size()) return nullptr;
  return b->runs[run];
}

extern "C" game_status game_batch_set_data(game_batch* b, int32_t run, const float* X,
                                           const float* t, int64_t n_patterns, int32_t n_features,
                                           int64_t n_train, int32_t device_ptrs) {
  if (!b || run < 0 || run >= (int)b->runs.size())
    return bfail(b, GAME_ERR_INVALID_ARG, "bad batch or run index");
  batch_free_plan(b);
  game_status s = game_set_data(b->runs[run], X, t, n_patterns, n_features, n_train, device_ptrs);
  if (s != GAME_OK) b->err = b->runs[run]->err;
  if (s == GAME_OK && b->runs[run]->otf) {
    b->runs[run]->have_data = false;
    return bfail(b, GAME_ERR_UNSUPPORTED,
                 "the grouped launch reads stored expansions; a run on the on-the-fly engine "
                 "cannot join a batch");
  }
  return s;
}

// Static schedule: every (run, slice) is cut into chunks of consecutive tiles of
// about equal cost (tiles x k-blocks x MMA products), and the work items go to
// the SM with the least work so far, largest first.
static game_status batch_plan(game_batch* b) {
  if (b->planned) return GAME_OK;
  cudaSetDevice(b->dev);
  const int nr = (int)b->runs.size();
  const int tile = batch_tile_rows();
  std::vector<double> tcost(nr);
  double total = 0.0;
  for (int r = 0; r < nr; ++r) {
    game_ctx* c = b->runs[r];
    if (!c->have_data) return bfail(b, GAME_ERR_STATE, "every run of the batch needs data first");
    const Shape& s = c->s;
    const double prods = s.precision == GAME_FP32 ? 3.0 : s.gene_planes * (s.precision == GAME_FP8 ? 0.5 : 1.0);
    tcost[r] = (double)s.kp * prods + 64.0;   // + fixed per-tile epilogue cost
    const long long tiles = (s.n_train + tile - 1) / tile;
    total += tcost[r] * (double)tiles * (s.pop_pad / 128);
  }
  const double target = total / ((double)b->n_sm * b->items_per_sm);
  std::vector<WorkItem> items;
  std::vector<double> icost;
  b->parts.assign(nr, 0);
  for (int r = 0; r < nr; ++r) {
    game_ctx* c = b->runs[r];
    const int tiles = (int)((c->s.n_train + tile - 1) / tile);
    int chunks = (int)ceil(tiles * tcost[r] / target);
    chunks = std::max(1, std::min(chunks, std::min(tiles, c->part_rows / 4)));
    b->parts[r] = chunks * 4;
    for (int sl = 0; sl < c->s.pop_pad / 128; ++sl)
      for (int k = 0; k < chunks; ++k) {
        const int t0 = (int)((long long)tiles * k / chunks), t1 = (int)((long long)tiles * (k + 1) / chunks);
        items.push_back(WorkItem{r, sl, t0, t1, k});
        icost.push_back((t1 - t0) * tcost[r]);
      }
  }
  std::vector<int> order(items.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
  std::sort(order.begin(), order.end(), [&](int x, int y) { return icost[x] > icost[y]; });
  const int g = std::min<int>(b->n_sm, (int)items.size());
  std::vector<double> load(g, 0.0);
  std::vector<std::vector<int>> per(g);
  for (int i : order) {
    const int m = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    load[m] += icost[i];
    per[m].push_back(i);
  }
  std::vector<WorkItem> flat;
  std::vector<int> off(1, 0);
  for (int m = 0; m < g; ++m) {
    for (int i : per[m]) flat.push_back(items[i]);
    off.push_back((int)flat.size());
  }
  std::vector<BatchRunDev> rd(nr);
  for (int r = 0; r < nr; ++r) {
    game_ctx* c = b->runs[r];
    cudaError_t e = batch_make_run(c->s, c->fit, c->p, c->e, c->d_partial, c->d_state, &rd[r]);
    if (e != cudaSuccess) return bfail(b, GAME_ERR_CUDA, "tensor maps of a batched run");
  }
  if (cudaMalloc(&b->d_runs, sizeof(BatchRunDev) * nr) != cudaSuccess ||
      cudaMalloc(&b->d_items, sizeof(WorkItem) * flat.size()) != cudaSuccess ||
      cudaMalloc(&b->d_item_off, sizeof(int) * off.size()) != cudaSuccess)
    return bfail(b, GAME_ERR_OOM, "batch schedule allocation");
  if (cudaMemcpy(b->d_runs, rd.data(), sizeof(BatchRunDev) * nr, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->d_items, flat.data(), sizeof(WorkItem) * flat.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->d_item_off, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return bfail(b, GAME_ERR_CUDA, "batch schedule upload");
  b->grid = g;
  b->n_items = (int)flat.size();
  b->planned = true;
  return GAME_OK;
}

// The per-run kernels of a phase run on parallel graph branches (one branch per
// side stream, runs dealt round-robin), joined before the grouped launch and at
// the end of the generation.
static game_status batch_fork_join(game_batch* b, cudaStream_t st, bool post) {
  const int ns = (int)b->side.size();
  if (cudaEventRecord(b->ev[0], st) != cudaSuccess) return bfail(b, GAME_ERR_CUDA, "fork");
  for (int k = 0; k < ns; ++k)
    if (cudaStreamWaitEvent(b->side[k], b->ev[0], 0) != cudaSuccess)
      return bfail(b, GAME_ERR_CUDA, "fork wait");
  for (size_t i = 0; i < b->runs.size(); ++i) {
    game_ctx* c = b->runs[i];
    cudaStream_t s = b->side[i % ns];
    game_status r = post ? enqueue_post(c, b->parts[i], s) : enqueue_pre(c, s);
    if (r != GAME_OK) return bfail(b, r, c->err.c_str());
  }
  for (int k = 0; k < ns; ++k)
    if (cudaEventRecord(b->ev[1 + k], b->side[k]) != cudaSuccess ||
        cudaStreamWaitEvent(st, b->ev[1 + k], 0) != cudaSuccess)
      return bfail(b, GAME_ERR_CUDA, "join");
  return GAME_OK;
}

static game_status batch_enqueue_generation(game_batch* b, cudaStream_t st) {
  game_status r = batch_fork_join(b, st, false);
  if (r != GAME_OK) return r;
  cudaError_t e = batch_fitness_launch(b->d_runs, b->d_items, b->d_item_off, b->grid, 1, st);
  if (e != cudaSuccess) return bfail(b, GAME_ERR_CUDA, cudaGetErrorString(e));
  return batch_fork_join(b, st, true);
}

static game_status batch_build_graph(game_batch* b) {
  if (b->graph) return GAME_OK;
  cudaStream_t cap;
  if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess)
    return bfail(b, GAME_ERR_CUDA, "stream for capture");
  cudaGraph_t g = nullptr;
  game_status r = GAME_OK;
  cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    r = batch_enqueue_generation(b, cap);
    e = cudaStreamEndCapture(cap, &g);
  }
  cudaStreamDestroy(cap);
  if (r != GAME_OK) {
    if (g) cudaGraphDestroy(g);
    return r;
  }
  if (e != cudaSuccess) return bfail(b, GAME_ERR_CUDA, cudaGetErrorString(e));
  b->gen_kernels = count_kernel_nodes(g);
  e = cudaGraphInstantiate(&b->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return bfail(b, GAME_ERR_CUDA, cudaGetErrorString(e));
  return GAME_OK;
}

extern "C" game_status game_batch_evolve(game_batch* b, int32_t max_generations,
                                         int32_t* generations_run) {
  if (!b) return bfail(nullptr, GAME_ERR_INVALID_ARG, "batch is NULL");
  if (max_generations < 0) return bfail(b, GAME_ERR_INVALID_ARG, "max_generations < 0");
  cudaSetDevice(b->dev);
  game_status r = batch_plan(b);
  if (r != GAME_OK) return r;
  if ((r = batch_build_graph(b)) != GAME_OK) return r;
  for (game_ctx* c : b->runs)
    if (launch_state_op(c->d_state, kStateBeginEvolve, b->st) != cudaSuccess)
      return bfail(b, GAME_ERR_CUDA, "state reset");
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, b->st);
  for (int i = 0; i < max_generations; ++i)
    if (cudaGraphLaunch(b->graph, b->st) != cudaSuccess) return bfail(b, GAME_ERR_CUDA, "graph launch");
  cudaEventRecord(e1, b->st);
  if (cudaStreamSynchronize(b->st) != cudaSuccess) return bfail(b, GAME_ERR_CUDA, cudaGetErrorString(cudaGetLastError()));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->timing = game_timing{};
  b->timing.ms_total = ms;
  b->timing.engine = GAME_ENGINE_TCGEN05;
  b->timing.launches = (int32_t)b->runs.size() + b->gen_kernels * max_generations;
  int status = 0;
  for (size_t i = 0; i < b->runs.size(); ++i) {
    DevState hs;
    if (cudaMemcpy(&hs, b->runs[i]->d_state, sizeof(hs), cudaMemcpyDeviceToHost) != cudaSuccess)
      return bfail(b, GAME_ERR_CUDA, "state read");
    if (generations_run) generations_run[i] = hs.gens_run;
    if (hs.status) status = hs.status;
    b->timing.generations = std::max(b->timing.generations, hs.gens_run);
  }
  if (status) return bfail(b, GAME_ERR_TIMEOUT, "device-side wait timed out");
  return GAME_OK;
}

extern "C" game_status game_batch_get_timing(game_batch* b, game_timing* out) {
  if (!b || !out) return bfail(b, GAME_ERR_INVALID_ARG, "batch and out must be non-NULL");
  *out = b->timing;
  return GAME_OK;
}

extern "C" game_status game_batch_set_granularity(game_batch* b, int32_t items_per_sm) {
  if (!b || items_per_sm < 1 || items_per_sm > 64)
    return bfail(b, GAME_ERR_INVALID_ARG, "items_per_sm must be in 1..64");
  if (b->items_per_sm != items_per_sm) batch_free_plan(b);
  b->items_per_sm = items_per_sm;
  return GAME_OK;
}

extern "C" game_status game_batch_autotune(game_batch* b, int32_t reps, int32_t* items_per_sm,
                                           double* ms) {
  if (!b) return bfail(nullptr, GAME_ERR_INVALID_ARG, "batch is NULL");
  if (reps < 1) reps = 1;
  cudaSetDevice(b->dev);
  for (game_ctx* c : b->runs) {
    if (!c->have_data) return bfail(b, GAME_ERR_STATE, "every run of the batch needs data first");
    if (launch_breed(c->s, c->cfg, c->p, c->d_fit, c->d_rank, c->d_state, 0, b->st, c->d_cum) != cudaSuccess ||
        launch_prepare(c->s, c->p, c->e, c->d_state, 0, b->st) != cudaSuccess)
      return bfail(b, GAME_ERR_CUDA, "operand preparation");
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int best_g = b->items_per_sm;
  double best_ms = 1e30;
  for (int gsz : {1, 2, 4, 8, 16}) {
    batch_free_plan(b);
    b->items_per_sm = gsz;
    game_status r = batch_plan(b);
    if (r != GAME_OK) return r;
    std::vector<float> t;
    for (int i = 0; i <= reps; ++i) {
      cudaEventRecord(e0, b->st);
      if (batch_fitness_launch(b->d_runs, b->d_items, b->d_item_off, b->grid, 0, b->st) != cudaSuccess)
        return bfail(b, GAME_ERR_CUDA, "grouped launch");
      cudaEventRecord(e1, b->st);
      cudaEventSynchronize(e1);
      float m = 0.f;
      cudaEventElapsedTime(&m, e0, e1);
      if (i > 0) t.push_back(m);
    }
    std::sort(t.begin(), t.end());
    if (t[t.size() / 2] < best_ms) {
      best_ms = t[t.size() / 2];
      best_g = gsz;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  batch_free_plan(b);
  b->items_per_sm = best_g;
  game_status r = batch_plan(b);
  if (r != GAME_OK) return r;
  if (items_per_sm) *items_per_sm = best_g;
  if (ms) *ms = best_ms;
  return GAME_OK;
}

extern "C" void game_batch_destroy(game_batch* b) {
  if (!b) return;
  cudaSetDevice(b->dev);
  cudaStreamSynchronize(b->st);
  batch_free_plan(b);
  for (game_ctx* c : b->runs) game_destroy(c);
  for (cudaStream_t s : b->side) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
  delete b;
}
