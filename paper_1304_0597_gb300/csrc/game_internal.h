// Internal declarations shared by the CUDA translation units of libgame.so.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <stdint.h>

#include <string>

#include "../../include/game.h"

namespace game {

// Philox stream ids (counter word 2).
enum : uint32_t {
  kStreamTournament = 0,
  kStreamCrossover = 1,
  kStreamMutMask = 2,
  kStreamMutNormal = 3,
  kStreamInit = 4,
  kStreamInitNormal = 5,
  kStreamImmigrant = 8,        // (6, 7: the surrogate's sampling and initial weights)
  kStreamImmigrantNormal = 9,
};

// Device-resident loop state.  Only single-thread "state" kernels and the
// single-CTA reduce/rank kernel write it, so every multi-CTA kernel of a
// generation reads one consistent value.
struct DevState {
  long long gen;      // breeding steps applied so far (Philox counter word 0)
  int cur;            // population buffer (0/1) holding the current population
  int evaluated;      // the current population has a fitness vector
  int bred;           // the breed kernel of this generation produced buf[cur^1]
  int stopped;        // best fitness reached stop_error
  int gens_run;       // populations evaluated since the last reset
  int status;         // device-side error code (0 ok)
  int evals;          // populations evaluated since game_set_data (never reset)
  double best;        // best fitness of the last evaluated population
  unsigned int rank_done;   // blocks of the running rank_count launch that finished (0 between)
};

// Everything a kernel needs to know about the problem and population shapes.
struct Shape {
  long long n_patterns;   // NP
  long long n_train;      // training rows (the first rows of P)
  int n_features;         // F
  int degree;             // d
  int basis;              // GAME_CHEBYSHEV | GAME_TRIG
  int bd;                 // basis columns per feature: B*d
  int shared;             // coefficients shared by all features (expansion summed over f)
  int kb;                 // basis columns in total: F*B*d, or B*d when shared (= n_genes - 1)
  int kp;                 // stored columns of P / of the gene planes (kb padded)
  int n_genes;            // kb + 1
  int kstride;            // row stride of the float32 gene buffers (n_genes padded to 4)
  int pop;                // population size
  int pop_pad;            // pop padded to the 128-row MMA tile
  int precision;          // GAME_FP32 | GAME_BF16 | GAME_FP8
  int gene_planes;        // terms of each gene in the operand planes (FP32: always 2)
  int tc_narrow = 0;      // tensor cores: the swapped kernel (patterns on M), see fitness_tc_narrow.cu
};

// Population double buffer plus the operand planes of the population being evaluated.
struct PopDev {
  float* g32[2];          // [pop_pad x kstride] master genes (float32)
  float* geval;           // [pop_pad x kp] basis genes of the population under evaluation
  float* bias;            // [pop_pad] gene 0 of the population under evaluation
  void* ghi;              // [pop_pad x kp] MMA operand plane (hi part)
  void* glo;              // [pop_pad x kp] MMA operand plane (lo part)
  float* rscale;          // [pop_pad] per-chromosome scale of the planes (FP32: a power of
                          // two, 1 unless a gene times its column scale passes 2^15)
  int pop_rows = 0;       // chromosomes in g32 (0: the shape's pop)
};

// Expansion matrix P (basis columns only; the bias column of ones is implicit).
struct ExpDev {
  void* p0;               // FP32: fp16 hi plane; BF16: bf16 values; FP8: e4m3 values
  void* p1;               // FP32: fp16 lo plane; otherwise unused
  float* colscale;        // [kp] per-column scale s_g: quantised P, or for FP32 a power of two
                          // (1 unless a column's values could pass 2^15)
  float* t;               // [n_patterns padded to 256] targets
  float* tcoef;           // [same] 2 log2(e) t_k, read by the fused +-1 / tanh epilogue
  int unit_scale32 = 1;   // FP32: colscale holds only ones (the expansion skips the multiply)
};

struct Fitness {
  int error;              // GAME_RMSE ...
  int activation;         // GAME_TANH | GAME_LINEAR
  float tmse_R;
  int pm1_targets;        // every training target is +-1 (enables the fused tanh form)
};

// ---- launchers (each returns cudaGetLastError of its launch) ----------------

// FP32 planes hold P / s_g with the power-of-two scales the caller has written to
// e.colscale (launch_fill_ones for none); the quantised forms compute theirs.
cudaError_t launch_expand(const float* X, const Shape& s, ExpDev& e, float* qmax_scratch,
                          cudaStream_t st);
cudaError_t launch_fill_ones(float* v, int n, cudaStream_t st);
// absmax_bits[f] = float bits of max_k |X[k][f]| (F <= 12288).
cudaError_t launch_feature_absmax(const float* X, long long n, int F, unsigned int* absmax_bits,
                                  int n_sm, cudaStream_t st);
// Outputs of one chromosome on n new patterns X [n x F] (device buffers).
cudaError_t launch_predict(const float* X, long long n, int F, const float* genes, int K,
                           int basis, int degree, int shared, int activation, float* out,
                           cudaStream_t st);
cudaError_t launch_expand_get(const Shape& s, const ExpDev& e, long long row0, long long nrows,
                              float* out, cudaStream_t st);
cudaError_t launch_target_coef(const float* t, float* c, long long n, cudaStream_t st);

cudaError_t launch_init_population(const Shape& s, int init_mode, uint64_t seed, uint64_t run,
                                   float* g32, cudaStream_t st);
cudaError_t launch_breed(const Shape& s, const game_config& cfg, const PopDev& p,
                         const double* fit, const int* rank, DevState* state, int allow,
                         cudaStream_t st, unsigned long long* cum);
// Roulette / ranking: cumulative integer weights of the current fitness (no-op
// for tournament selection).
cudaError_t launch_selection_weights(const game_config& cfg, const Shape& s, const double* fit,
                                     const int* rank, unsigned long long* cum, cudaStream_t st);
// use_bred_flag: bit 0 = read the bred buffer when this generation bred, bit 1 =
// inside game_evolve (skip when stopped).  rows (optional): row i of the planes
// takes chromosome rows[i] of src (default: p's own population buffers).
cudaError_t launch_prepare(const Shape& s, const PopDev& p, const ExpDev& e, DevState* state,
                           int use_bred_flag, cudaStream_t st, const int* rows = nullptr,
                           const PopDev* src = nullptr);
cudaError_t launch_rescore_merge(const Shape& sr, const game_config& cfg, const double* partial,
                                 int n_part, const int* rank, double* fit, const DevState* state,
                                 int in_evolve, cudaStream_t st);
// Populations of at least this size are ranked by counting over many CTAs
// (fit_reduce / rank_count / rank_state), smaller ones by one CTA's sort.
constexpr int kRankCountMin = 512;
// Random immigrants: the last cfg.immigrants rows of a bred population replaced.
cudaError_t launch_immigrants(const Shape& s, const game_config& cfg, const PopDev& p,
                              const DevState* state, cudaStream_t st);
cudaError_t launch_reduce_rank(const Shape& s, const game_config& cfg, const double* partial,
                               int n_part, double* fit, int* rank, DevState* state,
                               int mode, cudaStream_t st);
cudaError_t launch_state_op(DevState* state, int op, cudaStream_t st);
cudaError_t ga_init_attributes();   // once per device, outside stream capture

// Bounds-check words of the debug build (-DGAME_CHECKS): site << 48 | index of the
// first failed check since the last read, per translation unit (0 in other builds).
unsigned long long check_word_expand();
unsigned long long check_word_ga();
unsigned long long check_word_tc();

// State ops.
enum : int {
  kStateReset = 0,          // gen=0, cur=0, evaluated=0, bred=0, stopped=0, gens_run=0
  kStatePopulationSet = 1,  // evaluated=0, bred=0, stopped=0
  kStateBeginEvolve = 2,    // gens_run=0
  kStateAfterBreed = 3,     // if bred: cur^=1, gen++ ; evaluated=0, bred=0
  kStateClearStatus = 4,    // status = 0
};

// reduce_rank modes (low byte), flags: bit 8 inside game_evolve, bit 9 no stop test
enum : int {
  kRankEvaluate = 0,        // reduce partials -> fitness, sort, update state
  kRankSortOnly = 1,        // sort the given fitness vector, mark evaluated
  kRankResort = 2,          // sort the (re-scored) fitness vector, stop test
  kRankInEvolve = 1 << 8,
  kRankNoStop = 1 << 9,
};

// sum_{b < n_part} partial[b * stride + c], added in b order.  The loads are
// issued eight at a time ahead of the adds: one chain of dependent global loads
// would cost a memory latency per partial row.
__device__ __forceinline__ double sum_partials(const double* __restrict__ partial, int n_part,
                                               long long stride, long long c) {
  double s = 0.0;
  int b = 0;
  for (; b + 8 <= n_part; b += 8) {
    double v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = partial[(long long)(b + i) * stride + c];
#pragma unroll
    for (int i = 0; i < 8; ++i) s += v[i];
  }
  for (; b < n_part; ++b) s += partial[(long long)b * stride + c];
  return s;
}

// SIMT fitness (FFMA) over the training rows: partial sums [n_part x pop_pad].
// simt_narrow: the shape takes the one-pattern-per-thread kernel (pop <= 32,
// kp 16 or 32), which the automatic engine choice prefers to the tensor cores.
bool simt_narrow(const Shape& s);
int simt_partials(const Shape& s, int n_sm);
// state: read (stop flag) only inside game_evolve, else null; dev_state: the
// context's device state, where a timed-out wait records its status.
cudaError_t launch_fitness_simt(const Shape& s, const Fitness& f, const PopDev& p,
                                const ExpDev& e, double* partial, int n_part,
                                const DevState* state, DevState* dev_state, cudaStream_t st);
cudaError_t simt_init_attributes();   // the narrow kernel's shared-memory ring

// On-the-fly engine (fitness_otf.cu): P formed per tile from the features X, never
// stored.  Same partial-sum layout as the SIMT engine, otf_partials rows.
int otf_partials(const Shape& s, int n_sm);
cudaError_t launch_fitness_otf(const Shape& s, const Fitness& f, const PopDev& p, const float* X,
                               const ExpDev& e, double* partial, int n_part,
                               const DevState* state, cudaStream_t st);
cudaError_t launch_score_otf(const Shape& s, const Fitness& f, const float* X, const float* t,
                             const float* genes, long long r0, long long r1, double* block_out,
                             int n_blocks, double* result, cudaStream_t st);
cudaError_t launch_expand_get_otf(const Shape& s, const float* X, long long row0, long long nrows,
                                  float* out, cudaStream_t st);

// Float64 score of one chromosome on rows [r0, r1).
cudaError_t launch_score(const Shape& s, const Fitness& f, const ExpDev& e, const float* genes,
                         long long r0, long long r1, double* block_out, int n_blocks,
                         double* result, cudaStream_t st);
int score_blocks(long long rows, int n_sm);

}  // namespace game
