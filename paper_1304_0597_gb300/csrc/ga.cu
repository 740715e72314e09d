// Genetic-algorithm side of the GAME loop on the device: counter-based random
// numbers, population initialisation, the genetic operators, operand
// preparation, and the reduce + rank step that closes each generation.
//
// Paper Section 4.1 lists the loop: (1) random initial population, (2) fitness
// and sort of the chromosomes, (3) stop test, (4) genetic operators.  Section 2
// names the user options (error function, selection, elitism, three random
// generation criteria); Section 5 gives crossover, mutation, tournament and
// elitism settings.  The paper keeps selection and the operators on the host;
// here they run on the device so that a generation never leaves the GPU.
#include "checks.cuh"
#include "game_internal.h"
#include "rng.cuh"

#include <math_constants.h>

namespace game {

// ---------------------------------------------------------------------------
// Initial population (Section 2: pseudo-random in [-1,1], normal in [-1,1],
// pseudo-random in [0,1]).  One thread per gene.
// ---------------------------------------------------------------------------
// Gene g of a random chromosome c of the init distribution, Philox counter
// (gen, c, stream, word): U[-1,1], N(0,0.5^2) resampled into [-1,1] (64 rounds,
// then clamp), or U[0,1].
__device__ __forceinline__ float draw_gene(Key key, uint64_t gen, int c, int g, int n_genes,
                                           int mode, uint64_t stream_u, uint64_t stream_n) {
  if (mode == GAME_INIT_NORMAL_PM1) {
    for (int r = 0; r < 64; ++r) {
      uint32_t w0, w1;
      philox_word_pair(key, gen, (uint64_t)c, stream_n,
                       (uint64_t)r * (uint64_t)n_genes + (uint64_t)g, &w0, &w1);
      const float x = __fmul_rn(gauss_f32(w0, w1), 0.5f);
      if (fabsf(x) <= 1.0f) return x;
      if (r == 63) return fminf(fmaxf(x, -1.0f), 1.0f);
    }
    return 0.0f;
  }
  const float u = uniform24(philox_word(key, gen, (uint64_t)c, stream_u, (uint64_t)g));
  return (mode == GAME_INIT_UNIFORM_01) ? u : __fsub_rn(__fmul_rn(u, 2.0f), 1.0f);
}

__global__ void init_population_kernel(int pop, int n_genes, int kstride, int mode, Key key,
                                       float* __restrict__ g32) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)pop * n_genes) return;
  const int c = (int)(i / n_genes), g = (int)(i % n_genes);
  g32[(long long)c * kstride + g] =
      draw_gene(key, 0, c, g, n_genes, mode, kStreamInit, kStreamInitNormal);
}

// Random immigrants (Section 4.1): the last n rows of the population just bred
// (buffer cur ^ 1) are replaced by fresh chromosomes, counter generation gen + 1.
__global__ void immigrants_kernel(const DevState* st, float* g32_0, float* g32_1, int pop, int n,
                                  int n_genes, int kstride, int mode, Key key) {
  if (!st->bred) return;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)n * n_genes) return;
  const int c = pop - n + (int)(i / n_genes), g = (int)(i % n_genes);
  float* out = st->cur ? g32_0 : g32_1;
  out[(long long)c * kstride + g] = draw_gene(key, (uint64_t)st->gen + 1, c, g, n_genes, mode,
                                              kStreamImmigrant, kStreamImmigrantNormal);
}

cudaError_t launch_immigrants(const Shape& s, const game_config& cfg, const PopDev& p,
                              const DevState* state, cudaStream_t st) {
  const int n = cfg.immigrants < s.pop ? cfg.immigrants : s.pop;
  if (n <= 0) return cudaSuccess;
  const long long total = (long long)n * s.n_genes;
  immigrants_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(
      state, p.g32[0], p.g32[1], s.pop, n, s.n_genes, s.kstride, cfg.init,
      Key{cfg.seed, cfg.run});
  return cudaGetLastError();
}

cudaError_t launch_init_population(const Shape& s, int init_mode, uint64_t seed, uint64_t run,
                                   float* g32, cudaStream_t st) {
  const long long n = (long long)s.pop * s.n_genes;
  const int threads = 256;
  init_population_kernel<<<(unsigned)((n + threads - 1) / threads), threads, 0, st>>>(
      s.pop, s.n_genes, s.kstride, init_mode, Key{seed, run}, g32);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Genetic operators: one warp per child pair (plus one warp per elite slot).
// ---------------------------------------------------------------------------
struct BreedArgs {
  const float* g32_0;
  const float* g32_1;
  float* out_0;
  float* out_1;
  const double* fit;
  const int* rank;
  const unsigned long long* cum;   // roulette / ranking cumulative weights, or nullptr
  DevState* state;
  Key key;
  int pop, n_genes, kstride;
  int tournament_k, elitism, elite_mode, clamp;
  float p_c, p_m, sigma;
  int allow, in_evolve;
};

__global__ void breed_kernel(BreedArgs a) {
  DevState* st = a.state;
  const int decision = a.allow && st->evaluated && !(a.in_evolve && st->stopped);
  if (blockIdx.x == 0 && threadIdx.x == 0) st->bred = decision;
  if (!decision) return;
  const int cur = st->cur;
  const uint64_t gen = (uint64_t)st->gen;
  const float* __restrict__ G = cur ? a.g32_1 : a.g32_0;
  float* __restrict__ out = cur ? a.out_0 : a.out_1;
  const int warp = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  const int e = min(a.elitism, a.pop);
  const int n_child = a.pop - e;
  const int n_pairs = (n_child + 1) / 2;
  const int K = a.n_genes;

  if (warp < n_pairs) {
    const int slot_a = e + 2 * warp, slot_b = slot_a + 1;
    breed_pair(G, a.kstride, K, a.pop, a.fit, a.cum, a.key, gen, (uint64_t)warp, a.tournament_k,
               a.p_c, a.p_m, a.sigma, a.clamp, out + (long long)slot_a * a.kstride,
               out + (long long)slot_b * a.kstride, slot_b < a.pop, lane);
  } else if (warp < n_pairs + e) {
    const int slot = warp - n_pairs;
    const int src = (a.elite_mode == GAME_ELITE_TOP) ? a.rank[slot] : a.rank[0];
    if (!GAME_IN_BOUNDS_DBG(src >= 0 && src < a.pop, kSiteBreedParent, src)) return;
    const float* __restrict__ r = G + (long long)src * a.kstride;
    float* o = out + (long long)slot * a.kstride;
    for (int g = lane; g < K; g += 32) o[g] = r[g];
  }
}

// ---------------------------------------------------------------------------
// Roulette and ranking selection (Section 2): integer weights (so that the
// cumulative sums are exact in any order of addition) and their inclusive
// prefix sums, one CTA.
//   roulette: w_c = 1 / (1e-12 + f_c) (float64, correctly rounded), NaN -> 0,
//             q_c = floor(2^24 w_c / max w);
//   ranking:  q = 9 (N - 1) + 2 (N - 1 - r) at rank position r (linear ranking,
//             expected values 1.1 best to 0.9 worst).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) selection_weights_kernel(const double* fit,
                                                                 const int* rank, int pop,
                                                                 int mode,
                                                                 unsigned long long* cum) {
  __shared__ double wred[1024];
  __shared__ unsigned long long part[1024];
  const int tid = threadIdx.x, nt = blockDim.x;
  if (mode == GAME_SEL_RANKING) {
    for (int r = tid; r < pop; r += nt)
      cum[rank[r]] = 9ull * (unsigned long long)(pop - 1) + 2ull * (unsigned long long)(pop - 1 - r);
  } else {
    double m = 0.0;
    for (int c = tid; c < pop; c += nt) {
      const double f = fit[c];
      const double w = isnan(f) ? 0.0 : 1.0 / (1e-12 + f);
      if (w > m) m = w;
    }
    wred[tid] = m;
    __syncthreads();
    for (int o = nt >> 1; o > 0; o >>= 1) {
      if (tid < o && wred[tid + o] > wred[tid]) wred[tid] = wred[tid + o];
      __syncthreads();
    }
    const double wmax = wred[0];
    for (int c = tid; c < pop; c += nt) {
      const double f = fit[c];
      const double w = isnan(f) ? 0.0 : 1.0 / (1e-12 + f);
      cum[c] = wmax > 0.0 ? (unsigned long long)floor(w / wmax * 16777216.0) : 0ull;
    }
  }
  __syncthreads();
  // inclusive prefix sums: each thread a contiguous chunk, then a scan of the chunk totals
  const int chunk = (pop + nt - 1) / nt;
  const int b0 = min(pop, tid * chunk), b1 = min(pop, b0 + chunk);
  unsigned long long sum = 0;
  for (int i = b0; i < b1; ++i) sum += cum[i];
  part[tid] = sum;
  __syncthreads();
  for (int o = 1; o < nt; o <<= 1) {
    const unsigned long long v = tid >= o ? part[tid - o] : 0ull;
    __syncthreads();
    part[tid] += v;
    __syncthreads();
  }
  unsigned long long run = part[tid] - sum;
  for (int i = b0; i < b1; ++i) {
    run += cum[i];
    cum[i] = run;
  }
}

cudaError_t launch_selection_weights(const game_config& cfg, const Shape& s, const double* fit,
                                     const int* rank, unsigned long long* cum, cudaStream_t st) {
  if (cfg.selection == GAME_SEL_TOURNAMENT) return cudaSuccess;
  // a power-of-two block no wider than the population needs (the paper's 23 chromosomes:
  // one warp, so 5 + 10 barrier steps instead of 10 + 20); integer weights and a maximum,
  // so the result does not depend on the block size
  int nt = 32;
  while (nt < s.pop && nt < 1024) nt <<= 1;
  selection_weights_kernel<<<1, nt, 0, st>>>(fit, rank, s.pop, cfg.selection, cum);
  return cudaGetLastError();
}

cudaError_t launch_breed(const Shape& s, const game_config& cfg, const PopDev& p,
                         const double* fit, const int* rank, DevState* state, int allow,
                         cudaStream_t st, unsigned long long* cum) {
  if ((allow & 1) && cfg.selection != GAME_SEL_TOURNAMENT) {
    cudaError_t e = launch_selection_weights(cfg, s, fit, rank, cum, st);
    if (e != cudaSuccess) return e;
  }
  BreedArgs a;
  a.cum = cfg.selection != GAME_SEL_TOURNAMENT ? cum : nullptr;
  a.g32_0 = p.g32[0];
  a.g32_1 = p.g32[1];
  a.out_0 = p.g32[0];
  a.out_1 = p.g32[1];
  a.fit = fit;
  a.rank = rank;
  a.state = state;
  a.key = Key{cfg.seed, cfg.run};
  a.pop = s.pop;
  a.n_genes = s.n_genes;
  a.kstride = s.kstride;
  a.tournament_k = cfg.tournament_k;
  a.elitism = cfg.elitism;
  a.elite_mode = cfg.elite_mode;
  a.clamp = cfg.clamp_genes;
  a.p_c = cfg.p_crossover;
  a.p_m = cfg.p_mutation;
  a.sigma = cfg.sigma_mutation;
  a.allow = allow & 1;
  a.in_evolve = (allow >> 1) & 1;
  const int e = cfg.elitism < s.pop ? cfg.elitism : s.pop;
  const int warps = (s.pop - e + 1) / 2 + e;
  const int threads = 256;
  const int blocks = allow & 1 ? (warps * 32 + threads - 1) / threads : 1;
  breed_kernel<<<blocks > 0 ? blocks : 1, threads, 0, st>>>(a);
  if ((allow & 1) && cfg.immigrants > 0) return launch_immigrants(s, cfg, p, state, st);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Operand preparation: basis genes of the population under evaluation, in the
// float32 layout of the SIMT path and in the tensor-core planes of the chosen
// precision.  One warp per chromosome row (rows >= pop are zero).
//   FP32: g' = g * s_col / r_c with s_col the power-of-two column scale of P and r_c
//   the smallest power of two >= 1 that keeps max_col |g * s_col| / r_c <= 2^15 (so both
//   are 1 for features in range and genes in [-1, 1]); plane hi = fp16(g'),
//   lo = fp16(g' - hi): g' = hi + lo to ~22 bits.  The epilogue multiplies by r_c.
//   BF16 / FP8: g' = g * s_col / r_c with r_c = max_col |g * s_col| / qmax;
//   hi = q(g'), lo = q(g' - hi); the contraction result is scaled back by r_c.
// ---------------------------------------------------------------------------
struct PrepArgs {
  const int* rows;        // optional: row i takes chromosome rows[i] (i < pop), else row i
  const float* g32_0;
  const float* g32_1;
  const float* colscale;
  float* geval;
  float* bias;
  void* ghi;
  void* glo;
  float* rscale;
  const DevState* state;
  int pop, pop_pad, kb, kp, kstride, precision, use_bred_flag, in_evolve;
  int src_pop;            // rows of the source population (bounds of rows[])
};

__global__ void prepare_kernel(PrepArgs a) {
  const DevState* st = a.state;
  if (a.in_evolve && st->stopped) return;
  const int row = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= a.pop_pad) return;
  int buf = st->cur;
  if (a.use_bred_flag && st->bred) buf ^= 1;
  const bool live = row < a.pop;
  const int src = (live && a.rows) ? a.rows[row] : row;
  if (!GAME_IN_BOUNDS_DBG(!live || (src >= 0 && src < a.src_pop), kSitePrepareSrc, src)) return;
  const float* G = (buf ? a.g32_1 : a.g32_0) + (long long)src * a.kstride;
  float* ge = a.geval + (long long)row * a.kp;
  if (lane == 0) a.bias[row] = live ? G[0] : 0.0f;
  // Genes and column scales are read in batches of kPrepU per lane, all loads of a batch
  // before its stores (a chain of load-store rounds costs a memory latency each).
  constexpr int kPrepU = 8;
  float m = 0.0f;
  if (live)
    for (int c0 = 0; c0 < a.kb; c0 += 32 * kPrepU) {
      float v[kPrepU];
#pragma unroll
      for (int u = 0; u < kPrepU; ++u) {
        const int c = c0 + lane + 32 * u;
        v[u] = c < a.kb ? G[1 + c] * a.colscale[c] : 0.0f;
      }
#pragma unroll
      for (int u = 0; u < kPrepU; ++u) m = fmaxf(m, fabsf(v[u]));
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (a.precision == GAME_FP32) {
    __half* hi = (__half*)a.ghi + (long long)row * a.kp;
    __half* lo = (__half*)a.glo + (long long)row * a.kp;
    int ex = 0;
    frexpf(m, &ex);                                  // m < 2^ex
    const float r = ex > 15 ? ldexpf(1.0f, ex - 15) : 1.0f;
    const float inv_r = 1.0f / r;                    // powers of two: exact
    for (int c0 = 0; c0 < a.kp; c0 += 32 * kPrepU) {
      float v[kPrepU], cs[kPrepU];
#pragma unroll
      for (int u = 0; u < kPrepU; ++u) {
        const int c = c0 + lane + 32 * u;
        v[u] = (live && c < a.kb) ? G[1 + c] : 0.0f;
        cs[u] = c < a.kb ? a.colscale[c] : 0.0f;
      }
#pragma unroll
      for (int u = 0; u < kPrepU; ++u) {
        const int c = c0 + lane + 32 * u;
        if (c >= a.kp) break;
        ge[c] = v[u];
        const float w = c < a.kb ? (v[u] * cs[u]) * inv_r : 0.0f;
        const __half h = __float2half_rn(w);
        hi[c] = h;
        lo[c] = __float2half_rn(__fsub_rn(w, __half2float(h)));
      }
    }
    if (lane == 0) a.rscale[row] = r;
    return;
  }
  const float qmax = a.precision == GAME_BF16 ? 1.0f : 448.0f;
  const float r = m > 0.0f ? m / qmax : 1.0f;
  if (lane == 0) a.rscale[row] = r;
  for (int c0 = 0; c0 < a.kp; c0 += 32 * kPrepU) {
    float vv[kPrepU], cs[kPrepU];
#pragma unroll
    for (int u = 0; u < kPrepU; ++u) {
      const int c = c0 + lane + 32 * u;
      vv[u] = (live && c < a.kb) ? G[1 + c] : 0.0f;
      cs[u] = c < a.kb ? a.colscale[c] : 0.0f;
    }
#pragma unroll
    for (int u = 0; u < kPrepU; ++u) {
      const int c = c0 + lane + 32 * u;
      if (c >= a.kp) break;
      const float v = vv[u];
      ge[c] = v;
      const float w = (c < a.kb) ? (v * cs[u]) / r : 0.0f;
      if (a.precision == GAME_BF16) {
        __nv_bfloat16* hi = (__nv_bfloat16*)a.ghi + (long long)row * a.kp;
        __nv_bfloat16* lo = (__nv_bfloat16*)a.glo + (long long)row * a.kp;
        const __nv_bfloat16 h = __float2bfloat16_rn(w);
        hi[c] = h;
        lo[c] = __float2bfloat16_rn(w - __bfloat162float(h));
      } else {
        __nv_fp8_e4m3* hi = (__nv_fp8_e4m3*)a.ghi + (long long)row * a.kp;
        __nv_fp8_e4m3* lo = (__nv_fp8_e4m3*)a.glo + (long long)row * a.kp;
        const __nv_fp8_e4m3 h(w);
        hi[c] = h;
        lo[c] = __nv_fp8_e4m3(w - (float)h);
      }
    }
  }
}

cudaError_t launch_prepare(const Shape& s, const PopDev& p, const ExpDev& e, DevState* state,
                           int use_bred_flag, cudaStream_t st, const int* rows,
                           const PopDev* src) {
  PrepArgs a;
  a.rows = rows;
  a.g32_0 = src ? src->g32[0] : p.g32[0];
  a.g32_1 = src ? src->g32[1] : p.g32[1];
  a.colscale = e.colscale;
  a.geval = p.geval;
  a.bias = p.bias;
  a.ghi = p.ghi;
  a.glo = p.glo;
  a.rscale = p.rscale;
  a.state = state;
  a.pop = s.pop;
  a.pop_pad = s.pop_pad;
  a.kb = s.kb;
  a.kp = s.kp;
  a.kstride = s.kstride;
  a.precision = s.precision;
  a.use_bred_flag = use_bred_flag & 1;
  a.in_evolve = (use_bred_flag >> 1) & 1;
  a.src_pop = (src && src->pop_rows) ? src->pop_rows : s.pop;
  const int threads = 256;
  const int blocks = (s.pop_pad * 32 + threads - 1) / threads;
  prepare_kernel<<<blocks, threads, 0, st>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Reduce + rank (one CTA): per-chromosome sums of the fitness partials in a
// fixed order (float64), fitness (eq.4 / eq.5 / eq.10), then a bitonic sort of
// (fitness, index) and the end-of-generation state update with the stop test
// (Section 4.1 steps 2-3).
// ---------------------------------------------------------------------------
struct RankArgs {
  const double* partial;
  double* fit;
  int* rank;
  DevState* state;
  int n_part, pop, pop_pad, n2, error, mode, in_evolve, no_stop;
  double inv_m, stop_error;
};

// Order-preserving map of a float64 (NaN already replaced by +inf) to uint64,
// so that the sort compares integers (float64 units are scarce on this part).
__device__ __forceinline__ unsigned long long ordered_key(double f) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(f);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__global__ void __launch_bounds__(1024) reduce_rank_kernel(RankArgs a) {
  DevState* st = a.state;
  if (a.in_evolve && st->stopped) return;
  extern __shared__ unsigned char smem_raw[];
  unsigned long long* key = reinterpret_cast<unsigned long long*>(smem_raw);
  int* idx = reinterpret_cast<int*>(key + a.n2);
  __shared__ double best_f;
  const int tid = threadIdx.x;
  if (a.mode == kRankEvaluate && a.n_part <= 32) {
    // few partial rows: one thread per chromosome adds them in row order
    for (int c = tid; c < a.pop; c += blockDim.x) {
      const double mse = sum_partials(a.partial, a.n_part, a.pop_pad, c) * a.inv_m;
      a.fit[c] = (a.error == GAME_RMSE) ? sqrt(mse) : mse;
    }
    __syncthreads();
  } else if (a.mode == kRankEvaluate) {
    // many (one per CTA of the narrow kernels): one warp per chromosome, lane l
    // adds rows l, l + 32, ... in order, then a fixed butterfly adds the 32 lane
    // sums (deterministic; the lanes' loads overlap instead of forming one chain
    // of memory latencies)
    const int lane = tid & 31;
    for (int c = tid >> 5; c < a.pop; c += blockDim.x >> 5) {
      // eight rows are loaded before they are added, in the same order as one at a time
      double sse = 0.0;
      int b = lane;
      for (; b + 32 * 7 < a.n_part; b += 32 * 8) {
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = a.partial[(long long)(b + 32 * u) * a.pop_pad + c];
#pragma unroll
        for (int u = 0; u < 8; ++u) sse += v[u];
      }
      for (; b < a.n_part; b += 32) sse += a.partial[(long long)b * a.pop_pad + c];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sse += __shfl_xor_sync(0xffffffffu, sse, o);
      if (lane == 0) {
        const double mse = sse * a.inv_m;
        a.fit[c] = (a.error == GAME_RMSE) ? sqrt(mse) : mse;
      }
    }
    __syncthreads();
  }
  for (int c = tid; c < a.n2; c += blockDim.x) {
    double f = CUDART_INF;
    if (c < a.pop) {
      f = a.fit[c];
      if (isnan(f)) f = CUDART_INF;
    }
    key[c] = ordered_key(f);
    idx[c] = c < a.pop ? c : 0x7fffffff;
  }
  __syncthreads();
  for (int k = 2; k <= a.n2; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = tid; i < a.n2; i += blockDim.x) {
        const int l = i ^ j;
        if (l > i) {
          const bool up = (i & k) == 0;
          const unsigned long long ki = key[i], kl = key[l];
          const int ii = idx[i], il = idx[l];
          const bool lt = kl < ki || (kl == ki && il < ii);
          if (lt == up) {
            key[i] = kl;
            key[l] = ki;
            idx[i] = il;
            idx[l] = ii;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int c = tid; c < a.pop; c += blockDim.x) a.rank[c] = idx[c];
  if (tid == 0) {
    const double f0 = a.fit[idx[0]];
    best_f = isnan(f0) ? CUDART_INF : f0;
    st->best = best_f;
    if (a.mode == kRankEvaluate) {
      if (st->bred) {
        st->cur ^= 1;
        st->gen += 1;
      }
      st->bred = 0;
      st->gens_run += 1;
      st->evals += 1;
    }
    if (a.mode != kRankSortOnly && !a.no_stop && a.in_evolve && best_f <= a.stop_error)
      st->stopped = 1;
    st->evaluated = 1;
  }
}

// ---- large populations: the same result without a single-CTA sort ----
// fit[c] from the partial sums (many CTAs).
// 256-thread blocks over 32 consecutive chromosomes: warp g adds partial rows g, g + 8,
// g + 16, ... (each load coalesced over the 32 chromosomes, four in flight), then the
// eight group sums are added in group order.  The order is fixed by n_part alone.
constexpr int kRedGroups = 8;

__device__ __forceinline__ double group_partial_sum(const double* __restrict__ partial,
                                                    int n_part, long long stride, long long c,
                                                    int g) {
  double s = 0.0;
  int b = g;
  for (; b + 3 * kRedGroups < n_part; b += 4 * kRedGroups) {
    double v[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = partial[(long long)(b + i * kRedGroups) * stride + c];
#pragma unroll
    for (int i = 0; i < 4; ++i) s += v[i];
  }
  for (; b < n_part; b += kRedGroups) s += partial[(long long)b * stride + c];
  return s;
}

// sse of chromosome blockIdx.x * 32 + lane, valid in warp 0 (n: chromosomes).
__device__ __forceinline__ double block_sse(const double* __restrict__ partial, int n_part,
                                            long long stride, int n, double (*part)[32]) {
  const int l = threadIdx.x & 31, g = threadIdx.x >> 5;
  const int c = blockIdx.x * 32 + l;
  part[g][l] = c < n ? group_partial_sum(partial, n_part, stride, c, g) : 0.0;
  __syncthreads();
  double s = part[0][l];
#pragma unroll
  for (int i = 1; i < kRedGroups; ++i) s += part[i][l];
  return s;
}

__global__ void __launch_bounds__(256) fit_reduce_kernel(RankArgs a) {
  if (a.in_evolve && a.state->stopped) return;   // uniform over the block
  __shared__ double part[kRedGroups][32];
  const double sse = block_sse(a.partial, a.n_part, a.pop_pad, a.pop, part);
  const int c = blockIdx.x * 32 + (threadIdx.x & 31);
  if (threadIdx.x < 32 && c < a.pop) {
    const double mse = sse * a.inv_m;
    a.fit[c] = (a.error == GAME_RMSE) ? sqrt(mse) : mse;
  }
}

// The state transition of a ranking (one thread), as in reduce_rank_kernel; rank0 is
// the chromosome at the first rank position.
__device__ void apply_rank_state(const RankArgs& a, int rank0) {
  DevState* st = a.state;
  const double f0 = a.fit[rank0];
  const double best = isnan(f0) ? CUDART_INF : f0;
  st->best = best;
  if (a.mode == kRankEvaluate) {
    if (st->bred) {
      st->cur ^= 1;
      st->gen += 1;
    }
    st->bred = 0;
    st->gens_run += 1;
    st->evals += 1;
  }
  if (a.mode != kRankSortOnly && !a.no_stop && a.in_evolve && best <= a.stop_error)
    st->stopped = 1;
  st->evaluated = 1;
}

// Rank by counting: the position of chromosome c is the number of chromosomes
// before it in the order (fitness, index) (NaN as +inf), so rank[pos] = c.  One
// warp per c splits the comparisons; keys are staged per 1024.  The last block to
// finish (a fenced counter; nothing waits on it) applies the state transition.
__global__ void __launch_bounds__(256) rank_count_kernel(RankArgs a) {
  if (a.in_evolve && a.state->stopped) return;
  __shared__ unsigned long long tile[1024];
  const int lane = threadIdx.x & 31;
  const int c = blockIdx.x * 8 + (threadIdx.x >> 5);
  unsigned long long kc = 0;
  if (c < a.pop) {
    const double f = a.fit[c];
    kc = ordered_key(isnan(f) ? CUDART_INF : f);
  }
  int pos = 0;
  for (int t0 = 0; t0 < a.pop; t0 += 1024) {
    const int n = min(1024, a.pop - t0);
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const double f = a.fit[t0 + i];
      tile[i] = ordered_key(isnan(f) ? CUDART_INF : f);
    }
    __syncthreads();
    if (c < a.pop)
      for (int i = lane; i < n; i += 32) {
        const unsigned long long kj = tile[i];
        pos += (kj < kc) || (kj == kc && t0 + i < c);
      }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) pos += __shfl_xor_sync(0xffffffffu, pos, o);
  if (c < a.pop && lane == 0 && GAME_IN_BOUNDS_DBG(pos >= 0 && pos < a.pop, kSiteRankIndex, pos))
    a.rank[pos] = c;
  // this block's rank writes are visible device-wide before it is counted
  __threadfence();
  __syncthreads();
  __shared__ unsigned int done_before;
  if (threadIdx.x == 0) done_before = atomicAdd(&a.state->rank_done, 1u);
  __syncthreads();
  if (threadIdx.x == 0 && done_before == gridDim.x - 1) {
    __threadfence();
    a.state->rank_done = 0;                       // ready for the next launch
    apply_rank_state(a, __ldcg(a.rank));
  }
}

static int next_pow2(int n) {
  int p = 2;
  while (p < n) p <<= 1;
  return p;
}

cudaError_t launch_reduce_rank(const Shape& s, const game_config& cfg, const double* partial,
                               int n_part, double* fit, int* rank, DevState* state, int mode,
                               cudaStream_t st) {
  RankArgs a;
  a.partial = partial;
  a.fit = fit;
  a.rank = rank;
  a.state = state;
  a.n_part = n_part;
  a.pop = s.pop;
  a.pop_pad = s.pop_pad;
  a.n2 = next_pow2(s.pop);
  a.error = cfg.error;
  a.mode = mode & 0xff;
  a.in_evolve = (mode >> 8) & 1;
  a.no_stop = (mode >> 9) & 1;
  a.inv_m = 1.0 / (double)s.n_train;
  a.stop_error = cfg.stop_error;
  if (s.pop >= kRankCountMin) {
    if (a.mode == kRankEvaluate) fit_reduce_kernel<<<(s.pop + 31) / 32, 256, 0, st>>>(a);
    rank_count_kernel<<<(s.pop + 7) / 8, 256, 0, st>>>(a);
    return cudaGetLastError();
  }
  const size_t smem = (size_t)a.n2 * (sizeof(unsigned long long) + sizeof(int));
  // n2 threads for the sort; with many partial rows, one warp per chromosome
  int threads = a.n2 < 32 ? 32 : a.n2;
  if (n_part > 32 && threads < 32 * s.pop) threads = 32 * s.pop;
  if (threads > 1024) threads = 1024;
  reduce_rank_kernel<<<1, threads, smem, st>>>(a);
  return cudaGetLastError();
}

// FP32 re-score of the elites: fitness of rank[i] (i < n) from the partial sums of
// the FP32 engine over the gathered rows.
__global__ void __launch_bounds__(256) rescore_merge_kernel(const double* partial, int n_part,
                                                            int pop_pad, int n, const int* rank,
                                                            double* fit, double inv_m, int error,
                                                            const DevState* st, int in_evolve) {
  if (in_evolve && st->stopped) return;          // uniform over the block
  __shared__ double part[kRedGroups][32];
  const double sse = block_sse(partial, n_part, pop_pad, n, part);
  const int i = blockIdx.x * 32 + (threadIdx.x & 31);
  if (threadIdx.x < 32 && i < n) {
    const double mse = sse * inv_m;
    fit[rank[i]] = error == GAME_RMSE ? sqrt(mse) : mse;
  }
}

cudaError_t launch_rescore_merge(const Shape& sr, const game_config& cfg, const double* partial,
                                 int n_part, const int* rank, double* fit, const DevState* state,
                                 int in_evolve, cudaStream_t st) {
  rescore_merge_kernel<<<(sr.pop + 31) / 32, 256, 0, st>>>(
      partial, n_part, sr.pop_pad, sr.pop, rank, fit, 1.0 / (double)sr.n_train, cfg.error, state,
      in_evolve);
  return cudaGetLastError();
}

cudaError_t ga_init_attributes() {
  return cudaFuncSetAttribute(reduce_rank_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              8192 * (int)(sizeof(double) + sizeof(int)));
}

// ---------------------------------------------------------------------------
// Single-thread state transitions.
// ---------------------------------------------------------------------------
__global__ void state_kernel(DevState* st, int op) {
  switch (op) {
    case kStateReset:
      st->gen = 0;
      st->cur = 0;
      st->evaluated = 0;
      st->bred = 0;
      st->stopped = 0;
      st->gens_run = 0;
      st->evals = 0;
      st->status = 0;
      st->best = CUDART_INF;
      break;
    case kStatePopulationSet:
      st->evaluated = 0;
      st->bred = 0;
      st->stopped = 0;
      break;
    case kStateBeginEvolve:
      st->gens_run = 0;
      break;
    case kStateClearStatus:
      st->status = 0;
      break;
    case kStateAfterBreed:
      if (st->bred) {
        st->cur ^= 1;
        st->gen += 1;
      }
      st->bred = 0;
      st->evaluated = 0;
      break;
    default:
      break;
  }
}

cudaError_t launch_state_op(DevState* state, int op, cudaStream_t st) {
  state_kernel<<<1, 1, 0, st>>>(state, op);
  return cudaGetLastError();
}

}  // namespace game

namespace game {
GAME_DEFINE_CHECK_READER(check_word_ga)
}  // namespace game
