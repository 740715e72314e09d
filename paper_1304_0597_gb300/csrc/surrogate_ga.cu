// Kernels of the surrogate-driven generation: an oversized offspring pool bred
// with the same operators as plain breeding, selection of the children the
// surrogate ranks best, assembly of the next population, the replay ring of
// exact (chromosome, fitness) pairs, the accuracy monitor (Spearman correlation
// of predicted against exact fitness, with a fallback to plain selection) and
// the training batches.
#include "rng.cuh"
#include "surrogate.h"

namespace game {

namespace {

constexpr size_t kSelectSmem = 160 * 1024;   // pools up to 40,960 children keep keys on chip

__device__ __forceinline__ uint32_t ordered_f32(float f) {
  if (f != f) return 0xFFFFFFFFu;   // NaN ranks last
  const uint32_t b = __float_as_uint(f);
  return (b >> 31) ? ~b : (b | 0x80000000u);
}

// ---- pool breeding: pair j writes pool rows 2j and 2j+1 ----
__global__ void pool_breed_kernel(PoolArgs a) {
  const DevState* st = a.state;
  if (!(st->evaluated && !st->stopped)) return;
  const int warp = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  const int n_pairs = (a.n_pool + 1) / 2;
  if (warp >= n_pairs) return;
  const float* G = st->cur ? a.g32_1 : a.g32_0;
  const int sa = 2 * warp, sb = sa + 1;
  breed_pair(G, a.kstride, a.n_genes, a.pop, a.fit, a.cum, Key{a.k0, a.k1}, (uint64_t)st->gen,
             (uint64_t)warp, a.tournament_k, a.p_c, a.p_m, a.sigma, a.clamp,
             a.pool + (long long)sa * a.kstride, a.pool + (long long)sb * a.kstride, sb < a.n_pool,
             lane);
}

// ---- selection (one CTA): the n_sel lowest scores, ties by lower index ----
// Block-wide exclusive scan of one int per thread (1024 threads); returns the
// total.  wt holds 32 + 1 ints of shared scratch.
__device__ __forceinline__ int block_excl_scan(int v, int* wt, int* excl) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) wt[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const int t = lane < (int)(blockDim.x >> 5) ? wt[lane] : 0;
    int ti = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, ti, o);
      if (lane >= o) ti += y;
    }
    wt[lane] = ti - t;
    if (lane == 31) wt[32] = ti;
  }
  __syncthreads();
  *excl = wt[warp] + incl - v;
  const int total = wt[32];
  __syncthreads();   // wt is reused by the next call
  return total;
}

__global__ void __launch_bounds__(1024) select_kernel(const float* __restrict__ score, int n_pool,
                                                      int n_sel, int* __restrict__ sel,
                                                      DevState* st, const int* fallback,
                                                      int random_select, int keys_in_smem) {
  const int decision = st->evaluated && !st->stopped;
  if (threadIdx.x == 0) st->bred = decision;
  if (!decision) return;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (random_select || *fallback) {
    for (int i = tid; i < n_sel; i += nt) sel[i] = i;
    return;
  }
  __shared__ int hist[256];
  __shared__ int wt[33];
  __shared__ uint32_t sel_prefix;
  __shared__ int sel_left;
  // keys staged in shared memory when the pool fits (dynamic size n_pool words)
  extern __shared__ uint32_t skey[];
  if (keys_in_smem) {
    for (int i = tid; i < n_pool; i += nt) skey[i] = ordered_f32(score[i]);
  }
  auto key_at = [&](int i) -> uint32_t {
    return keys_in_smem ? skey[i] : ordered_f32(score[i]);
  };
  // tau = the n_sel-th smallest key (smallest tau with count(key <= tau) >= n_sel),
  // by radix selection over the four bytes of the key, most significant first
  if (tid == 0) {
    sel_prefix = 0u;
    sel_left = n_sel;
  }
  for (int shift = 24; shift >= 0; shift -= 8) {
    for (int i = tid; i < 256; i += nt) hist[i] = 0;
    __syncthreads();
    const uint32_t prefix = sel_prefix;
    const uint32_t hmask = shift == 24 ? 0u : (0xFFFFFFFFu << (shift + 8));
    // children's scores share their leading bytes: a thread adds each run of equal
    // bins with one atomic
    int prev = -1, run = 0;
    for (int i = tid; i < n_pool; i += nt) {
      const uint32_t k = key_at(i);
      const int bin = (k & hmask) == (prefix & hmask) ? (int)((k >> shift) & 255u) : -1;
      if (bin != prev) {
        if (run) atomicAdd(&hist[prev], run);
        prev = bin;
        run = 0;
      }
      if (bin >= 0) ++run;
    }
    if (run) atomicAdd(&hist[prev], run);
    __syncthreads();
    if (tid < 32) {
      // lane l owns bins 8l .. 8l+7; find the bin where the running count reaches sel_left
      int c[8], tot = 0;
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        c[b] = hist[tid * 8 + b];
        tot += c[b];
      }
      int incl = tot;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (tid >= o) incl += y;
      }
      const int left = sel_left;
      const unsigned hit = __ballot_sync(0xffffffffu, incl >= left);
      const int owner = __ffs(hit) - 1;   // hist sums to >= left, so some lane hits
      if (tid == owner) {
        int run2 = incl - tot;
        int b = 0;
        while (b < 7 && run2 + c[b] < left) run2 += c[b++];
        sel_prefix = prefix | ((uint32_t)(tid * 8 + b) << shift);
        sel_left = left - run2;
      }
    }
    __syncthreads();
  }
  const uint32_t tau = sel_prefix;
  // Ordered compaction, 4 consecutive keys per thread per chunk of 4 nt: pass 0
  // takes every key < tau, pass 1 the first keys == tau until n_sel are taken.
  int start = 0;
  for (int pass = 0; pass < 2; ++pass) {
    for (int c0 = 0; c0 < n_pool; c0 += 4 * nt) {
      const int i0 = c0 + 4 * tid;
      bool pr[4];
      int cnt = 0;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = i0 + q;
        bool p = false;
        if (i < n_pool) {
          const uint32_t k = key_at(i);
          p = pass == 0 ? (k < tau) : (k == tau);
        }
        pr[q] = p;
        cnt += p;
      }
      int excl;
      const int total = block_excl_scan(cnt, wt, &excl);
      int pos = start + excl;
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (pr[q]) {
          if (pos < n_sel) sel[pos] = i0 + q;
          ++pos;
        }
      start += total;
    }
  }
}

// ---- next population: elites of the current one, then the selected children ----
__global__ void assemble_kernel(const float* __restrict__ pool, const int* __restrict__ sel,
                                const float* __restrict__ score, const float* g32_0,
                                const float* g32_1, float* out_0, float* out_1,
                                const int* __restrict__ rank, const DevState* st, int pop, int e,
                                int elite_copies, int n_genes, int kstride,
                                float* __restrict__ pred) {
  if (!st->bred) return;
  const int row = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= pop) return;
  const float* G = st->cur ? g32_1 : g32_0;
  float* out = st->cur ? out_0 : out_1;
  const float* src;
  float pv;
  if (row < e) {
    src = G + (long long)(elite_copies ? rank[0] : rank[row]) * kstride;
    pv = CUDART_NAN_F;
  } else {
    const int k = sel[row - e];
    src = pool + (long long)k * kstride;
    pv = score[k];
  }
  float* dst = out + (long long)row * kstride;
  for (int g = lane; g < n_genes; g += 32) dst[g] = src[g];
  if (lane == 0) pred[row] = pv;
}

// ---- replay ring: append the evaluated population (many CTAs) ----
__global__ void replay_copy_kernel(const float* g32_0, const float* g32_1, const double* fit,
                                   const DevState* st, int pop, int n_genes, int kstride,
                                   float* ring_x, float* ring_f, const int* ring_meta,
                                   int ring_cap, const float* norm) {
  if (st->evals == ring_meta[2]) return;   // nothing evaluated since the last append
  const int row = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= pop) return;
  const float* G = (st->cur ? g32_1 : g32_0) + (long long)row * kstride;
  const int slot = (ring_meta[0] + row) % ring_cap;
  float* dst = ring_x + (long long)slot * kstride;
  for (int g = lane; g < n_genes; g += 32) dst[g] = G[g];
  // target: log fitness standardised within its own generation, so that the
  // network learns what ranks children of the same population
  if (lane == 0)
    ring_f[slot] = (logf(fmaxf((float)fit[row], 1e-30f)) - norm[0]) / norm[1];
}

// Ring bookkeeping after the copy (one thread).
__global__ void replay_commit_kernel(const DevState* st, int pop, int* ring_meta, int ring_cap) {
  if (st->evals == ring_meta[2]) return;
  ring_meta[0] = (ring_meta[0] + pop) % ring_cap;
  ring_meta[1] = min(ring_cap, ring_meta[1] + pop);
  ring_meta[2] = st->evals;
}

// ---- monitor: rank difference of every non-elite row (many CTAs) ----
// Ranks by counting over keys (value, row) ordered as floats, row as the tie
// break: rank = number of rows with a smaller key.  One warp per row.
__device__ __forceinline__ unsigned long long spearman_key(const float* pred, const double* fit,
                                                           int e, int i, int which) {
  const float v = which == 0 ? pred[e + i] : (float)fit[e + i];
  return ((unsigned long long)ordered_f32(v) << 32) | (uint32_t)i;
}

__global__ void __launch_bounds__(256) spearman_dsq_kernel(const double* fit, const float* pred,
                                                           const DevState* st, int pop, int e,
                                                           const int* ring_meta,
                                                           long long* dsq) {
  if (st->evals == ring_meta[2]) return;
  const int n = pop - e;
  if (!(n >= 3 && !(pred[e] != pred[e]))) return;
  __shared__ unsigned long long tp[1024], tf[1024];
  const int sub = threadIdx.x & 31;
  const int i = blockIdx.x * 8 + (threadIdx.x >> 5);
  const unsigned long long kp = i < n ? spearman_key(pred, fit, e, i, 0) : 0ull;
  const unsigned long long kf = i < n ? spearman_key(pred, fit, e, i, 1) : 0ull;
  int rp = 0, rf = 0;
  for (int t0 = 0; t0 < n; t0 += 1024) {
    const int m = min(1024, n - t0);
    __syncthreads();
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
      tp[j] = spearman_key(pred, fit, e, t0 + j, 0);
      tf[j] = spearman_key(pred, fit, e, t0 + j, 1);
    }
    __syncthreads();
    if (i < n)
      for (int j = sub; j < m; j += 32) {
        rp += tp[j] < kp;
        rf += tf[j] < kf;
      }
  }
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    rp += __shfl_xor_sync(0xffffffffu, rp, o);
    rf += __shfl_xor_sync(0xffffffffu, rf, o);
  }
  if (i < n && sub == 0) {
    const long long d = (long long)(rp - rf);
    dsq[i] = d * d;
  }
}

// ---- monitor and the generation's target standardisation (one CTA) ----
__global__ void __launch_bounds__(1024) replay_stats_kernel(const double* fit, const float* pred,
                                                            const DevState* st, int pop, int e,
                                                            int* ring_meta, float* norm,
                                                            double* monitor, int* fallback,
                                                            float fallback_rho,
                                                            const long long* dsq) {
  if (st->evals == ring_meta[2]) return;
  const int tid = threadIdx.x, nt = blockDim.x;
  __shared__ double red[1024];
  __shared__ double red2[1024];
  // Spearman correlation of predicted and exact fitness over rows e..pop-1 with a
  // prediction (rows of an untrained or fallback generation still carry one):
  // 1 - 6 sum d^2 / (n (n^2 - 1)), d the rank differences (integers: the sum is exact).
  const int n = pop - e;
  double rho = CUDART_NAN;
  const bool have_pred = n >= 3 && !(pred[e] != pred[e]);
  if (have_pred) {
    long long sdd = 0;
    for (int i = tid; i < n; i += nt) sdd += dsq[i];
    red[tid] = (double)sdd;
    __syncthreads();
    for (int o = nt >> 1; o > 0; o >>= 1) {
      if (tid < o) red[tid] += red[tid + o];
      __syncthreads();
    }
    rho = 1.0 - 6.0 * red[0] / ((double)n * ((double)n * n - 1.0));
    __syncthreads();
  }
  // mean / std of log fitness over this generation's population
  // (float32 logarithm, the one the ring's targets use; float64 sums)
  double s1 = 0.0, s2 = 0.0;
  for (int i = tid; i < pop; i += nt) {
    const double l = (double)logf(fmaxf((float)fit[i], 1e-30f));
    s1 += l;
    s2 += l * l;
  }
  red[tid] = s1;
  red2[tid] = s2;
  __syncthreads();
  for (int o = nt >> 1; o > 0; o >>= 1) {
    if (tid < o) {
      red[tid] += red[tid + o];
      red2[tid] += red2[tid + o];
    }
    __syncthreads();
  }
  if (tid == 0) {
    const double mu = red[0] / pop;
    const double var = fmax(red2[0] / pop - mu * mu, 1e-18);
    norm[0] = (float)mu;
    norm[1] = (float)sqrt(var);
    const int g = ring_meta[3];
    monitor[g % 4096] = rho;
    ring_meta[3] = g + 1;
    // fall back to plain selection while the surrogate ranks children poorly
    if (have_pred) *fallback = (rho == rho && rho < (double)fallback_rho) ? 1 : 0;
  }
}

// ---- training batch: B rows drawn uniformly from the ring ----
__global__ void sample_batch_kernel(const float* __restrict__ ring_x, const float* __restrict__ ring_f,
                                    const int* __restrict__ ring_meta, int kstride, int n_genes,
                                    const float* __restrict__ norm, int B, Key key, uint64_t salt,
                                    int step, const DevState* st, float* __restrict__ bx,
                                    float* __restrict__ bt) {
  const int row = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= B) return;
  const int count = ring_meta[1];
  const uint32_t w = philox_word(key, (uint64_t)st->evals, salt + (uint64_t)step, 6, (uint64_t)row);
  const int idx = count > 0 ? index_draw(w, count) : 0;
  const float* src = ring_x + (long long)idx * kstride;
  float* dst = bx + (long long)row * kstride;
  for (int g = lane; g < n_genes; g += 32) dst[g] = src[g];
  if (lane == 0) bt[row] = ring_f[idx];
}

// ---- input standardisation of the bf16 form: running per-gene statistics ----
constexpr float kStatsWeight = 0.3f;   // weight of the newest population in the running average
// Block of 32 genes x 32 row groups; the mean and variance of the population just
// evaluated enter an exponential average (weight 0.3; the first generation sets
// it), and scale = 1 / sqrt(var + 1e-6).
__global__ void gene_stats_kernel(const float* g32_0, const float* g32_1, const DevState* st,
                                  const int* ring_meta, int pop, int D, int kstride,
                                  float* gnorm) {
  if (st->evals == ring_meta[2]) return;   // nothing evaluated since the last update
  __shared__ float s1[32][33], s2[32][33];
  const float* G = st->cur ? g32_1 : g32_0;
  const int d = blockIdx.x * 32 + threadIdx.x;
  float a = 0.0f, b = 0.0f;
  if (d < D)
    for (int r = threadIdx.y; r < pop; r += 32) {
      const float v = G[(long long)r * kstride + d];
      a += v;
      b += v * v;
    }
  s1[threadIdx.y][threadIdx.x] = a;
  s2[threadIdx.y][threadIdx.x] = b;
  __syncthreads();
  if (threadIdx.y == 0 && d < D) {
    float ta = 0.0f, tb = 0.0f;
    for (int i = 0; i < 32; ++i) {
      ta += s1[i][threadIdx.x];
      tb += s2[i][threadIdx.x];
    }
    const float mu = ta / (float)pop;
    const float var = fmaxf(tb / (float)pop - mu * mu, 0.0f);
    const float w = ring_meta[3] > 0 ? kStatsWeight : 1.0f;   // monitor's generation count (read only)
    const float m2 = (1.0f - w) * gnorm[d] + w * mu;
    const float v2 = (1.0f - w) * gnorm[2 * D + d] + w * var;
    gnorm[d] = m2;
    gnorm[2 * D + d] = v2;
    gnorm[D + d] = rsqrtf(v2 + 1e-6f);
  }
}

// ---- training batch straight into the tensor-core operands (bf16 form) ----
// Same draws as sample_batch_kernel; a CTA takes 32 rows x 32 genes through a
// shared tile so that both the row-major and the transposed bf16 stores coalesce.
__global__ void sample_batch_tc_kernel(const float* __restrict__ ring_x,
                                       const float* __restrict__ ring_f,
                                       const int* __restrict__ ring_meta, int kstride, int D,
                                       int B, Key key, uint64_t salt, int step, const DevState* st,
                                       __nv_bfloat16* __restrict__ Xb, int Dp,
                                       __nv_bfloat16* __restrict__ XT, long long ldt,
                                       float* __restrict__ bt, const float* __restrict__ gnorm) {
  __shared__ float tile[32][33];
  __shared__ int rows[32];
  const int d0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  if (ty == 0) {
    const int r = r0 + tx;
    int idx = 0;
    if (r < B) {
      const int count = ring_meta[1];
      const uint32_t w = philox_word(key, (uint64_t)st->evals, salt + (uint64_t)step, 6, (uint64_t)r);
      idx = count > 0 ? index_draw(w, count) : 0;
      if (blockIdx.x == 0) bt[r] = ring_f[idx];
    }
    rows[tx] = idx;
  }
  __syncthreads();
  for (int i = ty; i < 32; i += 8) {
    const int r = r0 + i, d = d0 + tx;
    float v = 0.0f;
    if (r < B && d < D) {
      v = ring_x[(long long)rows[i] * kstride + d];
      v = (v - gnorm[d]) * gnorm[D + d];   // running per-gene standardisation
      Xb[(long long)r * Dp + d] = __float2bfloat16_rn(v);
    }
    tile[i][tx] = v;
  }
  __syncthreads();
  for (int i = ty; i < 32; i += 8) {
    const int d = d0 + i, r = r0 + tx;
    if (d < D && r < B) XT[(long long)d * ldt + r] = __float2bfloat16_rn(tile[tx][i]);
  }
}

// ---- initial weights: U[-a, a], a = sqrt(3 / fan_in); biases 0 ----
__global__ void surrogate_init_kernel(float* p, __nv_bfloat16* ph, float* m, float* v, long long n,
                                      long long n_w1, long long n_b1, long long n_w2,
                                      long long n_b2, long long n_w3, int D, int H, Key key) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float a = 0.0f;
  if (i < n_w1) a = sqrtf(3.0f / D);
  else if (i >= n_w1 + n_b1 && i < n_w1 + n_b1 + n_w2) a = sqrtf(3.0f / H);
  else if (i >= n_w1 + n_b1 + n_w2 + n_b2 && i < n_w1 + n_b1 + n_w2 + n_b2 + n_w3) a = sqrtf(3.0f / H);
  const float u = uniform24(philox_word(key, 0, (uint64_t)i, 7, 0));
  const float w = a * (2.0f * u - 1.0f);
  p[i] = w;
  ph[i] = __float2bfloat16_rn(w);
  m[i] = 0.0f;
  v[i] = 0.0f;
}

}  // namespace

cudaError_t launch_pool_breed(const PoolArgs& a, cudaStream_t st) {
  const int pairs = (a.n_pool + 1) / 2;
  pool_breed_kernel<<<(pairs * 32 + 255) / 256, 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_select(const float* score, int n_pool, int n_sel, int* sel, DevState* state,
                          const int* fallback, int random_select, cudaStream_t st) {
  const int in_smem = (size_t)n_pool * sizeof(uint32_t) <= kSelectSmem ? 1 : 0;
  select_kernel<<<1, 1024, in_smem ? (size_t)n_pool * sizeof(uint32_t) : 0, st>>>(
      score, n_pool, n_sel, sel, state, fallback, random_select, in_smem);
  return cudaGetLastError();
}

cudaError_t launch_assemble(const float* pool, const int* sel, const float* score, const PopDev& p,
                            const Shape& s, int elitism, int elite_copies, const int* rank,
                            const DevState* state, float* pred, cudaStream_t st) {
  assemble_kernel<<<(s.pop * 32 + 255) / 256, 256, 0, st>>>(
      pool, sel, score, p.g32[0], p.g32[1], p.g32[0], p.g32[1], rank, state, s.pop, elitism,
      elite_copies, s.n_genes, s.kstride, pred);
  return cudaGetLastError();
}

cudaError_t launch_replay_update(const PopDev& p, const Shape& s, int elitism, const double* fit,
                                 const float* pred, DevState* state, float* ring_x,
                                 float* ring_f, int* ring_meta, int ring_cap, float* norm,
                                 double* monitor, int* fallback, float fallback_rho,
                                 long long* dsq, cudaStream_t st) {
  const int n = s.pop - elitism;
  if (n > 0)
    spearman_dsq_kernel<<<(n + 7) / 8, 256, 0, st>>>(fit, pred, state, s.pop, elitism, ring_meta,
                                                       dsq);
  replay_stats_kernel<<<1, 1024, 0, st>>>(fit, pred, state, s.pop, elitism, ring_meta, norm,
                                          monitor, fallback, fallback_rho, dsq);
  replay_copy_kernel<<<(s.pop * 32 + 255) / 256, 256, 0, st>>>(
      p.g32[0], p.g32[1], fit, state, s.pop, s.n_genes, s.kstride, ring_x, ring_f, ring_meta,
      ring_cap, norm);
  replay_commit_kernel<<<1, 1, 0, st>>>(state, s.pop, ring_meta, ring_cap);
  return cudaGetLastError();
}

cudaError_t launch_sample_batch(const float* ring_x, const float* ring_f, const int* ring_meta,
                                int kstride, int n_genes, const float* norm, int B, uint64_t k0,
                                uint64_t k1, uint64_t gen_salt, int step, const DevState* state,
                                float* bx, float* bt, cudaStream_t st) {
  sample_batch_kernel<<<(B * 32 + 255) / 256, 256, 0, st>>>(ring_x, ring_f, ring_meta, kstride,
                                                             n_genes, norm, B, Key{k0, k1},
                                                             gen_salt, step, state, bx, bt);
  return cudaGetLastError();
}

cudaError_t launch_sample_batch_tc(const float* ring_x, const float* ring_f, const int* ring_meta,
                                   int kstride, const Surrogate& sg, int B, uint64_t k0,
                                   uint64_t k1, uint64_t gen_salt, int step, const DevState* state,
                                   float* bt, cudaStream_t st) {
  const dim3 grid((sg.D + 31) / 32, (B + 31) / 32);
  sample_batch_tc_kernel<<<grid, dim3(32, 8), 0, st>>>(ring_x, ring_f, ring_meta, kstride, sg.D, B,
                                                       Key{k0, k1}, gen_salt, step, state, sg.Xb,
                                                       sg.Dp, sg.XTb, sg.ldt, bt, sg.gnorm);
  return cudaGetLastError();
}

cudaError_t launch_gene_stats(const PopDev& p, const Shape& s, const DevState* state,
                              const int* ring_meta, Surrogate& sg, cudaStream_t st) {
  gene_stats_kernel<<<(s.n_genes + 31) / 32, dim3(32, 32), 0, st>>>(
      p.g32[0], p.g32[1], state, ring_meta, s.pop, s.n_genes, s.kstride, sg.gnorm);
  return cudaGetLastError();
}

cudaError_t surrogate_ga_init_attributes() {
  return cudaFuncSetAttribute(select_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)kSelectSmem);
}

cudaError_t launch_surrogate_init(Surrogate& sg, uint64_t seed, cudaStream_t st) {
  const long long n = (long long)sg.n_params();
  const long long n_w1 = (long long)sg.H * sg.D, n_b1 = sg.H, n_w2 = (long long)sg.H * sg.H,
                  n_b2 = sg.H, n_w3 = sg.H;
  surrogate_init_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
      sg.p, sg.ph, sg.m, sg.v, n, n_w1, n_b1, n_w2, n_b2, n_w3, sg.D, sg.H, Key{seed, 0x5u});
  cudaError_t e = cudaMemsetAsync(sg.step, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace game
