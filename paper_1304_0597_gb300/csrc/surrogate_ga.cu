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
  breed_pair(G, a.kstride, a.n_genes, a.pop, a.fit, Key{a.k0, a.k1}, (uint64_t)st->gen,
             (uint64_t)warp, a.tournament_k, a.p_c, a.p_m, a.sigma, a.clamp,
             a.pool + (long long)sa * a.kstride, a.pool + (long long)sb * a.kstride, sb < a.n_pool,
             lane);
}

// ---- selection (one CTA): the n_sel lowest scores, ties by lower index ----
__global__ void __launch_bounds__(1024) select_kernel(const float* __restrict__ score, int n_pool,
                                                      int n_sel, int* __restrict__ sel,
                                                      DevState* st, const int* fallback,
                                                      int random_select) {
  const int decision = st->evaluated && !st->stopped;
  if (threadIdx.x == 0) st->bred = decision;
  if (!decision) return;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (random_select || *fallback) {
    for (int i = tid; i < n_sel; i += nt) sel[i] = i;
    return;
  }
  __shared__ int cnt;
  __shared__ int scan[1024];
  // smallest threshold tau with count(key <= tau) >= n_sel (binary search on the key)
  uint32_t lo = 0u, hi = 0xFFFFFFFFu;
  while (lo < hi) {
    const uint32_t mid = lo + ((hi - lo) >> 1);
    if (tid == 0) cnt = 0;
    __syncthreads();
    int c = 0;
    for (int i = tid; i < n_pool; i += nt) c += ordered_f32(score[i]) <= mid;
    atomicAdd(&cnt, c);
    __syncthreads();
    const int total = cnt;
    __syncthreads();
    if (total >= n_sel) hi = mid;
    else lo = mid + 1;
  }
  const uint32_t tau = lo;
  // compaction in index order: thread t owns the contiguous range [t*chunk, (t+1)*chunk);
  // pass 0 takes every key < tau, pass 1 the first keys == tau up to n_sel.
  const int chunk = (n_pool + nt - 1) / nt;
  const int b0 = min(n_pool, tid * chunk), b1 = min(n_pool, b0 + chunk);
  __shared__ int start_s;
  if (tid == 0) start_s = 0;
  __syncthreads();
  for (int pass = 0; pass < 2; ++pass) {
    int c = 0;
    for (int i = b0; i < b1; ++i) {
      const uint32_t k = ordered_f32(score[i]);
      c += pass == 0 ? (k < tau) : (k == tau);
    }
    scan[tid] = c;
    __syncthreads();
    for (int o = 1; o < nt; o <<= 1) {
      const int v = tid >= o ? scan[tid - o] : 0;
      __syncthreads();
      scan[tid] += v;
      __syncthreads();
    }
    int pos = start_s + scan[tid] - c;
    for (int i = b0; i < b1; ++i) {
      const uint32_t k = ordered_f32(score[i]);
      if (pass == 0 ? (k < tau) : (k == tau)) {
        if (pos < n_sel) sel[pos] = i;
        ++pos;
      }
    }
    __syncthreads();
    if (tid == 0) start_s += scan[nt - 1];
    __syncthreads();
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

// ---- monitor and the generation's target standardisation (one CTA) ----
__global__ void __launch_bounds__(1024) replay_stats_kernel(const double* fit, const float* pred,
                                                            const DevState* st, int pop, int e,
                                                            int* ring_meta, float* norm,
                                                            double* monitor, int* fallback,
                                                            float fallback_rho) {
  if (st->evals == ring_meta[2]) return;
  extern __shared__ unsigned char sm[];
  unsigned long long* key = reinterpret_cast<unsigned long long*>(sm);
  const int tid = threadIdx.x, nt = blockDim.x;
  __shared__ double red[1024];
  __shared__ double red2[1024];
  // Spearman correlation of predicted and exact fitness over rows e..pop-1 with a
  // prediction (rows of an untrained or fallback generation still carry one).
  const int n = pop - e;
  int n2 = 2;
  while (n2 < n) n2 <<= 1;
  int* rk_pred = reinterpret_cast<int*>(key + n2);
  double rho = CUDART_NAN;
  const bool have_pred = n >= 3 && !(pred[e] != pred[e]);
  if (have_pred) {
    for (int pass = 0; pass < 2; ++pass) {
      for (int i = tid; i < n2; i += nt) {
        uint64_t k = 0xFFFFFFFFFFFFFFFFull;
        if (i < n) {
          const float v = pass == 0 ? pred[e + i] : (float)fit[e + i];
          k = ((uint64_t)ordered_f32(v) << 32) | (uint32_t)i;
        }
        key[i] = k;
      }
      __syncthreads();
      for (int k = 2; k <= n2; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
          for (int i = tid; i < n2; i += nt) {
            const int l = i ^ j;
            if (l > i) {
              const bool up = (i & k) == 0;
              const unsigned long long a = key[i], b = key[l];
              if ((b < a) == up) {
                key[i] = b;
                key[l] = a;
              }
            }
          }
          __syncthreads();
        }
      double s = 0.0;
      for (int r = tid; r < n; r += nt) {
        const int i = (int)(key[r] & 0xFFFFFFFFu);
        if (pass == 0) {
          rk_pred[i] = r;
        } else {
          const double d = (double)(rk_pred[i] - r);
          s += d * d;
        }
      }
      __syncthreads();
      if (pass == 1) {
        red[tid] = s;
        __syncthreads();
        for (int o = nt >> 1; o > 0; o >>= 1) {
          if (tid < o) red[tid] += red[tid + o];
          __syncthreads();
        }
        rho = 1.0 - 6.0 * red[0] / ((double)n * ((double)n * n - 1.0));
      }
      __syncthreads();
    }
  }
  // mean / std of log fitness over this generation's population
  double s1 = 0.0, s2 = 0.0;
  for (int i = tid; i < pop; i += nt) {
    const double l = log(fmax(fit[i], 1e-30));
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
  select_kernel<<<1, 1024, 0, st>>>(score, n_pool, n_sel, sel, state, fallback, random_select);
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
                                 cudaStream_t st) {
  int n2 = 2;
  while (n2 < s.pop) n2 <<= 1;
  const size_t smem = (size_t)n2 * (sizeof(unsigned long long) + sizeof(int));
  replay_stats_kernel<<<1, 1024, smem, st>>>(fit, pred, state, s.pop, elitism, ring_meta, norm,
                                             monitor, fallback, fallback_rho);
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

cudaError_t surrogate_ga_init_attributes() {
  return cudaFuncSetAttribute(replay_stats_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              8192 * (int)(sizeof(unsigned long long) + sizeof(int)));
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
