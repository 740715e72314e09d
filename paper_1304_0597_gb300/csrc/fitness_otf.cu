// On-the-fly fitness engine: the expansion matrix P is never stored.  Each block
// forms the slab of P it is about to use -- 64 patterns x 32 basis columns -- in
// shared memory from the features X, with the same float-float Chebyshev recurrence
// and trig angle addition as the stored expansion (basis.cuh), then runs the
// CUDA-core contraction of the SIMT engine on it.
//
// The paper lists, among its future work (Section 6), forming the population
// matrix in place on the GPU instead of holding it in memory; Section 4.1 keeps the
// precomputed sines and cosines on the device.  Here the device memory of the
// expansion (NP x K_pad x 4 bytes in the FP32 form) drops to that of X (NP x F x 4
// bytes), at the price of recomputing each slab once per block that reads it.  What
// it computes is the same as the stored path (eq.2 -> eq.3 -> eq.4 / eq.5 / eq.10),
// with P in float32 instead of the stored fp16 hi + lo pair.
#include "basis.cuh"
#include "game_internal.h"

namespace game {

namespace {

struct OtfArgs {
  const float* X;         // [n_patterns x F] features, row-major
  const float* t;
  const float* geval;     // [pop_pad x kp] basis genes (float32)
  const float* bias;
  double* partial;
  const DevState* state;
  long long m;            // training rows
  int F, d, basis, bd, shared, kb, kp, pop, pop_pad, act, err, in_evolve;
  float R;
};

__device__ __forceinline__ float otf_error(float t, float s, int act, int err, float R) {
  const float y = act == GAME_TANH ? tanhf(s) : s;
  const float d = t - y;
  const float e = d * d;
  if (err == GAME_TMSE) return fabsf(d) > R ? e : 0.0f;
  if (err == GAME_TMSE_SQ) return e > R ? e : 0.0f;
  return e;
}

// Ps[r][j] = P[m0 + r][k0 + j] for r < 64, j < 32 (zero past the rows or the kb
// columns).  Per-feature coefficients: one item per (row, feature touched by the
// slab), each running its feature's recurrence up to the slab's last column.
// Shared coefficients (the paper's eq.2 / eq.9 form, kb = B d): one thread per row
// adds the features' values in feature order as float-float pairs (dacc), then rounds
// once, as the stored shared expansion does.
__device__ void otf_slab(const OtfArgs& a, long long m0, int k0, float (*Ps)[33],
                         float2 (*dacc)[33]) {
  const int tid = threadIdx.x;
  const int c_end = min(k0 + 32, a.kb);
  if (!a.shared) {
    if (k0 < c_end) {
      const int f_lo = k0 / a.bd, f_hi = (c_end - 1) / a.bd;
      const int items = 64 * (f_hi - f_lo + 1);
      for (int it = tid; it < items; it += blockDim.x) {
        const int r = it & 63;
        const int f = f_lo + (it >> 6);
        const int cb = max(k0, f * a.bd), ce = min(c_end, (f + 1) * a.bd);
        const long long row = m0 + r;
        int col = cb - k0;
        if (row < a.m) {
          basis_range(a.basis, a.d, __ldg(a.X + row * a.F + f), cb - f * a.bd, ce - f * a.bd,
                      [&](float v) { Ps[r][col++] = v; });
        } else {
          for (; col < ce - k0; ++col) Ps[r][col] = 0.0f;
        }
      }
    }
    // columns past kb (disjoint from the items' columns)
    for (int i = tid; i < 64 * 32; i += blockDim.x) {
      const int r = i >> 5, j = i & 31;
      if (k0 + j >= c_end) Ps[r][j] = 0.0f;
    }
  } else if (tid < 64) {
    const int r = tid;
    const long long row = m0 + r;
    for (int j = 0; j < 32; ++j) dacc[r][j] = make_float2(0.0f, 0.0f);
    if (row < a.m && k0 < c_end) {
      for (int f = 0; f < a.F; ++f) {
        int col = 0;
        basis_range(a.basis, a.d, __ldg(a.X + row * a.F + f), k0, c_end, [&](float v) {
          float s, e;
          two_sum(dacc[r][col].x, v, s, e);
          dacc[r][col] = make_float2(s, __fadd_rn(dacc[r][col].y, e));
          ++col;
        });
      }
    }
    for (int j = 0; j < 32; ++j) Ps[r][j] = __fadd_rn(dacc[r][j].x, dacc[r][j].y);   // zero past kb
  }
}

// 64 patterns x 64 chromosomes per block, 4 x 4 per thread; blocks stride over the
// pattern tiles and write one float64 partial row each (as the SIMT engine).
__global__ void __launch_bounds__(256) fitness_otf_kernel(OtfArgs a) {
  if (a.in_evolve && a.state->stopped) return;
  __shared__ float Ps[64][33];
  __shared__ float Gs[64][33];
  __shared__ float red[16][65];
  __shared__ double acc64[64];
  __shared__ float2 dacc[64][33];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int c0 = blockIdx.y * 64;
  if (tid < 64) acc64[tid] = 0.0;
  float bias[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) bias[j] = a.bias[c0 + tx * 4 + j];
  for (long long m0 = (long long)blockIdx.x * 64; m0 < a.m; m0 += (long long)gridDim.x * 64) {
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
    for (int k0 = 0; k0 < a.kb; k0 += 32) {
      otf_slab(a, m0, k0, Ps, dacc);
      for (int i = tid; i < 64 * 32; i += 256) {
        const int r = i >> 5, cc = i & 31;
        const int col = k0 + cc;
        Gs[r][cc] = (col < a.kb) ? a.geval[(long long)(c0 + r) * a.kp + col] : 0.0f;
      }
      __syncthreads();
#pragma unroll 8
      for (int kk = 0; kk < 32; ++kk) {
        float pa[4], gb[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) pa[i] = Ps[ty * 4 + i][kk];
#pragma unroll
        for (int j = 0; j < 4; ++j) gb[j] = Gs[tx * 4 + j][kk];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(pa[i], gb[j], acc[i][j]);
      }
      __syncthreads();
    }
    float cs[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const long long row = m0 + ty * 4 + i;
      if (row < a.m) {
        const float tt = a.t[row];
#pragma unroll
        for (int j = 0; j < 4; ++j) cs[j] += otf_error(tt, acc[i][j] + bias[j], a.act, a.err, a.R);
      }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) red[ty][tx * 4 + j] = cs[j];
    __syncthreads();
    if (tid < 64) {
      double s = 0.0;
      for (int r = 0; r < 16; ++r) s += (double)red[r][tid];
      acc64[tid] += s;
    }
    __syncthreads();
  }
  if (tid < 64) a.partial[(long long)blockIdx.x * a.pop_pad + c0 + tid] = acc64[tid];
}

// Float64 report of one chromosome (Section 5 figures of merit) with P formed per
// row: squared error, correct decisions, TP, FP, FN summed per block.
__global__ void __launch_bounds__(256) score_otf_kernel(const float* __restrict__ X, int F, int d,
                                                        int basis, int bd, int shared,
                                                        const float* __restrict__ t,
                                                        const float* __restrict__ genes,
                                                        long long r0, long long r1, int act,
                                                        double* block_out) {
  __shared__ double red[5][256];
  double v[5] = {0, 0, 0, 0, 0};
  for (long long r = r0 + (long long)blockIdx.x * blockDim.x + threadIdx.x; r < r1;
       r += (long long)gridDim.x * blockDim.x) {
    double s = (double)genes[0];
    for (int f = 0; f < F; ++f) {
      const float* g = genes + 1 + (shared ? 0 : f * bd);
      basis_values(basis, d, __ldg(X + r * F + f),
                   [&](int b, float p) { s = fma((double)g[b], (double)p, s); });
    }
    const double y = act == GAME_TANH ? tanh(s) : s;
    const double tt = (double)t[r];
    const double e = tt - y;
    v[0] += e * e;
    const double cls = act == GAME_TANH ? (y >= 0.0 ? 1.0 : -1.0) : (y >= 0.5 ? 1.0 : 0.0);
    v[1] += (cls == tt) ? 1.0 : 0.0;
    v[2] += (cls == 1.0 && tt == 1.0) ? 1.0 : 0.0;
    v[3] += (cls == 1.0 && tt != 1.0) ? 1.0 : 0.0;
    v[4] += (cls != 1.0 && tt == 1.0) ? 1.0 : 0.0;
  }
#pragma unroll
  for (int i = 0; i < 5; ++i) red[i][threadIdx.x] = v[i];
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o)
#pragma unroll
      for (int i = 0; i < 5; ++i) red[i][threadIdx.x] += red[i][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x < 5) block_out[blockIdx.x * 5 + threadIdx.x] = red[threadIdx.x][0];
}

__global__ void score_otf_final_kernel(const double* block_out, int n_blocks, double* result) {
  if (threadIdx.x >= 5) return;
  double s = 0.0;
  for (int b = 0; b < n_blocks; ++b) s += block_out[b * 5 + threadIdx.x];
  result[threadIdx.x] = s;
}

// Rows [row0, row0 + nrows) of P (basis columns) as float32, formed from X: one
// thread per (row, feature) (per-feature coefficients) or per row (shared; float-float
// sums over the features, rounded once).
__global__ void expand_get_otf_kernel(const float* __restrict__ X, int F, int d, int basis, int bd,
                                      int shared, int kb, long long row0, long long nrows,
                                      float* __restrict__ out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (!shared) {
    if (i >= nrows * F) return;
    const long long r = i / F;
    const int f = (int)(i % F);
    float* o = out + r * kb + f * bd;
    basis_values(basis, d, __ldg(X + (row0 + r) * F + f), [&](int b, float v) { o[b] = v; });
  } else {
    if (i >= nrows) return;
    for (int b = 0; b < kb; ++b) {
      float hi = 0.0f, lo = 0.0f;
      for (int f = 0; f < F; ++f) {
        float v = 0.0f;
        basis_range(basis, d, __ldg(X + (row0 + i) * F + f), b, b + 1, [&](float u) { v = u; });
        float s, e;
        two_sum(hi, v, s, e);
        hi = s;
        lo = __fadd_rn(lo, e);
      }
      out[i * kb + b] = __fadd_rn(hi, lo);
    }
  }
}

}  // namespace

cudaError_t launch_fitness_otf(const Shape& s, const Fitness& f, const PopDev& p, const float* X,
                               const ExpDev& e, double* partial, int n_part,
                               const DevState* state, cudaStream_t st) {
  OtfArgs a;
  a.X = X;
  a.t = e.t;
  a.geval = p.geval;
  a.bias = p.bias;
  a.partial = partial;
  a.state = state;
  a.m = s.n_train;
  a.F = s.n_features;
  a.d = s.degree;
  a.basis = s.basis;
  a.bd = s.bd;
  a.shared = s.shared;
  a.kb = s.kb;
  a.kp = s.kp;
  a.pop = s.pop;
  a.pop_pad = s.pop_pad;
  a.act = f.activation;
  a.err = f.error;
  a.in_evolve = state != nullptr;
  a.R = f.tmse_R;
  fitness_otf_kernel<<<dim3(n_part, s.pop_pad / 64), 256, 0, st>>>(a);
  return cudaGetLastError();
}

int otf_partials(const Shape& s, int n_sm) {
  const long long mt = (s.n_train + 63) / 64;
  const int ct = s.pop_pad / 64;
  long long g = (4LL * n_sm + ct - 1) / ct;   // two 38 KB blocks per SM and a second wave
  if (g > mt) g = mt;
  return g < 1 ? 1 : (int)g;
}

cudaError_t launch_score_otf(const Shape& s, const Fitness& f, const float* X, const float* t,
                             const float* genes, long long r0, long long r1, double* block_out,
                             int n_blocks, double* result, cudaStream_t st) {
  score_otf_kernel<<<n_blocks, 256, 0, st>>>(X, s.n_features, s.degree, s.basis, s.bd, s.shared,
                                              t, genes, r0, r1, f.activation, block_out);
  score_otf_final_kernel<<<1, 32, 0, st>>>(block_out, n_blocks, result);
  return cudaGetLastError();
}

cudaError_t launch_expand_get_otf(const Shape& s, const float* X, long long row0, long long nrows,
                                  float* out, cudaStream_t st) {
  const long long n = s.shared ? nrows : nrows * s.n_features;
  if (n == 0) return cudaSuccess;
  expand_get_otf_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
      X, s.n_features, s.degree, s.basis, s.bd, s.shared, s.kb, row0, nrows, out);
  return cudaGetLastError();
}

}  // namespace game
