// SIMT (FFMA) fitness of the whole population and the float64 report of one
// chromosome.
//
// Fitness (paper Section 2): Out(pat_k) = a_0 + sum_g P[k,g] G[c,g] (eq.2),
// E_k = (t_k - act(Out))^2 (eq.3) or its threshold form (eq.10), summed over the
// training patterns and turned into MSE / RMSE by the reduce step (eq.4, eq.5).
// This kernel is the float32 CUDA-core path: register-tiled 64 x 64 blocks
// (patterns x chromosomes), fused epilogue, per-CTA column sums in float64
// written to a partial-sum buffer that the reduce step adds in a fixed order.
// It serves small populations and is the engine-independent cross-check of the
// tensor-core kernel.  Populations of at most 32 with at most 32 basis columns
// (the paper's own settings: 2N+1 chromosomes, Section 5) take the narrow
// kernel instead (fitness_narrow.cu), a stream over P.
#include "simt.h"
#include "tc_ptx.cuh"

#include <math_constants.h>

namespace game {

__device__ __forceinline__ float pattern_error(float t, float s, int act, int err, float R) {
  const float y = act == GAME_TANH ? tanhf(s) : s;
  const float d = t - y;
  const float e = d * d;
  if (err == GAME_TMSE) return fabsf(d) > R ? e : 0.0f;
  if (err == GAME_TMSE_SQ) return e > R ? e : 0.0f;
  return e;
}

template <int PREC>
__device__ __forceinline__ float load_p(const void* p0, const void* p1, const float* cs,
                                        long long o, int c) {
  if (PREC == GAME_FP32)   // hi + lo, times the column's power-of-two scale (1 in range)
    return (__half2float(((const __half*)p0)[o]) + __half2float(((const __half*)p1)[o])) * cs[c];
  if (PREC == GAME_BF16) return __bfloat162float(((const __nv_bfloat16*)p0)[o]) * cs[c];
  return (float)(((const __nv_fp8_e4m3*)p0)[o]) * cs[c];
}

template <int PREC>
__global__ void __launch_bounds__(256) fitness_simt_kernel(SimtArgs a) {
  if (a.in_evolve && a.state->stopped) return;
  __shared__ float Ps[64][33];
  __shared__ float Gs[64][33];
  __shared__ float red[16][65];
  __shared__ double acc64[64];
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
      for (int i = tid; i < 64 * 32; i += 256) {
        const int r = i >> 5, cc = i & 31;
        const long long row = m0 + r;
        const int col = k0 + cc;
        Ps[r][cc] = (row < a.m && col < a.kb)
                        ? load_p<PREC>(a.p0, a.p1, a.colscale, row * a.kp + col, col)
                        : 0.0f;
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
        const float t = a.t[row];
#pragma unroll
        for (int j = 0; j < 4; ++j) cs[j] += pattern_error(t, acc[i][j] + bias[j], a.act, a.err, a.R);
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

int simt_partials(const Shape& s, int n_sm) {
  if (narrow_shape_ok(s.pop, s.kp)) return narrow_partials(s, n_sm);
  const long long mt = (s.n_train + 63) / 64;
  const int ct = s.pop_pad / 64;
  long long g = (2LL * n_sm + ct - 1) / ct;
  if (g > mt) g = mt;
  if (g < 1) g = 1;
  return (int)g;
}

cudaError_t launch_fitness_simt(const Shape& s, const Fitness& f, const PopDev& p,
                                const ExpDev& e, double* partial, int n_part,
                                const DevState* state, DevState* dev_state, cudaStream_t st) {
  SimtArgs a;
  a.p0 = e.p0;
  a.p1 = e.p1;
  a.colscale = e.colscale;
  a.t = e.t;
  a.geval = p.geval;
  a.bias = p.bias;
  a.ghi = p.ghi;
  a.glo = p.glo;
  a.rscale = p.rscale;
  a.partial = partial;
  a.state = state;
  a.dev_state = dev_state;
  a.m = s.n_train;
  a.kb = s.kb;
  a.kp = s.kp;
  a.pop = s.pop;
  a.pop_pad = s.pop_pad;
  a.act = f.activation;
  a.err = f.error;
  a.R = f.tmse_R;
  a.in_evolve = state != nullptr;   // state is read only inside game_evolve
  if (narrow_shape_ok(s.pop, s.kp)) return launch_narrow(a, s, n_part, st);
  dim3 grid(n_part, s.pop_pad / 64);
  if (s.precision == GAME_FP32)
    fitness_simt_kernel<GAME_FP32><<<grid, 256, 0, st>>>(a);
  else if (s.precision == GAME_BF16)
    fitness_simt_kernel<GAME_BF16><<<grid, 256, 0, st>>>(a);
  else
    fitness_simt_kernel<GAME_FP8><<<grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Float64 report of one chromosome (Section 5 figures of merit): per-block
// sums of squared error, correct decisions, TP, FP, FN; a second one-block
// kernel adds the blocks in index order.
// ---------------------------------------------------------------------------
template <int PREC>
__global__ void __launch_bounds__(256) score_kernel(const void* p0, const void* p1,
                                                    const float* cs, const float* t,
                                                    const float* genes, long long r0,
                                                    long long r1, int kb, int kp, int act,
                                                    double* block_out) {
  __shared__ double red[5][256];
  double v[5] = {0, 0, 0, 0, 0};
  for (long long r = r0 + (long long)blockIdx.x * blockDim.x + threadIdx.x; r < r1;
       r += (long long)gridDim.x * blockDim.x) {
    // four interleaved float64 partial sums: one dependent chain of kb float64 FMAs
    // per row would leave the (narrow) float64 pipe waiting on its own latency
    double part[4] = {0.0, 0.0, 0.0, 0.0};
    int c = 0;
    for (; c + 4 <= kb; c += 4) {
#pragma unroll
      for (int j = 0; j < 4; ++j)
        part[j] += (double)load_p<PREC>(p0, p1, cs, r * kp + c + j, c + j) * (double)genes[1 + c + j];
    }
    for (; c < kb; ++c) part[0] += (double)load_p<PREC>(p0, p1, cs, r * kp + c, c) * (double)genes[1 + c];
    const double s = (double)genes[0] + ((part[0] + part[1]) + (part[2] + part[3]));
    const double y = act == GAME_TANH ? tanh(s) : s;
    const double tt = (double)t[r];
    const double d = tt - y;
    v[0] += d * d;
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

__global__ void score_final_kernel(const double* block_out, int n_blocks, double* result) {
  if (threadIdx.x >= 5) return;
  double s = 0.0;
  for (int b = 0; b < n_blocks; ++b) s += block_out[b * 5 + threadIdx.x];
  result[threadIdx.x] = s;
}

int score_blocks(long long rows, int n_sm) {
  long long b = (rows + 255) / 256;
  if (b > 4LL * n_sm) b = 4LL * n_sm;
  return b < 1 ? 1 : (int)b;
}

cudaError_t launch_score(const Shape& s, const Fitness& f, const ExpDev& e, const float* genes,
                         long long r0, long long r1, double* block_out, int n_blocks,
                         double* result, cudaStream_t st) {
  if (s.precision == GAME_FP32)
    score_kernel<GAME_FP32><<<n_blocks, 256, 0, st>>>(e.p0, e.p1, e.colscale, e.t, genes, r0, r1,
                                                      s.kb, s.kp, f.activation, block_out);
  else if (s.precision == GAME_BF16)
    score_kernel<GAME_BF16><<<n_blocks, 256, 0, st>>>(e.p0, e.p1, e.colscale, e.t, genes, r0, r1,
                                                      s.kb, s.kp, f.activation, block_out);
  else
    score_kernel<GAME_FP8><<<n_blocks, 256, 0, st>>>(e.p0, e.p1, e.colscale, e.t, genes, r0, r1,
                                                     s.kb, s.kp, f.activation, block_out);
  score_final_kernel<<<1, 32, 0, st>>>(block_out, n_blocks, result);
  return cudaGetLastError();
}

}  // namespace game
