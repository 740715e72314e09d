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
// kernel below instead, a stream over P with one pattern per thread.
#include "game_internal.h"
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

struct SimtArgs {
  const void* p0;
  const void* p1;
  const float* colscale;
  const float* t;
  const float* geval;
  const float* bias;
  double* partial;
  const DevState* state;
  long long m;          // training rows
  int kb, kp, pop, pop_pad, act, err, in_evolve;
  float R;
};

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

// ---------------------------------------------------------------------------
// Narrow populations: pop <= 32 and kp in {16, 32}.  With 23 chromosomes the
// 64-chromosome blocks above, or the 128-chromosome tensor-core tiles, would be
// mostly padding, and the work is a pass over P.  Here a thread takes one
// pattern at a time and reads its whole row with 16-byte loads (the rows of a
// warp are contiguous), the genes of every chromosome sit transposed in shared
// memory (each read is a broadcast, four chromosomes per load), and two
// chromosomes share each packed f32x2 FMA.  Each thread sums its errors per
// chromosome in float32 over blocks of 32 patterns; a butterfly across the
// warp then leaves lane c with chromosome c's block total, which is added to a
// float64 sum.  Fixed assignment and order: the result is deterministic.
// ---------------------------------------------------------------------------
constexpr int kNarrowPop = 32;
constexpr int kNarrowThreads = 256;

__host__ __device__ constexpr bool narrow_shape(int pop, int kp) {
  return pop >= 1 && pop <= kNarrowPop && (kp == 16 || kp == 32);
}

// Rows per thread and pass: each gene read from shared memory then feeds this
// many patterns.  Two FP32 rows of 16 columns would need more than the 128
// registers that two resident CTAs of 256 threads leave, and one CTA per SM
// hides latency worse than the shared-memory reads cost (measured).
__host__ __device__ constexpr int narrow_rows(int prec, int kp) {
  return kp == 16 && prec != GAME_FP32 ? 2 : 1;
}

// One row of P as 16-byte words: FP32 = hi and lo fp16 planes, BF16 = one bf16
// plane, FP8 = one e4m3 plane.
template <int PREC, int KP>
struct NarrowRow {
  static constexpr int kWords = PREC == GAME_FP32 ? KP / 4 : PREC == GAME_BF16 ? KP / 8 : KP / 16;
  uint4 w[kWords];
};

template <int PREC, int KP>
__device__ __forceinline__ void narrow_load(const SimtArgs& a, long long k, NarrowRow<PREC, KP>& r) {
  if (PREC == GAME_FP32) {
    const uint4* hi = reinterpret_cast<const uint4*>(static_cast<const __half*>(a.p0) + k * KP);
    const uint4* lo = reinterpret_cast<const uint4*>(static_cast<const __half*>(a.p1) + k * KP);
#pragma unroll
    for (int q = 0; q < KP / 8; ++q) {
      r.w[q] = __ldg(hi + q);
      r.w[KP / 8 + q] = __ldg(lo + q);
    }
  } else {
    const size_t esz = PREC == GAME_BF16 ? 2 : 1;
    const uint4* src =
        reinterpret_cast<const uint4*>(static_cast<const uint8_t*>(a.p0) + (size_t)k * KP * esz);
#pragma unroll
    for (int q = 0; q < NarrowRow<PREC, KP>::kWords; ++q) r.w[q] = __ldg(src + q);
  }
}

// Values of the row (the column scales of BF16 / FP8 are folded into the genes).
template <int PREC, int KP>
__device__ __forceinline__ void narrow_unpack(const NarrowRow<PREC, KP>& r, float p[KP]) {
  if (PREC == GAME_FP32) {
#pragma unroll
    for (int q = 0; q < KP / 8; ++q) {
      const __half2* h = reinterpret_cast<const __half2*>(&r.w[q]);
      const __half2* l = reinterpret_cast<const __half2*>(&r.w[KP / 8 + q]);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float2 fh = __half22float2(h[i]), fl = __half22float2(l[i]);
        p[q * 8 + 2 * i] = fh.x + fl.x;   // exact: 11 + 11 significant bits
        p[q * 8 + 2 * i + 1] = fh.y + fl.y;
      }
    }
  } else if (PREC == GAME_BF16) {
#pragma unroll
    for (int q = 0; q < KP / 8; ++q) {
      const __nv_bfloat162* b = reinterpret_cast<const __nv_bfloat162*>(&r.w[q]);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float2 f = __bfloat1622float2(b[i]);
        p[q * 8 + 2 * i] = f.x;
        p[q * 8 + 2 * i + 1] = f.y;
      }
    }
  } else {
#pragma unroll
    for (int q = 0; q < KP / 16; ++q) {
      const __nv_fp8x2_storage_t* b = reinterpret_cast<const __nv_fp8x2_storage_t*>(&r.w[q]);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const float2 f = __half22float2(__half2(__nv_cvt_fp8x2_to_halfraw2(b[i], __NV_E4M3)));
        p[q * 16 + 2 * i] = f.x;
        p[q * 16 + 2 * i + 1] = f.y;
      }
    }
  }
}

template <bool TANH>
__device__ __forceinline__ float narrow_error(float t, float s, int err, float R) {
  const float y = TANH ? tanhf(s) : s;
  const float d = t - y;
  const float e = d * d;
  if (err == GAME_TMSE) return fabsf(d) > R ? e : 0.0f;
  if (err == GAME_TMSE_SQ) return e > R ? e : 0.0f;
  return e;
}

template <int PREC, int KP, bool TANH>
__global__ void __launch_bounds__(kNarrowThreads, 2) fitness_narrow_kernel(SimtArgs a) {
  if (a.in_evolve && a.state->stopped) return;
  constexpr int kRows = narrow_rows(PREC, KP);
  __shared__ __align__(16) float Gt[KP][kNarrowPop];   // Gt[g][c] = G[c][g] (x s_g)
  __shared__ __align__(16) float bs[kNarrowPop];
  __shared__ double red[kNarrowThreads / 32][kNarrowPop];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < KP * kNarrowPop; i += kNarrowThreads) {
    const int g = i / kNarrowPop, c = i % kNarrowPop;
    float v = 0.0f;
    if (c < a.pop && g < a.kb) {
      v = a.geval[(long long)c * a.kp + g] * a.colscale[g];
    }
    Gt[g][c] = v;
  }
  if (tid < kNarrowPop) bs[tid] = tid < a.pop ? a.bias[tid] : 0.0f;
  __syncthreads();

  const int ngroups = (a.pop + 3) >> 2;   // chromosomes in groups of four
  float acc[kNarrowPop];
#pragma unroll
  for (int c = 0; c < kNarrowPop; ++c) acc[c] = 0.0f;
  double tot = 0.0;
  int nblk = 0;
  // A warp takes 32 * kRows consecutive rows per pass (lane l: rows l, l + 32, ...);
  // the loop is warp-uniform.  The next pass's rows are loaded into registers
  // while this one runs.
  const long long step = (long long)gridDim.x * kNarrowThreads * kRows;
  long long k0 = ((long long)blockIdx.x * kNarrowThreads + warp * 32) * kRows;
  NarrowRow<PREC, KP> nxt[kRows];
  float tn[kRows];   // the targets travel with their rows
#pragma unroll
  for (int r = 0; r < kRows; ++r) {
    tn[r] = 0.0f;
    if (k0 + lane + 32 * r < a.m) {
      narrow_load<PREC, KP>(a, k0 + lane + 32 * r, nxt[r]);
      tn[r] = __ldg(a.t + k0 + lane + 32 * r);
    }
  }
  for (; k0 < a.m; k0 += step) {
    float p[kRows][KP];
    float t[kRows];
    bool valid[kRows];
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
      const long long k = k0 + lane + 32 * r;
      valid[r] = k < a.m;
      if (valid[r]) {
        narrow_unpack<PREC, KP>(nxt[r], p[r]);
      } else {
#pragma unroll
        for (int g = 0; g < KP; ++g) p[r][g] = 0.0f;
      }
      t[r] = tn[r];
      if (k + step < a.m) {
        narrow_load<PREC, KP>(a, k + step, nxt[r]);
        tn[r] = __ldg(a.t + k + step);
      }
    }
#pragma unroll
    for (int q = 0; q < kNarrowPop / 4; ++q) {
      if (q < ngroups) {
        const float4 b4 = *reinterpret_cast<const float4*>(&bs[4 * q]);
        unsigned long long s01[kRows], s23[kRows];
#pragma unroll
        for (int r = 0; r < kRows; ++r) {
          s01[r] = tc::pack2(b4.x, b4.y);
          s23[r] = tc::pack2(b4.z, b4.w);
        }
#pragma unroll
        for (int g = 0; g < KP; ++g) {
          const float4 gv = *reinterpret_cast<const float4*>(&Gt[g][4 * q]);
          const unsigned long long g01 = tc::pack2(gv.x, gv.y), g23 = tc::pack2(gv.z, gv.w);
#pragma unroll
          for (int r = 0; r < kRows; ++r) {
            const unsigned long long pp = tc::pack2(p[r][g], p[r][g]);
            s01[r] = tc::fma2(pp, g01, s01[r]);
            s23[r] = tc::fma2(pp, g23, s23[r]);
          }
        }
#pragma unroll
        for (int r = 0; r < kRows; ++r) {
          float sv[4];
          tc::unpack2(s01[r], sv[0], sv[1]);
          tc::unpack2(s23[r], sv[2], sv[3]);
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const float e = narrow_error<TANH>(t[r], sv[j], a.err, a.R);
            acc[4 * q + j] += valid[r] ? e : 0.0f;
          }
        }
      }
    }
    nblk += kRows;
    if (nblk == 32) {   // float32 sums over at most 32 patterns
      tot += (double)tc::warp_column_sums32(acc, lane);
      nblk = 0;
    }
  }
  tot += (double)tc::warp_column_sums32(acc, lane);
  red[warp][lane] = tot;
  __syncthreads();
  if (tid < kNarrowPop) {
    double sum = 0.0;
#pragma unroll
    for (int w = 0; w < kNarrowThreads / 32; ++w) sum += red[w][tid];
    a.partial[(long long)blockIdx.x * a.pop_pad + tid] = sum;
  }
}

template <int PREC, int KP>
void launch_narrow(const SimtArgs& a, int grid, bool tanh_act, cudaStream_t st) {
  if (tanh_act)
    fitness_narrow_kernel<PREC, KP, true><<<grid, kNarrowThreads, 0, st>>>(a);
  else
    fitness_narrow_kernel<PREC, KP, false><<<grid, kNarrowThreads, 0, st>>>(a);
}

bool simt_narrow(const Shape& s) { return narrow_shape(s.pop, s.kp); }

int simt_partials(const Shape& s, int n_sm) {
  if (narrow_shape(s.pop, s.kp)) {
    const int rows = narrow_rows(s.precision, s.kp);
    const long long need = (s.n_train + kNarrowThreads * rows - 1) / (kNarrowThreads * rows);
    const long long g = 2LL * n_sm;
    return (int)(need < 1 ? 1 : need < g ? need : g);
  }
  const long long mt = (s.n_train + 63) / 64;
  const int ct = s.pop_pad / 64;
  long long g = (2LL * n_sm + ct - 1) / ct;
  if (g > mt) g = mt;
  if (g < 1) g = 1;
  return (int)g;
}

cudaError_t launch_fitness_simt(const Shape& s, const Fitness& f, const PopDev& p,
                                const ExpDev& e, double* partial, int n_part,
                                const DevState* state, cudaStream_t st) {
  SimtArgs a;
  a.p0 = e.p0;
  a.p1 = e.p1;
  a.colscale = e.colscale;
  a.t = e.t;
  a.geval = p.geval;
  a.bias = p.bias;
  a.partial = partial;
  a.state = state;
  a.m = s.n_train;
  a.kb = s.kb;
  a.kp = s.kp;
  a.pop = s.pop;
  a.pop_pad = s.pop_pad;
  a.act = f.activation;
  a.err = f.error;
  a.R = f.tmse_R;
  a.in_evolve = state != nullptr;   // state is read only inside game_evolve
  if (narrow_shape(s.pop, s.kp)) {
    const bool th = f.activation == GAME_TANH;
    if (s.kp == 16) {
      if (s.precision == GAME_FP32)
        launch_narrow<GAME_FP32, 16>(a, n_part, th, st);
      else if (s.precision == GAME_BF16)
        launch_narrow<GAME_BF16, 16>(a, n_part, th, st);
      else
        return cudaErrorInvalidValue;   // e4m3 rows are padded to 32 columns
    } else {
      if (s.precision == GAME_FP32)
        launch_narrow<GAME_FP32, 32>(a, n_part, th, st);
      else if (s.precision == GAME_BF16)
        launch_narrow<GAME_BF16, 32>(a, n_part, th, st);
      else
        launch_narrow<GAME_FP8, 32>(a, n_part, th, st);
    }
    return cudaGetLastError();
  }
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
