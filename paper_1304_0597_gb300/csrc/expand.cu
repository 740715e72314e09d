// Expansion matrix P: every feature of every pattern expanded once into its
// polynomial sequence and kept on the device for the whole run.
//
// Paper Section 2, eq.1 (per-feature sequence a_1 g(f_i) + ... + a_d g^d(f_i),
// with g^j the j-th member of the basis, eq.9), eq.8 / eq.9 (polytrigo:
// cos(m x), sin(m x), m = 1..d).  Section 4.1 computes the sines and cosines in
// advance and reuses them every iteration, which is what this kernel does; the
// bias a_0 multiplies a column of ones that is never stored (its gene is added
// in the fitness epilogue).
//
// Values come from recurrences carried well beyond float32 precision
// (Chebyshev: T_{k+1} = 2x T_k - T_{k-1} in float-float; trig: angle addition
// from one float64 sincos(x)), rounded once to float32, then stored in the
// precision of the run:
//   FP32: two fp16 planes of v' = v / s_g, hi = fp16(v'), lo = fp16(v' - hi) (v' = hi + lo
//         to ~22 bits); s_g is a power of two, 1 unless the column's values could pass
//         2^15 (Chebyshev features beyond [-1, 1]), so that hi never overflows fp16
//   BF16: bf16(v / s_g), s_g = max_k |P[k,g]|          (per-column scale)
//   FP8 : e4m3(v / s_g), s_g = max_k |P[k,g]| / 448
#include "basis.cuh"
#include "checks.cuh"
#include "game_internal.h"

#include <algorithm>

namespace game {

struct ExpArgs {
  const float* X;
  long long n;
  int F, d, basis, bd, kb, kp, precision, shared;
  void* p0;
  void* p1;
  const float* colscale;
  unsigned int* colmax_bits;
  int unit_scale;         // FP32: every column scale is 1 (no multiply)
};

// Column maxima of |P|: block-local maxima in shared memory (non-negative floats
// order like their bit patterns), one global atomic per block and column.
__global__ void expand_colmax_kernel(ExpArgs a) {
  extern __shared__ unsigned int cmax[];
  for (int c = threadIdx.x; c < a.kb; c += blockDim.x) cmax[c] = 0u;
  __syncthreads();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < a.n * a.F;
       i += (long long)gridDim.x * blockDim.x) {
    const int f = (int)(i % a.F);
    unsigned int* cm = cmax + f * a.bd;
    basis_values(a.basis, a.d, a.X[i],
                 [&](int b, float v) { atomicMax(cm + b, __float_as_uint(fabsf(v))); });
  }
  __syncthreads();
  for (int c = threadIdx.x; c < a.kb; c += blockDim.x)
    if (cmax[c]) atomicMax(a.colmax_bits + c, cmax[c]);
}

__global__ void expand_scale_kernel(const unsigned int* colmax_bits, float* colscale, int kb,
                                    int kp, float qmax) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= kp) return;
  const float m = c < kb ? __uint_as_float(colmax_bits[c]) : 0.0f;
  colscale[c] = m > 0.0f ? m / qmax : 1.0f;
}

// Vectorised expansion: one thread per (pattern row, 16-byte chunk of the stored row),
// consecutive threads on consecutive chunks of a row, so that every store is a full
// coalesced 16-byte vector.  Blocks are (chunks of a row) x (rows): threadIdx.x is the
// chunk, so no thread divides by the chunk count.  A chunk holds EPC = 16 / element-size columns; the thread
// runs the recurrence of each feature its columns belong to (from T_1 / m = 1, stopping
// at the chunk's last column) and shifts every value into packed registers in column
// order.  Columns past kb are zero.
template <int PREC>
__global__ void __launch_bounds__(256) expand_chunk_kernel(ExpArgs a) {
  constexpr int kEsz = PREC == GAME_FP8 ? 1 : 2;
  constexpr int kEpc = 16 / kEsz;
  constexpr int kBits = 8 * kEsz;
  const long long row = (long long)blockIdx.x * blockDim.y + threadIdx.y;
  const int col0 = (int)(blockIdx.y * blockDim.x + threadIdx.x) * kEpc;
  if (row >= a.n || col0 >= a.kp) return;
  if (!GAME_IN_BOUNDS_DBG(col0 + kEpc <= a.kp, kSiteExpandCol, row)) return;
  uint32_t w0[4] = {0u, 0u, 0u, 0u}, w1[4] = {0u, 0u, 0u, 0u};   // plane 0 / plane 1 words
  // shift the 128-bit chunk right by one element and put e (its low kBits) on top
  auto push = [&](uint32_t* w, uint32_t e) {
    w[0] = __funnelshift_r(w[0], w[1], kBits);
    w[1] = __funnelshift_r(w[1], w[2], kBits);
    w[2] = __funnelshift_r(w[2], w[3], kBits);
    w[3] = __funnelshift_r(w[3], e, kBits);
  };
  int col = col0;
  auto emit = [&](float v) {
    if (PREC == GAME_FP32) {
      v = v * (1.0f / a.colscale[col]);                  // a power of two: exact
      const __half h = __float2half_rn(v);
      const __half l = __float2half_rn(__fsub_rn(v, __half2float(h)));
      push(w0, (uint32_t)__half_as_ushort(h));
      push(w1, (uint32_t)__half_as_ushort(l));
    } else if (PREC == GAME_BF16) {
      push(w0, (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v / a.colscale[col])));
    } else {
      push(w0, (uint32_t)__nv_fp8_e4m3(v / a.colscale[col]).__x);
    }
    ++col;
  };
  const int c_end = min(col0 + kEpc, a.kb);
  const float* x = a.X + row * a.F;
  while (col < c_end) {
    const int f = col / a.bd;
    const int b_lo = col - f * a.bd;
    const int b_hi = min(a.bd, c_end - f * a.bd);
    basis_range(a.basis, a.d, __ldg(x + f), b_lo, b_hi, emit);
  }
  for (; col < col0 + kEpc; ++col) {   // zero padding (shifted in like values)
    push(w0, 0u);
    if (PREC == GAME_FP32) push(w1, 0u);
  }
  const long long o = (row * a.kp + col0) * kEsz;   // byte offset, a multiple of 16
  *reinterpret_cast<uint4*>((uint8_t*)a.p0 + o) = make_uint4(w0[0], w0[1], w0[2], w0[3]);
  if (PREC == GAME_FP32)
    *reinterpret_cast<uint4*>((uint8_t*)a.p1 + o) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
}

// The same for Chebyshev bases whose kb columns per feature are a whole number of
// chunks (B d a multiple of EPC, e.g. d = 8 with 16-bit storage): a chunk lies inside
// one feature, starts at a multiple of EPC and is wholly values or wholly padding, so
// the EPC values are computed in an unrolled loop and packed at fixed positions.
template <int PREC>
__global__ void __launch_bounds__(256) expand_cheb_aligned_kernel(ExpArgs a) {
  constexpr int kEsz = PREC == GAME_FP8 ? 1 : 2;
  constexpr int kEpc = 16 / kEsz;
  constexpr int kRows = 2;   // rows per thread: two independent recurrences in flight
  const int col0 = (int)(blockIdx.y * blockDim.x + threadIdx.x) * kEpc;
  if (col0 >= a.kp) return;
  if (!GAME_IN_BOUNDS_DBG(col0 + kEpc <= a.kp, kSiteExpandCol, col0)) return;
  // per-thread constants: the chunk's feature, its first basis index, its column scales
  const bool val = col0 < a.kb;
  int f = 0, b0 = 0;
  float sc[kEpc];
#pragma unroll
  for (int j = 0; j < kEpc; ++j) sc[j] = 1.0f;
  if (val) {
    f = col0 / a.bd;
    b0 = col0 - f * a.bd;
    if (PREC != GAME_FP32 || !a.unit_scale) {
#pragma unroll
      for (int j = 0; j < kEpc; ++j)
        sc[j] = PREC == GAME_FP32 ? 1.0f / __ldg(a.colscale + col0 + j)   // powers of two
                                  : __ldg(a.colscale + col0 + j);
    }
  }
  const long long rbase = (long long)blockIdx.x * blockDim.y * kRows + threadIdx.y;
  float v[kRows][kEpc];
  float x[kRows];
#pragma unroll
  for (int u = 0; u < kRows; ++u) {
    const long long row = rbase + (long long)u * blockDim.y;
    x[u] = val && row < a.n ? __ldg(a.X + row * a.F + f) : 0.0f;
  }
  if (val) {
    // T_{b+1}(x) for b = b0 .. b0 + EPC - 1 by the float-float recurrence, both rows
    // advanced in the same loop
    float y[kRows], mh[kRows], ml[kRows], th[kRows], tl[kRows];
#pragma unroll
    for (int u = 0; u < kRows; ++u) {
      y[u] = __fmul_rn(2.0f, x[u]);
      mh[u] = 1.0f;
      ml[u] = 0.0f;
      th[u] = x[u];
      tl[u] = 0.0f;
    }
    auto step = [&](int u) {
      float p, pe, s2, se;
      two_prod(y[u], th[u], p, pe);
      two_sum(p, -mh[u], s2, se);
      const float low = __fsub_rn(__fadd_rn(__fadd_rn(se, pe), __fmul_rn(y[u], tl[u])), ml[u]);
      const float nh = __fadd_rn(s2, low);
      const float nl = __fsub_rn(low, __fsub_rn(nh, s2));
      mh[u] = th[u];
      ml[u] = tl[u];
      th[u] = nh;
      tl[u] = nl;
    };
    for (int b = 0; b < b0; ++b) {
#pragma unroll
      for (int u = 0; u < kRows; ++u) step(u);
    }
#pragma unroll
    for (int j = 0; j < kEpc; ++j) {
#pragma unroll
      for (int u = 0; u < kRows; ++u) {
        v[u][j] = __fadd_rn(th[u], tl[u]);
        if (j + 1 < kEpc) step(u);
      }
    }
    if (PREC != GAME_FP32 || !a.unit_scale) {
#pragma unroll
      for (int u = 0; u < kRows; ++u)
#pragma unroll
        for (int j = 0; j < kEpc; ++j)
          v[u][j] = PREC == GAME_FP32 ? v[u][j] * sc[j] : v[u][j] / sc[j];
    }
  } else {
#pragma unroll
    for (int u = 0; u < kRows; ++u)
#pragma unroll
      for (int j = 0; j < kEpc; ++j) v[u][j] = 0.0f;
  }
#pragma unroll
  for (int u = 0; u < kRows; ++u) {
    const long long row = rbase + (long long)u * blockDim.y;
    if (row >= a.n) break;
    uint32_t w0[4], w1[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (PREC == GAME_FP32) {
        const __half h0 = __float2half_rn(v[u][2 * q]), h1 = __float2half_rn(v[u][2 * q + 1]);
        const __half l0 = __float2half_rn(__fsub_rn(v[u][2 * q], __half2float(h0)));
        const __half l1 = __float2half_rn(__fsub_rn(v[u][2 * q + 1], __half2float(h1)));
        w0[q] = (uint32_t)__half_as_ushort(h0) | ((uint32_t)__half_as_ushort(h1) << 16);
        w1[q] = (uint32_t)__half_as_ushort(l0) | ((uint32_t)__half_as_ushort(l1) << 16);
      } else if (PREC == GAME_BF16) {
        w0[q] = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v[u][2 * q])) |
                ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v[u][2 * q + 1])) << 16);
      } else {
        uint32_t w = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) w |= (uint32_t)__nv_fp8_e4m3(v[u][4 * q + j]).__x << (8 * j);
        w0[q] = w;
      }
    }
    const long long o = (row * a.kp + col0) * kEsz;
    *reinterpret_cast<uint4*>((uint8_t*)a.p0 + o) = make_uint4(w0[0], w0[1], w0[2], w0[3]);
    if (PREC == GAME_FP32)
      *reinterpret_cast<uint4*>((uint8_t*)a.p1 + o) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
  }
}

// Shared coefficients (the paper's eq.2 / eq.9 form): column b of pattern k is the
// sum over the features of the b-th basis value, the float32 values of the
// per-feature expansion added in float-float and rounded once.
constexpr int kSharedRows = 64;   // patterns (threads) per block of the shared-form kernels

// Column sums of one pattern in the shared form: acc[b * kSharedRows] (this
// thread's slot of a column-major block array in shared memory) = the sum over the
// features, in feature order, of the float32 b-th basis values, kept as a float-float
// pair (Knuth's TwoSum: about 48 bits, on the float32 pipes) and rounded once by the
// caller.
__device__ __forceinline__ void shared_row_sums(const ExpArgs& a, long long k, float2* acc) {
  for (int b = 0; b < a.kb; ++b) acc[b * kSharedRows] = make_float2(0.0f, 0.0f);
  const float* x = a.X + k * a.F;
  for (int f = 0; f < a.F; ++f)
    basis_values(a.basis, a.d, x[f], [&](int b, float v) {
      float2 c = acc[b * kSharedRows];
      float s, e;
      two_sum(c.x, v, s, e);
      acc[b * kSharedRows] = make_float2(s, __fadd_rn(c.y, e));
    });
}

__device__ __forceinline__ float ff_round(float2 c) { return __fadd_rn(c.x, c.y); }

__global__ void __launch_bounds__(kSharedRows) expand_shared_colmax_kernel(ExpArgs a) {
  extern __shared__ float2 sacc[];   // [kb][kSharedRows]
  __shared__ unsigned int cmax[64];  // kb <= 2 * 32
  for (int c = threadIdx.x; c < a.kb; c += blockDim.x) cmax[c] = 0u;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  for (long long k0 = (long long)blockIdx.x * kSharedRows; k0 < a.n;
       k0 += (long long)gridDim.x * kSharedRows) {
    const long long k = k0 + threadIdx.x;
    float2* acc = sacc + threadIdx.x;
    if (k < a.n) shared_row_sums(a, k, acc);
    for (int b = 0; b < a.kb; ++b) {
      // non-negative floats order like their bit patterns
      const unsigned int v = k < a.n ? __float_as_uint(fabsf(ff_round(acc[b * kSharedRows]))) : 0u;
      const unsigned int m = __reduce_max_sync(0xffffffffu, v);
      if (lane == 0 && m) atomicMax(cmax + b, m);
    }
  }
  __syncthreads();
  for (int c = threadIdx.x; c < a.kb; c += blockDim.x)
    if (cmax[c]) atomicMax(a.colmax_bits + c, cmax[c]);
}

// One pattern per thread: the kb column sums, rounded once to float32, stored as
// the run's planes 16 bytes at a time (kp is a multiple of 16, or of 32 for e4m3).
__global__ void __launch_bounds__(kSharedRows) expand_shared_kernel(ExpArgs a) {
  extern __shared__ float2 sacc[];   // [kb][kSharedRows]
  const long long k = (long long)blockIdx.x * kSharedRows + threadIdx.x;
  if (k >= a.n) return;
  const float2* acc = sacc + threadIdx.x;
  shared_row_sums(a, k, sacc + threadIdx.x);
  const long long row = k * a.kp;
  auto val = [&](int b) { return b < a.kb ? ff_round(acc[b * kSharedRows]) : 0.0f; };
  if (a.precision == GAME_FP32) {
    // the power-of-two column scale divides exactly
    auto vs = [&](int b) { return b < a.kb ? val(b) * (1.0f / a.colscale[b]) : 0.0f; };
    for (int b0 = 0; b0 < a.kp; b0 += 8) {
      uint32_t hw[4], lw[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float v0 = vs(b0 + 2 * i), v1 = vs(b0 + 2 * i + 1);
        const __half h0 = __float2half_rn(v0), h1 = __float2half_rn(v1);
        const __half l0 = __float2half_rn(__fsub_rn(v0, __half2float(h0)));
        const __half l1 = __float2half_rn(__fsub_rn(v1, __half2float(h1)));
        const __half2 hh = __halves2half2(h0, h1), ll = __halves2half2(l0, l1);
        hw[i] = *reinterpret_cast<const uint32_t*>(&hh);
        lw[i] = *reinterpret_cast<const uint32_t*>(&ll);
      }
      *reinterpret_cast<uint4*>((__half*)a.p0 + row + b0) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
      *reinterpret_cast<uint4*>((__half*)a.p1 + row + b0) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
    }
  } else if (a.precision == GAME_BF16) {
    for (int b0 = 0; b0 < a.kp; b0 += 8) {
      uint32_t w[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int b = b0 + 2 * i;
        const __nv_bfloat162 q =
            __halves2bfloat162(__float2bfloat16_rn(b < a.kb ? val(b) / a.colscale[b] : 0.0f),
                               __float2bfloat16_rn(b + 1 < a.kb ? val(b + 1) / a.colscale[b + 1] : 0.0f));
        w[i] = *reinterpret_cast<const uint32_t*>(&q);
      }
      *reinterpret_cast<uint4*>((__nv_bfloat16*)a.p0 + row + b0) = make_uint4(w[0], w[1], w[2], w[3]);
    }
  } else {
    for (int b0 = 0; b0 < a.kp; b0 += 16) {
      uint32_t w[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        uint32_t word = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int b = b0 + 4 * i + j;
          const __nv_fp8_e4m3 q(b < a.kb ? val(b) / a.colscale[b] : 0.0f);
          word |= (uint32_t)q.__x << (8 * j);
        }
        w[i] = word;
      }
      *reinterpret_cast<uint4*>((__nv_fp8_e4m3*)a.p0 + row + b0) = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
}

// The same for a degree fixed at compile time (D <= 8, the paper's settings): the
// column sums live in registers (b is a constant in every emit) instead of shared
// memory, and the kernel stores the same bytes as expand_shared_kernel.  kp <= 32.
template <int D>
__global__ void __launch_bounds__(128) expand_shared_reg_kernel(ExpArgs a) {
  constexpr int kB = 2 * D;                      // room for both bases (trig: 2 d columns)
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= a.n) return;
  float2 acc[kB];
#pragma unroll
  for (int b = 0; b < kB; ++b) acc[b] = make_float2(0.0f, 0.0f);
  const float* x = a.X + k * a.F;
  for (int f = 0; f < a.F; ++f)
    basis_values<D>(a.basis, D, __ldg(x + f), [&](int b, float v) {
      float s, e;
      two_sum(acc[b].x, v, s, e);
      acc[b] = make_float2(s, __fadd_rn(acc[b].y, e));
    });
  const long long row = k * a.kp;
  auto val = [&](int b) { return b < kB && b < a.kb ? ff_round(acc[b < kB ? b : 0]) : 0.0f; };
  if (a.precision == GAME_FP32) {
#pragma unroll
    for (int b0 = 0; b0 < 16; b0 += 8) {
      if (b0 >= a.kp) break;
      uint32_t hw[4], lw[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int b = b0 + 2 * i;
        // the power-of-two column scale divides exactly
        const float v0 = b < a.kb ? val(b) * (1.0f / a.colscale[b]) : 0.0f;
        const float v1 = b + 1 < a.kb ? val(b + 1) * (1.0f / a.colscale[b + 1]) : 0.0f;
        const __half h0 = __float2half_rn(v0), h1 = __float2half_rn(v1);
        const __half l0 = __float2half_rn(__fsub_rn(v0, __half2float(h0)));
        const __half l1 = __float2half_rn(__fsub_rn(v1, __half2float(h1)));
        const __half2 hh = __halves2half2(h0, h1), ll = __halves2half2(l0, l1);
        hw[i] = *reinterpret_cast<const uint32_t*>(&hh);
        lw[i] = *reinterpret_cast<const uint32_t*>(&ll);
      }
      *reinterpret_cast<uint4*>((__half*)a.p0 + row + b0) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
      *reinterpret_cast<uint4*>((__half*)a.p1 + row + b0) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
    }
  } else if (a.precision == GAME_BF16) {
#pragma unroll
    for (int b0 = 0; b0 < 16; b0 += 8) {
      if (b0 >= a.kp) break;
      uint32_t w[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int b = b0 + 2 * i;
        const __nv_bfloat162 q =
            __halves2bfloat162(__float2bfloat16_rn(b < a.kb ? val(b) / a.colscale[b] : 0.0f),
                               __float2bfloat16_rn(b + 1 < a.kb ? val(b + 1) / a.colscale[b + 1] : 0.0f));
        w[i] = *reinterpret_cast<const uint32_t*>(&q);
      }
      *reinterpret_cast<uint4*>((__nv_bfloat16*)a.p0 + row + b0) = make_uint4(w[0], w[1], w[2], w[3]);
    }
  } else {
#pragma unroll
    for (int b0 = 0; b0 < 32; b0 += 16) {
      if (b0 >= a.kp) break;
      uint32_t w[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        uint32_t word = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int b = b0 + 4 * i + j;
          const __nv_fp8_e4m3 q(b < a.kb ? val(b) / a.colscale[b] : 0.0f);
          word |= (uint32_t)q.__x << (8 * j);
        }
        w[i] = word;
      }
      *reinterpret_cast<uint4*>((__nv_fp8_e4m3*)a.p0 + row + b0) = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
}

__global__ void target_coef_kernel(const float* t, float* c, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) c[i] = 2.8853900817779268f * t[i];   // 2 log2(e) t
}

cudaError_t launch_target_coef(const float* t, float* c, long long n, cudaStream_t st) {
  target_coef_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(t, c, n);
  return cudaGetLastError();
}

__global__ void fill_ones_kernel(float* v, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = 1.0f;
}

cudaError_t launch_fill_ones(float* v, int n, cudaStream_t st) {
  fill_ones_kernel<<<(n + 255) / 256, 256, 0, st>>>(v, n);
  return cudaGetLastError();
}

// Largest |x| of every feature over all patterns (bits of non-negative floats order
// like the floats).  Lane l of a warp owns feature fc + l of each 32-feature group and
// keeps a running maximum over the warp's rows (row r reads 32 consecutive floats);
// the block's warps meet in shared memory, then one global atomic per block and
// feature.  absmax_bits [F] must be zero on entry.
__global__ void feature_absmax_kernel(const float* __restrict__ X, long long n, int F,
                                      unsigned int* absmax_bits) {
  extern __shared__ unsigned int fm[];
  for (int f = threadIdx.x; f < F; f += blockDim.x) fm[f] = 0u;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const long long wg = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (int fc = 0; fc < F; fc += 32) {
    const int f = fc + lane;
    if (f >= F) continue;
    float m = 0.0f;
#pragma unroll 4
    for (long long r = wg; r < n; r += nw) m = fmaxf(m, fabsf(__ldg(X + r * F + f)));
    atomicMax(fm + f, __float_as_uint(m));
  }
  __syncthreads();
  for (int f = threadIdx.x; f < F; f += blockDim.x)
    if (fm[f]) atomicMax(absmax_bits + f, fm[f]);
}

cudaError_t launch_feature_absmax(const float* X, long long n, int F, unsigned int* absmax_bits,
                                  int n_sm, cudaStream_t st) {
  cudaError_t err = cudaMemsetAsync(absmax_bits, 0, sizeof(unsigned int) * F, st);
  if (err != cudaSuccess) return err;
  const long long blocks = std::min<long long>((n + 7) / 8, 4LL * n_sm);   // 8 warps a block
  feature_absmax_kernel<<<(unsigned)std::max<long long>(blocks, 1), 256,
                          sizeof(unsigned int) * F, st>>>(X, n, F, absmax_bits);
  return cudaGetLastError();
}

cudaError_t launch_expand(const float* X, const Shape& s, ExpDev& e, float* qmax_scratch,
                          cudaStream_t st) {
  ExpArgs a;
  a.X = X;
  a.n = s.n_patterns;
  a.F = s.n_features;
  a.d = s.degree;
  a.basis = s.basis;
  a.bd = s.bd;
  a.kb = s.kb;
  a.kp = s.kp;
  a.precision = s.precision;
  a.p0 = e.p0;
  a.p1 = e.p1;
  a.colscale = e.colscale;
  a.colmax_bits = reinterpret_cast<unsigned int*>(qmax_scratch);
  a.shared = s.shared;
  const int threads = 256;
  if (s.shared) {
    // one thread per pattern, F basis sequences each; column sums in shared memory
    if (s.kb > 64) return cudaErrorInvalidValue;   // B * d <= 2 * 32
    const size_t smem = sizeof(float2) * s.kb * kSharedRows;
    const long long nblk = (s.n_patterns + kSharedRows - 1) / kSharedRows;
    if (s.precision != GAME_FP32) {   // FP32: the caller has set the power-of-two scales
      cudaError_t err = cudaMemsetAsync(qmax_scratch, 0, sizeof(float) * s.kp, st);
      if (err != cudaSuccess) return err;
      const unsigned cblocks = (unsigned)(nblk < 4864 ? nblk : 4864);
      expand_shared_colmax_kernel<<<cblocks, kSharedRows, smem, st>>>(a);
      expand_scale_kernel<<<(s.kp + 255) / 256, 256, 0, st>>>(
          a.colmax_bits, e.colscale, s.kb, s.kp, s.precision == GAME_BF16 ? 1.0f : 448.0f);
    }
    // degrees up to 8: the register form (kp <= 16 for 16-bit storage, <= 32 for e4m3)
    const unsigned rblk = (unsigned)((s.n_patterns + 127) / 128);
    switch (s.degree) {
#define GAME_SHARED_REG(DV)                                          \
  case DV:                                                           \
    expand_shared_reg_kernel<DV><<<rblk, 128, 0, st>>>(a);           \
    return cudaGetLastError();
      GAME_SHARED_REG(1)
      GAME_SHARED_REG(2)
      GAME_SHARED_REG(3)
      GAME_SHARED_REG(4)
      GAME_SHARED_REG(5)
      GAME_SHARED_REG(6)
      GAME_SHARED_REG(7)
      GAME_SHARED_REG(8)
#undef GAME_SHARED_REG
      default:
        break;
    }
    expand_shared_kernel<<<(unsigned)nblk, kSharedRows, smem, st>>>(a);
    return cudaGetLastError();
  }
  const long long n = s.n_patterns * s.n_features;
  const unsigned blocks = (unsigned)((n + threads - 1) / threads);
  if (s.precision != GAME_FP32) {   // FP32: the caller has set the power-of-two scales
    cudaError_t err = cudaMemsetAsync(qmax_scratch, 0, sizeof(float) * s.kp, st);
    if (err != cudaSuccess) return err;
    const unsigned cblocks = blocks < 1216u ? blocks : 1216u;
    expand_colmax_kernel<<<cblocks, threads, sizeof(unsigned int) * s.kb, st>>>(a);
    expand_scale_kernel<<<(s.kp + 255) / 256, 256, 0, st>>>(
        a.colmax_bits, e.colscale, s.kb, s.kp, s.precision == GAME_BF16 ? 1.0f : 448.0f);
  }
  // Blocks of (chunks of a row) x (rows): x = min(chunks, 256) consecutive chunks, y = rows,
  // grid y over the chunk groups of wider rows.
  const int epc = s.precision == GAME_FP8 ? 16 : 8;
  const int nc = s.kp / epc;
  const int bx = nc < threads ? nc : threads;
  const int by = threads / bx;
  const unsigned gy = (unsigned)((nc + bx - 1) / bx);
  a.unit_scale = e.unit_scale32;
  if (s.basis == GAME_CHEBYSHEV && s.bd % epc == 0) {
    const dim3 grid((unsigned)((s.n_patterns + 2LL * by - 1) / (2LL * by)), gy);   // 2 rows/thread
    if (s.precision == GAME_FP32)
      expand_cheb_aligned_kernel<GAME_FP32><<<grid, dim3(bx, by), 0, st>>>(a);
    else if (s.precision == GAME_BF16)
      expand_cheb_aligned_kernel<GAME_BF16><<<grid, dim3(bx, by), 0, st>>>(a);
    else
      expand_cheb_aligned_kernel<GAME_FP8><<<grid, dim3(bx, by), 0, st>>>(a);
    return cudaGetLastError();
  }
  const dim3 grid((unsigned)((s.n_patterns + by - 1) / by), gy);
  if (s.precision == GAME_FP32)
    expand_chunk_kernel<GAME_FP32><<<grid, dim3(bx, by), 0, st>>>(a);
  else if (s.precision == GAME_BF16)
    expand_chunk_kernel<GAME_BF16><<<grid, dim3(bx, by), 0, st>>>(a);
  else
    expand_chunk_kernel<GAME_FP8><<<grid, dim3(bx, by), 0, st>>>(a);
  return cudaGetLastError();
}

// Float32 reconstruction of rows [row0, row0 + nrows) of P (basis columns).
__global__ void expand_get_kernel(const void* p0, const void* p1, const float* colscale,
                                  int precision, int kb, int kp, long long row0, long long nrows,
                                  float* out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nrows * kb) return;
  const long long r = row0 + i / kb;
  const int c = (int)(i % kb);
  const long long o = r * kp + c;
  float v;
  if (precision == GAME_FP32)
    v = (__half2float(((const __half*)p0)[o]) + __half2float(((const __half*)p1)[o])) * colscale[c];
  else if (precision == GAME_BF16)
    v = __bfloat162float(((const __nv_bfloat16*)p0)[o]) * colscale[c];
  else
    v = (float)(((const __nv_fp8_e4m3*)p0)[o]) * colscale[c];
  out[i] = v;
}

cudaError_t launch_expand_get(const Shape& s, const ExpDev& e, long long row0, long long nrows,
                              float* out, cudaStream_t st) {
  const long long n = nrows * s.kb;
  if (n == 0) return cudaSuccess;
  expand_get_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
      e.p0, e.p1, e.colscale, s.precision, s.kb, s.kp, row0, nrows, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Prediction on new patterns (the paper's test / run use of a trained
// chromosome): Out(x) = a_0 + sum_f sum_b g[1 + f B d + b] g_b(x_f) (eq.2, eq.8,
// eq.9 with per-feature coefficients; g[1 + b] for every f when shared), then the
// activation.  One thread per
// pattern; the expansion is computed on the fly in float64 (Chebyshev
// recurrence; cos / sin of (b+1) x by angle addition from one sincos).
// ---------------------------------------------------------------------------
__global__ void predict_kernel(const float* __restrict__ X, long long n, int F,
                               const float* __restrict__ genes, int K, int basis, int degree,
                               int shared, int activation, float* __restrict__ out) {
  extern __shared__ float gs[];
  for (int i = threadIdx.x; i < K; i += blockDim.x) gs[i] = genes[i];
  __syncthreads();
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const float* x = X + k * F;
  double s = (double)gs[0];
  if (basis == GAME_CHEBYSHEV) {
    for (int f = 0; f < F; ++f) {
      const double v = (double)x[f];
      const float* g = gs + 1 + (shared ? 0 : f * degree);
      double tm = 1.0, t = v;                     // T_0, T_1
      for (int b = 0; b < degree; ++b) {
        s = fma((double)g[b], t, s);
        const double tn = 2.0 * v * t - tm;
        tm = t;
        t = tn;
      }
    }
  } else {
    for (int f = 0; f < F; ++f) {
      const double v = (double)x[f];
      const float* g = gs + 1 + (shared ? 0 : f * 2 * degree);
      double s1, c1;
      sincos(v, &s1, &c1);
      double c = c1, sn = s1;                     // cos((b+1) v), sin((b+1) v)
      for (int b = 0; b < degree; ++b) {
        s = fma((double)g[b], c, s);
        s = fma((double)g[degree + b], sn, s);
        const double cn = c * c1 - sn * s1;
        sn = sn * c1 + c * s1;
        c = cn;
      }
    }
  }
  out[k] = (float)(activation == GAME_TANH ? tanh(s) : s);
}

cudaError_t launch_predict(const float* X, long long n, int F, const float* genes, int K,
                           int basis, int degree, int shared, int activation, float* out,
                           cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int threads = 256;
  predict_kernel<<<(unsigned)((n + threads - 1) / threads), threads, sizeof(float) * K, st>>>(
      X, n, F, genes, K, basis, degree, shared, activation, out);
  return cudaGetLastError();
}

}  // namespace game

namespace game {
GAME_DEFINE_CHECK_READER(check_word_expand)
}  // namespace game
