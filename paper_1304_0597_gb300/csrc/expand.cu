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
#include "game_internal.h"

#include <algorithm>

namespace game {

// Error-free transformations on float32 (Dekker's product via FMA, Knuth's sum):
// a*b = p + e and a+b = s + e exactly.
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = fmaf(a, b, -p);
}
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Calls emit(b, v) with the float32 rounding of the b-th basis value of x.
// Chebyshev: T_{k+1} = 2x T_k - T_{k-1} carried as a float-float pair (about
// 44 significant bits, all on the float32 pipes).  Trig: one float64 sincos and
// float64 angle addition.
template <typename Emit>
__device__ __forceinline__ void basis_values(int basis, int d, float x, Emit emit) {
  if (basis == GAME_CHEBYSHEV) {
    const float y = __fmul_rn(2.0f, x);          // exact
    float mh = 1.0f, ml = 0.0f;                  // T_{k-1}
    float th = x, tl = 0.0f;                     // T_k
    for (int b = 0; b < d; ++b) {
      emit(b, __fadd_rn(th, tl));
      float p, pe, s, se;
      two_prod(y, th, p, pe);
      two_sum(p, -mh, s, se);
      const float low = __fsub_rn(__fadd_rn(__fadd_rn(se, pe), __fmul_rn(y, tl)), ml);
      const float nh = __fadd_rn(s, low);
      const float nl = __fsub_rn(low, __fsub_rn(nh, s));
      mh = th;
      ml = tl;
      th = nh;
      tl = nl;
    }
  } else {
    double s1, c1;
    sincos((double)x, &s1, &c1);
    double c = c1, s = s1;
    for (int k = 0; k < d; ++k) {
      emit(k, (float)c);
      emit(d + k, (float)s);
      const double cn = c * c1 - s * s1;
      const double sn = s * c1 + c * s1;
      c = cn;
      s = sn;
    }
  }
}

struct ExpArgs {
  const float* X;
  long long n;
  int F, d, basis, bd, kb, kp, precision, shared;
  void* p0;
  void* p1;
  const float* colscale;
  unsigned int* colmax_bits;
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

__global__ void expand_kernel(ExpArgs a) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n * a.F) return;
  const long long k = i / a.F;
  const int f = (int)(i % a.F);
  const float x = a.X[i];
  const long long row = k * a.kp;
  const int col0 = f * a.bd;
  if (a.precision == GAME_FP32) {
    __half* hi = (__half*)a.p0 + row + col0;
    __half* lo = (__half*)a.p1 + row + col0;
    const float* sc = a.colscale + col0;
    basis_values(a.basis, a.d, x, [&](int b, float v) {
      v = v * (1.0f / sc[b]);                     // a power of two: exact
      const __half h = __float2half_rn(v);
      hi[b] = h;
      lo[b] = __float2half_rn(__fsub_rn(v, __half2float(h)));
    });
    if (f == a.F - 1)
      for (int c = a.kb; c < a.kp; ++c) {
        ((__half*)a.p0)[row + c] = __float2half_rn(0.0f);
        ((__half*)a.p1)[row + c] = __float2half_rn(0.0f);
      }
  } else if (a.precision == GAME_BF16) {
    __nv_bfloat16* q = (__nv_bfloat16*)a.p0 + row + col0;
    const float* sc = a.colscale + col0;
    basis_values(a.basis, a.d, x, [&](int b, float v) { q[b] = __float2bfloat16_rn(v / sc[b]); });
    if (f == a.F - 1)
      for (int c = a.kb; c < a.kp; ++c) ((__nv_bfloat16*)a.p0)[row + c] = __float2bfloat16_rn(0.0f);
  } else {
    __nv_fp8_e4m3* q = (__nv_fp8_e4m3*)a.p0 + row + col0;
    const float* sc = a.colscale + col0;
    basis_values(a.basis, a.d, x, [&](int b, float v) { q[b] = __nv_fp8_e4m3(v / sc[b]); });
    if (f == a.F - 1)
      for (int c = a.kb; c < a.kp; ++c) ((__nv_fp8_e4m3*)a.p0)[row + c] = __nv_fp8_e4m3(0.0f);
  }
}

// Shared coefficients (the paper's eq.2 / eq.9 form): column b of pattern k is the
// sum over the features of the b-th basis value, the float32 values of the
// per-feature expansion added in float64 and rounded once.
constexpr int kSharedRows = 64;   // patterns (threads) per block of the shared-form kernels

// Column sums of one pattern in the shared form: acc[b * kSharedRows] (this
// thread's slot of a column-major block array in shared memory) = the float64
// sum over the features, in feature order, of the float32 b-th basis values.
__device__ __forceinline__ void shared_row_sums(const ExpArgs& a, long long k, double* acc) {
  for (int b = 0; b < a.kb; ++b) acc[b * kSharedRows] = 0.0;
  const float* x = a.X + k * a.F;
  for (int f = 0; f < a.F; ++f)
    basis_values(a.basis, a.d, x[f], [&](int b, float v) { acc[b * kSharedRows] += (double)v; });
}

__global__ void __launch_bounds__(kSharedRows) expand_shared_colmax_kernel(ExpArgs a) {
  extern __shared__ double sacc[];   // [kb][kSharedRows]
  __shared__ unsigned int cmax[64];  // kb <= 2 * 32
  for (int c = threadIdx.x; c < a.kb; c += blockDim.x) cmax[c] = 0u;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  for (long long k0 = (long long)blockIdx.x * kSharedRows; k0 < a.n;
       k0 += (long long)gridDim.x * kSharedRows) {
    const long long k = k0 + threadIdx.x;
    double* acc = sacc + threadIdx.x;
    if (k < a.n) shared_row_sums(a, k, acc);
    for (int b = 0; b < a.kb; ++b) {
      // non-negative floats order like their bit patterns
      const unsigned int v = k < a.n ? __float_as_uint(fabsf((float)acc[b * kSharedRows])) : 0u;
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
  extern __shared__ double sacc[];   // [kb][kSharedRows]
  const long long k = (long long)blockIdx.x * kSharedRows + threadIdx.x;
  if (k >= a.n) return;
  const double* acc = sacc + threadIdx.x;
  shared_row_sums(a, k, sacc + threadIdx.x);
  const long long row = k * a.kp;
  auto val = [&](int b) { return b < a.kb ? (float)acc[b * kSharedRows] : 0.0f; };
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
// like the floats): block maxima in shared memory, one global atomic per block and
// feature.  absmax_bits [F] must be zero on entry.
__global__ void feature_absmax_kernel(const float* X, long long n_elems, int F,
                                      unsigned int* absmax_bits) {
  extern __shared__ unsigned int fm[];
  for (int f = threadIdx.x; f < F; f += blockDim.x) fm[f] = 0u;
  __syncthreads();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n_elems;
       i += (long long)gridDim.x * blockDim.x)
    atomicMax(fm + (int)(i % F), __float_as_uint(fabsf(X[i])));
  __syncthreads();
  for (int f = threadIdx.x; f < F; f += blockDim.x)
    if (fm[f]) atomicMax(absmax_bits + f, fm[f]);
}

cudaError_t launch_feature_absmax(const float* X, long long n, int F, unsigned int* absmax_bits,
                                  int n_sm, cudaStream_t st) {
  cudaError_t err = cudaMemsetAsync(absmax_bits, 0, sizeof(unsigned int) * F, st);
  if (err != cudaSuccess) return err;
  const long long blocks = std::min<long long>((n * F + 255) / 256, 2LL * n_sm);
  feature_absmax_kernel<<<(unsigned)std::max<long long>(blocks, 1), 256,
                          sizeof(unsigned int) * F, st>>>(X, n * F, F, absmax_bits);
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
    const size_t smem = sizeof(double) * s.kb * kSharedRows;
    const long long nblk = (s.n_patterns + kSharedRows - 1) / kSharedRows;
    if (s.precision != GAME_FP32) {   // FP32: the caller has set the power-of-two scales
      cudaError_t err = cudaMemsetAsync(qmax_scratch, 0, sizeof(float) * s.kp, st);
      if (err != cudaSuccess) return err;
      const unsigned cblocks = (unsigned)(nblk < 4864 ? nblk : 4864);
      expand_shared_colmax_kernel<<<cblocks, kSharedRows, smem, st>>>(a);
      expand_scale_kernel<<<(s.kp + 255) / 256, 256, 0, st>>>(
          a.colmax_bits, e.colscale, s.kb, s.kp, s.precision == GAME_BF16 ? 1.0f : 448.0f);
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
  expand_kernel<<<blocks, threads, 0, st>>>(a);
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
