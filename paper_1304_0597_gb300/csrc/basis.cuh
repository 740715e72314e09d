// Basis values of one feature (paper Section 2, eq.1 / eq.8 / eq.9), shared by the
// stored expansion (expand.cu) and the on-the-fly fitness engine (fitness_otf.cu), so
// that both form the same float32 values.
#pragma once

#include "game_internal.h"

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

// ---- float-float arithmetic: a value hi + lo with |lo| <= ulp(hi) / 2 ------------
struct FF {
  float hi, lo;
};
__device__ __forceinline__ FF ff_quick(float a, float b) {   // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return FF{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ FF ff_add(FF a, FF b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return ff_quick(s, e);
}
__device__ __forceinline__ FF ff_neg(FF a) { return FF{-a.hi, -a.lo}; }
__device__ __forceinline__ FF ff_mul(FF a, FF b) {
  float p, e;
  two_prod(a.hi, b.hi, p, e);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return ff_quick(p, e);
}

// sin x and cos x as float-float pairs (about 2^-44 absolute) on the float32 pipes.
// Cody and Waite's argument reduction: k = nearest integer to x 2/pi, r = x - k pi/2
// with pi/2 split into three floats (C1 + C2 + C3, 76 bits) and the products k C1,
// k C2 taken exactly (two_prod); then the Taylor series of sin r and cos r (|r| <=
// pi/4; terms to r^13 / r^14, the first omitted one below 2^-45) by Horner's rule in
// r^2, float-float except for the two smallest terms; the quadrant k mod 4 picks the
// signs.  Beyond |x| = 2^15 (k no longer small) one float64 sincos is used instead.
__device__ __forceinline__ void ff_sincos(float x, FF& s, FF& c) {
  if (!(fabsf(x) <= 32768.0f)) {
    double sd, cd;
    sincos((double)x, &sd, &cd);
    s.hi = (float)sd;
    s.lo = (float)(sd - (double)s.hi);
    c.hi = (float)cd;
    c.lo = (float)(cd - (double)c.hi);
    return;
  }
  constexpr float kC1 = 0x1.921fb6p+0f, kC2 = -0x1.777a5cp-25f, kC3 = -0x1.ee59dap-50f;
  const float k = rintf(x * 0x1.45f306p-1f);
  FF r{x, 0.0f};
  float p, e;
  two_prod(k, kC1, p, e);
  r = ff_add(r, FF{-p, -e});
  two_prod(k, kC2, p, e);
  r = ff_add(r, FF{-p, -e});
  r = ff_add(r, FF{-k * kC3, 0.0f});
  const FF r2 = ff_mul(r, r);
  // 1/n! as float-float pairs (hi = float nearest, lo = float nearest of the rest)
  const FF i3{0x1.555556p-3f, -0x1.555556p-28f}, i5{0x1.111112p-7f, -0x1.dddddep-32f},
      i7{0x1.a01a02p-13f, -0x1.7f97fap-39f}, i9{0x1.71de3ap-19f, 0x1.55b1ccp-45f};
  const FF i2{0.5f, 0.0f}, i4{0x1.555556p-5f, -0x1.555556p-30f},
      i6{0x1.6c16c2p-10f, -0x1.27d27ep-35f}, i8{0x1.a01a02p-16f, -0x1.7f97fap-42f},
      i10{0x1.27e4fcp-22f, -0x1.10ec14p-47f};
  // sin r = r + r r^2 (-1/3! + r^2 (1/5! + r^2 (-1/7! + r^2 (1/9! + r^2 (-1/11! + r^2/13!)))))
  FF S{fmaf(r2.hi, 0x1.612462p-33f, -0x1.ae6456p-26f), 0.0f};
  S = ff_add(i9, ff_mul(r2, S));
  S = ff_add(ff_neg(i7), ff_mul(r2, S));
  S = ff_add(i5, ff_mul(r2, S));
  S = ff_add(ff_neg(i3), ff_mul(r2, S));
  const FF sr = ff_add(r, ff_mul(ff_mul(r, r2), S));
  // cos r = 1 + r^2 (-1/2 + r^2 (1/4! + r^2 (-1/6! + r^2 (1/8! + r^2 (-1/10! + r^2 (1/12! - r^2/14!))))))
  FF Cq{fmaf(r2.hi, -0x1.93974ap-37f, 0x1.1eed8ep-29f), 0.0f};
  Cq = ff_add(ff_neg(i10), ff_mul(r2, Cq));
  Cq = ff_add(i8, ff_mul(r2, Cq));
  Cq = ff_add(ff_neg(i6), ff_mul(r2, Cq));
  Cq = ff_add(i4, ff_mul(r2, Cq));
  Cq = ff_add(ff_neg(i2), ff_mul(r2, Cq));
  const FF cr = ff_add(FF{1.0f, 0.0f}, ff_mul(r2, Cq));
  switch (((int)k) & 3) {
    case 0: s = sr; c = cr; break;
    case 1: s = cr; c = ff_neg(sr); break;
    case 2: s = ff_neg(sr); c = ff_neg(cr); break;
    default: s = ff_neg(cr); c = sr; break;
  }
}

// One step of the three-term recurrence v_{k+1} = y v_k - v_{k-1} (y = 2 cos x):
// cos((k+1) x) and sin((k+1) x) from their two predecessors.
__device__ __forceinline__ void ff_step(FF y, FF& prev, FF& cur) {
  const FF next = ff_add(ff_mul(y, cur), ff_neg(prev));
  prev = cur;
  cur = next;
}

// Calls emit(b, v) with the float32 rounding of the b-th basis value of x.
// Chebyshev: T_{k+1} = 2x T_k - T_{k-1} carried as a float-float pair (about
// 44 significant bits, all on the float32 pipes).  Trig: cos(m x) = T_m(cos x) and
// sin(m x) = sin x U_{m-1}(cos x) by the same three-term recurrence with y = 2 cos x,
// from a float-float sincos, also on the float32 pipes (float64 is a narrow unit on
// this part).
// DC > 0 fixes the degree at compile time (the loops unroll and b is a constant in
// emit); DC = 0 takes the run-time d.
template <int DC = 0, typename Emit>
__device__ __forceinline__ void basis_values(int basis, int d_rt, float x, Emit emit) {
  const int d = DC > 0 ? DC : d_rt;
  if (basis == GAME_CHEBYSHEV) {
    const float y = __fmul_rn(2.0f, x);          // exact
    float mh = 1.0f, ml = 0.0f;                  // T_{k-1}
    float th = x, tl = 0.0f;                     // T_k
#pragma unroll
    for (int b = 0; b < d; ++b) {
      emit(b, __fadd_rn(th, tl));
      if (b + 1 == d) break;                     // no step past the last value
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
    // cos(m x), sin(m x), m = 1..d: float-float sincos, then the recurrences
    FF s1, c1;
    ff_sincos(x, s1, c1);
    const FF y{__fmul_rn(2.0f, c1.hi), __fmul_rn(2.0f, c1.lo)};   // exact
    FF cm{1.0f, 0.0f}, cc = c1, sm{0.0f, 0.0f}, sc = s1;
#pragma unroll
    for (int k = 0; k < d; ++k) {
      emit(k, cc.hi);
      emit(d + k, sc.hi);
      if (k + 1 == d) break;                     // no step past the last value
      ff_step(y, cm, cc);
      ff_step(y, sm, sc);
    }
  }
}

// Calls emit(v) with the float32 basis values of x for b = b_lo .. b_hi - 1 in order
// (0 <= b_lo < b_hi <= B*d): the same arithmetic as basis_values, stopped at b_hi.
template <typename Emit>
__device__ __forceinline__ void basis_range(int basis, int d, float x, int b_lo, int b_hi,
                                            Emit emit) {
  if (basis == GAME_CHEBYSHEV) {
    const float y = __fmul_rn(2.0f, x);
    float mh = 1.0f, ml = 0.0f, th = x, tl = 0.0f;
    for (int b = 0; b < b_hi; ++b) {
      if (b >= b_lo) emit(__fadd_rn(th, tl));
      float p, pe, s2, se;
      two_prod(y, th, p, pe);
      two_sum(p, -mh, s2, se);
      const float low = __fsub_rn(__fadd_rn(__fadd_rn(se, pe), __fmul_rn(y, tl)), ml);
      const float nh = __fadd_rn(s2, low);
      const float nl = __fsub_rn(low, __fsub_rn(nh, s2));
      mh = th;
      ml = tl;
      th = nh;
      tl = nl;
    }
  } else {
    FF s1, c1;
    ff_sincos(x, s1, c1);
    const FF y{__fmul_rn(2.0f, c1.hi), __fmul_rn(2.0f, c1.lo)};
    // cos((k+1) x) for the columns below d, then sin((k+1) x) for those from d
    for (int half = 0; half < 2; ++half) {
      const int lo = half ? max(b_lo, d) - d : b_lo;
      const int hi = half ? b_hi - d : min(b_hi, d);
      FF prev = half ? FF{0.0f, 0.0f} : FF{1.0f, 0.0f}, cur = half ? s1 : c1;
      for (int k = 0; k < hi; ++k) {
        if (k >= lo) emit(cur.hi);
        ff_step(y, prev, cur);
      }
    }
  }
}

}  // namespace game

namespace game {

// One 16-byte chunk of a pattern's FP32 expansion planes: the basis columns
// [col0, col0 + 8) (zero from kb on) of the pattern whose features start at x, divided
// by their power-of-two column scales (skipped when every scale is 1), each value v
// split as hi = fp16(v), lo = fp16(v - hi).  hi[i] / lo[i] hold columns col0 + 2i (low
// half) and col0 + 2i + 1 (high half), the stored planes' byte order.  The same
// recurrences and rounding as the stored expansion, so the halves are the stored ones.
__device__ __forceinline__ void fp32_planes_chunk(const float* __restrict__ x, int basis, int d,
                                                  int bd, int kb, int col0,
                                                  const float* __restrict__ colscale,
                                                  bool unit_scale, uint32_t hi[4], uint32_t lo[4]) {
  float v[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = 0.0f;
  int n = 0;   // values written so far
  const int c_end = min(col0 + 8, kb);
  int col = col0;
  while (col < c_end) {
    const int f = col / bd;
    const int b_lo = col - f * bd;
    const int b_hi = min(bd, c_end - f * bd);
    basis_range(basis, d, __ldg(x + f), b_lo, b_hi, [&](float val) {
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if (j == n) v[j] = val;
      ++n;
    });
    col = f * bd + b_hi;
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    float a = v[2 * i], b = v[2 * i + 1];
    if (!unit_scale) {
      if (col0 + 2 * i < kb) a = a * (1.0f / __ldg(colscale + col0 + 2 * i));
      if (col0 + 2 * i + 1 < kb) b = b * (1.0f / __ldg(colscale + col0 + 2 * i + 1));
    }
    const __half ha = __float2half_rn(a), hb = __float2half_rn(b);
    const __half la = __float2half_rn(__fsub_rn(a, __half2float(ha)));
    const __half lb = __float2half_rn(__fsub_rn(b, __half2float(hb)));
    hi[i] = (uint32_t)__half_as_ushort(ha) | ((uint32_t)__half_as_ushort(hb) << 16);
    lo[i] = (uint32_t)__half_as_ushort(la) | ((uint32_t)__half_as_ushort(lb) << 16);
  }
}

}  // namespace game

namespace game {

// T_{b0+1}(x) .. T_{b0+8}(x) for N patterns at once (N independent float-float
// recurrences advanced in the same loop, so that their latencies overlap): the same
// arithmetic, step by step, as the stored expansion's Chebyshev kernels.
template <int N>
__device__ __forceinline__ void cheb8_rows(const float (&x)[N], int b0, float (&v)[N][8]) {
  float y[N], mh[N], ml[N], th[N], tl[N];
#pragma unroll
  for (int u = 0; u < N; ++u) {
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
    for (int u = 0; u < N; ++u) step(u);
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) {
#pragma unroll
    for (int u = 0; u < N; ++u) {
      v[u][j] = __fadd_rn(th[u], tl[u]);
      if (j + 1 < 8) step(u);
    }
  }
}

// hi / lo fp16 planes of 8 consecutive float32 values (times the column scales' inverses
// inv[j], powers of two), packed as the stored planes are.
__device__ __forceinline__ void fp32_split8(const float (&v)[8], const float (&inv)[8],
                                            bool unit_scale, uint32_t hi[4], uint32_t lo[4]) {
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float a = unit_scale ? v[2 * i] : v[2 * i] * inv[2 * i];
    const float b = unit_scale ? v[2 * i + 1] : v[2 * i + 1] * inv[2 * i + 1];
    const __half ha = __float2half_rn(a), hb = __float2half_rn(b);
    const __half la = __float2half_rn(__fsub_rn(a, __half2float(ha)));
    const __half lb = __float2half_rn(__fsub_rn(b, __half2float(hb)));
    hi[i] = (uint32_t)__half_as_ushort(ha) | ((uint32_t)__half_as_ushort(hb) << 16);
    lo[i] = (uint32_t)__half_as_ushort(la) | ((uint32_t)__half_as_ushort(lb) << 16);
  }
}

}  // namespace game
