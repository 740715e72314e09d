// Counter-based random numbers and the per-gene operators of the GA, shared by
// the generation kernels (plain breeding and the surrogate's offspring pool).
#pragma once

#include <math_constants.h>

#include "game_internal.h"

namespace game {

// ---------------------------------------------------------------------------
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11).  Key = (seed, run);
// counter = (generation, pair or chromosome, stream, block).  A block gives
// 4 x 64 bits = 8 words of 32 bits: word w is the low (w even) or high (w odd)
// half of lane w/2.
// ---------------------------------------------------------------------------
struct Key {
  uint64_t k0, k1;
};

__device__ __forceinline__ void philox_block(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                             Key key, uint64_t out[4]) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
  uint64_t k0 = key.k0, k1 = key.k1;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += W0;
      k1 += W1;
    }
    const uint64_t hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
    const uint64_t hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
    const uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

__device__ __forceinline__ uint64_t pick_lane(const uint64_t v[4], uint32_t lane) {
  return lane == 0 ? v[0] : lane == 1 ? v[1] : lane == 2 ? v[2] : v[3];
}

__device__ __forceinline__ uint32_t philox_word(Key key, uint64_t gen, uint64_t pair,
                                                uint64_t stream, uint64_t word) {
  uint64_t v[4];
  philox_block(gen, pair, stream, word >> 3, key, v);
  const uint64_t x = pick_lane(v, (uint32_t)(word & 7) >> 1);
  return (word & 1) ? (uint32_t)(x >> 32) : (uint32_t)x;
}

// Both words 2w and 2w+1 (one 64-bit lane of one block).
__device__ __forceinline__ void philox_word_pair(Key key, uint64_t gen, uint64_t pair,
                                                 uint64_t stream, uint64_t w, uint32_t* a,
                                                 uint32_t* b) {
  uint64_t v[4];
  const uint64_t word = 2 * w;
  philox_block(gen, pair, stream, word >> 3, key, v);
  const uint64_t x = pick_lane(v, (uint32_t)(word & 7) >> 1);
  *a = (uint32_t)x;
  *b = (uint32_t)(x >> 32);
}

__device__ __forceinline__ float uniform24(uint32_t w) {
  return __fmul_rn((float)(w >> 8), 0x1p-24f);
}

__device__ __forceinline__ int index_draw(uint32_t w, int n) {
  return (int)(((uint64_t)w * (uint64_t)n) >> 32);
}

// ---------------------------------------------------------------------------
// Box-Muller (Box & Muller, 1958) with its own float32 logarithm and cosine,
// evaluated with explicitly rounded operations (no FMA contraction) so that the
// draw is the same on every IEEE-754 machine that performs the same steps.
//   ln u:   u = m 2^e, m in [sqrt(1/2), sqrt(2)); ln m = 2 atanh(s),
//           s = (m-1)/(m+1), series 2s(1 + s^2/3 + ... + s^10/11).
//   cos 2 pi v: quadrant q = floor(4v), a = (4v - q) pi/2 in [0, pi/2);
//           Taylor series of cos a (to a^16) and sin a (to a^15).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float ln_f32(float u) {
  const uint32_t b = __float_as_uint(u);
  int e = (int)((b >> 23) & 0xffu) - 126;
  float m = __uint_as_float((b & 0x7fffffu) | 0x3f000000u);   // [0.5, 1)
  if (m < 0x1.6a09e6p-1f) {
    m = __fmul_rn(m, 2.0f);
    e -= 1;
  }
  const float f = __fsub_rn(m, 1.0f);
  const float s = __fdiv_rn(f, __fadd_rn(f, 2.0f));
  const float z = __fmul_rn(s, s);
  float p = 0x1.745d18p-4f;                       // 1/11
  p = __fadd_rn(__fmul_rn(p, z), 0x1.c71c72p-4f);  // 1/9
  p = __fadd_rn(__fmul_rn(p, z), 0x1.24924ap-3f);  // 1/7
  p = __fadd_rn(__fmul_rn(p, z), 0x1.99999ap-3f);  // 1/5
  p = __fadd_rn(__fmul_rn(p, z), 0x1.555556p-2f);  // 1/3
  p = __fadd_rn(__fmul_rn(p, z), 1.0f);
  float a = __fmul_rn(s, p);
  a = __fadd_rn(a, a);
  return __fadd_rn(__fmul_rn((float)e, 0x1.62e430p-1f), a);
}

__device__ __forceinline__ float cos2pi_f32(float v) {
  const float v4 = __fmul_rn(v, 4.0f);
  const float q = floorf(v4);
  const float a = __fmul_rn(__fsub_rn(v4, q), 0x1.921fb6p+0f);
  const float a2 = __fmul_rn(a, a);
  float c = 0x1.ae7f3ep-45f;
  c = __fadd_rn(__fmul_rn(c, a2), -0x1.93974ap-37f);
  c = __fadd_rn(__fmul_rn(c, a2), 0x1.1eed8ep-29f);
  c = __fadd_rn(__fmul_rn(c, a2), -0x1.27e4fcp-22f);
  c = __fadd_rn(__fmul_rn(c, a2), 0x1.a01a02p-16f);
  c = __fadd_rn(__fmul_rn(c, a2), -0x1.6c16c2p-10f);
  c = __fadd_rn(__fmul_rn(c, a2), 0x1.555556p-5f);
  c = __fadd_rn(__fmul_rn(c, a2), -0x1.000000p-1f);
  c = __fadd_rn(__fmul_rn(c, a2), 1.0f);
  float s = -0x1.ae7f3ep-41f;
  s = __fadd_rn(__fmul_rn(s, a2), 0x1.612462p-33f);
  s = __fadd_rn(__fmul_rn(s, a2), -0x1.ae6456p-26f);
  s = __fadd_rn(__fmul_rn(s, a2), 0x1.71de3ap-19f);
  s = __fadd_rn(__fmul_rn(s, a2), -0x1.a01a02p-13f);
  s = __fadd_rn(__fmul_rn(s, a2), 0x1.111112p-7f);
  s = __fadd_rn(__fmul_rn(s, a2), -0x1.555556p-3f);
  s = __fadd_rn(__fmul_rn(s, a2), 1.0f);
  s = __fmul_rn(a, s);
  const int qi = (int)q;
  return qi == 0 ? c : qi == 1 ? -s : qi == 2 ? -c : s;
}

__device__ __forceinline__ float gauss_f32(uint32_t w0, uint32_t w1) {
  const float u1 = __fmul_rn((float)((w0 >> 8) + 1u), 0x1p-24f);   // (0, 1]
  const float u2 = uniform24(w1);                                  // [0, 1)
  const float r = __fsqrt_rn(__fmul_rn(ln_f32(u1), -2.0f));
  return __fmul_rn(r, cos2pi_f32(u2));
}

__device__ __forceinline__ double fit_key(const double* fit, int i) {
  const double f = fit[i];
  return isnan(f) ? CUDART_INF : f;
}

__device__ __forceinline__ bool better(double fa, int ia, double fb, int ib) {
  return fa < fb || (fa == fb && ia < ib);
}

// Mutation of one gene (taken with probability p_m): add sigma N(0,1), the normal
// from the words 2w, 2w+1 of the normal stream, then clamp.  Out of line: one copy
// of the normal draw keeps the breeding loop's instruction footprint small.
static __device__ __noinline__ float mutation_step(float v, Key key, uint64_t gen, uint64_t pair,
                                                   uint64_t w, float sigma, int clamp) {
  uint32_t a, b;
  philox_word_pair(key, gen, pair, kStreamMutNormal, w, &a, &b);
  v = __fadd_rn(v, __fmul_rn(sigma, gauss_f32(a, b)));
  if (clamp) v = fminf(fmaxf(v, -1.0f), 1.0f);
  return v;
}

// The 8 words of one Philox block in word order.
__device__ __forceinline__ void block_words(const uint64_t v[4], uint32_t w[8]) {
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    w[2 * i] = (uint32_t)v[i];
    w[2 * i + 1] = (uint32_t)(v[i] >> 32);
  }
}

// w[i] <- w[i + o] for i < 8, o in [0, 8), over the 16 words of two consecutive
// blocks; shifts by 4, 2, 1 with static indices (no local-memory indexing).
__device__ __forceinline__ void shift_words(uint32_t w[16], int o) {
  if (o & 4) {
#pragma unroll
    for (int i = 0; i < 12; ++i) w[i] = w[i + 4];
  }
  if (o & 2) {
#pragma unroll
    for (int i = 0; i < 14; ++i) w[i] = w[i + 2];
  }
  if (o & 1) {
#pragma unroll
    for (int i = 0; i < 15; ++i) w[i] = w[i + 1];
  }
}

// One child pair j (one warp): two parents by tournaments of k draws with
// replacement (winner = min (fitness, index)), or by roulette / ranking draws on
// cum when given; single-point crossover with probability p_c
// (cut in [1, K-1]), per-gene Gaussian mutation with probability p_m, clamp.
// Child a goes to oa, child b to ob (when has_b).
// Roulette / ranking draw on inclusive cumulative integer weights cum[0..pop):
// t = (u24 Q) >> 24 with u24 the word's top 24 bits and Q = cum[pop-1]; the first
// index whose cumulative weight exceeds t.  A zero total draws uniformly.
__device__ __forceinline__ int wheel_draw(const unsigned long long* __restrict__ cum, int pop,
                                          uint32_t w) {
  const unsigned long long total = cum[pop - 1];
  if (total == 0ull) return index_draw(w, pop);
  const unsigned long long t = ((unsigned long long)(w >> 8) * total) >> 24;
  int lo = 0, hi = pop - 1;   // cum[hi] = total > t
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (cum[mid] > t)
      hi = mid;
    else
      lo = mid + 1;
  }
  return lo;
}

__device__ __forceinline__ void breed_pair(const float* __restrict__ G, int kstride, int K, int pop,
                                           const double* fit, const unsigned long long* cum,
                                           Key key, uint64_t gen, uint64_t j, int tk, float p_c,
                                           float p_m, float sigma, int clamp, float* oa, float* ob,
                                           bool has_b, int lane) {
  int bi0, bi1;
  if (cum) {
    // roulette / ranking: lane 0 draws the first parent, lane 1 the second
    int mine = 0;
    if (lane < 2) mine = wheel_draw(cum, pop, philox_word(key, gen, j, kStreamTournament, lane));
    bi0 = __shfl_sync(0xffffffffu, mine, 0);
    bi1 = __shfl_sync(0xffffffffu, mine, 1);
  } else {
    double bf0 = CUDART_INF, bf1 = CUDART_INF;
    bi0 = 0x7fffffff;
    bi1 = 0x7fffffff;
    for (int i = lane; i < 2 * tk; i += 32) {
      const int idx = index_draw(philox_word(key, gen, j, kStreamTournament, (uint64_t)i), pop);
      const double f = fit_key(fit, idx);
      if (i < tk) {
        if (better(f, idx, bf0, bi0)) { bf0 = f; bi0 = idx; }
      } else {
        if (better(f, idx, bf1, bi1)) { bf1 = f; bi1 = idx; }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double f0 = __shfl_xor_sync(0xffffffffu, bf0, o);
      const int i0 = __shfl_xor_sync(0xffffffffu, bi0, o);
      const double f1 = __shfl_xor_sync(0xffffffffu, bf1, o);
      const int i1 = __shfl_xor_sync(0xffffffffu, bi1, o);
      if (better(f0, i0, bf0, bi0)) { bf0 = f0; bi0 = i0; }
      if (better(f1, i1, bf1, bi1)) { bf1 = f1; bi1 = i1; }
    }
  }
  uint32_t wc, wk;   // crossover decision and cut: words 0 and 1 of one block
  philox_word_pair(key, gen, j, kStreamCrossover, 0, &wc, &wk);
  int cut = K;
  if (uniform24(wc) < p_c && K >= 2) cut = 1 + index_draw(wk, K - 1);
  const float* __restrict__ r1 = G + (long long)bi0 * kstride;
  const float* __restrict__ r2 = G + (long long)bi1 * kstride;
  // Rounds of 256 genes: lane l takes genes g0 .. g0+7, g0 = base + 8 l.  Child
  // a's mask words g are exactly one Philox block (g0 / 8); child b's words K + g
  // span at most two.  Genes that do not mutate are written at once; the round's
  // mutations (probability p_m each) are then packed over the warp, one per lane,
  // so that the normal draws run in parallel rather than once per gene slot.
  const int ob_off = K & 7;
  for (int base = 0; base < K; base += 256) {
    const int g0 = base + 8 * lane;
    uint32_t flags = 0;   // bit i: child a's gene g0 + i mutates; bit 8 + i: child b's
    if (g0 < K) {
      uint64_t v[4];
      uint32_t wa[8], wb[16];
      philox_block(gen, j, kStreamMutMask, (uint64_t)(g0 >> 3), key, v);
      block_words(v, wa);
      if (has_b) {
        const uint64_t bb = ((uint64_t)K + (uint64_t)g0) >> 3;
        philox_block(gen, j, kStreamMutMask, bb, key, v);
        block_words(v, wb);
        if (ob_off) {
          philox_block(gen, j, kStreamMutMask, bb + 1, key, v);
          block_words(v, wb + 8);
          shift_words(wb, ob_off);
        }
      }
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int g = g0 + i;
        if (g < K) {
          const bool head = g < cut;
          const float x1 = r1[g], x2 = r2[g];
          if (uniform24(wa[i]) < p_m)
            flags |= 1u << i;
          else
            oa[g] = head ? x1 : x2;
          if (has_b) {
            if (uniform24(wb[i]) < p_m)
              flags |= 1u << (8 + i);
            else
              ob[g] = head ? x2 : x1;
          }
        }
      }
    }
    int incl = __popc(flags);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    for (int jb = 0; jb < total; jb += 32) {
      const int job = jb + lane;
      // owner = first lane whose inclusive count exceeds job
      int owner = 0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1)
        if (__shfl_sync(0xffffffffu, incl, owner + step - 1) <= job) owner += step;
      const uint32_t of = __shfl_sync(0xffffffffu, flags, owner);
      const int oexcl = __shfl_sync(0xffffffffu, incl, owner) - __popc(of);
      if (job < total) {
        const int bit = (int)__fns(of, 0, job - oexcl + 1);
        const int g = base + 8 * owner + (bit & 7);
        const bool head = g < cut;
        if (bit < 8)
          oa[g] = mutation_step(head ? r1[g] : r2[g], key, gen, j, (uint64_t)g, sigma, clamp);
        else
          ob[g] = mutation_step(head ? r2[g] : r1[g], key, gen, j, (uint64_t)K + (uint64_t)g, sigma,
                                clamp);
      }
    }
  }
}

}  // namespace game
