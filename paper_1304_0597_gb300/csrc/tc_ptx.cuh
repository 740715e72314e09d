// Inline-PTX building blocks of the sm_103a tensor-core kernels: mbarriers,
// TMA (cp.async.bulk.tensor), tcgen05 MMA / commit / TMEM loads, clusters.
#pragma once

#include <cuda.h>
#include <stdint.h>

#include "game_internal.h"

namespace game {
namespace tc {

constexpr unsigned long long kWaitNs = 2000000000ull;   // bound of every mbarrier wait

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on one phase of an mbarrier.  On timeout raises the CTA error
// flag and the device status, and returns false.  Also returns false as soon
// as another role of the CTA has raised the flag.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* err,
                                          DevState* st) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*err) return false;
    if (globaltimer() - t0 > kWaitNs) {
      *err = 1;
      atomicExch(&st->status, (int)GAME_ERR_TIMEOUT);
      return false;
    }
  }
}

// Bounded wait with a growing sleep between polls (32 ns up to 512 ns), for
// waiters whose reaction time does not matter: it leaves the issue slots of the
// sub-partition to the warps that do the work.
__device__ __forceinline__ bool mbar_wait_backoff(uint64_t* bar, uint32_t parity, volatile int* err,
                                                  DevState* st) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  unsigned ns = 32;
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*err) return false;
    if (globaltimer() - t0 > kWaitNs) {
      *err = 1;
      atomicExch(&st->status, (int)GAME_ERR_TIMEOUT);
      return false;
    }
    __nanosleep(ns);
    if (ns < 512) ns <<= 1;
  }
}

__device__ __forceinline__ bool warp_wait_backoff(uint64_t* bar, uint32_t parity, volatile int* err,
                                                  DevState* st, int lane) {
  int ok = 0;
  if (lane == 0) ok = mbar_wait_backoff(bar, parity, err, st) ? 1 : 0;
  return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

// Warp-uniform bounded wait: lane 0 polls, the outcome is broadcast.
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, volatile int* err,
                                          DevState* st, int lane) {
  int ok = 0;
  if (lane == 0) ok = mbar_wait(bar, parity, err, st) ? 1 : 0;
  return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int c0, int c1,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(c0), "r"(c1), "r"(smem_u32(bar))
      : "memory");
}

// 3-D box (c0 innermost): several 128-byte k-blocks of a run of rows in one request,
// landing as [c2][rows][128 B] in shared memory.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
      : "memory");
}

// L2 prefetch of one box (no shared memory, no completion): warms L2 for a load
// issued later, so that the ring's loads see L2 rather than DRAM latency.
__device__ __forceinline__ void tma_prefetch_2d(const CUtensorMap* map, int c0, int c1) {
  asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];" ::"l"(map),
               "r"(c0), "r"(c1)
               : "memory");
}

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                   : "memory");
}

// Distributed shared memory: the address of the same shared-memory location in
// CTA `rank` of the cluster, a float32 store there, and an arrive on a peer's
// mbarrier that releases this thread's earlier cluster-scope writes.
__device__ __forceinline__ uint32_t mapa_shared(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}
__device__ __forceinline__ void st_cluster_f32(uint32_t addr, float v) {
  asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t remote_bar) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(remote_bar)
               : "memory");
}
// Bounded per-thread wait with cluster-scope acquire (the arrivals come from
// peer CTAs).  Same timeout behaviour as mbar_wait.
__device__ __forceinline__ bool mbar_wait_cluster(uint64_t* bar, uint32_t parity, volatile int* err,
                                                  DevState* st) {
  const unsigned long long t0 = globaltimer();
  while (true) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
    if (globaltimer() - t0 > kWaitNs) {
      *err = 1;
      atomicExch(&st->status, (int)GAME_ERR_TIMEOUT);
      return false;
    }
  }
}

// ---- CTA pairs (cta_group::2): one MMA over the shared memory of two CTAs ----
// A pair is a cluster of two CTAs; rank 0 (the leader) issues the MMAs.  An MMA of
// M = 256 takes A rows 0-127 from the leader's and rows 128-255 from the peer's shared
// memory, B rows (N) half from each, at the same offsets, and writes D rows 0-127 to
// the leader's TMEM and rows 128-255 to the peer's.

// TMA load into this CTA's shared memory whose bytes complete on the mbarrier at the
// shared::cluster address bar_cl (the leader's barrier, also for the peer's loads).
__device__ __forceinline__ void tma_load_2d_pair(void* dst, const CUtensorMap* map, int c0, int c1,
                                                 uint32_t bar_cl) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      ".cta_group::2 [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(c0), "r"(c1), "r"(bar_cl)
      : "memory");
}

__device__ __forceinline__ void tma_load_3d_pair(void* dst, const CUtensorMap* map, int c0, int c1,
                                                 int c2, uint32_t bar_cl) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      ".cta_group::2 [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(bar_cl)
      : "memory");
}

template <int PREC>
__device__ __forceinline__ void mma_pair(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accum) {
  if (PREC == GAME_FP8) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accum));
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accum));
  }
}

// Arrive on the mbarrier at shared::cluster address bar_cl (this CTA's or the peer's)
// when every pair MMA this thread has issued so far has completed.
__device__ __forceinline__ void mma_commit_pair(uint32_t bar_cl) {
  asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   bar_cl)
               : "memory");
}

// Warp-uniform bounded wait whose arrivals may come from the peer CTA (acquire at
// cluster scope): lane 0 polls, the outcome is broadcast.
__device__ __forceinline__ bool warp_wait_cluster(uint64_t* bar, uint32_t parity, volatile int* err,
                                                  DevState* st, int lane) {
  int ok = 0;
  if (lane == 0) ok = mbar_wait_cluster(bar, parity, err, st) ? 1 : 0;
  return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (stride byte offset), descriptor version 1 (tcgen05).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;                      // leading byte offset (unused with swizzle)
  d |= (uint64_t)(1024 >> 4) << 32;            // stride byte offset
  d |= (uint64_t)1 << 46;                      // version
  d |= (uint64_t)2 << 61;                      // SWIZZLE_128B
  return d;
}

// Instruction descriptor: D f32, A/B format, both K-major, N >> 3, M >> 4.
__host__ __device__ constexpr uint32_t make_idesc(int M, int N, uint32_t ab_fmt) {
  return (1u << 4) | (ab_fmt << 7) | (ab_fmt << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

template <int PREC>
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                    uint32_t accum) {
  if (PREC == GAME_FP8) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accum));
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accum));
  }
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float v[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
        "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// W = 16 or 32 consecutive TMEM columns of this thread's lane.
template <int W>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, float* v) {
  static_assert(W == 16 || W == 32, "tcgen05.ld width");
  if constexpr (W == 32)
    tmem_ld32(taddr, v);
  else
    tmem_ld16(taddr, v);
}

__device__ __forceinline__ void prefetch_l1(const void* p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// One MUFU op; relative error about 2^-11 (the PTX ISA's stated bound).
__device__ __forceinline__ float tanh_approx(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}


// A running sum kept as an unevaluated float32 pair hi + lo (TwoSum, Knuth): about
// 48 significant bits on the FP32 pipe, where float64 adds and conversions would
// queue on this part's narrow FP64 unit.  Explicit rounding intrinsics keep the
// compiler from reassociating the error term away.
struct F2Sum {
  float hi = 0.0f, lo = 0.0f;
  __device__ __forceinline__ void add(float t) {
    const float s = __fadd_rn(hi, t);
    const float bp = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(t, bp));
    hi = s;
    lo = __fadd_rn(lo, e);
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// acc[c] of every lane of the warp -> the return value on lane c is the sum over
// the 32 lanes of acc[c]; acc is cleared.  Five halving exchange rounds (31
// shuffles), in a fixed order.
__device__ __forceinline__ float warp_column_sums32(float acc[32], int lane) {
#pragma unroll
  for (int w = 16; w >= 1; w >>= 1) {
    const bool upper = (lane & w) != 0;
#pragma unroll
    for (int i = 0; i < w; ++i) {
      const float send = upper ? acc[i] : acc[i + w];
      const float keep = upper ? acc[i + w] : acc[i];
      acc[i] = keep + __shfl_xor_sync(0xffffffffu, send, w);
    }
  }
  const float r = acc[0];
#pragma unroll
  for (int i = 0; i < 32; ++i) acc[i] = 0.0f;
  return r;
}

__device__ __forceinline__ float general_error(float t, float s, int act, int err, float R) {
  const float y = act == GAME_TANH ? tanhf(s) : s;
  const float d = t - y;
  const float e = d * d;
  if (err == GAME_TMSE) return fabsf(d) > R ? e : 0.0f;
  if (err == GAME_TMSE_SQ) return e > R ? e : 0.0f;
  return e;
}

// Sum over 32 consecutive patterns of one chromosome's error.  The per-pattern
// inputs (c_k = 2 log2(e) t_k for the fused path, t_k otherwise) are loaded
// before the TMEM read so that the two latencies overlap.
// FAST (targets +-1, tanh, MSE/RMSE): |t - tanh(s)| = 2 / (1 + exp(2 t s)), so
// E = 4 r^2 with r = 1 / (1 + 2^(c_k s)); the factor 4 is applied by the caller.
// Packed float32 pairs (sm_100+ f32x2 arithmetic): one instruction for two lanes
// of work.  A pair lives in a 64-bit register.
__device__ __forceinline__ unsigned long long pack2(float a, float b) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void unpack2(unsigned long long r, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b,
                                                   unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ unsigned long long mul2(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long add2(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

// TANH (with FAST, for the BF16 / FP8 forms, whose operands already carry 2^-9 or
// coarser rounding): E = (t y - 1)^2 with y = tanh.approx(s) and pk = t_k, one MUFU
// op and 2.5 instructions per element, where the exact form takes 2 MUFU ops and 4.
template <bool FAST, bool PACKED = false, bool TANH = false>
__device__ __forceinline__ float chunk_error(uint32_t taddr, const float* __restrict__ pk,
                                             long long p0, long long m, float rs, float bias,
                                             int act, int err, float R) {
  float cq[32];
  const float4* c4 = reinterpret_cast<const float4*>(pk + p0);
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const float4 x = __ldg(c4 + q);
    cq[4 * q] = x.x;
    cq[4 * q + 1] = x.y;
    cq[4 * q + 2] = x.z;
    cq[4 * q + 3] = x.w;
  }
  float v[32];
  tmem_ld32(taddr, v);
  float sum = 0.0f;
  if (FAST && TANH) {
    const unsigned long long rs2 = pack2(rs, rs), b2 = pack2(bias, bias), m2 = pack2(-1.0f, -1.0f);
    unsigned long long acc2 = pack2(0.0f, 0.0f);
    if (p0 + 32 <= m) {
#pragma unroll
      for (int j = 0; j < 32; j += 2) {
        const unsigned long long s2 = fma2(pack2(v[j], v[j + 1]), rs2, b2);
        float s0, s1;
        unpack2(s2, s0, s1);
        const unsigned long long e2 =
            fma2(pack2(cq[j], cq[j + 1]), pack2(tanh_approx(s0), tanh_approx(s1)), m2);
        acc2 = fma2(e2, e2, acc2);
      }
    } else {
#pragma unroll
      for (int j = 0; j < 32; j += 2) {
        const unsigned long long s2 = fma2(pack2(v[j], v[j + 1]), rs2, b2);
        float s0, s1;
        unpack2(s2, s0, s1);
        float e0, e1;
        unpack2(fma2(pack2(cq[j], cq[j + 1]), pack2(tanh_approx(s0), tanh_approx(s1)), m2), e0, e1);
        const unsigned long long e2 = pack2(p0 + j < m ? e0 : 0.0f, p0 + j + 1 < m ? e1 : 0.0f);
        acc2 = fma2(e2, e2, acc2);
      }
    }
    float a0, a1;
    unpack2(acc2, a0, a1);
    return a0 + a1;
  }
  if (FAST && PACKED && p0 + 32 <= m) {
    // two patterns per float32x2 instruction: s = v rs + b, u = c s, d = 1 + 2^u,
    // r = 1/d, sum += r^2 (the two running sums are added at the end)
    const unsigned long long rs2 = pack2(rs, rs), b2 = pack2(bias, bias), one2 = pack2(1.0f, 1.0f);
    unsigned long long acc2 = pack2(0.0f, 0.0f);
#pragma unroll
    for (int j = 0; j < 32; j += 2) {
      const unsigned long long s2 = fma2(pack2(v[j], v[j + 1]), rs2, b2);
      const unsigned long long u2 = mul2(pack2(cq[j], cq[j + 1]), s2);
      float u0, u1;
      unpack2(u2, u0, u1);
      const unsigned long long d2 = add2(pack2(ex2_approx(u0), ex2_approx(u1)), one2);
      float d0, d1;
      unpack2(d2, d0, d1);
      const unsigned long long r2 = pack2(rcp_approx(d0), rcp_approx(d1));
      acc2 = fma2(r2, r2, acc2);
    }
    float a0, a1;
    unpack2(acc2, a0, a1);
    return 4.0f * (a0 + a1);
  }
  if (p0 + 32 <= m) {
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const float s = fmaf(v[j], rs, bias);
      if (FAST) {
        // fewest instructions per element: epilogue issue slots are the limit
        const float r = rcp_approx(1.0f + ex2_approx(cq[j] * s));
        sum = fmaf(r, r, sum);
      } else {
        sum += general_error(cq[j], s, act, err, R);
      }
    }
  } else {
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const float s = fmaf(v[j], rs, bias);
      float e;
      if (FAST) {
        const float r = rcp_approx(1.0f + ex2_approx(cq[j] * s));
        e = r * r;
      } else {
        e = general_error(cq[j], s, act, err, R);
      }
      if (p0 + j < m) sum += e;
    }
  }
  return FAST ? 4.0f * sum : sum;
}

}  // namespace tc
}  // namespace game
