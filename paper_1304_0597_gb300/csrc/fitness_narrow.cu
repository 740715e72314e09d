// Population fitness for narrow populations: at most 32 chromosomes with 16 or
// 32 stored basis columns, the paper's own settings (2N + 1 chromosomes with the
// shared polytrigo expansion, Section 5).  Out(pat_k) = a_0 + sum_g P[k,g] G[c,g]
// (eq.2), E_k = (t_k - act(Out))^2 (eq.3) or its threshold form (eq.10), summed
// per chromosome into float64 partial rows that the reduce step adds in a fixed
// order (eq.4, eq.5).
//
// With 23 chromosomes a 128-chromosome tensor-core tile, or a 64-chromosome
// SIMT block, would be mostly padding, and the work is one pass over P: at 16
// columns a pattern brings 64 bytes (FP32 planes) for 23 x 16 multiply-adds.
// In both kernels here each warp streams its own ranges of rows through a
// two-stage ring in shared memory, and the float32 error sums of a lane cover
// at most 32 patterns before they are added across lanes and into float64
// (fixed assignment and order, so the result is deterministic).
// * FP32 and BF16 forms (fitness_narrow_mma_kernel): warp-level MMAs; each stage
//   is bulk copies (the P planes, then the targets) issued by one lane and
//   completed on an mbarrier.
// * FP8 form (fitness_narrow_kernel), whose genes stay float32: CUDA cores; each
//   stage is 16-byte cp.async copies, consecutive in global memory and stored
//   chunk-major (chunk j of row r at (j * rows + r) * 16), so that each thread
//   later reads its own rows without bank conflicts.
#include "simt.h"
#include "tc_ptx.cuh"

namespace game {
namespace {

constexpr int kNarrowPop = 32;
constexpr int kNarrowThreads = 256;
constexpr int kNarrowWarps = kNarrowThreads / 32;
constexpr int kNarrowStages = 2;

// CUDA-core form: chromosome groups of four the kernel carries (the population
// rounded up to 8), and rows per thread and pass (each gene read from shared
// memory feeds this many patterns; two rows fit 128 registers only at 16
// columns with up to 24 chromosomes, so the FP8 form's 32-column rows take one).
constexpr int narrow_groups(int pop) { return (pop + 7) / 8 * 2; }
constexpr int narrow_rows(int kp, int ng) { return kp == 16 && ng <= 6 ? 2 : 1; }

// Size of one warp's ring stage: W rows of every plane, then their targets
// (chunk-major in the CUDA-core kernel, row-major per plane in the warp-MMA one).
template <int PREC, int KP, int W>
struct NarrowGeom {
  static constexpr int kPlanes = PREC == GAME_FP32 ? 2 : 1;            // FP32: hi and lo fp16
  static constexpr int kPlaneBytes = PREC == GAME_FP8 ? KP : 2 * KP;   // a row of one plane
  static constexpr int kPlaneChunks = kPlaneBytes / 16;
  static constexpr int kChunks = kPlanes * kPlaneChunks;               // 16-byte chunks a row
  static constexpr int kWarpRows = W;                                  // rows a warp and pass
  static constexpr int kTargetOff = kWarpRows * kChunks * 16;          // targets after the rows
  static constexpr int kStageBytes = kTargetOff + 4 * kWarpRows;
  static constexpr int kSmem = kNarrowWarps * kNarrowStages * kStageBytes;
};

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src),
               "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(uint32_t dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(uint32_t dst, const void* src, int src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src),
               "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Copies rows [k0, k0 + kWarpRows) of every plane, and their targets, into one
// stage of the warp's ring.  A pass inside the data takes the plain form (one
// address add per copy); the last, ragged pass zero-fills the rows at or past m
// (source clamped to row 0, no byte of it read).
template <int PREC, int KP, int W>
__device__ __forceinline__ void narrow_stage(const SimtArgs& a, long long k0, uint32_t stage,
                                             int lane) {
  using Gm = NarrowGeom<PREC, KP, W>;
  constexpr int kPer = Gm::kWarpRows * Gm::kPlaneChunks;   // chunks of one plane
  const bool full = k0 + W <= a.m;
#pragma unroll
  for (int pl = 0; pl < Gm::kPlanes; ++pl) {
    const uint8_t* base = static_cast<const uint8_t*>(pl == 0 ? a.p0 : a.p1);
    const uint8_t* pass = base + k0 * Gm::kPlaneBytes;
#pragma unroll
    for (int u = 0; u < kPer / 32; ++u) {
      const int i = lane + 32 * u;
      const int r = i / Gm::kPlaneChunks, j = i % Gm::kPlaneChunks;
      const uint32_t dst = stage + ((pl * Gm::kPlaneChunks + j) * Gm::kWarpRows + r) * 16;
      if (full) {
        cp_async16(dst, pass + i * 16);   // row r, chunk j: (r * chunks + j) * 16
      } else {
        const bool ok = k0 + r < a.m;
        cp_async16(dst, ok ? pass + i * 16 : base, ok ? 16 : 0);
      }
    }
  }
#pragma unroll
  for (int u = 0; u < (W + 31) / 32; ++u) {
    const int r = lane + 32 * u;
    if (W % 32 != 0 && r >= W) break;
    if (full) {
      cp_async4(stage + Gm::kTargetOff + 4 * r, a.t + k0 + r);
    } else {
      const bool ok = k0 + r < a.m;
      cp_async4(stage + Gm::kTargetOff + 4 * r, ok ? a.t + k0 + r : a.t, ok ? 4 : 0);
    }
  }
}

// Values 8j .. 8j+7 of row r of an FP8 stage (the column scales are folded into
// the genes).
template <int PREC, int KP, int W>
__device__ __forceinline__ void narrow_values8(const uint8_t* stage, int r, int j, float v[8]) {
  using Gm = NarrowGeom<PREC, KP, W>;
  {   // e4m3: 16 values a chunk, this is its half j % 2
    const uint2 w = *reinterpret_cast<const uint2*>(
        stage + ((j >> 1) * Gm::kWarpRows + r) * 16 + 8 * (j & 1));
    const __nv_fp8x2_storage_t* b = reinterpret_cast<const __nv_fp8x2_storage_t*>(&w);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float2 f = __half22float2(__half2(__nv_cvt_fp8x2_to_halfraw2(b[i], __NV_E4M3)));
      v[2 * i] = f.x;
      v[2 * i + 1] = f.y;
    }
  }
}

__device__ __forceinline__ float narrow_error(float t, float s, int err, float R) {
  const float d = t - tanhf(s);
  const float e = d * d;
  if (err == GAME_TMSE) return fabsf(d) > R ? e : 0.0f;
  if (err == GAME_TMSE_SQ) return e > R ? e : 0.0f;
  return e;
}

// CUDA-core form (FP8 P, float32 genes x column scales).  A thread takes
// kRows patterns a pass.  The genes sit transposed in shared memory; each
// 16-byte read is a broadcast of four chromosomes that feeds kRows patterns, two
// chromosomes per packed f32x2 FMA.  The loop runs over the columns outside and
// the chromosome groups inside, so every group's sums are independent chains,
// and the P values stream through registers eight at a time.  The number of
// groups is a template parameter (the population rounded up to a multiple of 8).
// Errors are summed per chromosome in float32 pairs; a butterfly across the warp
// leaves lane c with chromosome c's block total.
template <int PREC, int KP, int NG, bool TANH>
__global__ void __launch_bounds__(kNarrowThreads, 2) fitness_narrow_kernel(SimtArgs a) {
  static_assert(PREC == GAME_FP8, "the FP32 and BF16 forms run on fitness_narrow_mma_kernel");
  if (a.in_evolve && a.state->stopped) return;
  constexpr int kRows = narrow_rows(KP, NG);
  using Gm = NarrowGeom<PREC, KP, 32 * kRows>;
  constexpr int kC = 4 * NG;   // chromosomes carried (the population, padded)
  extern __shared__ __align__(16) uint8_t narrow_ring[];   // [warp][stage][kStageBytes]
  __shared__ __align__(16) float Gt[KP][kC];                // Gt[g][c] = G[c][g] (x s_g)
  __shared__ __align__(16) float bs[kC];
  __shared__ double red[kNarrowWarps][kNarrowPop];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint8_t* ring = narrow_ring + warp * kNarrowStages * Gm::kStageBytes;
  const uint32_t ring_s = static_cast<uint32_t>(__cvta_generic_to_shared(ring));

  // The warp's passes: rows [k0, k0 + kWarpRows), k0 advancing by step; the
  // first stages are in flight while the genes are staged.
  const long long step = (long long)gridDim.x * kNarrowWarps * Gm::kWarpRows;
  long long k0 = ((long long)blockIdx.x * kNarrowWarps + warp) * Gm::kWarpRows;
#pragma unroll
  for (int s = 0; s < kNarrowStages; ++s) {
    if (k0 + s * step < a.m)
      narrow_stage<PREC, KP, 32 * kRows>(a, k0 + s * step, ring_s + s * Gm::kStageBytes, lane);
    cp_async_commit();
  }
  for (int i = tid; i < KP * kC; i += kNarrowThreads) {
    const int g = i / kC, c = i % kC;
    float v = 0.0f;
    if (c < a.pop && g < a.kb) v = a.geval[(long long)c * a.kp + g] * a.colscale[g];
    Gt[g][c] = v;
  }
  if (tid < kC) bs[tid] = tid < a.pop ? a.bias[tid] : 0.0f;
  __syncthreads();

  // Error sums: acc[2q] holds chromosomes (4q, 4q+1), acc[2q+1] (4q+2, 4q+3).
  unsigned long long acc[2 * NG];
#pragma unroll
  for (int i = 0; i < 2 * NG; ++i) acc[i] = tc::pack2(0.0f, 0.0f);
  const unsigned long long m1 = tc::pack2(-1.0f, -1.0f);
  double tot = 0.0;
  int nblk = 0;
  int stage = 0;
  for (; k0 < a.m; k0 += step) {
    cp_async_wait<kNarrowStages - 1>();   // this thread's copies of the pass have landed
    __syncwarp();                          // and every lane's
    const uint8_t* sp = ring + stage * Gm::kStageBytes;
    unsigned long long s[NG][kRows][2];
#pragma unroll
    for (int q = 0; q < NG; ++q) {
      const float4 b4 = *reinterpret_cast<const float4*>(&bs[4 * q]);
#pragma unroll
      for (int r = 0; r < kRows; ++r) {
        s[q][r][0] = tc::pack2(b4.x, b4.y);
        s[q][r][1] = tc::pack2(b4.z, b4.w);
      }
    }
#pragma unroll
    for (int j = 0; j < KP / 8; ++j) {
      float v[kRows][8];
#pragma unroll
      for (int r = 0; r < kRows; ++r) narrow_values8<PREC, KP, 32 * kRows>(sp, lane + 32 * r, j, v[r]);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        unsigned long long pp[kRows];
#pragma unroll
        for (int r = 0; r < kRows; ++r) pp[r] = tc::pack2(v[r][i], v[r][i]);
#pragma unroll
        for (int q = 0; q < NG; ++q) {
          const float4 gv = *reinterpret_cast<const float4*>(&Gt[8 * j + i][4 * q]);
          const unsigned long long g01 = tc::pack2(gv.x, gv.y), g23 = tc::pack2(gv.z, gv.w);
#pragma unroll
          for (int r = 0; r < kRows; ++r) {
            s[q][r][0] = tc::fma2(pp[r], g01, s[q][r][0]);
            s[q][r][1] = tc::fma2(pp[r], g23, s[q][r][1]);
          }
        }
      }
    }
    float t[kRows];
    bool valid[kRows];
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
      const int rr = lane + 32 * r;
      valid[r] = k0 + rr < a.m;
      t[r] = reinterpret_cast<const float*>(sp + Gm::kTargetOff)[rr];
    }
    __syncwarp();   // the stage is read: refill it with the pass kNarrowStages ahead
    if (k0 + kNarrowStages * step < a.m)
      narrow_stage<PREC, KP, 32 * kRows>(a, k0 + kNarrowStages * step, ring_s + stage * Gm::kStageBytes, lane);
    cp_async_commit();
    stage = stage + 1 == kNarrowStages ? 0 : stage + 1;

    // Epilogue: d = t - Out (linear) or t - tanh(Out); E = d^2, or its threshold forms.
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
      if (!valid[r]) continue;
      if (TANH) {
#pragma unroll
        for (int i = 0; i < 2 * NG; ++i) {
          float s0, s1;
          tc::unpack2(s[i >> 1][r][i & 1], s0, s1);
          acc[i] = tc::add2(acc[i], tc::pack2(narrow_error(t[r], s0, a.err, a.R),
                                              narrow_error(t[r], s1, a.err, a.R)));
        }
      } else {
        const unsigned long long t2 = tc::pack2(t[r], t[r]);
        if (a.err == GAME_TMSE || a.err == GAME_TMSE_SQ) {
          const bool sq = a.err == GAME_TMSE_SQ;
#pragma unroll
          for (int i = 0; i < 2 * NG; ++i) {
            const unsigned long long d2 = tc::fma2(s[i >> 1][r][i & 1], m1, t2);   // t - Out
            float d0, d1, e0, e1;
            tc::unpack2(d2, d0, d1);
            tc::unpack2(tc::mul2(d2, d2), e0, e1);
            const bool k0e = sq ? e0 > a.R : fabsf(d0) > a.R;
            const bool k1e = sq ? e1 > a.R : fabsf(d1) > a.R;
            acc[i] = tc::add2(acc[i], tc::pack2(k0e ? e0 : 0.0f, k1e ? e1 : 0.0f));
          }
        } else {
#pragma unroll
          for (int i = 0; i < 2 * NG; ++i) {
            const unsigned long long d2 = tc::fma2(s[i >> 1][r][i & 1], m1, t2);
            acc[i] = tc::add2(acc[i], tc::mul2(d2, d2));
          }
        }
      }
    }
    nblk += kRows;
    if (nblk == 32) {   // float32 sums over at most 32 patterns
      float f[kNarrowPop];
#pragma unroll
      for (int c = 0; c < kNarrowPop; ++c) f[c] = 0.0f;
#pragma unroll
      for (int i = 0; i < 2 * NG; ++i) {
        tc::unpack2(acc[i], f[2 * i], f[2 * i + 1]);
        acc[i] = tc::pack2(0.0f, 0.0f);
      }
      tot += (double)tc::warp_column_sums32(f, lane);
      nblk = 0;
    }
  }
  cp_async_wait<0>();
  {
    float f[kNarrowPop];
#pragma unroll
    for (int c = 0; c < kNarrowPop; ++c) f[c] = 0.0f;
#pragma unroll
    for (int i = 0; i < 2 * NG; ++i) tc::unpack2(acc[i], f[2 * i], f[2 * i + 1]);
    tot += (double)tc::warp_column_sums32(f, lane);
  }
  red[warp][lane] = tot;
  __syncthreads();
  if (tid < kNarrowPop) {
    double sum = 0.0;
#pragma unroll
    for (int w = 0; w < kNarrowWarps; ++w) sum += red[w][tid];
    a.partial[(long long)blockIdx.x * a.pop_pad + tid] = sum;
  }
}

template <int PREC, int KP, int NG>
void launch_ng(const SimtArgs& a, int grid, bool tanh_act, cudaStream_t st) {
  constexpr int smem = NarrowGeom<PREC, KP, 32 * narrow_rows(KP, NG)>::kSmem;
  if (tanh_act)
    fitness_narrow_kernel<PREC, KP, NG, true><<<grid, kNarrowThreads, smem, st>>>(a);
  else
    fitness_narrow_kernel<PREC, KP, NG, false><<<grid, kNarrowThreads, smem, st>>>(a);
}

template <int PREC, int KP>
void launch_prec(const SimtArgs& a, int grid, bool tanh_act, cudaStream_t st) {
  switch (narrow_groups(a.pop)) {
    case 2: launch_ng<PREC, KP, 2>(a, grid, tanh_act, st); break;
    case 4: launch_ng<PREC, KP, 4>(a, grid, tanh_act, st); break;
    case 6: launch_ng<PREC, KP, 6>(a, grid, tanh_act, st); break;
    default: launch_ng<PREC, KP, 8>(a, grid, tanh_act, st); break;
  }
}

template <int PREC, int KP, int NG>
cudaError_t attributes_ng() {
  constexpr int smem = NarrowGeom<PREC, KP, 32 * narrow_rows(KP, NG)>::kSmem;
  for (auto k : {fitness_narrow_kernel<PREC, KP, NG, true>,
                 fitness_narrow_kernel<PREC, KP, NG, false>}) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                               cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <int PREC, int KP>
cudaError_t attributes_prec() {
  cudaError_t e = attributes_ng<PREC, KP, 2>();
  if (e == cudaSuccess) e = attributes_ng<PREC, KP, 4>();
  if (e == cudaSuccess) e = attributes_ng<PREC, KP, 6>();
  if (e == cudaSuccess) e = attributes_ng<PREC, KP, 8>();
  return e;
}


// ---------------------------------------------------------------------------
// FP32 and BF16 forms on warp-level MMAs.  The contraction of a 23-chromosome population
// is 16 x 23 FMAs a pattern, which keeps the FMA pipe of the CUDA-core form
// above busy for longer than HBM takes to deliver the rows; here the tensor
// cores take it through mma.sync m16n8k16 (f16 operands, f32 accumulate), fed
// from a shared-memory ring of bulk copies, so the threads only run the epilogue.
// * A (16 patterns x 16 columns) comes from the staged P planes, B (16 columns x
//   8 chromosomes) from prepare_kernel's gene planes, kept in registers.  The
//   sum over a k-step does not depend on the column order, so the columns are
//   permuted within each k-step: the fragment's logical columns 2i, 2i+1,
//   2i+8, 2i+9 (i = lane % 4) are the stored columns 4i .. 4i+3, one 8-byte
//   load for A's row and for B's chromosome alike.  With rows staged row-major
//   (2 KP bytes) the 8-byte loads of a fragment cover eight consecutive rows.
// * FP32 from fp16 pieces, as in the tensor-core kernel: P = P_hi + P_lo
//   exactly, g' = g s_col / r_c = G_hi + G_lo; D = P_hi G_hi + P_hi G_lo +
//   P_lo G_hi, three products on one accumulator that starts at a_0 / r_c, so
//   Out = r_c D.  BF16: one P plane; the float32 genes times the column scales
//   are split into three bf16 pieces that add up to them exactly, so the three
//   products P w1 + P w2 + P w3 give what float32 genes would (each product is
//   exact in float32; only the order of the sums differs).
// * A thread ends with rows lane/4 and lane/4 + 8 of each 16-row block for
//   chromosomes 2i, 2i+1 of each 8-chromosome block: it sums their errors in
//   float32 pairs over 32 patterns, then the 8 lanes that share i add theirs
//   (3 shuffles) into float64.
// ---------------------------------------------------------------------------
// One bulk (TMA engine) copy global -> shared, completing on an mbarrier.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      :
      : "r"(dst), "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

// Stage of the warp-MMA kernel: rows [k0, k0 + W) of each plane (FP32: hi, then
// lo; BF16: the one plane; row-major, 2 KP bytes a row), then their targets; bulk
// copies issued by one lane.  A ragged last pass copies its rows only (a
// multiple of 16 bytes) and leaves its targets to be read from global memory;
// the stale rows past m feed only outputs that are never summed.
template <int PREC, int KP, int W>
__device__ __forceinline__ void mma_stage(const SimtArgs& a, long long k0, uint32_t stage,
                                          uint64_t* bar) {
  constexpr uint32_t RB = 2 * KP;
  constexpr uint32_t kPlanes = PREC == GAME_FP32 ? 2 : 1;
  const long long rows = a.m - k0 < W ? a.m - k0 : W;
  const uint32_t bp = (uint32_t)rows * RB;
  const bool full = rows == W;
  tc::mbar_expect_tx(bar, kPlanes * bp + (full ? 4 * W : 0));
  const uint32_t b = tc::smem_u32(bar);
  bulk_g2s(stage, static_cast<const uint8_t*>(a.p0) + k0 * RB, bp, b);
  if (kPlanes == 2) bulk_g2s(stage + W * RB, static_cast<const uint8_t*>(a.p1) + k0 * RB, bp, b);
  if (full) bulk_g2s(stage + kPlanes * W * RB, a.t + k0, 4 * W, b);
}

// Bounded wait that ignores the CTA's error flag: after a timeout the warp still
// lets its own copies in flight land before it exits.
__device__ __forceinline__ void drain_wait(uint64_t* bar, uint32_t parity, int lane) {
  if (lane == 0) {
    const unsigned long long t0 = tc::globaltimer();
    while (!tc::mbar_try_wait(bar, parity) && tc::globaltimer() - t0 < tc::kWaitNs) {
    }
  }
  __syncwarp();
}

// 16-row blocks a warp takes a pass: as many as the 128 registers of two resident
// CTAs hold without spilling (the per-pass wait, refill and loop cost is shared by
// more rows; 64 rows instead of 32 took the paper's 16-column shape from 0.080 to
// 0.066 ms).
constexpr int mma_blocks(int kp, int nb) {
  return kp == 16 ? (nb <= 3 ? 4 : 2) : (nb <= 3 ? 2 : 1);
}

// m16n8k16 with f32 accumulate; BF: bf16 operands, else f16.  a_r0 = {a0a1, a4a5}
// (row lane/4), a_r1 = {a2a3, a6a7} (row lane/4 + 8).
template <bool BF>
__device__ __forceinline__ void mma_16816_c(float d[4], const uint2 a_r0, const uint2 a_r1,
                                            const uint2 b, float c0, float c1) {
  // d = A B + (c0, c1, c0, c1): the accumulator starts from registers held for the pass
  if (BF)
    asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, "
        "{%4, %5, %6, %7}, {%8, %9}, {%10, %11, %10, %11};"
        : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
        : "r"(a_r0.x), "r"(a_r1.x), "r"(a_r0.y), "r"(a_r1.y), "r"(b.x), "r"(b.y), "f"(c0),
          "f"(c1));
  else
    asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, "
        "{%4, %5, %6, %7}, {%8, %9}, {%10, %11, %10, %11};"
        : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
        : "r"(a_r0.x), "r"(a_r1.x), "r"(a_r0.y), "r"(a_r1.y), "r"(b.x), "r"(b.y), "f"(c0),
          "f"(c1));
}

template <bool BF>
__device__ __forceinline__ void mma_16816(float d[4], const uint2 a_r0, const uint2 a_r1,
                                          const uint2 b) {
  if (BF)
    asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, "
        "{%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a_r0.x), "r"(a_r1.x), "r"(a_r0.y), "r"(a_r1.y), "r"(b.x), "r"(b.y));
  else
    asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, "
        "{%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a_r0.x), "r"(a_r1.x), "r"(a_r0.y), "r"(a_r1.y), "r"(b.x), "r"(b.y));
}

// Four float32 gene values as three bf16 pieces that add up to them exactly: each
// remainder is exact in float32, and the third piece has at most 8 significant bits.
__device__ __forceinline__ void bf16_pieces4(const float w[4], uint2& p1, uint2& p2, uint2& p3) {
  __nv_bfloat16 h1[4], h2[4], h3[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    h1[e] = __float2bfloat16_rn(w[e]);
    const float r1 = w[e] - __bfloat162float(h1[e]);
    h2[e] = __float2bfloat16_rn(r1);
    h3[e] = __float2bfloat16_rn(r1 - __bfloat162float(h2[e]));
  }
  auto pack = [](__nv_bfloat16 lo, __nv_bfloat16 hi) {
    const __nv_bfloat162 v = __halves2bfloat162(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
  };
  p1 = make_uint2(pack(h1[0], h1[1]), pack(h1[2], h1[3]));
  p2 = make_uint2(pack(h2[0], h2[1]), pack(h2[2], h2[3]));
  p3 = make_uint2(pack(h3[0], h3[1]), pack(h3[2], h3[3]));
}

template <int ERR, bool TANH>
__device__ __forceinline__ unsigned long long mma_error2(const float d0, const float d1,
                                                         unsigned long long nr2, float t,
                                                         float R, unsigned long long acc) {
  if (TANH) {
    float nr0, nr1;   // -r_c
    tc::unpack2(nr2, nr0, nr1);
    const float y0 = tanhf(-nr0 * d0), y1 = tanhf(-nr1 * d1);   // tanh(Out)
    const float e0 = (t - y0) * (t - y0), e1 = (t - y1) * (t - y1);
    const float u0 = ERR == GAME_TMSE ? (fabsf(t - y0) > R ? e0 : 0.0f)
                     : ERR == GAME_TMSE_SQ ? (e0 > R ? e0 : 0.0f) : e0;
    const float u1 = ERR == GAME_TMSE ? (fabsf(t - y1) > R ? e1 : 0.0f)
                     : ERR == GAME_TMSE_SQ ? (e1 > R ? e1 : 0.0f) : e1;
    return tc::add2(acc, tc::pack2(u0, u1));
  }
  const unsigned long long dd = tc::fma2(tc::pack2(d0, d1), nr2, tc::pack2(t, t));   // t - Out
  if (ERR == GAME_TMSE || ERR == GAME_TMSE_SQ) {   // branch-free: d, or 0 below the threshold
    float x0, x1;
    tc::unpack2(dd, x0, x1);
    const bool k0 = ERR == GAME_TMSE_SQ ? x0 * x0 > R : fabsf(x0) > R;
    const bool k1 = ERR == GAME_TMSE_SQ ? x1 * x1 > R : fabsf(x1) > R;
    const unsigned long long z = tc::pack2(k0 ? x0 : 0.0f, k1 ? x1 : 0.0f);
    return tc::fma2(z, z, acc);
  }
  return tc::fma2(dd, dd, acc);
}

template <int PREC, int KP, int NB, int ERR, bool TANH>
__global__ void __launch_bounds__(kNarrowThreads, 2) fitness_narrow_mma_kernel(SimtArgs a) {
  if (a.in_evolve && a.state->stopped) return;
  constexpr int MB = mma_blocks(KP, NB);   // 16-row blocks a warp and pass
  constexpr int W = 16 * MB;
  constexpr int KS = KP / 16;              // k-steps of 16 columns
  constexpr bool BF = PREC == GAME_BF16;
  constexpr int kPlanes = BF ? 1 : 2;
  using Gm = NarrowGeom<PREC, KP, W>;
  constexpr int RB = 2 * KP;               // bytes of a row of one plane
  extern __shared__ __align__(16) uint8_t narrow_ring[];   // [warp][stage][kStageBytes]
  __shared__ double red[kNarrowWarps][kNarrowPop];
  __shared__ __align__(8) uint64_t full_bar[kNarrowWarps][kNarrowStages];
  __shared__ int err;   // raised by the first timed-out wait of the CTA
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int gq = lane >> 2, qi = lane & 3;
  const uint8_t* ring = narrow_ring + warp * kNarrowStages * Gm::kStageBytes;
  const uint32_t ring_s = static_cast<uint32_t>(__cvta_generic_to_shared(ring));

  const long long step = (long long)gridDim.x * kNarrowWarps * W;
  long long k0 = ((long long)blockIdx.x * kNarrowWarps + warp) * W;
  if (tid == 0) err = 0;
  if (lane == 0) {
    for (int s = 0; s < kNarrowStages; ++s) tc::mbar_init(&full_bar[warp][s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  uint32_t pending = 0;   // stages with copies in flight (warp-uniform)
  uint32_t phase = 0;     // parity of each stage's next completion
  for (int s = 0; s < kNarrowStages; ++s)
    if (k0 + s * step < a.m) {
      if (lane == 0)
        mma_stage<PREC, KP, W>(a, k0 + s * step, ring_s + s * Gm::kStageBytes, &full_bar[warp][s]);
      pending |= 1u << s;
    }
  // B fragments: chromosome 8 nb + lane/4, stored columns 16 ks + 4i .. +3.  FP32:
  // prepare_kernel's gene planes (hi, lo; rows past pop are zero), accumulator start
  // a_0 / r_c and epilogue factor -r_c.  BF16: the float32 genes times the column
  // scales as three bf16 pieces, accumulator start a_0 and factor -1.
  uint2 b0[NB][KS], b1[NB][KS], b2[NB][KS];
  float cb[NB][2];
  unsigned long long nr2[NB];
#pragma unroll
  for (int nb = 0; nb < NB; ++nb) {
    const int cg = 8 * nb + gq;
    const long long row = (long long)cg * a.kp;
#pragma unroll
    for (int ks = 0; ks < KS; ++ks) {
      if (BF) {
        float w[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int col = 16 * ks + 4 * qi + e;
          w[e] = (cg < a.pop && col < a.kb) ? a.geval[row + col] * a.colscale[col] : 0.0f;
        }
        bf16_pieces4(w, b0[nb][ks], b1[nb][ks], b2[nb][ks]);
      } else {
        b0[nb][ks] = *reinterpret_cast<const uint2*>(static_cast<const __half*>(a.ghi) + row +
                                                     16 * ks + 4 * qi);
        b1[nb][ks] = *reinterpret_cast<const uint2*>(static_cast<const __half*>(a.glo) + row +
                                                     16 * ks + 4 * qi);
        b2[nb][ks] = make_uint2(0u, 0u);
      }
    }
    float r[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int c = 8 * nb + 2 * qi + h;
      r[h] = (!BF && c < a.pop) ? a.rscale[c] : 1.0f;
      cb[nb][h] = c < a.pop ? a.bias[c] / r[h] : 0.0f;   // r: a power of two, exact
    }
    nr2[nb] = tc::pack2(-r[0], -r[1]);
  }

  unsigned long long acc[NB];   // error sums of chromosomes (8 nb + 2i, 8 nb + 2i + 1)
#pragma unroll
  for (int nb = 0; nb < NB; ++nb) acc[nb] = tc::pack2(0.0f, 0.0f);
  double* wred = red[warp];      // the warp's float64 totals, one per chromosome
  wred[lane] = 0.0;
  __syncwarp();
  auto flush = [&]() {   // float32 block sums over at most 32 patterns a lane
#pragma unroll
    for (int nb = 0; nb < NB; ++nb) {
      float f0, f1;
      tc::unpack2(acc[nb], f0, f1);
#pragma unroll
      for (int o = 4; o < 32; o <<= 1) {
        f0 += __shfl_xor_sync(0xffffffffu, f0, o);
        f1 += __shfl_xor_sync(0xffffffffu, f1, o);
      }
      if (gq == 0) {   // lanes 0..3: chromosomes 8 nb + 2i, 8 nb + 2i + 1
        wred[8 * nb + 2 * qi] += (double)f0;
        wred[8 * nb + 2 * qi + 1] += (double)f1;
      }
      acc[nb] = tc::pack2(0.0f, 0.0f);
    }
  };
  constexpr int kFlush = 32 / (2 * MB);   // passes per float32 block
  int nblk = 0;
  int stage = 0;
  for (; k0 < a.m; k0 += step) {
    if (!tc::warp_wait(&full_bar[warp][stage], (phase >> stage) & 1, &err, a.dev_state, lane)) break;
    phase ^= 1u << stage;
    pending &= ~(1u << stage);
    const int cur = stage;
    const bool full = k0 + W <= a.m;
    const uint8_t* sp = ring + stage * Gm::kStageBytes;
    uint2 ah[MB][KS][2], al[MB][KS][2];   // [.][.][0]: row lane/4, [1]: row lane/4 + 8
    float t[MB][2];
#pragma unroll
    for (int mb = 0; mb < MB; ++mb) {
#pragma unroll
      for (int ks = 0; ks < KS; ++ks) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int r = 16 * mb + gq + 8 * h;   // columns 16 ks + 4i .. + 3
          ah[mb][ks][h] = *reinterpret_cast<const uint2*>(sp + r * RB + 32 * ks + 8 * qi);
          if (!BF)
            al[mb][ks][h] = *reinterpret_cast<const uint2*>(sp + (W + r) * RB + 32 * ks + 8 * qi);
        }
      }
    }
    if (full) {   // targets: from the stage, or for the ragged last pass from global memory
#pragma unroll
      for (int mb = 0; mb < MB; ++mb)
#pragma unroll
        for (int h = 0; h < 2; ++h)
          t[mb][h] = reinterpret_cast<const float*>(sp + kPlanes * W * RB)[16 * mb + gq + 8 * h];
    } else {
#pragma unroll
      for (int mb = 0; mb < MB; ++mb)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int rr = 16 * mb + gq + 8 * h;
          t[mb][h] = k0 + rr < a.m ? a.t[k0 + rr] : 0.0f;
        }
    }
    stage = stage + 1 == kNarrowStages ? 0 : stage + 1;

#pragma unroll
    for (int mb = 0; mb < MB; ++mb) {
      float d[NB][4];
#pragma unroll
      for (int ks = 0; ks < KS; ++ks)
#pragma unroll
        for (int nb = 0; nb < NB; ++nb) {
          // FP32: P_hi G_hi + P_hi G_lo + P_lo G_hi.  BF16: P (w1 + w2 + w3).
          if (ks == 0)
            mma_16816_c<BF>(d[nb], ah[mb][0][0], ah[mb][0][1], b0[nb][0], cb[nb][0], cb[nb][1]);
          else
            mma_16816<BF>(d[nb], ah[mb][ks][0], ah[mb][ks][1], b0[nb][ks]);
          mma_16816<BF>(d[nb], ah[mb][ks][0], ah[mb][ks][1], b1[nb][ks]);
          if (BF)
            mma_16816<BF>(d[nb], ah[mb][ks][0], ah[mb][ks][1], b2[nb][ks]);
          else
            mma_16816<BF>(d[nb], al[mb][ks][0], al[mb][ks][1], b0[nb][ks]);
        }
      if (full) {   // every pass but the last: no row checks
#pragma unroll
        for (int nb = 0; nb < NB; ++nb) {
          acc[nb] = mma_error2<ERR, TANH>(d[nb][0], d[nb][1], nr2[nb], t[mb][0], a.R, acc[nb]);
          acc[nb] = mma_error2<ERR, TANH>(d[nb][2], d[nb][3], nr2[nb], t[mb][1], a.R, acc[nb]);
        }
      } else {
        const bool v0 = k0 + 16 * mb + gq < a.m;
        const bool v1 = k0 + 16 * mb + gq + 8 < a.m;
#pragma unroll
        for (int nb = 0; nb < NB; ++nb) {
          if (v0) acc[nb] = mma_error2<ERR, TANH>(d[nb][0], d[nb][1], nr2[nb], t[mb][0], a.R, acc[nb]);
          if (v1) acc[nb] = mma_error2<ERR, TANH>(d[nb][2], d[nb][3], nr2[nb], t[mb][1], a.R, acc[nb]);
        }
      }
    }
    __syncwarp();   // the stage's values are used: refill it with the pass kNarrowStages ahead
    if (k0 + kNarrowStages * step < a.m) {
      if (lane == 0)
        mma_stage<PREC, KP, W>(a, k0 + kNarrowStages * step, ring_s + cur * Gm::kStageBytes,
                         &full_bar[warp][cur]);
      pending |= 1u << cur;
    }
    if (++nblk == kFlush) {
      flush();
      nblk = 0;
    }
  }
  for (int s = 0; s < kNarrowStages; ++s)   // only after a timeout: copies still in flight
    if (pending & (1u << s)) drain_wait(&full_bar[warp][s], (phase >> s) & 1, lane);
  flush();   // chromosomes past 8 NB keep the zero they started with
  __syncthreads();
  if (tid < kNarrowPop) {
    double sum = 0.0;
#pragma unroll
    for (int w = 0; w < kNarrowWarps; ++w) sum += red[w][tid];
    a.partial[(long long)blockIdx.x * a.pop_pad + tid] = sum;
  }
}

template <int PREC, int KP, int NB, int ERR>
void launch_mma_err(const SimtArgs& a, int grid, bool tanh_act, cudaStream_t st) {
  constexpr int smem = NarrowGeom<PREC, KP, 16 * mma_blocks(KP, NB)>::kSmem;
  if (tanh_act)
    fitness_narrow_mma_kernel<PREC, KP, NB, ERR, true><<<grid, kNarrowThreads, smem, st>>>(a);
  else
    fitness_narrow_mma_kernel<PREC, KP, NB, ERR, false><<<grid, kNarrowThreads, smem, st>>>(a);
}

template <int PREC, int KP, int NB>
void launch_mma_nb(const SimtArgs& a, int grid, bool tanh_act, cudaStream_t st) {
  if (a.err == GAME_TMSE)
    launch_mma_err<PREC, KP, NB, GAME_TMSE>(a, grid, tanh_act, st);
  else if (a.err == GAME_TMSE_SQ)
    launch_mma_err<PREC, KP, NB, GAME_TMSE_SQ>(a, grid, tanh_act, st);
  else
    launch_mma_err<PREC, KP, NB, GAME_MSE>(a, grid, tanh_act, st);
}

template <int PREC, int KP>
void launch_mma(const SimtArgs& a, int grid, bool tanh_act, cudaStream_t st) {
  switch ((a.pop + 7) / 8) {
    case 1: launch_mma_nb<PREC, KP, 1>(a, grid, tanh_act, st); break;
    case 2: launch_mma_nb<PREC, KP, 2>(a, grid, tanh_act, st); break;
    case 3: launch_mma_nb<PREC, KP, 3>(a, grid, tanh_act, st); break;
    default: launch_mma_nb<PREC, KP, 4>(a, grid, tanh_act, st); break;
  }
}

template <int PREC, int KP, int NB, int ERR>
cudaError_t mma_attributes_err() {
  constexpr int smem = NarrowGeom<PREC, KP, 16 * mma_blocks(KP, NB)>::kSmem;
  for (auto k : {fitness_narrow_mma_kernel<PREC, KP, NB, ERR, true>,
                 fitness_narrow_mma_kernel<PREC, KP, NB, ERR, false>}) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                               cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <int PREC, int KP, int NB>
cudaError_t mma_attributes_nb() {
  cudaError_t e = mma_attributes_err<PREC, KP, NB, GAME_MSE>();
  if (e == cudaSuccess) e = mma_attributes_err<PREC, KP, NB, GAME_TMSE>();
  if (e == cudaSuccess) e = mma_attributes_err<PREC, KP, NB, GAME_TMSE_SQ>();
  return e;
}

template <int PREC, int KP>
cudaError_t mma_attributes() {
  cudaError_t e = mma_attributes_nb<PREC, KP, 1>();
  if (e == cudaSuccess) e = mma_attributes_nb<PREC, KP, 2>();
  if (e == cudaSuccess) e = mma_attributes_nb<PREC, KP, 3>();
  if (e == cudaSuccess) e = mma_attributes_nb<PREC, KP, 4>();
  return e;
}
}  // namespace

bool narrow_shape_ok(int pop, int kp) {
  return pop >= 1 && pop <= kNarrowPop && (kp == 16 || kp == 32);
}

bool simt_narrow(const Shape& s) { return narrow_shape_ok(s.pop, s.kp); }

int narrow_partials(const Shape& s, int n_sm) {
  const int rows = s.precision == GAME_FP8
                       ? kNarrowThreads * narrow_rows(s.kp, narrow_groups(s.pop))
                       : kNarrowWarps * 16 * mma_blocks(s.kp, (s.pop + 7) / 8);
  const long long need = (s.n_train + rows - 1) / rows;
  const long long g = 2LL * n_sm;
  return (int)(need < 1 ? 1 : need < g ? need : g);
}

cudaError_t launch_narrow(const SimtArgs& a, const Shape& s, int grid, cudaStream_t st) {
  const bool th = a.act == GAME_TANH;
  if (s.precision == GAME_FP32) {   // warp-level MMAs
    if (s.kp == 16)
      launch_mma<GAME_FP32, 16>(a, grid, th, st);
    else
      launch_mma<GAME_FP32, 32>(a, grid, th, st);
  } else if (s.precision == GAME_BF16) {
    if (s.kp == 16)
      launch_mma<GAME_BF16, 16>(a, grid, th, st);
    else
      launch_mma<GAME_BF16, 32>(a, grid, th, st);
  } else {
    if (s.kp != 32) return cudaErrorInvalidValue;   // e4m3 rows are padded to 32 columns
    launch_prec<GAME_FP8, 32>(a, grid, th, st);
  }
  return cudaGetLastError();
}

cudaError_t simt_init_attributes() {
  cudaError_t e = mma_attributes<GAME_FP32, 16>();
  if (e == cudaSuccess) e = mma_attributes<GAME_FP32, 32>();
  if (e == cudaSuccess) e = mma_attributes<GAME_BF16, 16>();
  if (e == cudaSuccess) e = mma_attributes<GAME_BF16, 32>();
  if (e == cudaSuccess) e = attributes_prec<GAME_FP8, 32>();
  return e;
}

}  // namespace game
