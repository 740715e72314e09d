// On-the-fly tensor-core fitness (the FP32 form): the expansion matrix P is never
// stored.  Expansion warps form each 128-pattern tile of P, one 128-byte k-block at a
// time, straight from the features X into the 128-byte-swizzled shared-memory layout
// the tcgen05 MMA reads (fp16 hi and lo planes, the same values as the stored
// expansion), while the MMA warp contracts the previous k-blocks with the resident gene
// planes and the epilogue warps reduce finished accumulators.
//
// The paper lists, among its future work (Section 6), forming the population matrix in
// place on the GPU instead of holding it in memory; Section 4.1 keeps the precomputed
// sines and cosines on the device.  What this computes is the stored path's eq.2 ->
// eq.3 -> eq.4 / eq.5 / eq.10: S = P G^T with the fp16 hi / lo split of both operands
// (three products per term), the fused error epilogue, float-float per-chromosome sums
// and float64 partial rows, one per CTA that shares a slice.
//
// Roles of the 544 threads of a CTA (one CTA per SM; one 128-chromosome slice):
//   warp 0      TMEM allocation, the gene planes by TMA, the MMAs (lane 0 issues);
//   warps 1-8   expansion: a stage is one k-block of a tile, 128 rows x 8 chunks of 16
//               bytes, four chunks per thread, both planes;
//   warps 9-16  epilogue: TMEM lane quadrant warp % 4, half of the tile's columns each.
// Ring of S stages of 32 KB (hi plane then lo plane); full[s] counts the expansion
// warps (each fences its writes to the async proxy before arriving), empty[s] is the
// MMA commit.  Every wait is bounded (2 s) and records GAME_ERR_TIMEOUT.
#include <algorithm>

#include "basis.cuh"
#include "checks.cuh"
#include "fitness_tc.h"
#include "tc_ptx.cuh"

namespace game {

namespace {

using namespace tc;

constexpr int kBN = 128;                     // patterns per tile (MMA N)
constexpr int kExpWarps = 8;
constexpr int kEpiWarps = 8;
constexpr int kOtfThreads = 32 * (1 + kExpWarps + kEpiWarps);
constexpr int kTileA = 128 * 128;            // one gene plane's k-block: 128 rows x 128 B
constexpr int kPlaneB = kBN * 128;           // one pattern plane's k-block: 16 KB
constexpr int kStage = 2 * kPlaneB;          // hi plane, then lo plane
constexpr int kSmemMaxO = 232448;
constexpr int kSmemMiscO = 1024 + 512;
constexpr uint32_t kTmemColsO = 2 * kBN;     // two accumulator buffers

struct OtfTcParams {
  CUtensorMap a[2];        // gene planes (hi, lo) [pop_pad x kp], box 128 rows x 128 B
  const float* X;          // [n_patterns x F] features
  const float* pk;         // per-pattern epilogue input (2 log2(e) t when FAST, else t)
  const float* colscale;   // [kp] power-of-two column scales of P
  const float* bias;
  const float* rscale;
  double* partial;         // [cps x pop_pad]
  DevState* state;
  long long m;             // training rows
  int F, d, basis, bd, kb, kp, kblocks, stages, n_slices, cps, n_tiles, pop_pad;
  int unit_scale, act, err, in_evolve;
  int aligned;             // Chebyshev with whole 8-column chunks per feature (B d % 8 == 0)
  float R;
};

template <bool FAST>
__global__ void __launch_bounds__(kOtfThreads, 1)
    fitness_tc_otf_kernel(const __grid_constant__ OtfTcParams p) {
  if (p.in_evolve && p.state->stopped) return;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~(uintptr_t)1023);
  const int S = p.stages;
  uint8_t* sA = smem;                                        // [plane][k-block] gene tiles
  uint8_t* sB = sA + 2 * p.kblocks * kTileA;                 // [stage][plane] pattern tiles
  uint64_t* bars = reinterpret_cast<uint64_t*>(sB + S * kStage);
  uint64_t* a_full = bars;
  uint64_t* full = bars + 1;
  uint64_t* empty = full + S;
  uint64_t* acc_full = empty + S;
  uint64_t* acc_empty = acc_full + 2;
  uint64_t* fin = acc_empty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(fin + 1);
  volatile int* err = reinterpret_cast<volatile int*>(tmem_slot + 1);
  double* red = reinterpret_cast<double*>(sB);   // [2][128], once the ring is idle

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int slice = (int)blockIdx.x % p.n_slices;
  const int member = (int)blockIdx.x / p.n_slices;
  const int my_tiles = member < p.n_tiles ? (p.n_tiles - 1 - member) / p.cps + 1 : 0;

  if (threadIdx.x == 0) {
    mbar_init(a_full, 1);
    for (int s = 0; s < S; ++s) {
      mbar_init(full + s, kExpWarps);   // one arrival per expansion warp
      mbar_init(empty + s, 1);          // the MMA commit that frees the stage
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(acc_full + b, 1);
      mbar_init(acc_empty + b, kEpiWarps);
    }
    mbar_init(fin, 1);
    *err = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kTmemColsO));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  F2Sum acc;   // epilogue threads: the chromosome's error sum over its columns

  if (warp == 0) {
    // ---- the gene planes by TMA, then the MMAs (warp-uniform loop, lane 0 issues) ----
    if (lane == 0) {
      mbar_expect_tx(a_full, 2u * (uint32_t)p.kblocks * kTileA);
      for (int pl = 0; pl < 2; ++pl)
        for (int kb = 0; kb < p.kblocks; ++kb)
          tma_load_2d(sA + (pl * p.kblocks + kb) * kTileA, &p.a[pl], kb * 64, slice * 128, a_full);
    }
    __syncwarp();
    constexpr uint32_t kIdesc = make_idesc(128, kBN, 0u);   // fp16 operands, f32 accumulate
    const int a_steps_total = p.kp / 16;                    // 16 fp16 per MMA k-step
    bool ok = warp_wait(a_full, 0, err, p.state, lane);
    if (ok) {
      fence_after();
      int stage = 0;
      uint32_t phase = 0;
      const uint32_t a_addr = smem_u32(sA), b_addr = smem_u32(sB);
      for (int it = 0; it < my_tiles && ok; ++it) {
        const int buf = it & 1;
        const uint32_t ap = (uint32_t)((it >> 1) & 1);
        if (!warp_wait(acc_empty + buf, ap ^ 1u, err, p.state, lane)) {
          ok = false;
          break;
        }
        fence_after();
        const uint32_t d = tmem + (uint32_t)(buf * kBN);
        uint32_t accum = 0;   // the tile's first product starts the accumulator
        for (int kb = 0; kb < p.kblocks; ++kb) {
          if (!warp_wait(full + stage, phase, err, p.state, lane)) {
            ok = false;
            break;
          }
          fence_after();
          const int steps = min(4, a_steps_total - kb * 4);
          const uint64_t bhi = sw128_desc(b_addr + (uint32_t)(stage * kStage));
          const uint64_t blo = sw128_desc(b_addr + (uint32_t)(stage * kStage + kPlaneB));
          const uint64_t ahi = sw128_desc(a_addr + (uint32_t)(kb * kTileA));
          const uint64_t alo = sw128_desc(a_addr + (uint32_t)((p.kblocks + kb) * kTileA));
          // FP32 split: G_hi P_hi + G_lo P_hi + G_hi P_lo; +32 bytes along K inside the
          // 128-byte swizzle row = +2 in the descriptor's address field
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            if (k < steps) {
              if (lane == 0) {
                mma<GAME_FP32>(d, ahi + 2 * k, bhi + 2 * k, kIdesc, accum);
                mma<GAME_FP32>(d, alo + 2 * k, bhi + 2 * k, kIdesc, 1u);
                mma<GAME_FP32>(d, ahi + 2 * k, blo + 2 * k, kIdesc, 1u);
              }
              accum = 1;
            }
          }
          if (lane == 0) mma_commit(empty + stage);   // the stage is free once these complete
          if (++stage == S) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (!ok) break;
        if (lane == 0) mma_commit(acc_full + buf);
      }
    }
    // Drain: the gene copies have landed and every issued MMA has completed before TMEM
    // is released and the ring is reused (both bounded).
    if (lane == 0) {
      const unsigned long long t0 = globaltimer();
      while (!mbar_try_wait(a_full, 0) && globaltimer() - t0 < kWaitNs) {
      }
      mma_commit(fin);
      const unsigned long long t1 = globaltimer();
      while (!mbar_try_wait(fin, 0) && globaltimer() - t1 < kWaitNs) {
      }
    }
    __syncwarp();
  } else if (warp <= kExpWarps) {
    // ---- expansion: k-block kb of the tile into a ring stage, both planes ----
    // Thread e fills 16-byte chunk c = e mod 8 of rows e / 8 + 32 i (i < 4); a warp covers
    // 4 rows x 8 chunks per i.
    const int e = (warp - 1) * 32 + lane;
    const int c = e & 7, rbase = e >> 3;
    // 128-byte swizzle: chunk c of row r sits at chunk c ^ (r mod 8) of its line
    auto put = [&](uint8_t* st, int r, const uint32_t (&hi)[4], const uint32_t (&lo)[4]) {
      const int off = r * 128 + ((c ^ (r & 7)) << 4);   // < kPlaneB
      *reinterpret_cast<uint4*>(st + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
      *reinterpret_cast<uint4*>(st + kPlaneB + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    };
    int stage = 0;
    uint32_t phase = 0;
    bool ok = true;
    for (int it = 0; it < my_tiles && ok; ++it) {
      const long long row0 = (long long)(member + it * p.cps) * kBN;
      for (int kb = 0; kb < p.kblocks; ++kb) {
        const int col0 = kb * 64 + c * 8;
        const bool live = col0 < p.kb;
        // Chebyshev in whole chunks: the four rows' features are loaded before the stage
        // wait, and their recurrences run side by side
        float x[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        int b0 = 0;
        if (p.aligned && live) {
          const int f = col0 / p.bd;
          b0 = col0 - f * p.bd;
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const long long row = row0 + rbase + 32 * i;
            if (row < p.m) x[i] = __ldg(p.X + row * p.F + f);   // rows past m: masked later
          }
        }
        if (!warp_wait(empty + stage, phase ^ 1u, err, p.state, lane)) {
          ok = false;
          break;
        }
        uint8_t* st = sB + stage * kStage;
        if (p.aligned) {
          uint32_t hi[4][4], lo[4][4];
          if (live) {
            float v[4][8], inv[8];
#pragma unroll
            for (int j = 0; j < 8; ++j)
              inv[j] = p.unit_scale ? 1.0f : 1.0f / __ldg(p.colscale + col0 + j);
            cheb8_rows<4>(x, b0, v);
#pragma unroll
            for (int i = 0; i < 4; ++i) fp32_split8(v[i], inv, p.unit_scale != 0, hi[i], lo[i]);
          } else {
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
              for (int q = 0; q < 4; ++q) hi[i][q] = lo[i][q] = 0u;
          }
#pragma unroll
          for (int i = 0; i < 4; ++i) put(st, rbase + 32 * i, hi[i], lo[i]);
        } else {
#pragma unroll 1
          for (int i = 0; i < 4; ++i) {
            const long long row = row0 + rbase + 32 * i;
            uint32_t hi[4] = {0u, 0u, 0u, 0u}, lo[4] = {0u, 0u, 0u, 0u};
            if (row < p.m)   // rows past the training rows stay zero (masked later)
              fp32_planes_chunk(p.X + row * p.F, p.basis, p.d, p.bd, p.kb, col0, p.colscale,
                                p.unit_scale != 0, hi, lo);
            put(st, rbase + 32 * i, hi, lo);
          }
        }
        // the writes reach the tensor cores' (async) proxy before the stage is announced
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(full + stage);
        if (++stage == S) {
          stage = 0;
          phase ^= 1u;
        }
      }
    }
  } else {
    // ---- epilogue: lane quadrant q, columns h*64 .. h*64 + 63 of each tile ----
    const int q = warp & 3;
    const int h = (warp - 1 - kExpWarps) >> 2;
    const int c = slice * 128 + q * 32 + lane;
    const float bias = p.bias[c], rs = p.rscale[c];
    bool ok = true;
    for (int it = 0; it < my_tiles && ok; ++it) {
      const int buf = it & 1;
      const uint32_t ap = (uint32_t)((it >> 1) & 1);
      const long long tile = member + (long long)it * p.cps;
      if (!warp_wait_backoff(acc_full + buf, ap, err, p.state, lane)) {
        ok = false;
        break;
      }
      fence_after();
      const uint32_t tb = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * kBN + h * 64);
#pragma unroll
      for (int ch = 0; ch < 2; ++ch) {
        const long long p0 = tile * kBN + h * 64 + ch * 32;
        acc.add(chunk_error<FAST, true>(tb + ch * 32, p.pk, p0, p.m, rs, bias, p.act, p.err,
                                        p.R));
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acc_empty + buf);
    }
  }
  // Every MMA has completed (drained by warp 0): the ring is free for the reduction of
  // the two column halves and TMEM can be released.
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemColsO));
  if (warp > kExpWarps)
    red[((warp - 1 - kExpWarps) >> 2) * 128 + (warp & 3) * 32 + lane] = acc.value();
  __syncthreads();
  if (threadIdx.x < 128) {
    const double tot = red[threadIdx.x] + red[128 + threadIdx.x];
    const long long o = (long long)member * p.pop_pad + slice * 128 + threadIdx.x;
    if (GAME_IN_BOUNDS_DBG(member < p.cps && slice * 128 + (int)threadIdx.x < p.pop_pad,
                           kSiteTcPartial, o))
      p.partial[o] = tot;
  }
}

}  // namespace

bool otf_tc_supported(const Shape& s) {
  if (s.precision != GAME_FP32 || s.shared) return false;
  const int kblocks = (s.kp + 63) / 64;
  // the resident gene planes and at least two ring stages
  return 2 * kblocks * kTileA + 2 * kStage + kSmemMiscO <= kSmemMaxO;
}

cudaError_t otf_tc_plan(const Shape& s, const PopDev& p, int n_sm, OtfTcPlan* plan) {
  if (!otf_tc_supported(s) || s.n_train < 1) return cudaErrorNotSupported;
  OtfTcPlan& t = *plan;
  t.kblocks = (s.kp + 63) / 64;
  const int a_bytes = 2 * t.kblocks * kTileA;
  t.stages = std::min(8, (kSmemMaxO - kSmemMiscO - a_bytes) / kStage);
  if (t.stages < 2) return cudaErrorNotSupported;
  const int n_slices = s.pop_pad / 128;
  t.n_tiles = (int)((s.n_train + kBN - 1) / kBN);
  int cps = n_sm / n_slices;
  if (cps < 1) cps = 1;
  if (cps > t.n_tiles) cps = t.n_tiles;
  t.cps = cps;
  t.grid = n_slices * cps;
  t.smem = (size_t)a_bytes + (size_t)t.stages * kStage + kSmemMiscO;
  cudaError_t err;
  if ((err = tc_make_map(&t.a_map[0], p.ghi, GAME_FP32, s.pop_pad, s.kp, 128)) != cudaSuccess)
    return err;
  return tc_make_map(&t.a_map[1], p.glo, GAME_FP32, s.pop_pad, s.kp, 128);
}

cudaError_t otf_tc_launch(const OtfTcPlan& t, const Shape& s, const Fitness& f, const PopDev& pd,
                          const ExpDev& e, const float* X, double* partial, DevState* dev_state,
                          int in_evolve, cudaStream_t st) {
  OtfTcParams a;
  a.a[0] = t.a_map[0];
  a.a[1] = t.a_map[1];
  const bool fast = f.pm1_targets && f.activation == GAME_TANH &&
                    (f.error == GAME_RMSE || f.error == GAME_MSE);
  a.X = X;
  a.pk = fast ? e.tcoef : e.t;
  a.colscale = e.colscale;
  a.bias = pd.bias;
  a.rscale = pd.rscale;
  a.partial = partial;
  a.state = dev_state;
  a.m = s.n_train;
  a.F = s.n_features;
  a.d = s.degree;
  a.basis = s.basis;
  a.bd = s.bd;
  a.kb = s.kb;
  a.kp = s.kp;
  a.kblocks = t.kblocks;
  a.stages = t.stages;
  a.n_slices = s.pop_pad / 128;
  a.cps = t.cps;
  a.n_tiles = t.n_tiles;
  a.pop_pad = s.pop_pad;
  a.unit_scale = e.unit_scale32;
  a.aligned = s.basis == GAME_CHEBYSHEV && s.bd % 8 == 0;
  a.act = f.activation;
  a.err = f.error;
  a.R = f.tmse_R;
  a.in_evolve = in_evolve;
  if (!dev_state) return cudaErrorInvalidValue;   // the kernel records timeouts there
  if (fast)
    fitness_tc_otf_kernel<true><<<t.grid, kOtfThreads, t.smem, st>>>(a);
  else
    fitness_tc_otf_kernel<false><<<t.grid, kOtfThreads, t.smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t otf_tc_init_attributes() {
  cudaError_t e = cudaFuncSetAttribute(fitness_tc_otf_kernel<true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemMaxO);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(fitness_tc_otf_kernel<false>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemMaxO);
}

}  // namespace game
