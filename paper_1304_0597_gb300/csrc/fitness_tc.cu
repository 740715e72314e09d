// Tensor-core fitness of the whole population on sm_103a: tcgen05.mma with the
// accumulator in TMEM, operands staged in shared memory by TMA, fused epilogue.
//
// What it computes (paper Section 2): for every chromosome c and training
// pattern k, Out = a_0 + sum_g G[c,g] P[k,g] (eq.2), E = (t_k - tanh(Out))^2
// (eq.3; eq.10 for the threshold form), and per chromosome the sum of E over
// the training patterns, later turned into MSE / RMSE (eq.4, eq.5).
//
// Layout.  D[c, k] = sum_g A[c, g] B[k, g] with A = genes of a 128-chromosome
// slice (M = 128, TMEM lane = chromosome) and B = a tile of BN expansion rows
// (N = BN, TMEM column = pattern); both K-major, 128-byte swizzled.  A CTA owns
// SP slices (1, or 2 with 128-pattern tiles) for its whole life: their gene
// planes are loaded once and stay in shared memory, while pattern tiles stream
// through a ring of B stages and each tile feeds the MMAs of every slice.  The
// per-chromosome error sum is then a per-thread running sum over TMEM columns,
// with no cross-lane reduction.
//
// Precision.  FP32 fitness: P = P_hi + P_lo and G = G_hi + G_lo are fp16
// pairs (~22 significant bits) and D accumulates G_hi.P_hi + G_lo.P_hi +
// G_hi.P_lo in float32 (kind::f16).  BF16 / FP8: one quantised P plane with
// per-column scales folded into the genes, genes as a hi/lo pair with a
// per-chromosome scale applied in the epilogue (kind::f16 bf16 / kind::f8f6f4).
// With +-1 targets, tanh and (R)MSE the FP32 form takes E = 4 / (1 + 2^(c_k s))^2
// (ex2 and rcp, no cancellation), the low-precision forms (t_k tanh.approx(s) - 1)^2
// (one MUFU op); both are in chunk_error.
//
// Roles (576 threads): warp 0 = TMA producer, warp 1 = TMEM allocator + MMA
// issuer, warps 2..17 = epilogue (warp w reads TMEM lanes 32*(w%4) and a
// quarter of the columns).  Two TMEM accumulators let the epilogue of tile i overlap the
// MMAs of tile i+1.  Every mbarrier wait is bounded (2 s of %globaltimer); on
// a timeout the CTA records GAME_ERR_TIMEOUT in the device state, drains its
// outstanding copies and MMAs (again bounded), frees TMEM and exits.
#include "checks.cuh"
#include "fitness_tc.h"
#include "tc_ptx.cuh"

#include <cudaTypedefs.h>

namespace game {

namespace {

using namespace tc;

constexpr int kEpiWarps = 16;
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr int kColGroups = kEpiWarps / 4;     // epilogue warps sharing one TMEM lane quadrant
constexpr int kTileA = 128 * 128;         // bytes of one 128-row x 128-byte A tile

// Profiling build only (-DGAME_TC_TIMELINE): CTA 0 stamps clock64 at each role's
// waits and hand-offs for its first 32 tiles, read back by game_tc_timeline().
// Slot (event, tile, k-block) = event * 256 + tile * 8 + k-block; events: 0 producer
// issues a B k-block, 1 MMA warp past its ring wait, 2 MMA warp past the accumulator
// wait, 3 MMA warp committed the tile, 4 / 5 epilogue warp 2 starts / ends the tile,
// 6 / 7 the same for warp 17.
#ifdef GAME_TC_TIMELINE
__device__ long long g_tc_timeline[2048];
#define TC_STAMP(cond, ev, tile, kb)                                                   \
  do {                                                                                 \
    if ((cond) && blockIdx.x == 0 && (tile) < 32 && (kb) < 8)                          \
      g_tc_timeline[(ev) * 256 + (tile) * 8 + (kb)] = clock64();                       \
  } while (0)
#else
#define TC_STAMP(cond, ev, tile, kb) \
  do {                               \
  } while (0)
#endif

struct TcParams {
  CUtensorMap a[2];
  CUtensorMap b[2];
  const float* t;
  const float* tcoef;     // 2 log2(e) t_k (fused +-1 / tanh path)
  const float* bias;
  const float* rscale;
  double* partial;
  DevState* state;
  long long m;            // training rows
  int n_groups, cps, n_tiles, kblocks, kp, stages, pop_pad;   // group = SP slices
  int n_bplanes;          // FP32: 2 (P_hi, P_lo); else 1
  int act, err, in_evolve;
  float R;
  int prefetch;           // L2 prefetch of the next tile's boxes
  int kg;                 // k-blocks per pattern-tile stage (one 3-D TMA request when > 1)
  int a_rows;             // gene rows held per A tile (128, or the live rows of one slice)
};

template <int BN, int PREC, bool FAST, int NA, int SP, bool PAIR>
__global__ void __launch_bounds__(kThreads, 1) fitness_tc_kernel(const __grid_constant__ TcParams p) {
  static_assert(SP == 1 || (SP == 2 && BN == 128), "two slices per CTA use 128-pattern tiles");
  static_assert(!PAIR || SP == 1, "a CTA pair holds one slice per CTA");
  if (p.in_evolve && p.state->stopped) return;   // (both CTAs of a pair read the same flag)
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~(uintptr_t)1023);
  // A pair's CTA stages BN / 2 rows of each pattern tile (its half of the MMA's N).
  constexpr int kRowsB = PAIR ? BN / 2 : BN;
  constexpr int kTileB = kRowsB * 128;
  constexpr int kKB = PREC == GAME_FP8 ? 128 : 64;    // elements per 128-byte k-block
  constexpr int kKStep = PREC == GAME_FP8 ? 32 : 16;  // elements per MMA
  constexpr uint32_t kFmt = PREC == GAME_BF16 ? 1u : 0u;
  constexpr uint32_t kIdesc = make_idesc(PAIR ? 256 : 128, BN, kFmt);
  const int S = p.stages;
  uint8_t* sA = smem;
  // A tiles hold a_rows rows (a multiple of 8): 128, or, for a single slice of at most
  // 120 chromosomes, its live rows only.  The MMA still spans 128 rows; the 8-row groups
  // past a_rows read whatever shared memory follows (the next A tile or the ring, all
  // inside the CTA's allocation) and feed only padded chromosomes, whose sums are never
  // read; the epilogue skips the lane quadrants that hold no live row.
  const int a_tile = p.a_rows * 128;
  uint8_t* sB = sA + SP * NA * p.kblocks * a_tile;
  const int kg = p.kg;                                // k-blocks per stage
  const int stage_bytes = kg * kTileB;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sB + S * stage_bytes);
  uint64_t* a_full = bars;
  uint64_t* b_full = bars + 1;
  uint64_t* b_empty = b_full + S;
  uint64_t* acc_full = b_empty + S;
  uint64_t* acc_empty = acc_full + 2;
  uint64_t* fin = acc_empty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(fin + 1);
  volatile int* err = reinterpret_cast<volatile int*>(tmem_slot + 1);
  int* last_par = reinterpret_cast<int*>(tmem_slot + 2);          // [S]
  double* red = reinterpret_cast<double*>(sB);   // [SP][kColGroups][128], once the ring is idle

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // Work of this CTA: the slices slice0 .. slice0 + SP - 1 over the pattern tiles
  // member, member + cps, ...  A pair (ranks 0 / 1 of a 2-CTA cluster) takes the two
  // adjacent slices 2 g, 2 g + 1 over the same tiles.
  const uint32_t crank = PAIR ? cluster_rank() : 0u;
  const int unit = PAIR ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;
  const int group = unit % p.n_groups;
  const int member = unit / p.n_groups;
  const int slice0 = PAIR ? 2 * group + (int)crank : group * SP;
  const bool issuer = !PAIR || crank == 0;        // the CTA whose warp 1 issues the MMAs
  const int my_tiles = member < p.n_tiles ? (p.n_tiles - 1 - member) / p.cps + 1 : 0;
  constexpr uint32_t kTmemCols = 2 * SP * BN;      // [buffer][slice] accumulators of BN columns

  if (threadIdx.x == 0) {
    mbar_init(a_full, 1);
    for (int s = 0; s < S; ++s) {
      mbar_init(b_full + s, 1);
      mbar_init(b_empty + s, 1);        // the MMA commit that frees the stage
      last_par[s] = -1;
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(acc_full + b, 1);
      // a pair's leader waits for the epilogue warps of both CTAs
      mbar_init(acc_empty + b, PAIR ? 2 * kEpiWarps : kEpiWarps);
    }
    mbar_init(fin, 1);
    *err = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    if constexpr (PAIR) {
      // one warp of each CTA of the pair allocates, together, the same TMEM columns in both
      asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                       smem_u32(tmem_slot)),
                   "r"(kTmemCols));
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
    } else {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                       smem_u32(tmem_slot)),
                   "r"(kTmemCols));
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  // The peer completes bytes on and arrives at the leader's barriers: both CTAs'
  // barriers exist before either CTA goes on.
  if constexpr (PAIR) cluster_sync_all();
  const uint32_t tmem = *tmem_slot;
  // shared::cluster addresses of the leader's barriers (the CTA's own for a single CTA)
  auto lead = [&](uint64_t* bar) -> uint32_t {
    return PAIR ? mapa_shared(smem_u32(bar), 0u) : smem_u32(bar);
  };
  const int a_steps_total = p.kp / kKStep;
  F2Sum acc[SP];   // epilogue threads: each slice's chromosome error sum over its columns

  if (warp == 0) {
    // ---- TMA producer: the whole warp follows one control flow, lane 0 issues ----
    if (lane == 0) {
      const uint32_t a_bytes = (uint32_t)SP * NA * p.kblocks * a_tile;
      // The leader expects its own and (pair) the peer's bytes on its barrier.
      if (issuer) mbar_expect_tx(a_full, PAIR ? 2 * a_bytes : a_bytes);
      for (int sp = 0; sp < SP; ++sp)
        for (int pl = 0; pl < NA; ++pl)
          for (int kb = 0; kb < p.kblocks; ++kb) {
            void* dst = sA + ((sp * NA + pl) * p.kblocks + kb) * a_tile;
            if constexpr (PAIR)
              tma_load_2d_pair(dst, &p.a[pl], kb * kKB, slice0 * 128, lead(a_full));
            else
              tma_load_2d(dst, &p.a[pl], kb * kKB, (slice0 + sp) * 128, a_full);
          }
    }
    int stage = 0;
    uint32_t phase = 0;
    bool ok = true;
    for (int it = 0; it < my_tiles && ok; ++it) {
      const int row0 = (member + it * p.cps) * BN + (int)crank * kRowsB;
      for (int kb = 0; kb < p.kblocks && ok; kb += kg)
        for (int bp = 0; bp < p.n_bplanes; ++bp) {
          if (!warp_wait(b_empty + stage, phase ^ 1u, err, p.state, lane)) {
            ok = false;
            break;
          }
          TC_STAMP(lane == 0 && bp == 0, 0, it, kb);
          if (lane == 0) {
            // warm L2 with the same box of this CTA's next tile
            if (it + 1 < my_tiles && p.prefetch && kg == 1)
              tma_prefetch_2d(&p.b[bp], kb * kKB, row0 + p.cps * BN);
            if constexpr (PAIR) {
              if (issuer) mbar_expect_tx(b_full + stage, 2 * stage_bytes);
              if (kg == 1)
                tma_load_2d_pair(sB + stage * kTileB, &p.b[bp], kb * kKB, row0, lead(b_full + stage));
              else
                tma_load_3d_pair(sB + stage * stage_bytes, &p.b[bp], 0, row0, kb, lead(b_full + stage));
            } else if (kg == 1) {
              mbar_expect_tx(b_full + stage, kTileB);
              tma_load_2d(sB + stage * kTileB, &p.b[bp], kb * kKB, row0, b_full + stage);
            } else {
              // k-blocks kb .. kb + kg - 1 in one request (past the last: zero fill)
              mbar_expect_tx(b_full + stage, stage_bytes);
              tma_load_3d(sB + stage * stage_bytes, &p.b[bp], 0, row0, kb, b_full + stage);
            }
            last_par[stage] = (int)phase;
          }
          if (++stage == S) {
            stage = 0;
            phase ^= 1u;
          }
        }
    }
    // Drain: every issued copy has landed before the CTA may exit.  A pair's copies
    // complete on the leader's barriers, which the leader drains (both CTAs issue the
    // same stage sequence); the pair meets at a cluster barrier before either exits.
    if (lane == 0 && issuer) {
      mbar_wait(a_full, 0, err, p.state);
      for (int s2 = 0; s2 < S; ++s2)
        if (last_par[s2] >= 0) {
          const unsigned long long t0 = globaltimer();
          while (!mbar_try_wait(b_full + s2, (uint32_t)last_par[s2]) && globaltimer() - t0 < kWaitNs) {
          }
        }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---- MMA issuer: warp-uniform loop (descriptors in uniform registers), lane 0 issues ----
    if (issuer && warp_wait(a_full, 0, err, p.state, lane)) {
      fence_after();
      int stage = 0;
      uint32_t phase = 0;
      const uint32_t a_addr = smem_u32(sA);
      const uint32_t b_addr = smem_u32(sB);
      for (int it = 0; it < my_tiles; ++it) {
        const int buf = it & 1;
        const uint32_t ap = (uint32_t)((it >> 1) & 1);
        const bool freed = PAIR ? warp_wait_cluster(acc_empty + buf, ap ^ 1u, err, p.state, lane)
                                : warp_wait(acc_empty + buf, ap ^ 1u, err, p.state, lane);
        if (!freed) break;
        fence_after();
        TC_STAMP(lane == 0, 2, it, 0);
        uint32_t accum = 0;   // the first k-step of a tile starts every slice's accumulator
        bool ok = true;
        for (int kb0 = 0; kb0 < p.kblocks && ok; kb0 += kg) {
          for (int bp = 0; bp < p.n_bplanes; ++bp) {
            if (!warp_wait(b_full + stage, phase, err, p.state, lane)) {
              ok = false;
              break;
            }
            fence_after();
            TC_STAMP(lane == 0 && bp == 0, 1, it, kb0);
            for (int g = 0; g < kg && kb0 + g < p.kblocks; ++g) {
              const int kb = kb0 + g;
              const int steps = min(kKB / kKStep, a_steps_total - kb * (kKB / kKStep));
              const uint64_t bdesc =
                  sw128_desc(b_addr + (uint32_t)(stage * stage_bytes + g * kTileB));
              // FP32 split: B = P_hi meets A = G_hi and G_lo; B = P_lo meets G_hi.
              const int n_ap = (PREC == GAME_FP32 && bp == 1) ? 1 : NA;
#pragma unroll
              for (int sp = 0; sp < SP; ++sp) {
                const uint32_t d = tmem + (uint32_t)((buf * SP + sp) * BN);
                uint32_t acc_sp = accum;
                for (int ai = 0; ai < n_ap; ++ai) {
                  const uint64_t adesc =
                      sw128_desc(a_addr + (uint32_t)(((sp * NA + ai) * p.kblocks + kb) * a_tile));
#pragma unroll
                  for (int k = 0; k < kKB / kKStep; ++k) {
                    if (k < steps) {
                      // +32 bytes along K inside the 128-byte swizzle row = +2 in the address field
                      if (lane == 0) {
                        if constexpr (PAIR)
                          mma_pair<PREC>(d, adesc + 2 * k, bdesc + 2 * k, kIdesc, acc_sp);
                        else
                          mma<PREC>(d, adesc + 2 * k, bdesc + 2 * k, kIdesc, acc_sp);
                      }
                      acc_sp = 1;
                    }
                  }
                }
                if (sp == SP - 1) accum = acc_sp;
              }
            }
            if (lane == 0) {
              if constexpr (PAIR) {   // the stage is free in both CTAs
                mma_commit_pair(smem_u32(b_empty + stage));
                mma_commit_pair(mapa_shared(smem_u32(b_empty + stage), 1u));
              } else {
                mma_commit(b_empty + stage);
              }
            }
            if (++stage == S) {
              stage = 0;
              phase ^= 1u;
            }
          }
        }
        if (!ok) break;
        if (lane == 0) {
          if constexpr (PAIR) {       // both CTAs' accumulators hold the tile
            mma_commit_pair(smem_u32(acc_full + buf));
            mma_commit_pair(mapa_shared(smem_u32(acc_full + buf), 1u));
          } else {
            mma_commit(acc_full + buf);
          }
        }
        TC_STAMP(lane == 0, 3, it, 0);
      }
    }
    // Drain: all issued MMAs complete before TMEM is released.
    if (lane == 0 && issuer) {
      if constexpr (PAIR)
        mma_commit_pair(smem_u32(fin));
      else
        mma_commit(fin);
      const unsigned long long t0 = globaltimer();
      while (!mbar_try_wait(fin, 0) && globaltimer() - t0 < kWaitNs) {
      }
    }
    __syncwarp();
  } else {
    // ---- epilogue ----
    const int q = warp & 3;
    const int h = (warp - 2) >> 2;                    // column group 0..kColGroups-1
    // FP32 keeps the exact fast form (c_k = 2 log2(e) t_k); the low-precision forms
    // take the one-MUFU tanh form, which reads t_k.
    constexpr bool kTanh = FAST && PREC != GAME_FP32;
    const float* pk = FAST && !kTanh ? p.tcoef : p.t;
    float bias[SP], rs[SP];
#pragma unroll
    for (int sp = 0; sp < SP; ++sp) {
      const int c = (slice0 + sp) * 128 + q * 32 + lane;
      bias[sp] = p.bias[c];
      rs[sp] = p.rscale[c];
    }
    constexpr int kCols = BN / kColGroups;
    for (int it = 0; it < my_tiles; ++it) {
      const int buf = it & 1;
      const uint32_t ap = (uint32_t)((it >> 1) & 1);
      const long long tile = member + (long long)it * p.cps;
      // The low-precision forms are bound by the epilogue: the per-pattern
      // coefficients of this tile (one 128-byte line per lane) are brought into
      // L1 while the MMAs run, so that the loads after the wait hit.
      if (PREC != GAME_FP32 && lane < kCols / 32) prefetch_l1(pk + tile * BN + h * kCols + lane * 32);
      // FP32 (three products per term) is MMA-bound: the accumulator wait sleeps
      // between polls so that the issue slots go to the MMA warp on the same
      // sub-partition.  The low-precision forms are epilogue-bound and poll.
      const bool got = PREC == GAME_FP32 ? warp_wait_backoff(acc_full + buf, ap, err, p.state, lane)
                                         : warp_wait(acc_full + buf, ap, err, p.state, lane);
      if (!got) break;
      fence_after();
      TC_STAMP(lane == 0 && (warp == 2 || warp == 17), warp == 2 ? 4 : 6, it, 0);
#pragma unroll
      for (int sp = 0; sp < SP; ++sp) {
        if (q * 32 >= p.a_rows) continue;   // no live chromosome in this lane quadrant
        const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16) +
                               (uint32_t)((buf * SP + sp) * BN + h * kCols);
#pragma unroll
        for (int ch = 0; ch < kCols / 32; ++ch) {
          const long long p0 = tile * BN + h * kCols + ch * 32;
          acc[sp].add(chunk_error<FAST, true, kTanh>(tbase + ch * 32, pk, p0, p.m, rs[sp],
                                                     bias[sp], p.act, p.err, p.R));
        }
      }
      TC_STAMP(lane == 0 && (warp == 2 || warp == 17), warp == 2 ? 5 : 7, it, 0);
      fence_before();
      __syncwarp();
      if (lane == 0) {
        if constexpr (PAIR)
          mbar_arrive_cluster(lead(acc_empty + buf));   // the leader reuses the buffer
        else
          mbar_arrive(acc_empty + buf);
      }
    }
  }
  // Every copy and MMA of this CTA has completed (drained above): the B ring is
  // free for the cross-half reduction and TMEM can be released.
  fence_before();
  __syncthreads();
  fence_after();
  // A pair: the leader's MMAs (into both CTAs' TMEM) and copies (completing on the
  // leader's barriers) are done and the peer has made its last arrival at the leader
  // before either CTA releases TMEM or exits.
  if constexpr (PAIR) cluster_sync_all();
  if (warp == 1) {
    if constexpr (PAIR)
      asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                   "r"(kTmemCols));
    else
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                   "r"(kTmemCols));
  }
  if (warp >= 2) {
#pragma unroll
    for (int sp = 0; sp < SP; ++sp)
      red[(sp * kColGroups + ((warp - 2) >> 2)) * 128 + (warp & 3) * 32 + lane] = acc[sp].value();
  }
  __syncthreads();
  if (threadIdx.x < SP * 128) {
    const int sp = threadIdx.x >> 7, r = threadIdx.x & 127;
    double tot = 0.0;
#pragma unroll
    for (int g = 0; g < kColGroups; ++g) tot += red[(sp * kColGroups + g) * 128 + r];
    const long long o = (long long)member * p.pop_pad + (slice0 + sp) * 128 + r;
    if (GAME_IN_BOUNDS_DBG(member < p.cps && (slice0 + sp) * 128 + r < p.pop_pad, kSiteTcPartial, o))
      p.partial[o] = tot;
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void* ptr = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
  }
  return fn;
}

cudaError_t make_map(CUtensorMap* m, const void* base, int precision, long long rows, int cols,
                     int box_rows) {  // NOLINT
  auto fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  const CUtensorMapDataType dt = precision == GAME_FP32   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                 : precision == GAME_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                          : CU_TENSOR_MAP_DATA_TYPE_UINT8;
  const int esz = precision == GAME_FP8 ? 1 : 2;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)cols * esz};
  cuuint32_t box[2] = {(cuuint32_t)(128 / esz), (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(m, dt, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// The same plane viewed as [k-block][row][128 bytes]: one box brings kg k-blocks of
// box_rows rows, laid out in shared memory as kg 2-D boxes one after the other.
// Needs cols to be whole k-blocks (else a k-block would run into the next row).
cudaError_t make_map3(CUtensorMap* m, const void* base, int precision, long long rows, int cols,
                      int box_rows, int kg) {
  auto fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  const CUtensorMapDataType dt = precision == GAME_FP32   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                 : precision == GAME_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                          : CU_TENSOR_MAP_DATA_TYPE_UINT8;
  const int esz = precision == GAME_FP8 ? 1 : 2;
  const int kb_elems = 128 / esz;
  if (cols % kb_elems != 0) return cudaErrorInvalidValue;
  cuuint64_t dims[3] = {(cuuint64_t)kb_elems, (cuuint64_t)rows, (cuuint64_t)(cols / kb_elems)};
  cuuint64_t strides[2] = {(cuuint64_t)cols * esz, 128};
  cuuint32_t box[3] = {(cuuint32_t)kb_elems, (cuuint32_t)box_rows, (cuuint32_t)kg};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(m, dt, 3, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

constexpr int kSmemMax = 232448;     // 227 KB opt-in per block on sm_103
constexpr int kSmemMisc = 1024 + 512;   // alignment slack + barriers

int kblocks_of(const Shape& s) {
  const int kkb = s.precision == GAME_FP8 ? 128 : 64;
  return (s.kp + kkb - 1) / kkb;
}

template <int BN, int PREC, bool FAST, int NA, int SP, bool PAIR>
void* kernel_ptr() {
  return reinterpret_cast<void*>(&fitness_tc_kernel<BN, PREC, FAST, NA, SP, PAIR>);
}

// pair: 2-CTA clusters sharing each MMA (cta_group::2, M = 256 chromosomes)
void* pick_kernel(int bn, int prec, bool fast, int na, int sp, bool pair = false) {
#define GAME_TC_PAIR(BNV, PV, NAV)                                                          \
  if (pair && bn == BNV && prec == PV && na == NAV && sp == 1)                               \
    return fast ? kernel_ptr<BNV, PV, true, NAV, 1, true>()                                  \
                : kernel_ptr<BNV, PV, false, NAV, 1, true>();
  GAME_TC_PAIR(256, GAME_FP32, 2)
  GAME_TC_PAIR(256, GAME_BF16, 2)
  GAME_TC_PAIR(256, GAME_FP8, 2)
  GAME_TC_PAIR(256, GAME_BF16, 1)
  GAME_TC_PAIR(256, GAME_FP8, 1)
#undef GAME_TC_PAIR
  if (pair) return nullptr;
#define GAME_TC_PICK(BNV, PV, NAV, SPV)                                                     \
  if (bn == BNV && prec == PV && na == NAV && sp == SPV)                                     \
    return fast ? kernel_ptr<BNV, PV, true, NAV, SPV, false>()                               \
                : kernel_ptr<BNV, PV, false, NAV, SPV, false>();
  GAME_TC_PICK(256, GAME_FP32, 2, 1)
  GAME_TC_PICK(128, GAME_FP32, 2, 1)
  GAME_TC_PICK(256, GAME_BF16, 2, 1)
  GAME_TC_PICK(128, GAME_BF16, 2, 1)
  GAME_TC_PICK(256, GAME_FP8, 2, 1)
  GAME_TC_PICK(128, GAME_FP8, 2, 1)
  GAME_TC_PICK(256, GAME_BF16, 1, 1)
  GAME_TC_PICK(128, GAME_BF16, 1, 1)
  GAME_TC_PICK(256, GAME_FP8, 1, 1)
  GAME_TC_PICK(128, GAME_FP8, 1, 1)
  // two slices per CTA (128-pattern tiles)
  GAME_TC_PICK(128, GAME_FP32, 2, 2)
  GAME_TC_PICK(128, GAME_BF16, 2, 2)
  GAME_TC_PICK(128, GAME_FP8, 2, 2)
  GAME_TC_PICK(128, GAME_BF16, 1, 2)
  GAME_TC_PICK(128, GAME_FP8, 1, 2)
#undef GAME_TC_PICK
  return nullptr;
}

}  // namespace

cudaError_t tc_make_map(CUtensorMap* m, const void* base, int precision, long long rows, int cols,
                        int box_rows) {
  return make_map(m, base, precision, rows, cols, box_rows);
}

// Self-test of the bounded wait used by every tensor-core kernel: one thread
// waits on an mbarrier that nothing will ever complete, with a limit of wait_ns
// instead of the production 2 s, and records GAME_ERR_TIMEOUT in the state.
__global__ void timeout_selftest_kernel(DevState* st, unsigned long long wait_ns, int* out) {
  __shared__ uint64_t bar;
  __shared__ int err;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  err = 0;
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  const unsigned long long t0 = globaltimer();
  bool done = false;
  while (!(done = mbar_try_wait(&bar, 0)) && globaltimer() - t0 < wait_ns) {
  }
  if (!done) {
    err = 1;
    atomicExch(&st->status, (int)GAME_ERR_TIMEOUT);
  }
  out[0] = done ? 0 : 1;
  out[1] = (int)((globaltimer() - t0) / 1000ull);   // microseconds waited
  // complete the phase so that the barrier is left consistent
  mbar_arrive(&bar);
}

cudaError_t tc_timeout_selftest(DevState* st, unsigned long long wait_ns, int* out,
                                cudaStream_t s) {
  timeout_selftest_kernel<<<1, 32, 0, s>>>(st, wait_ns, out);
  return cudaGetLastError();
}

cudaError_t tc_init_attributes() {
  cudaError_t en = tc_narrow_init_attributes();
  if (en != cudaSuccess) return en;
  for (int bn : {128, 256})
    for (int prec : {GAME_FP32, GAME_BF16, GAME_FP8})
      for (bool fast : {false, true})
        for (int na : {1, 2})
          for (int sp : {1, 2})
            for (bool pair : {false, true}) {
              void* k = pick_kernel(bn, prec, fast, na, sp, pair);
              if (!k) continue;
              cudaError_t e =
                  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemMax);
              if (e != cudaSuccess) return e;
            }
  return cudaSuccess;
}

bool tc_supported(const Shape& s) {
  if (!encode_fn()) return false;
  const int a_bytes = s.gene_planes * kblocks_of(s) * kTileA;
  // at least two B stages of 128 rows next to the resident gene planes
  return a_bytes + 2 * 128 * 128 + kSmemMisc <= kSmemMax;
}

// Gene rows held per A tile: a single slice (at most 128 chromosomes) of a single CTA
// keeps only its live rows, rounded up to a whole 8-row group (the elites' FP32
// re-score: 16 of 128), which frees shared memory for a deeper pattern-tile ring.
static int a_rows_of(const Shape& s, bool pair, int sp) {
  if (pair || sp != 1 || s.pop_pad != 128) return 128;
  const int r = (s.pop + 7) / 8 * 8;
  return r < 8 ? 8 : r;
}

// Deepest pattern-tile ring next to the resident gene planes; rows = pattern rows a CTA
// stages per tile (BN, or BN / 2 for a CTA of a pair), kg = k-blocks per stage.
static int max_stages(const Shape& s, int rows, int sp, int kg = 1, int a_rows = 128) {
  const int room = kSmemMax - kSmemMisc - sp * s.gene_planes * kblocks_of(s) * a_rows * 128;
  int st = room / (kg * rows * 128);
  return st > 8 ? 8 : st;
}

// Grouped k-blocks: whole k-blocks per row (the 3-D view) and more than one of them.
static bool kg_ok(const Shape& s, int kg) {
  const int kkb = s.precision == GAME_FP8 ? 128 : 64;
  return kg == 1 || (kg == 2 && s.kp % kkb == 0 && kblocks_of(s) >= 2);
}

// CTA pairs: 256-pattern tiles, one slice per CTA, an even number of slices.
static bool pair_ok(const Shape& s) { return (s.pop_pad / 128) % 2 == 0; }

void tc_candidates(const Shape& s, std::vector<TileReq>* out) {
  if (tc_narrow_shape(s)) {
    tc_narrow_candidates(s, out);
    return;
  }
  const int n_slices = s.pop_pad / 128;
  for (int sp : {1, 2})
    for (int bn : {256, 128}) {
      if (sp == 2 && (bn != 128 || n_slices % 2 != 0)) continue;
      const int ar = a_rows_of(s, false, sp);
      const int ms = max_stages(s, bn, sp, 1, ar);
      for (int st = ms; st >= 2 && st >= ms - 1; --st)
        for (int pf : {1, 0}) out->push_back(TileReq{bn, st, 1, pf, sp, 1});
      if (kg_ok(s, 2)) {
        const int ms2 = max_stages(s, bn, sp, 2, ar);
        for (int st = ms2; st >= 2 && st >= ms2 - 2; --st) out->push_back(TileReq{bn, st, 1, 0, sp, 2});
      }
    }
  if (pair_ok(s)) {
    const int ms = max_stages(s, 128, 1);
    for (int st = ms; st >= 2 && st >= ms - 2; --st)
      for (int pf : {1, 0}) out->push_back(TileReq{256, st, 2, pf, 1, 1});
    if (kg_ok(s, 2))
      for (int st = max_stages(s, 128, 1, 2); st >= 2; --st)
        out->push_back(TileReq{256, st, 2, 0, 1, 2});
  }
}

cudaError_t tc_plan(const Shape& s, const ExpDev& e, const PopDev& p, int n_sm, TcPlan* plan,
                    TileReq req) {
  if (tc_narrow_shape(s)) return tc_narrow_plan(s, e, p, n_sm, plan, req);
  // Default cluster for the FP32 form: CTA pairs with two k-blocks per request where
  // nothing else is asked for and they fit (700k x 256 columns, pop 1024: single CTAs
  // 0.739 ms, pairs 0.642 ms); single CTAs when the pair plan cannot be made.
  if (req.cluster == 0 && s.precision == GAME_FP32 && pair_ok(s) && kg_ok(s, 2) &&
      (!req.n || req.n == 256) && (!req.sp || req.sp == 1) && (!req.kg || req.kg == 2)) {
    TileReq r2 = req;
    r2.cluster = 2;
    if (tc_plan(s, e, p, n_sm, plan, r2) == cudaSuccess) return cudaSuccess;
    cudaGetLastError();
    req.cluster = 1;
  }
  TcPlan& t = *plan;
  t.kblocks = kblocks_of(s);
  const int n_bplanes = s.precision == GAME_FP32 ? 2 : 1;
  t.n_slices = s.pop_pad / 128;
  // cluster 2: CTA pairs (cta_group::2), each CTA one slice, 256-pattern tiles
  if (req.cluster < 0 || req.cluster > 2) return cudaErrorInvalidValue;
  t.cluster = req.cluster == 2 ? 2 : 1;
  const bool pair = t.cluster == 2;
  if (pair && (!pair_ok(s) || (req.sp && req.sp != 1) || (req.n && req.n != 256)))
    return cudaErrorInvalidValue;
  t.sp = req.sp ? req.sp : 1;
  if (t.sp != 1 && t.sp != 2) return cudaErrorInvalidValue;
  if (t.sp == 2 && (t.n_slices % 2 != 0 || (req.n && req.n != 128))) return cudaErrorInvalidValue;
  // groups: units of work sharing the pattern tiles (a CTA's slices, or a pair's two)
  t.n_groups = pair ? t.n_slices / 2 : t.n_slices / t.sp;
  t.a_rows = a_rows_of(s, pair, t.sp);
  const int a_bytes = t.sp * s.gene_planes * t.kblocks * t.a_rows * 128;
  // Default shape: 256-pattern tiles when two stages fit, else 128
  // (128-pattern tiles cost as much per MMA instruction as 256-pattern ones).
  t.bn = pair ? 256 : t.sp == 2 ? 128
                               : (req.n ? req.n : (max_stages(s, 256, 1, 1, t.a_rows) >= 2 ? 256 : 128));
  if (t.bn != 128 && t.bn != 256) return cudaErrorInvalidValue;
  const int rows = pair ? t.bn / 2 : t.bn;          // pattern rows a CTA stages per tile
  // Default k-grouping: two k-blocks per request wherever two such stages fit (at 700k x
  // 256 columns, pop 1024: BF16 0.350 -> 0.274 ms, FP8 0.227 -> 0.213 ms, FP32 pairs
  // 0.778 -> 0.642 ms); the FP32 form's two gene planes leave room for one only at
  // 256-pattern tiles of single CTAs.
  t.kg = req.kg;
  if (!t.kg) {
    t.kg = 1;
    if (kg_ok(s, 2)) {
      const int ms2 = max_stages(s, rows, t.sp, 2, t.a_rows);
      if (ms2 >= 2 && (!req.stages || req.stages <= ms2)) t.kg = 2;
    }
  }
  if (!kg_ok(s, t.kg)) return cudaErrorInvalidValue;
  const int ms = max_stages(s, rows, t.sp, t.kg, t.a_rows);
  t.stages = req.stages ? req.stages : ms;
  if (t.stages < 2 || t.stages > ms) return cudaErrorNotSupported;
  // the prefetch addresses 2-D boxes; grouped stages go without it
  t.prefetch = req.prefetch == 0 || t.kg > 1 ? 0 : 1;
  t.n_tiles = (int)((s.n_train + t.bn - 1) / t.bn);
  t.smem = (size_t)a_bytes + (size_t)t.stages * t.kg * rows * 128 + kSmemMisc;
  // Co-resident work units: one CTA per SM (its shared memory fills the SM); pairs must
  // also find two SMs of one GPC, which the occupancy query counts.
  int resident = n_sm;
  if (pair) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = 2;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.gridDim = dim3(2 * n_sm);      // large enough not to cap the count
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = t.smem;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    int n_clusters = 0;
    const cudaError_t oe = cudaOccupancyMaxActiveClusters(
        &n_clusters, pick_kernel(t.bn, s.precision, true, s.gene_planes, 1, true), &cfg);
    if (oe != cudaSuccess || n_clusters < 1) {
      cudaGetLastError();
      return cudaErrorNotSupported;
    }
    resident = n_clusters;                           // pairs
  }
  int cps = resident / t.n_groups;
  if (cps < 1) cps = 1;
  if (cps > t.n_tiles) cps = t.n_tiles;
  t.ctas_per_slice = cps;
  t.grid = t.n_groups * cps * (pair ? 2 : 1);
  t.n_part = cps;
  cudaError_t err;
  if ((err = make_map(&t.a_map[0], p.ghi, s.precision, s.pop_pad, s.kp, t.a_rows)) != cudaSuccess) return err;
  if ((err = make_map(&t.a_map[1], p.glo, s.precision, s.pop_pad, s.kp, t.a_rows)) != cudaSuccess) return err;
  auto bmap = [&](CUtensorMap* m, const void* base) {
    return t.kg == 1 ? make_map(m, base, s.precision, s.n_train, s.kp, rows)
                     : make_map3(m, base, s.precision, s.n_train, s.kp, rows, t.kg);
  };
  if ((err = bmap(&t.b_map[0], e.p0)) != cudaSuccess) return err;
  if (n_bplanes == 2) {
    if ((err = bmap(&t.b_map[1], e.p1)) != cudaSuccess) return err;
  } else {
    t.b_map[1] = t.b_map[0];
  }
  return cudaSuccess;
}

cudaError_t tc_launch(const TcPlan& t, const Shape& s, const Fitness& f, const PopDev& pd,
                      const ExpDev& e, double* partial, const DevState* state, cudaStream_t st) {
  if (t.narrow) return tc_narrow_launch(t, s, f, pd, e, partial, state, st);
  TcParams p;
  p.a[0] = t.a_map[0];
  p.a[1] = t.a_map[1];
  p.b[0] = t.b_map[0];
  p.b[1] = t.b_map[1];
  p.t = e.t;
  p.tcoef = e.tcoef;
  p.bias = pd.bias;
  p.rscale = pd.rscale;
  p.partial = partial;
  p.state = const_cast<DevState*>(state);
  p.m = s.n_train;
  p.n_groups = t.n_groups;
  p.cps = t.ctas_per_slice;
  p.n_tiles = t.n_tiles;
  p.kblocks = t.kblocks;
  p.kp = s.kp;
  p.stages = t.stages;
  p.pop_pad = s.pop_pad;
  p.n_bplanes = s.precision == GAME_FP32 ? 2 : 1;
  p.act = f.activation;
  p.err = f.error;
  p.R = f.tmse_R;
  p.in_evolve = state != nullptr;
  p.prefetch = t.prefetch;
  p.kg = t.kg;
  p.a_rows = t.a_rows;
  const bool fast = f.pm1_targets && f.activation == GAME_TANH &&
                    (f.error == GAME_RMSE || f.error == GAME_MSE);
  const bool pair = t.cluster == 2;
  void* k = pick_kernel(t.bn, s.precision, fast, s.gene_planes, t.sp, pair);
  if (!k) return cudaErrorNotSupported;
  void* args[] = {&p};
  if (!pair) return cudaLaunchKernel(k, dim3(t.grid), dim3(kThreads), args, t.smem, st);
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeClusterDimension;
  attr.val.clusterDim.x = 2;
  attr.val.clusterDim.y = 1;
  attr.val.clusterDim.z = 1;
  cfg.gridDim = dim3(t.grid);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = t.smem;
  cfg.stream = st;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, k, args);
}

#ifdef GAME_TC_TIMELINE
// Copies the 2048 stamps to host memory (profiling build only).
extern "C" int game_tc_timeline(long long* host) {
  return (int)cudaMemcpyFromSymbol(host, g_tc_timeline, sizeof(long long) * 2048);
}
// Zeroes the stamps, so that a read after one launch shows that launch alone.
extern "C" int game_tc_timeline_clear() {
  static const long long zeros[2048] = {};
  return (int)cudaMemcpyToSymbol(g_tc_timeline, zeros, sizeof(zeros));
}
#endif

GAME_DEFINE_CHECK_READER(check_word_tc)

}  // namespace game
