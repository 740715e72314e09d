// Tensor-core fitness of a narrow population (at most 32 chromosomes, FP32
// form) on sm_103a: the operands of the main kernel swapped, patterns on the
// MMA's M side.
//
// What it computes is the same as the main tensor-core kernel (paper Section 2:
// Out = a_0 + sum_g G[c,g] P[k,g], eq.2; E = (t_k - act(Out))^2, eq.3, or the
// threshold form, eq.10; per-chromosome sums over the training rows, eq.4 /
// eq.5).  The paper's own runs use 2N + 1 = 23 chromosomes (Section 5): in a
// tile of 128 chromosomes on M, 105 of 128 TMEM lanes would carry padding and
// one warp quadrant would do all the epilogue work.  Here
//   D[k, c] = sum_g P[k, g] G[c, g],  M = 128 patterns, N = 32 chromosomes,
// so every lane of the accumulator is a real pattern and each epilogue thread
// owns one pattern and all chromosomes.
//
// FP32 split as in the main kernel: P = P_hi + P_lo and G = G_hi + G_lo as fp16
// pairs, D accumulates P_hi G_hi + P_lo G_hi + P_hi G_lo (kind::f16, float32 in
// TMEM).  The gene planes (32 rows) stay in shared memory; pattern tiles of 128
// rows stream through a ring of stages, one (k-block, plane) per stage.  A row of
// P takes SWA bytes of shared memory: 32 or 64 when the whole stored row fits
// (16 or 32 columns, 32- / 64-byte swizzle, one stage per tile and plane), else
// 128-byte k-blocks.  With short rows a 128-byte k-block would be mostly zero
// fill, and the ring would carry a quarter of the data it could.
//
// Roles (448 threads): warp 0 TMA producer, warp 1 TMEM allocator + MMA issuer,
// warps 2..13 epilogue in three sets of four (set s takes the tiles i = s mod 3;
// tile i sits in TMEM accumulator i mod 4, so the MMAs run up to three tiles ahead
// of the epilogue; warp w reads lanes 32 (w % 4)).  Each epilogue thread adds its
// pattern's error per chromosome in float32 over blocks of 32 tiles; a butterfly
// over the warp then gives lane c the block total of chromosome c, added in
// float64.  Every mbarrier wait is bounded (2 s); on a timeout the CTA records
// GAME_ERR_TIMEOUT, drains its copies and MMAs (bounded), frees TMEM and exits.
#include "fitness_tc.h"
#include "tc_ptx.cuh"

#include <cudaTypedefs.h>

namespace game {

namespace {

using namespace tc;

constexpr int kNSets = 3;                        // epilogue sets of four warps
constexpr int kNThreads = 64 + 32 * 4 * kNSets;
constexpr int kNPop = 32;                        // chromosomes per launch (MMA N)
constexpr int kNTileG = kNPop * 128;             // one 32-row x 128-byte gene block
constexpr int kNMaxKblocks = 12;
constexpr int kNMaxStages = 32;
constexpr int kNBuf = 8;                         // TMEM accumulators (32 columns each)
constexpr int kNR = 2;                           // 128-pattern tiles per stage (one 256-row box)
constexpr int kNSmemMax = 232448;
constexpr int kNGuard = 1024;                    // after the ring, before the barriers
// alignment, guard, barriers + TMEM slot + last parities, per-warp totals
constexpr int kNSmemMisc = 1024 + kNGuard + 1024 + 4 * kNSets * 32 * 8 + 2 * kNPop * 4;

// Shared-memory matrix descriptor for K-major rows of SW = 32, 64 or 128 bytes:
// that swizzle, 8-row groups 8 * SW bytes apart, descriptor version 1.
template <int SW>
__device__ __forceinline__ uint64_t swz_desc(uint32_t saddr) {
  static_assert(SW == 32 || SW == 64 || SW == 128, "swizzle span");
  constexpr uint64_t kLayout = SW == 128 ? 2 : SW == 64 ? 4 : 6;
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)((8 * SW) >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= kLayout << 61;
  return d;
}

struct NarrowParams {
  CUtensorMap a[2];       // expansion planes P_hi, P_lo (M operand, patterns x genes)
  CUtensorMap g[2];       // gene planes G_hi, G_lo (N operand, chromosomes x genes)
  const float* pk;        // 2 log2(e) t_k (fused +-1 / tanh form) or t_k
  const float* bias;
  const float* rscale;    // per-chromosome scale of the gene planes (a power of two)
  double* partial;
  DevState* state;
  long long m;
  int pop, pop_pad, n_tiles, per_cta, kblocks, ksteps, stages, act, err, in_evolve;
  float R;
};

// Error forms, fixed per launch so that the per-chromosome loop has no branches.
enum : int { kEfFast = 0, kEfMse = 1, kEfTmse = 2, kEfTmseSq = 3, kEfGeneral = 4 };

// E for one (pattern, chromosome): pk = 2 log2(e) t_k for kEfFast (then E / 4, see
// chunk_error), t_k otherwise; linear Out for kEfMse / kEfTmse / kEfTmseSq.
template <int EF>
__device__ __forceinline__ float narrow_tc_error(float pk, float s, int act, int err, float R) {
  if (EF == kEfFast) {
    const float r = rcp_approx(1.0f + ex2_approx(pk * s));
    return r * r;
  }
  if (EF == kEfGeneral) return general_error(pk, s, act, err, R);
  const float d = pk - s;
  const float e = d * d;
  if (EF == kEfTmse) return fabsf(d) > R ? e : 0.0f;
  if (EF == kEfTmseSq) return e > R ? e : 0.0f;
  return e;
}

template <int EF, int SWA>
__global__ void __launch_bounds__(kNThreads, 1) fitness_tc_narrow_kernel(const __grid_constant__ NarrowParams p) {
  if (p.in_evolve && p.state->stopped) return;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~(uintptr_t)1023);
  constexpr uint32_t kIdesc = make_idesc(128, kNPop, 0u);   // fp16 x fp16 -> f32
  constexpr int kTileA = 128 * SWA;                         // one 128-pattern tile
  constexpr int kStageA = kNR * kTileA;                     // one stage: kNR tiles
  constexpr int kStepsA = SWA / 32;                         // 16-element K steps per A row block
  const int a_blocks = (p.ksteps + kStepsA - 1) / kStepsA;  // A k-blocks per tile
  const int S = p.stages;
  uint8_t* sG = smem;                                      // [plane][kb] 4 KB blocks
  uint8_t* sA = sG + 2 * p.kblocks * kNTileG;              // [stage] kStageA
  uint64_t* bars = reinterpret_cast<uint64_t*>(sA + S * kStageA + kNGuard);
  uint64_t* g_full = bars;
  uint64_t* a_full = bars + 1;
  uint64_t* a_empty = a_full + S;
  uint64_t* acc_full = a_empty + S;
  uint64_t* acc_empty = acc_full + kNBuf;
  uint64_t* fin = acc_empty + kNBuf;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(fin + 1);
  volatile int* err = reinterpret_cast<volatile int*>(tmem_slot + 1);
  int* last_par = reinterpret_cast<int*>(tmem_slot + 2);   // [S]
  double* red = reinterpret_cast<double*>(last_par + kNMaxStages);  // [epilogue warps][32]
  float* bsm = reinterpret_cast<float*>(red + 4 * kNSets * 32);     // [32] gene 0 per chromosome
  float* rsm = bsm + kNPop;                                           // [32] plane scale per chromosome

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // This CTA's tiles are t0 .. t0 + my_tiles - 1 (contiguous, per_cta a multiple of kNR),
  // loaded and multiplied kNR at a time; a group past the last tile reads zero fill.
  const int t0 = (int)blockIdx.x * p.per_cta;
  const int my_tiles = max(0, min(p.per_cta, p.n_tiles - t0));
  const int my_groups = (my_tiles + kNR - 1) / kNR;

  if (threadIdx.x == 0) {
    mbar_init(g_full, 1);
    for (int s = 0; s < S; ++s) {
      mbar_init(a_full + s, 1);
      mbar_init(a_empty + s, 1);
      last_par[s] = -1;
    }
    for (int b = 0; b < kNBuf; ++b) {
      mbar_init(acc_full + b, 1);
      mbar_init(acc_empty + b, 4);   // the four warps of the set that reads the buffer
    }
    mbar_init(fin, 1);
    *err = 0;
    for (int c = 0; c < kNPop; ++c) {
      bsm[c] = c < p.pop ? p.bias[c] : 0.0f;
      rsm[c] = c < p.pop ? p.rscale[c] : 1.0f;
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"((uint32_t)(kNBuf * kNPop)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ---- TMA producer ----
    if (lane == 0) {
      mbar_expect_tx(g_full, (uint32_t)(2 * p.kblocks * kNTileG));
      for (int pl = 0; pl < 2; ++pl)
        for (int kb = 0; kb < p.kblocks; ++kb)
          tma_load_2d(sG + (pl * p.kblocks + kb) * kNTileG, &p.g[pl], kb * 64, 0, g_full);
    }
    int stage = 0;
    uint32_t phase = 0;
    bool ok = true;
    for (int gi = 0; gi < my_groups && ok; ++gi) {
      const int row0 = (t0 + gi * kNR) * 128;
      for (int kb = 0; kb < a_blocks && ok; ++kb)
        for (int pl = 0; pl < 2; ++pl) {
          if (!warp_wait(a_empty + stage, phase ^ 1u, err, p.state, lane)) {
            ok = false;
            break;
          }
          if (lane == 0) {
            mbar_expect_tx(a_full + stage, kStageA);
            tma_load_2d(sA + stage * kStageA, &p.a[pl], kb * (SWA / 2), row0, a_full + stage);
            last_par[stage] = (int)phase;
          }
          if (++stage == S) {
            stage = 0;
            phase ^= 1u;
          }
        }
    }
    // Drain: every issued copy has landed before the CTA may exit.
    if (lane == 0) {
      mbar_wait(g_full, 0, err, p.state);
      for (int s2 = 0; s2 < S; ++s2)
        if (last_par[s2] >= 0) {
          const unsigned long long w0 = globaltimer();
          while (!mbar_try_wait(a_full + s2, (uint32_t)last_par[s2]) && globaltimer() - w0 < kWaitNs) {
          }
        }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---- MMA issuer (warp-uniform loop, lane 0 issues) ----
    if (warp_wait(g_full, 0, err, p.state, lane)) {
      fence_after();
      int stage = 0;
      uint32_t phase = 0;
      const uint32_t a_addr = smem_u32(sA);
      const uint32_t g_addr = smem_u32(sG);
      bool ok = true;
      for (int gi = 0; gi < my_groups && ok; ++gi) {
        // the group's accumulators must be free before its first stage is multiplied
        for (int r = 0; r < kNR && ok; ++r) {
          const int it = gi * kNR + r;
          ok = warp_wait(acc_empty + (it & (kNBuf - 1)), (uint32_t)((it / kNBuf) & 1) ^ 1u, err,
                         p.state, lane);
        }
        if (!ok) break;
        fence_after();
        uint32_t accum = 0;
        for (int kb = 0; kb < a_blocks && ok; ++kb) {
          const int steps = min(kStepsA, p.ksteps - kb * kStepsA);
          for (int pl = 0; pl < 2; ++pl) {
            if (!warp_wait(a_full + stage, phase, err, p.state, lane)) {
              ok = false;
              break;
            }
            fence_after();
            // P_hi meets G_hi and G_lo; P_lo meets G_hi
            const int n_g = pl == 0 ? 2 : 1;
#pragma unroll
            for (int r = 0; r < kNR; ++r) {
              const uint32_t d = tmem + (uint32_t)(((gi * kNR + r) & (kNBuf - 1)) * kNPop);
              const uint64_t adesc =
                  swz_desc<SWA>(a_addr + (uint32_t)(stage * kStageA + r * kTileA));
              uint32_t acc_r = accum;
              for (int g = 0; g < n_g; ++g) {
#pragma unroll
                for (int k = 0; k < kStepsA; ++k) {
                  if (k < steps) {
                    // K step ks of the row: gene block ks / 4, +32 bytes per step inside
                    // a swizzled row = +2 in the address field (on both sides)
                    const int ks = kb * kStepsA + k;
                    const uint64_t gdesc = swz_desc<128>(
                        g_addr + (uint32_t)((g * p.kblocks + (ks >> 2)) * kNTileG));
                    if (lane == 0)
                      mma<GAME_FP32>(d, adesc + 2 * k, gdesc + 2 * (ks & 3), kIdesc, acc_r);
                    acc_r = 1;
                  }
                }
              }
              if (r == kNR - 1) accum = acc_r;
            }
            if (lane == 0) mma_commit(a_empty + stage);
            if (++stage == S) {
              stage = 0;
              phase ^= 1u;
            }
          }
        }
        if (!ok) break;
        if (lane == 0)
          for (int r = 0; r < kNR; ++r) mma_commit(acc_full + ((gi * kNR + r) & (kNBuf - 1)));
      }
    }
    // Drain: all issued MMAs complete before TMEM is released.
    if (lane == 0) {
      mma_commit(fin);
      const unsigned long long w0 = globaltimer();
      while (!mbar_try_wait(fin, 0) && globaltimer() - w0 < kWaitNs) {
      }
    }
    __syncwarp();
  } else {
    // ---- epilogue: thread = one pattern of the tile, all chromosomes ----
    const int ew = warp - 2;
    const int set = ew >> 2;               // tiles it = set (mod kNSets)
    const int q = warp & 3;                // TMEM lane quadrant

    float acc[kNPop];
#pragma unroll
    for (int c = 0; c < kNPop; ++c) acc[c] = 0.0f;
    double tot = 0.0;
    int nblk = 0;
    const uint32_t tlane = tmem + ((uint32_t)(q * 32) << 16);
    // This thread's pattern in the set's tiles it = set, set + kNSets, ...: k advances
    // by kNSets * 128 per tile.  Its target is loaded two tiles ahead (a DRAM miss: the
    // pattern stream evicts the targets from L2); the target arrays are padded past the
    // last tile.
    const long long kstep = (long long)kNSets * 128;
    long long k = (long long)(t0 + set) * 128 + q * 32 + lane;
    float pk0 = set < my_tiles ? p.pk[k] : 0.0f;
    float pk1 = set + kNSets < my_tiles ? p.pk[k + kstep] : 0.0f;
    for (int it = set; it < my_tiles; it += kNSets, k += kstep) {
      const int buf = it & (kNBuf - 1);
      const uint32_t ap = (uint32_t)((it / kNBuf) & 1);
      const float pk = pk0;
      pk0 = pk1;
      pk1 = it + 2 * kNSets < my_tiles ? p.pk[k + 2 * kstep] : 0.0f;
      if (!warp_wait(acc_full + buf, ap, err, p.state, lane)) break;
      fence_after();
      float v[kNPop];
      tmem_ld32(tlane + (uint32_t)(buf * kNPop), v);
      // the accumulator is in registers: hand the buffer back to the MMA warp
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acc_empty + buf);
      const bool valid = k < p.m;
      // all 32 columns, without branches: columns past the population are never read
#pragma unroll
      for (int c = 0; c < kNPop; ++c) {
        const float e = narrow_tc_error<EF>(pk, fmaf(v[c], rsm[c], bsm[c]), p.act, p.err, p.R);
        acc[c] += valid ? e : 0.0f;
      }
      if (++nblk == 32) {
        tot += (double)warp_column_sums32(acc, lane);
        nblk = 0;
      }
    }
    tot += (double)warp_column_sums32(acc, lane);
    red[ew * 32 + lane] = EF == kEfFast ? 4.0 * tot : tot;
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)(kNBuf * kNPop)));
  if (threadIdx.x < kNPop) {
    double sum = 0.0;
#pragma unroll
    for (int w = 0; w < 4 * kNSets; ++w) sum += red[w * 32 + threadIdx.x];
    p.partial[(long long)blockIdx.x * p.pop_pad + threadIdx.x] = sum;
  }
}

template <int SWA>
void* narrow_kernel_sw(int ef) {
  switch (ef) {
    case kEfFast: return reinterpret_cast<void*>(&fitness_tc_narrow_kernel<kEfFast, SWA>);
    case kEfMse: return reinterpret_cast<void*>(&fitness_tc_narrow_kernel<kEfMse, SWA>);
    case kEfTmse: return reinterpret_cast<void*>(&fitness_tc_narrow_kernel<kEfTmse, SWA>);
    case kEfTmseSq: return reinterpret_cast<void*>(&fitness_tc_narrow_kernel<kEfTmseSq, SWA>);
    default: return reinterpret_cast<void*>(&fitness_tc_narrow_kernel<kEfGeneral, SWA>);
  }
}

void* narrow_kernel(int ef, int swa) {
  return swa == 32 ? narrow_kernel_sw<32>(ef) : swa == 64 ? narrow_kernel_sw<64>(ef)
                                                          : narrow_kernel_sw<128>(ef);
}

int narrow_kblocks(const Shape& s) { return (s.kp + 63) / 64; }

// Tiles per CTA over `ctas` CTAs, rounded up to whole stages of kNR tiles.  For the
// grid this gives, every CTA gets at least one tile and the ranges cover all.
int narrow_per_cta(int n_tiles, int ctas) {
  const int per = (n_tiles + ctas - 1) / ctas;
  return (per + kNR - 1) / kNR * kNR;
}

// Bytes of shared memory per stored row of P: the whole row when it is 32 or 64 bytes.
int narrow_swa(const Shape& s) { return s.kp * 2 <= 32 ? 32 : s.kp * 2 <= 64 ? 64 : 128; }

size_t narrow_smem(const Shape& s, int stages) {
  return (size_t)2 * narrow_kblocks(s) * kNTileG + (size_t)stages * kNR * 128 * narrow_swa(s) +
         kNSmemMisc;
}

int narrow_max_stages(const Shape& s) {
  const long long room = kNSmemMax - kNSmemMisc - 2LL * narrow_kblocks(s) * kNTileG;
  const long long st = room / ((long long)kNR * 128 * narrow_swa(s));
  // 128-byte rows: up to 6 stages of 32 KB; shorter rows: up to 32 stages
  const long long cap = narrow_swa(s) == 128 ? 10 : 32;
  return (int)(st > cap ? cap : st);
}

cudaError_t narrow_map(CUtensorMap* m, const void* base, long long rows, int cols, int swa) {
  if (swa == 128) return tc_make_map(m, base, GAME_FP32, rows, cols, 128 * kNR);
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void* ptr = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return cudaErrorNotSupported;
    fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
  }
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
  cuuint32_t box[2] = {(cuuint32_t)(swa / 2), (cuuint32_t)(128 * kNR)};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void*>(base), dims, strides,
                  box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  swa == 32 ? CU_TENSOR_MAP_SWIZZLE_32B : CU_TENSOR_MAP_SWIZZLE_64B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace

bool tc_narrow_fits(const Shape& s) {
  return s.precision == GAME_FP32 && s.pop >= 1 && s.pop <= kNPop && s.kp % 16 == 0 &&
         narrow_kblocks(s) <= kNMaxKblocks && narrow_max_stages(s) >= 2;
}

bool tc_narrow_shape(const Shape& s) { return s.tc_narrow && tc_narrow_fits(s); }

void tc_narrow_candidates(const Shape& s, std::vector<TileReq>* out) {
  const int ms = narrow_max_stages(s);
  for (int st : {ms, 16, 6, 4})
    if (st >= 2 && st <= ms) {
      bool dup = false;
      for (const TileReq& r : *out) dup |= r.stages == st;
      if (!dup) out->push_back(TileReq{128, st, 1, 0, 1});
    }
}

cudaError_t tc_narrow_plan(const Shape& s, const ExpDev& e, const PopDev& p, int n_sm,
                           TcPlan* plan, TileReq req) {
  TcPlan& t = *plan;
  if (!tc_narrow_shape(s)) return cudaErrorInvalidValue;
  if ((req.n && req.n != 128) || req.cluster > 1 || req.sp > 1) return cudaErrorInvalidValue;
  t.narrow = 1;
  t.bn = 128;
  t.sp = 1;
  t.cluster = 1;
  t.prefetch = 0;
  t.kblocks = narrow_kblocks(s);
  const int ms = narrow_max_stages(s);
  const int dflt = narrow_swa(s) == 128 ? 6 : 16;
  t.stages = req.stages ? req.stages : (ms < dflt ? ms : dflt);
  if (t.stages < 2 || t.stages > ms) return cudaErrorNotSupported;
  t.n_slices = 1;
  t.n_groups = 1;
  t.n_tiles = (int)((s.n_train + 127) / 128);
  // contiguous tile ranges, a multiple of kNR tiles each, over at most one CTA per SM
  t.grid = (t.n_tiles + narrow_per_cta(t.n_tiles, n_sm) - 1) / narrow_per_cta(t.n_tiles, n_sm);
  t.ctas_per_slice = t.grid;
  t.n_part = t.grid;
  t.smem = narrow_smem(s, t.stages);
  cudaError_t err;
  const int swa = narrow_swa(s);
  if ((err = narrow_map(&t.b_map[0], e.p0, s.n_train, s.kp, swa)) != cudaSuccess) return err;
  if ((err = narrow_map(&t.b_map[1], e.p1, s.n_train, s.kp, swa)) != cudaSuccess) return err;
  if ((err = tc_make_map(&t.a_map[0], p.ghi, GAME_FP32, s.pop_pad, s.kp, kNPop)) != cudaSuccess) return err;
  if ((err = tc_make_map(&t.a_map[1], p.glo, GAME_FP32, s.pop_pad, s.kp, kNPop)) != cudaSuccess) return err;
  return cudaSuccess;
}

cudaError_t tc_narrow_launch(const TcPlan& t, const Shape& s, const Fitness& f, const PopDev& pd,
                             const ExpDev& e, double* partial, const DevState* state,
                             cudaStream_t st) {
  NarrowParams p;
  p.a[0] = t.b_map[0];   // patterns: the expansion planes
  p.a[1] = t.b_map[1];
  p.g[0] = t.a_map[0];   // chromosomes: the gene planes
  p.g[1] = t.a_map[1];
  const bool fast = f.pm1_targets && f.activation == GAME_TANH &&
                    (f.error == GAME_RMSE || f.error == GAME_MSE);
  p.pk = fast ? e.tcoef : e.t;
  p.bias = pd.bias;
  p.rscale = pd.rscale;
  p.partial = partial;
  p.state = const_cast<DevState*>(state);
  p.m = s.n_train;
  p.pop = s.pop;
  p.pop_pad = s.pop_pad;
  p.n_tiles = t.n_tiles;
  p.per_cta = narrow_per_cta(t.n_tiles, t.grid);
  p.kblocks = t.kblocks;
  p.ksteps = s.kp / 16;
  p.stages = t.stages;
  p.act = f.activation;
  p.err = f.error;
  p.R = f.tmse_R;
  p.in_evolve = state != nullptr;
  int ef = kEfGeneral;
  if (fast)
    ef = kEfFast;
  else if (f.activation == GAME_LINEAR)
    ef = f.error == GAME_TMSE ? kEfTmse : f.error == GAME_TMSE_SQ ? kEfTmseSq : kEfMse;
  void* args[] = {&p};
  return cudaLaunchKernel(narrow_kernel(ef, narrow_swa(s)), dim3(t.grid), dim3(kNThreads), args,
                          t.smem, st);
}

cudaError_t tc_narrow_init_attributes() {
  for (int swa : {32, 64, 128})
    for (int ef = kEfFast; ef <= kEfGeneral; ++ef) {
      cudaError_t e = cudaFuncSetAttribute(narrow_kernel(ef, swa),
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, kNSmemMax);
      if (e != cudaSuccess) return e;
    }
  return cudaSuccess;
}

}  // namespace game
