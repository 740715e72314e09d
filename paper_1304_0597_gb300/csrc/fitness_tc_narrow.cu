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
// rows stream through a ring of stages, one (k-block, plane) per stage.
//
// Roles (320 threads): warp 0 TMA producer, warp 1 TMEM allocator + MMA issuer,
// warps 2..9 epilogue in two sets of four (set s takes the tiles of parity s and
// TMEM buffer s; warp w reads lanes 32 (w % 4)).  Each epilogue thread adds its
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

constexpr int kNThreads = 64 + 32 * 8;
constexpr int kNPop = 32;                        // chromosomes per launch (MMA N)
constexpr int kNTileA = 128 * 128;               // one 128-pattern x 128-byte stage
constexpr int kNTileG = kNPop * 128;             // one 32-row x 128-byte gene block
constexpr int kNMaxKblocks = 12;
constexpr int kNSmemMax = 232448;
constexpr int kNSmemMisc = 1024 + 512 + 8 * 32 * 8;   // alignment, barriers, warp totals

struct NarrowParams {
  CUtensorMap a[2];       // expansion planes P_hi, P_lo (M operand, patterns x genes)
  CUtensorMap g[2];       // gene planes G_hi, G_lo (N operand, chromosomes x genes)
  const float* pk;        // 2 log2(e) t_k (fused +-1 / tanh form) or t_k
  const float* bias;
  double* partial;
  DevState* state;
  long long m;
  int pop, pop_pad, n_tiles, kblocks, ksteps, stages, act, err, in_evolve;
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

template <int EF>
__global__ void __launch_bounds__(kNThreads, 1) fitness_tc_narrow_kernel(const __grid_constant__ NarrowParams p) {
  if (p.in_evolve && p.state->stopped) return;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~(uintptr_t)1023);
  constexpr uint32_t kIdesc = make_idesc(128, kNPop, 0u);   // fp16 x fp16 -> f32
  const int S = p.stages;
  uint8_t* sG = smem;                                      // [plane][kb] 4 KB blocks
  uint8_t* sA = sG + 2 * p.kblocks * kNTileG;              // [stage] 16 KB
  uint64_t* bars = reinterpret_cast<uint64_t*>(sA + S * kNTileA);
  uint64_t* g_full = bars;
  uint64_t* a_full = bars + 1;
  uint64_t* a_empty = a_full + S;
  uint64_t* acc_full = a_empty + S;
  uint64_t* acc_empty = acc_full + 2;
  uint64_t* fin = acc_empty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(fin + 1);
  volatile int* err = reinterpret_cast<volatile int*>(tmem_slot + 1);
  int* last_par = reinterpret_cast<int*>(tmem_slot + 2);   // [S]
  double* red = reinterpret_cast<double*>(last_par + 16);  // [8][32]

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int my_tiles =
      (int)blockIdx.x < p.n_tiles ? (p.n_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

  if (threadIdx.x == 0) {
    mbar_init(g_full, 1);
    for (int s = 0; s < S; ++s) {
      mbar_init(a_full + s, 1);
      mbar_init(a_empty + s, 1);
      last_par[s] = -1;
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(acc_full + b, 1);
      mbar_init(acc_empty + b, 4);   // the four warps of the buffer's set
    }
    mbar_init(fin, 1);
    *err = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(2u * kNPop));
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
    for (int it = 0; it < my_tiles && ok; ++it) {
      const int row0 = ((int)blockIdx.x + it * (int)gridDim.x) * 128;
      for (int kb = 0; kb < p.kblocks && ok; ++kb)
        for (int pl = 0; pl < 2; ++pl) {
          if (!warp_wait(a_empty + stage, phase ^ 1u, err, p.state, lane)) {
            ok = false;
            break;
          }
          if (lane == 0) {
            mbar_expect_tx(a_full + stage, kNTileA);
            tma_load_2d(sA + stage * kNTileA, &p.a[pl], kb * 64, row0, a_full + stage);
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
          const unsigned long long t0 = globaltimer();
          while (!mbar_try_wait(a_full + s2, (uint32_t)last_par[s2]) && globaltimer() - t0 < kWaitNs) {
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
      for (int it = 0; it < my_tiles; ++it) {
        const int buf = it & 1;
        const uint32_t ap = (uint32_t)((it >> 1) & 1);
        if (!warp_wait(acc_empty + buf, ap ^ 1u, err, p.state, lane)) break;
        fence_after();
        const uint32_t d = tmem + (uint32_t)(buf * kNPop);
        uint32_t accum = 0;
        bool ok = true;
        for (int kb = 0; kb < p.kblocks && ok; ++kb) {
          const int steps = min(4, p.ksteps - kb * 4);
          for (int pl = 0; pl < 2; ++pl) {
            if (!warp_wait(a_full + stage, phase, err, p.state, lane)) {
              ok = false;
              break;
            }
            fence_after();
            const uint64_t adesc = sw128_desc(a_addr + (uint32_t)(stage * kNTileA));
            // P_hi meets G_hi and G_lo; P_lo meets G_hi
            const int n_g = pl == 0 ? 2 : 1;
            for (int gi = 0; gi < n_g; ++gi) {
              const uint64_t gdesc =
                  sw128_desc(g_addr + (uint32_t)((gi * p.kblocks + kb) * kNTileG));
#pragma unroll
              for (int k = 0; k < 4; ++k) {
                if (k < steps) {
                  // +32 bytes along K inside the 128-byte swizzle row = +2 in the address field
                  if (lane == 0) mma<GAME_FP32>(d, adesc + 2 * k, gdesc + 2 * k, kIdesc, accum);
                  accum = 1;
                }
              }
            }
            if (lane == 0) mma_commit(a_empty + stage);
            if (++stage == S) {
              stage = 0;
              phase ^= 1u;
            }
          }
        }
        if (!ok) break;
        if (lane == 0) mma_commit(acc_full + buf);
      }
    }
    // Drain: all issued MMAs complete before TMEM is released.
    if (lane == 0) {
      mma_commit(fin);
      const unsigned long long t0 = globaltimer();
      while (!mbar_try_wait(fin, 0) && globaltimer() - t0 < kWaitNs) {
      }
    }
    __syncwarp();
  } else {
    // ---- epilogue: thread = one pattern of the tile, all chromosomes ----
    const int ew = warp - 2;
    const int set = ew >> 2;               // tiles of parity `set`, TMEM buffer `set`
    const int q = warp & 3;                // TMEM lane quadrant
    float bias[kNPop];
#pragma unroll
    for (int c = 0; c < kNPop; ++c) bias[c] = c < p.pop ? p.bias[c] : 0.0f;
    float acc[kNPop];
#pragma unroll
    for (int c = 0; c < kNPop; ++c) acc[c] = 0.0f;
    double tot = 0.0;
    int nblk = 0;
    const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(set * kNPop);
    // This thread's pattern in the set's tiles it = set, set + 2, ...: k advances by
    // 2 * grid * 128 per tile.  Its target is loaded two tiles ahead (a DRAM miss:
    // the pattern stream evicts the targets from L2); the target arrays are padded
    // past the last tile.
    const long long kstep = 2LL * gridDim.x * 128;
    long long k = ((long long)blockIdx.x + (long long)set * gridDim.x) * 128 + q * 32 + lane;
    float pk0 = set < my_tiles ? p.pk[k] : 0.0f;
    float pk1 = set + 2 < my_tiles ? p.pk[k + kstep] : 0.0f;
    for (int it = set; it < my_tiles; it += 2, k += kstep) {
      const uint32_t ap = (uint32_t)((it >> 1) & 1);
      const float pk = pk0;
      pk0 = pk1;
      pk1 = it + 4 < my_tiles ? p.pk[k + 2 * kstep] : 0.0f;
      if (!warp_wait(acc_full + set, ap, err, p.state, lane)) break;
      fence_after();
      float v[kNPop];
      tmem_ld32(taddr, v);
      // the accumulator is in registers: hand the buffer back to the MMA warp
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acc_empty + set);
      const bool valid = k < p.m;
      // all 32 columns, without branches: columns past the population are never read
#pragma unroll
      for (int c = 0; c < kNPop; ++c) {
        const float e = narrow_tc_error<EF>(pk, v[c] + bias[c], p.act, p.err, p.R);
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
                 "r"(2u * kNPop));
  if (threadIdx.x < kNPop) {
    double sum = 0.0;
#pragma unroll
    for (int w = 0; w < 8; ++w) sum += red[w * 32 + threadIdx.x];
    p.partial[(long long)blockIdx.x * p.pop_pad + threadIdx.x] = sum;
  }
}

void* narrow_kernel(int ef) {
  switch (ef) {
    case kEfFast: return reinterpret_cast<void*>(&fitness_tc_narrow_kernel<kEfFast>);
    case kEfMse: return reinterpret_cast<void*>(&fitness_tc_narrow_kernel<kEfMse>);
    case kEfTmse: return reinterpret_cast<void*>(&fitness_tc_narrow_kernel<kEfTmse>);
    case kEfTmseSq: return reinterpret_cast<void*>(&fitness_tc_narrow_kernel<kEfTmseSq>);
    default: return reinterpret_cast<void*>(&fitness_tc_narrow_kernel<kEfGeneral>);
  }
}

int narrow_kblocks(const Shape& s) { return (s.kp + 63) / 64; }

size_t narrow_smem(const Shape& s, int stages) {
  return (size_t)2 * narrow_kblocks(s) * kNTileG + (size_t)stages * kNTileA + kNSmemMisc;
}

int narrow_max_stages(const Shape& s) {
  const long long room = kNSmemMax - kNSmemMisc - 2LL * narrow_kblocks(s) * kNTileG;
  const long long st = room / kNTileA;
  return (int)(st > 10 ? 10 : st);
}

}  // namespace

bool tc_narrow_fits(const Shape& s) {
  return s.precision == GAME_FP32 && s.pop >= 1 && s.pop <= kNPop && s.kp % 16 == 0 &&
         narrow_kblocks(s) <= kNMaxKblocks && narrow_max_stages(s) >= 2;
}

bool tc_narrow_shape(const Shape& s) { return s.tc_narrow && tc_narrow_fits(s); }

void tc_narrow_candidates(const Shape& s, std::vector<TileReq>* out) {
  const int ms = narrow_max_stages(s);
  for (int st : {ms, 6, 4, 3})
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
  t.stages = req.stages ? req.stages : (ms < 6 ? ms : 6);
  if (t.stages < 2 || t.stages > ms) return cudaErrorNotSupported;
  t.n_slices = 1;
  t.n_groups = 1;
  t.n_tiles = (int)((s.n_train + 127) / 128);
  t.grid = t.n_tiles < n_sm ? t.n_tiles : n_sm;
  t.ctas_per_slice = t.grid;
  t.n_part = t.grid;
  t.smem = narrow_smem(s, t.stages);
  cudaError_t err;
  if ((err = tc_make_map(&t.b_map[0], e.p0, GAME_FP32, s.n_train, s.kp, 128)) != cudaSuccess) return err;
  if ((err = tc_make_map(&t.b_map[1], e.p1, GAME_FP32, s.n_train, s.kp, 128)) != cudaSuccess) return err;
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
  p.partial = partial;
  p.state = const_cast<DevState*>(state);
  p.m = s.n_train;
  p.pop = s.pop;
  p.pop_pad = s.pop_pad;
  p.n_tiles = t.n_tiles;
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
  return cudaLaunchKernel(narrow_kernel(ef), dim3(t.grid), dim3(kNThreads), args, t.smem, st);
}

cudaError_t tc_narrow_init_attributes() {
  for (int ef = kEfFast; ef <= kEfGeneral; ++ef) {
    cudaError_t e = cudaFuncSetAttribute(narrow_kernel(ef),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kNSmemMax);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace game
