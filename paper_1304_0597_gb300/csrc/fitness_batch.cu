// Grouped tensor-core fitness of many independent GAME runs in one persistent
// launch (the batched form).  Every run keeps its own expansion planes, gene
// planes, targets and partial-sum rows; the launch walks a static list of work
// items (run, 128-chromosome slice, range of 256-pattern tiles) that the host
// balanced over the SMs.
//
// Unlike the single-run kernel, the gene planes are not resident: each ring
// stage carries one k-block of both operands (A = genes of the slice, B = the
// pattern tile), so runs of any gene count fit the same shared-memory layout
// (2 x 16 KB of A + 2 x 32 KB of B per stage).  The arithmetic per run is the
// single-run kernel's (FP32 split / BF16 / FP8 kinds, fused epilogue, float64
// per-chromosome sums), so each run's fitness is what it would be alone.
#include "fitness_tc.h"
#include "tc_ptx.cuh"

namespace game {

namespace {

using namespace tc;

constexpr int kEpiWarps = 16;
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr int kColGroups = kEpiWarps / 4;
constexpr int kBN = 256;
constexpr int kTileA = 128 * 128;
constexpr int kTileB = kBN * 128;
constexpr int kStage = 2 * kTileA + 2 * kTileB;     // 96 KB
constexpr int kSmemMaxB = 232448;

template <int PREC>
__device__ __forceinline__ void issue_kblock(uint32_t d, uint32_t a_addr, uint32_t b_addr,
                                             int n_ap, int n_bp, int steps, uint32_t& accum,
                                             int lane) {
  constexpr uint32_t kFmt = PREC == GAME_BF16 ? 1u : 0u;
  constexpr uint32_t kIdesc = make_idesc(128, kBN, kFmt);
  for (int bp = 0; bp < n_bp; ++bp) {
    const uint64_t bdesc = sw128_desc(b_addr + (uint32_t)(bp * kTileB));
    // FP32 split: P_hi meets G_hi and G_lo, P_lo meets G_hi.
    const int na = bp == 1 ? 1 : n_ap;
    for (int ai = 0; ai < na; ++ai) {
      const uint64_t adesc = sw128_desc(a_addr + (uint32_t)(ai * kTileA));
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (k < steps) {
          if (lane == 0) mma<PREC>(d, adesc + 2 * k, bdesc + 2 * k, kIdesc, accum);
          accum = 1;
        }
    }
  }
}

__global__ void __launch_bounds__(kThreads, 1)
    batch_fitness_kernel(const BatchRunDev* __restrict__ runs, const WorkItem* __restrict__ items,
                         const int* __restrict__ item_off, int S, int in_evolve) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~(uintptr_t)1023);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + S * kStage);
  uint64_t* full = bars;
  uint64_t* empty = full + S;
  uint64_t* acc_full = empty + S;
  uint64_t* acc_empty = acc_full + 2;
  uint64_t* fin = acc_empty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(fin + 1);
  volatile int* err = reinterpret_cast<volatile int*>(tmem_slot + 1);
  int* last_par = reinterpret_cast<int*>(tmem_slot + 2);
  DevState* any_state = const_cast<DevState*>(runs[0].state);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i0 = item_off[blockIdx.x], i1 = item_off[blockIdx.x + 1];
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
      last_par[s] = -1;
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
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(2 * kBN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ---- TMA producer ----
    int stage = 0;
    uint32_t phase = 0;
    bool ok = true;
    for (int w = i0; w < i1 && ok; ++w) {
      const WorkItem it = items[w];
      const BatchRunDev& r = runs[it.run];
      if (in_evolve && r.state->stopped) continue;
      const int kkb = r.prec == GAME_FP8 ? 128 : 64;
      const uint32_t bytes = (uint32_t)(r.n_aplanes * kTileA + r.n_bplanes * kTileB);
      for (int tile = it.tile0; tile < it.tile1 && ok; ++tile)
        for (int kb = 0; kb < r.kblocks; ++kb) {
          if (!warp_wait(empty + stage, phase ^ 1u, err, any_state, lane)) {
            ok = false;
            break;
          }
          if (lane == 0) {
            uint8_t* st = smem + stage * kStage;
            mbar_expect_tx(full + stage, bytes);
            for (int pl = 0; pl < r.n_aplanes; ++pl)
              tma_load_2d(st + pl * kTileA, &r.a[pl], kb * kkb, it.slice * 128, full + stage);
            for (int pl = 0; pl < r.n_bplanes; ++pl)
              tma_load_2d(st + 2 * kTileA + pl * kTileB, &r.b[pl], kb * kkb, tile * kBN,
                          full + stage);
            last_par[stage] = (int)phase;
          }
          if (++stage == S) {
            stage = 0;
            phase ^= 1u;
          }
        }
    }
    if (lane == 0)
      for (int s2 = 0; s2 < S; ++s2)
        if (last_par[s2] >= 0) {
          const unsigned long long t0 = globaltimer();
          while (!mbar_try_wait(full + s2, (uint32_t)last_par[s2]) && globaltimer() - t0 < kWaitNs) {
          }
        }
    __syncwarp();
  } else if (warp == 1) {
    // ---- MMA issuer (warp-uniform, lane 0 issues) ----
    int stage = 0;
    uint32_t phase = 0;
    int gt = 0;   // tiles processed by this CTA so far (accumulator parity)
    bool ok = true;
    const uint32_t base = smem_u32(smem);
    for (int w = i0; w < i1 && ok; ++w) {
      const WorkItem it = items[w];
      const BatchRunDev& r = runs[it.run];
      if (in_evolve && r.state->stopped) continue;
      const int kpb = r.prec == GAME_FP8 ? 4 : 4;    // MMA K-steps per 128-byte k-block
      for (int tile = it.tile0; tile < it.tile1 && ok; ++tile, ++gt) {
        const int buf = gt & 1;
        const uint32_t ap = (uint32_t)((gt >> 1) & 1);
        if (!warp_wait(acc_empty + buf, ap ^ 1u, err, any_state, lane)) {
          ok = false;
          break;
        }
        fence_after();
        const uint32_t d = tmem + (uint32_t)(buf * kBN);
        uint32_t accum = 0;
        for (int kb = 0; kb < r.kblocks; ++kb) {
          const int steps = min(kpb, r.ksteps - kb * kpb);
          if (!warp_wait(full + stage, phase, err, any_state, lane)) {
            ok = false;
            break;
          }
          fence_after();
          const uint32_t sa = base + (uint32_t)(stage * kStage);
          const uint32_t sb = sa + 2 * kTileA;
          if (r.prec == GAME_FP8)
            issue_kblock<GAME_FP8>(d, sa, sb, r.n_aplanes, r.n_bplanes, steps, accum, lane);
          else if (r.prec == GAME_BF16)
            issue_kblock<GAME_BF16>(d, sa, sb, r.n_aplanes, r.n_bplanes, steps, accum, lane);
          else
            issue_kblock<GAME_FP32>(d, sa, sb, r.n_aplanes, r.n_bplanes, steps, accum, lane);
          if (lane == 0) mma_commit(empty + stage);
          if (++stage == S) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (!ok) break;
        if (lane == 0) mma_commit(acc_full + buf);
      }
    }
    if (lane == 0) {
      mma_commit(fin);
      const unsigned long long t0 = globaltimer();
      while (!mbar_try_wait(fin, 0) && globaltimer() - t0 < kWaitNs) {
      }
    }
    __syncwarp();
  } else {
    // ---- epilogue ----
    const int q = warp & 3;
    const int h = (warp - 2) >> 2;
    int gt = 0;
    bool ok = true;
    for (int w = i0; w < i1 && ok; ++w) {
      const WorkItem it = items[w];
      const BatchRunDev& r = runs[it.run];
      if (in_evolve && r.state->stopped) continue;
      const int c = it.slice * 128 + q * 32 + lane;
      const float bias = r.bias[c];
      const float rs = r.rscale[c];
      F2Sum acc;
      for (int tile = it.tile0; tile < it.tile1; ++tile, ++gt) {
        const int buf = gt & 1;
        const uint32_t ap = (uint32_t)((gt >> 1) & 1);
        if (!warp_wait(acc_full + buf, ap, err, any_state, lane)) {
          ok = false;
          break;
        }
        fence_after();
        constexpr int kCols = kBN / kColGroups;
        const uint32_t tb = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * kBN + h * kCols);
#pragma unroll 1
        for (int ch = 0; ch < kCols / 32; ++ch) {
          const long long p0 = (long long)tile * kBN + h * kCols + ch * 32;
          // same arithmetic as the single-run kernels
          if (r.fast == 2)
            acc.add(chunk_error<true, true, true>(tb + ch * 32, r.pk, p0, r.m, rs, bias, r.act,
                                                  r.err, r.R));
          else if (r.fast)
            acc.add(chunk_error<true, true>(tb + ch * 32, r.pk, p0, r.m, rs, bias, r.act, r.err,
                                            r.R));
          else
            acc.add(chunk_error<false>(tb + ch * 32, r.pk, p0, r.m, rs, bias, r.act, r.err, r.R));
        }
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(acc_empty + buf);
      }
      if (!ok) break;
      r.partial[(long long)(it.chunk * kColGroups + h) * r.pop_pad + c] = acc.value();
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kBN));
}

}  // namespace

int batch_stages() { return (kSmemMaxB - 2048) / kStage; }

size_t batch_smem_bytes() { return (size_t)batch_stages() * kStage + 2048; }

cudaError_t batch_init_attributes() {
  return cudaFuncSetAttribute(batch_fitness_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)batch_smem_bytes());
}

cudaError_t batch_make_run(const Shape& s, const Fitness& f, const PopDev& p, const ExpDev& e,
                           double* partial, const DevState* state, BatchRunDev* out) {
  BatchRunDev r{};
  cudaError_t err;
  if ((err = tc_make_map(&r.a[0], p.ghi, s.precision, s.pop_pad, s.kp, 128)) != cudaSuccess) return err;
  if ((err = tc_make_map(&r.a[1], p.glo, s.precision, s.pop_pad, s.kp, 128)) != cudaSuccess) return err;
  if ((err = tc_make_map(&r.b[0], e.p0, s.precision, s.n_train, s.kp, kBN)) != cudaSuccess) return err;
  if (s.precision == GAME_FP32) {
    if ((err = tc_make_map(&r.b[1], e.p1, s.precision, s.n_train, s.kp, kBN)) != cudaSuccess) return err;
  } else {
    r.b[1] = r.b[0];
  }
  r.fast = f.pm1_targets && f.activation == GAME_TANH && (f.error == GAME_RMSE || f.error == GAME_MSE);
  if (r.fast && s.precision != GAME_FP32) r.fast = 2;
  r.pk = r.fast == 1 ? e.tcoef : e.t;
  r.bias = p.bias;
  r.rscale = p.rscale;
  r.partial = partial;
  r.state = state;
  r.m = s.n_train;
  r.pop_pad = s.pop_pad;
  const int kkb = s.precision == GAME_FP8 ? 128 : 64;
  const int kstep = s.precision == GAME_FP8 ? 32 : 16;
  r.kblocks = (s.kp + kkb - 1) / kkb;
  r.ksteps = s.kp / kstep;
  r.n_bplanes = s.precision == GAME_FP32 ? 2 : 1;
  r.n_aplanes = s.gene_planes;
  r.prec = s.precision;
  r.act = f.activation;
  r.err = f.error;
  r.R = f.tmse_R;
  *out = r;
  return cudaSuccess;
}

cudaError_t batch_fitness_launch(const BatchRunDev* d_runs, const WorkItem* d_items,
                                 const int* d_item_off, int grid, int in_evolve, cudaStream_t st) {
  batch_fitness_kernel<<<grid, kThreads, batch_smem_bytes(), st>>>(d_runs, d_items, d_item_off,
                                                                   batch_stages(), in_evolve);
  return cudaGetLastError();
}

int batch_tile_rows() { return kBN; }

}  // namespace game
