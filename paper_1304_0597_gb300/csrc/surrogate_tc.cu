// Tensor-core path of the surrogate network (bfloat16 weights, bfloat16 GEMM
// operands, float32 accumulation in TMEM) on sm_103a.
//
// Every GEMM of the network's forward and backward pass has the form
//   D[m, n] = sum_k A[m, k] B[n, k]
// with both operands K-major bfloat16 in global memory, fed by TMA into a ring
// of shared-memory stages and multiplied by tcgen05.mma (M = 128 rows per CTA,
// N = BN columns, K in 64-element blocks).  Sixteen epilogue warps read the
// accumulator with tcgen05.ld: warp w takes TMEM lanes 32 (w % 4) (one output
// row per thread) and a quarter of the columns, and applies one of four fused
// epilogues.  These GEMMs are small (K <= 320) and their epilogues cost more
// than the MMAs, so a small batch takes 64- or 128-column tiles to spread over
// more CTAs; the output layer then needs the partial sums of the other column
// tiles, which the CTAs of a thread-block cluster swap through distributed
// shared memory.  The epilogues:
//   L1    z = acc + b1; H1 = gelu(z) (bf16, the next layer's operand); when
//         training also gelu'(z) and the transposed H1 for the weight gradient;
//   L2    z = acc + b2; y = w3 . gelu(z) + b3; when training, from the same
//         accumulator, dy = 2 (y - t) / B, dZ2 = dy w3 gelu'(z) (bf16, row-major
//         and transposed) and dy * gelu(z) for the output-weight gradient;
//   B1    dZ1 = acc * gelu'(Z1), stored transposed;
//   GRAD  weight gradient rows; the bias gradient is the extra column that a
//         row of ones appended to the B operand produces.
// The transposed operands make the weight gradients (reductions over the
// batch) plain K-major GEMMs as well.  All waits are bounded: on a timeout the
// CTA records GAME_ERR_TIMEOUT in the device state and leaves.
#include <cudaTypedefs.h>

#include "surrogate.h"
#include "tc_ptx.cuh"

namespace game {

namespace {

using namespace tc;

enum MlpEpi { kEpiL1 = 0, kEpiL2 = 1, kEpiB1 = 2, kEpiGrad = 3 };

constexpr int kEpiWarpsTc = 16;
constexpr int kThreadsTc = 64 + 32 * kEpiWarpsTc;   // warp 0 TMA, warp 1 MMA, then the epilogue
constexpr int kStagesTc = 4;
constexpr int kTileA = 128 * 128;    // 128 rows x 64 bf16
constexpr int kGradSplits = 8;       // K slices of the weight-gradient GEMMs

struct MlpParams {
  CUtensorMap a, b;
  int M, N, kblocks, train;
  const float* bias;           // L1: b1, L2: b2
  const __nv_bfloat16* w3;     // L2
  const float* b3;             // L2
  const float* t;              // L2 (train): targets of the batch
  float two_over_b;            // L2 (train): 2 / B
  float* y;                    // L2: network output [M]
  float* dy;                   // L2 (train): [M]
  float* sq;                   // L2 (train): (y - t)^2 [M]
  float* dyh2;                 // L2 (train): dy * gelu(z2) [M x 256]
  __nv_bfloat16* out_b;        // L1: H1 [M x 256]; L2 (train): dZ2 [M x 256]
  __nv_bfloat16* out_t;        // L1 (train): H1^T; L2 (train): dZ2^T; B1: dZ1^T  [256 x ldt]
  float* gp;                   // L1 (train): gelu'(Z1) out; B1: in  [M x 256]
  long long ldt;
  float* g_main;               // GRAD: weight gradient rows [M x n_main], row stride ld_main
  float* g_bias;               // GRAD: bias gradient [M] (column n_main)
  int n_main;
  long long ld_main;
  int kbps;                    // k-blocks per split (blockIdx.z); kblocks when unsplit
  long long zstride;           // GRAD: floats between the partial planes of the splits
  DevState* state;
  int a_box, b_box;            // host check: rows of the A / B boxes (128 / BN)
};

template <int W>
__device__ __forceinline__ void store_bf16xw(__nv_bfloat16* dst, const float* v) {
  uint4* d4 = reinterpret_cast<uint4*>(dst);
#pragma unroll
  for (int q = 0; q < W / 8; ++q) {
    uint32_t w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const __nv_bfloat162 h = __floats2bfloat162_rn(v[q * 8 + 2 * i], v[q * 8 + 2 * i + 1]);
      w[i] = *reinterpret_cast<const uint32_t*>(&h);
    }
    d4[q] = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

template <int W>
__device__ __forceinline__ void store_f32xw(float* dst, const float* v) {
  float4* d4 = reinterpret_cast<float4*>(dst);
#pragma unroll
  for (int q = 0; q < W / 4; ++q)
    d4[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
}

// Shared memory: the ring of stages, then the cross-CTA partial outputs of L2
// (kExchBytes, outside the ring because peers write them while this CTA's MMAs
// may still run), then the barriers.
constexpr int kExchBytes = 4 * 128 * 4;

template <int BN, int EPI>
__global__ void __launch_bounds__(kThreadsTc, 1) mlp_tc_kernel(const __grid_constant__ MlpParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~(uintptr_t)1023);
  constexpr int kTileB = BN * 128;
  constexpr int kStage = kTileA + kTileB;
  constexpr uint32_t kIdesc = make_idesc(128, BN, 1u);   // bf16 x bf16 -> f32
  // L2 needs all 256 hidden columns of a row for y: with BN < 256 the CTAs of a
  // cluster (1, kCN, 1) split the columns and swap their partial dot products.
  constexpr int kCN = EPI == kEpiL2 ? 256 / BN : 1;
  float* xpart = reinterpret_cast<float*>(smem + kStagesTc * kStage);   // [kCN][128]
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStagesTc * kStage + kExchBytes);
  uint64_t* empty = full + kStagesTc;
  uint64_t* acc_full = empty + kStagesTc;
  uint64_t* fin = acc_full + 1;
  uint64_t* xbar = fin + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(xbar + 1);
  volatile int* err = reinterpret_cast<volatile int*>(tmem_slot + 1);
  int* last_par = reinterpret_cast<int*>(tmem_slot + 2);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * 128, n0 = blockIdx.y * BN;
  // split K: this CTA reduces k-blocks [kb0, kb1) (never empty)
  const int kb0 = blockIdx.z * p.kbps;
  const int kb1 = min(p.kblocks, kb0 + p.kbps);

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStagesTc; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
      last_par[s] = -1;
    }
    mbar_init(acc_full, 1);
    mbar_init(fin, 1);
    mbar_init(xbar, 128 * kCN);
    *err = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"((uint32_t)BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  // peers arrive on xbar only after it is initialised in every CTA of the cluster
  if constexpr (kCN > 1) cluster_sync_all();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ---- TMA producer ----
    int stage = 0;
    uint32_t phase = 0;
    for (int kb = kb0; kb < kb1; ++kb) {
      if (!warp_wait(empty + stage, phase ^ 1u, err, p.state, lane)) break;
      if (lane == 0) {
        uint8_t* sa = smem + stage * kStage;
        mbar_expect_tx(full + stage, kStage);
        tma_load_2d(sa, &p.a, kb * 64, m0, full + stage);
        tma_load_2d(sa + kTileA, &p.b, kb * 64, n0, full + stage);
        last_par[stage] = (int)phase;
      }
      if (++stage == kStagesTc) {
        stage = 0;
        phase ^= 1u;
      }
    }
    // Drain: every issued copy has landed before the CTA may exit.
    if (lane == 0)
      for (int s = 0; s < kStagesTc; ++s)
        if (last_par[s] >= 0) {
          const unsigned long long t0 = globaltimer();
          while (!mbar_try_wait(full + s, (uint32_t)last_par[s]) && globaltimer() - t0 < kWaitNs) {
          }
        }
    __syncwarp();
  } else if (warp == 1) {
    // ---- MMA issuer ----
    int stage = 0;
    uint32_t phase = 0;
    uint32_t accum = 0;
    bool ok = true;
    for (int kb = kb0; kb < kb1; ++kb) {
      if (!warp_wait(full + stage, phase, err, p.state, lane)) {
        ok = false;
        break;
      }
      fence_after();
      const uint32_t sa = smem_u32(smem + stage * kStage);
      const uint64_t adesc = sw128_desc(sa);
      const uint64_t bdesc = sw128_desc(sa + kTileA);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        // +32 bytes along K inside the 128-byte swizzle row = +2 in the address field
        if (lane == 0) mma<GAME_BF16>(tmem, adesc + 2 * k, bdesc + 2 * k, kIdesc, accum);
        accum = 1;
      }
      if (lane == 0) mma_commit(empty + stage);
      if (++stage == kStagesTc) {
        stage = 0;
        phase ^= 1u;
      }
    }
    if (lane == 0) {
      if (ok) mma_commit(acc_full);
      // Drain: all issued MMAs complete before TMEM is released.
      mma_commit(fin);
      const unsigned long long t0 = globaltimer();
      while (!mbar_try_wait(fin, 0) && globaltimer() - t0 < kWaitNs) {
      }
    }
    __syncwarp();
  } else {
    // ---- epilogue: thread = output row r, columns [c0, c0 + kCols) of the tile ----
    constexpr int kCols = BN / 4;
    constexpr int kW = kCols < 32 ? kCols : 32;   // TMEM columns per load
    const int q = warp & 3;
    const int h = (warp - 2) >> 2;
    const int r = m0 + q * 32 + lane;
    const bool rv = r < p.M;
    const int c0 = h * kCols;
    const uint32_t tb = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0;
    const bool ok = warp_wait(acc_full, 0, err, p.state, lane);
    if (ok) fence_after();
    float v[kW];
    if (EPI == kEpiL1) {
      if (ok) {
#pragma unroll 1
        for (int ch = 0; ch < kCols / kW; ++ch) {
          tmem_ld<kW>(tb + ch * kW, v);
          const int nb = n0 + c0 + ch * kW;
          if (!p.train) {
#pragma unroll
            for (int j = 0; j < kW; ++j) v[j] = gelu_f(v[j] + p.bias[nb + j]);
            if (rv) store_bf16xw<kW>(p.out_b + (long long)r * 256 + nb, v);
            continue;
          }
          // 16 columns at a time keep gelu' within the register budget
#pragma unroll
          for (int hh = 0; hh < kW; hh += 16) {
            float gp[16];
#pragma unroll
            for (int j = 0; j < 16; ++j)
              gelu_and_grad_f(v[hh + j] + p.bias[nb + hh + j], v[hh + j], gp[j]);
            if (rv) {
              store_bf16xw<16>(p.out_b + (long long)r * 256 + nb + hh, v + hh);
              store_f32xw<16>(p.gp + (long long)r * 256 + nb + hh, gp);
#pragma unroll
              for (int j = 0; j < 16; ++j)
                p.out_t[(long long)(nb + hh + j) * p.ldt + r] = __float2bfloat16_rn(v[hh + j]);
            }
          }
        }
      }
    } else if (EPI == kEpiL2) {
      // y needs all 256 columns: partial dots of the four column groups meet in
      // shared memory (the ring is idle once the accumulator is complete), then
      // the kCN CTAs of the cluster swap their sums.  Every epilogue thread
      // reaches the named barrier and the exchange, also after a failed wait.
      float* part = reinterpret_cast<float*>(smem);   // [4][128]
      float yp = 0.0f;
      if (ok) {
#pragma unroll 1
        for (int ch = 0; ch < kCols / kW; ++ch) {
          tmem_ld<kW>(tb + ch * kW, v);
#pragma unroll
          for (int j = 0; j < kW; ++j) {
            const int n = n0 + c0 + ch * kW + j;
            yp = fmaf(gelu_f(v[j] + p.bias[n]), __bfloat162float(p.w3[n]), yp);
          }
        }
      }
      part[h * 128 + q * 32 + lane] = yp;
      asm volatile("bar.sync 1, %0;" ::"r"(32 * kEpiWarpsTc) : "memory");
      const int rl = q * 32 + lane;
      float y;
      bool xok = true;
      if constexpr (kCN == 1) {
        y = p.b3[0] + ((part[rl] + part[128 + rl]) + (part[256 + rl] + part[384 + rl]));
      } else {
        const uint32_t rank = cluster_rank();
        if (h == 0) {
          const float own = (part[rl] + part[128 + rl]) + (part[256 + rl] + part[384 + rl]);
          const uint32_t slot = smem_u32(xpart + rank * 128 + rl);
#pragma unroll
          for (int c = 0; c < kCN; ++c) {
            st_cluster_f32(mapa_shared(slot, (uint32_t)c), own);
            mbar_arrive_cluster(mapa_shared(smem_u32(xbar), (uint32_t)c));
          }
        }
        xok = mbar_wait_cluster(xbar, 0, err, p.state);
        float sum = 0.0f;
#pragma unroll
        for (int c = 0; c < kCN; ++c) sum += xpart[c * 128 + rl];
        y = p.b3[0] + sum;
      }
      const bool lead = h == 0 && blockIdx.y == 0;   // one writer per row
      if (ok && xok && lead && rv) p.y[r] = y;
      if (ok && xok && p.train) {
        const float e = y - (rv ? p.t[r] : 0.0f);
        const float d = e * p.two_over_b;
        if (lead && rv) {
          p.dy[r] = d;
          p.sq[r] = e * e;
        }
#pragma unroll 1
        for (int ch = 0; ch < kCols / kW; ++ch) {
          tmem_ld<kW>(tb + ch * kW, v);
          const int nb = n0 + c0 + ch * kW;
          float dh[kW];
#pragma unroll
          for (int j = 0; j < kW; ++j) {
            float g, gd;
            gelu_and_grad_f(v[j] + p.bias[nb + j], g, gd);
            dh[j] = d * g;
            v[j] = d * __bfloat162float(p.w3[nb + j]) * gd;
          }
          if (rv) {
            store_bf16xw<kW>(p.out_b + (long long)r * 256 + nb, v);
            store_f32xw<kW>(p.dyh2 + (long long)r * 256 + nb, dh);
#pragma unroll
            for (int j = 0; j < kW; ++j)
              p.out_t[(long long)(nb + j) * p.ldt + r] = __float2bfloat16_rn(v[j]);
          }
        }
      }
    } else if (EPI == kEpiB1) {
      if (ok) {
#pragma unroll 1
        for (int ch = 0; ch < kCols / kW; ++ch) {
          tmem_ld<kW>(tb + ch * kW, v);
          const int nb = n0 + c0 + ch * kW;
          if (rv) {
            const float4* g4 = reinterpret_cast<const float4*>(p.gp + (long long)r * 256 + nb);
#pragma unroll
            for (int j4 = 0; j4 < kW / 4; ++j4) {
              const float4 gg = g4[j4];
              v[4 * j4] *= gg.x;
              v[4 * j4 + 1] *= gg.y;
              v[4 * j4 + 2] *= gg.z;
              v[4 * j4 + 3] *= gg.w;
            }
#pragma unroll
            for (int j = 0; j < kW; ++j)
              p.out_t[(long long)(nb + j) * p.ldt + r] = __float2bfloat16_rn(v[j]);
          }
        }
      }
    } else {
      // weight-gradient rows: each warp turns its 32 x kW block around in shared
      // memory (the idle ring) so that the global stores run along a row
      float* tile = reinterpret_cast<float*>(smem) + (warp - 2) * (32 * 33);
      float* gm = p.g_main + blockIdx.z * p.zstride;
      float* gb = p.g_bias + blockIdx.z * p.zstride;
      if (ok) {
#pragma unroll 1
        for (int ch = 0; ch < kCols / kW; ++ch) {
          tmem_ld<kW>(tb + ch * kW, v);
#pragma unroll
          for (int j = 0; j < kW; ++j) tile[lane * 33 + j] = v[j];
          __syncwarp();
          const int n = n0 + c0 + ch * kW + lane;
          if (lane < kW)
            for (int i = 0; i < 32; ++i) {
              const int rr = m0 + q * 32 + i;
              if (rr < p.M) {
                const float w = tile[i * 33 + lane];
                if (n < p.n_main)
                  gm[(long long)rr * p.ld_main + n] = w;
                else if (n == p.n_main)
                  gb[rr] = w;
              }
            }
          __syncwarp();
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)BN));
  // No CTA leaves while a peer may still write its partial sums here.
  if constexpr (kCN > 1) cluster_sync_all();
}

template <int BN>
constexpr size_t smem_bytes() {
  return (size_t)kStagesTc * (kTileA + BN * 128) + kExchBytes + 1024 + 256;
}

// X (float32, row stride ldx, first D columns) -> Xb (bf16, row stride Dp) and,
// when XT is given, the transposed copy XT[d * ldt + r].  32 x 32 tiles through
// shared memory so that both stores are coalesced.
__global__ void cast_rows_kernel(const float* __restrict__ X, long long ldx, int M, int D,
                                 __nv_bfloat16* __restrict__ Xb, int Dp,
                                 __nv_bfloat16* __restrict__ XT, long long ldt,
                                 const float* __restrict__ gnorm) {
  __shared__ float tile[32][33];
  const int d0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int i = ty; i < 32; i += 8) {
    const int r = r0 + i, d = d0 + tx;
    float v = 0.0f;
    if (r < M && d < D) {
      v = X[(long long)r * ldx + d];
      v = (v - gnorm[d]) * gnorm[D + d];   // running per-gene standardisation
    }
    tile[i][tx] = v;
    if (r < M && d < D) Xb[(long long)r * Dp + d] = __float2bfloat16_rn(v);
  }
  if (!XT) return;
  __syncthreads();
  for (int i = ty; i < 32; i += 8) {
    const int d = d0 + i, r = r0 + tx;
    if (d < D && r < M) XT[(long long)d * ldt + r] = __float2bfloat16_rn(tile[tx][i]);
  }
}

__global__ void fill_f32_tc_kernel(float* p, long long n, float v) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

__global__ void fill_bf16_kernel(__nv_bfloat16* p, long long n, float v) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = __float2bfloat16_rn(v);
}

// The GEMM copies of the weights: W1 [H x D] -> W1b [H x Dp], W2 -> W2b and W2^T.
__global__ void weights_bf16_kernel(const float* __restrict__ p, int D, int Dp, int H,
                                    __nv_bfloat16* __restrict__ W1b,
                                    __nv_bfloat16* __restrict__ W2b,
                                    __nv_bfloat16* __restrict__ W2Tb) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long n1 = (long long)H * D;
  if (i < n1) {
    W1b[(i / D) * Dp + i % D] = __float2bfloat16_rn(p[i]);
    return;
  }
  const long long j = i - n1;
  if (j < (long long)H * H) {
    const float w = p[n1 + H + j];   // W2 follows W1 and b1
    const int row = (int)(j / H), col = (int)(j % H);
    W2b[j] = __float2bfloat16_rn(w);
    W2Tb[(long long)col * H + row] = __float2bfloat16_rn(w);
  }
}

// Output-layer gradients and the loss of one batch in one launch (fixed-order
// tree sums): CTA n < H gives gw3[n] = sum_b dy[b] gelu(z2[b, n]); CTA H gives
// gb3 = sum_b dy[b] and the loss mean((y - t)^2).
__global__ void out_grads_kernel(const float* __restrict__ dyh2, const float* __restrict__ dy,
                                 const float* __restrict__ sq, int B, int H,
                                 float* __restrict__ gw3, float* __restrict__ gb3,
                                 float* __restrict__ loss) {
  __shared__ float red[2][256];
  const int n = blockIdx.x;
  float a = 0.0f, b = 0.0f;
  for (int r = threadIdx.x; r < B; r += blockDim.x) {
    if (n < H) {
      a += dyh2[(long long)r * H + n];
    } else {
      a += dy[r];
      b += sq[r];
    }
  }
  red[0][threadIdx.x] = a;
  red[1][threadIdx.x] = b;
  __syncthreads();
  for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      red[0][threadIdx.x] += red[0][threadIdx.x + o];
      red[1][threadIdx.x] += red[1][threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (n < H) {
      gw3[n] = red[0][0];
    } else {
      *gb3 = red[0][0];
      *loss = red[1][0] / (float)B;
    }
  }
}

// Adam (Kingma & Ba 2015) over the flat parameters, with the bf16 copies that the
// tensor-core GEMMs read (flat, W1 padded to Dp, W2 and W2^T).  Every block reads
// the step count first; the last block to finish advances it.
// With ws != nullptr the gradient of [W1 | b1 | W2 | b2] (the first n12 entries) is
// the in-order sum of the split-K planes ws[z * n12 + i] (what grad_sum_kernel would
// write to g first); w3 and b3 come from g.
__global__ void adam_tc_kernel(float* __restrict__ p, const float* __restrict__ g,
                               float* __restrict__ m, float* __restrict__ v,
                               __nv_bfloat16* __restrict__ ph, long long n, int* step,
                               unsigned int* done, float lr, float beta1, float beta2, float eps,
                               int D, int Dp, int H, __nv_bfloat16* __restrict__ W1b,
                               __nv_bfloat16* __restrict__ W2b, __nv_bfloat16* __restrict__ W2Tb,
                               const float* __restrict__ ws, int splits, long long n12) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int t = *step + 1;
  if (i < n) {
    float gi;
    if (ws && i < n12) {
      gi = ws[i];
      for (int z = 1; z < splits; ++z) gi += ws[z * n12 + i];
    } else {
      gi = g[i];
    }
    const float mi = beta1 * m[i] + (1.0f - beta1) * gi;
    const float vi = beta2 * v[i] + (1.0f - beta2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / (1.0f - powf(beta1, (float)t));
    const float vh = vi / (1.0f - powf(beta2, (float)t));
    const float pi = p[i] - lr * mh / (sqrtf(vh) + eps);
    p[i] = pi;
    const __nv_bfloat16 hb = __float2bfloat16_rn(pi);
    ph[i] = hb;
    const long long n1 = (long long)H * D;
    if (i < n1) {
      W1b[(i / D) * Dp + i % D] = hb;
    } else if (i >= n1 + H && i < n1 + H + (long long)H * H) {
      const long long j = i - n1 - H;
      W2b[j] = hb;
      W2Tb[(j % H) * H + j / H] = hb;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(done, 1u) == gridDim.x - 1) {
      *step = t;
      *done = 0u;
    }
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_tiled() {
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

// K-major bf16 operand [rows x cols] with row stride ld elements (multiple of 8);
// boxes of 64 columns x box_rows rows, 128-byte swizzle; reads outside
// [rows x cols] return zeros.
cudaError_t bf16_map(CUtensorMap* m, const void* base, long long rows, long long cols, long long ld,
                     int box_rows) {
  auto fn = encode_tiled();
  if (!fn) return cudaErrorNotSupported;
  if (rows < 1 || cols < 1 || ld % 8 != 0 || ((uintptr_t)base & 15u)) return cudaErrorInvalidValue;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {64u, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides,
                  box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// The operand maps of one GEMM: A boxes are 128 rows (the MMA's M), B boxes
// one column tile of BN rows; a stage expects exactly these bytes.
cudaError_t map_a(MlpParams& p, const void* base, long long rows, long long cols, long long ld) {
  p.a_box = 128;
  return bf16_map(&p.a, base, rows, cols, ld, 128);
}
cudaError_t map_b(MlpParams& p, const void* base, long long rows, long long cols, long long ld,
                  int box) {
  p.b_box = box;
  return bf16_map(&p.b, base, rows, cols, ld, box);
}

template <int BN, int EPI>
cudaError_t launch_mlp(MlpParams& p, int grid_m, int grid_n, cudaStream_t st, int splits = 1) {
  if (p.a_box != 128 || p.b_box != BN) return cudaErrorInvalidValue;
  if (splits <= 1) p.kbps = p.kblocks;
  constexpr int kCN = EPI == kEpiL2 ? 256 / BN : 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid_m, grid_n, splits);
  cfg.blockDim = dim3(kThreadsTc);
  cfg.dynamicSmemBytes = smem_bytes<BN>();
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  if (kCN > 1) {
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 1;
    at[0].val.clusterDim.y = kCN;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
  }
  return cudaLaunchKernelEx(&cfg, mlp_tc_kernel<BN, EPI>, p);
}

// Column-tile width of the hidden-layer GEMMs by the number of 128-row tiles:
// the epilogue, not the MMA, bounds them, so a small batch (a training step)
// takes narrow tiles and more CTAs, a large one (the candidate pool) wide ones.
int hidden_bn(int grid_m, bool l2) {
  if (l2 && grid_m >= 128) return 256;
  return grid_m >= 32 ? 128 : 64;
}

// g[i] = sum over the splits z of ws[z * n + i], in order (deterministic).
__global__ void grad_sum_kernel(const float* __restrict__ ws, int splits, long long n,
                                float* __restrict__ g) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float s = ws[i];
  for (int z = 1; z < splits; ++z) s += ws[z * n + i];
  g[i] = s;
}

int ceil_div(long long a, int b) { return (int)((a + b - 1) / b); }

}  // namespace

cudaError_t surrogate_tc_init_attributes() {
  cudaError_t e;
#define GAME_MLP_ATTR(BN, EPI)                                                                 \
  if ((e = cudaFuncSetAttribute(mlp_tc_kernel<BN, EPI>,                                        \
                                cudaFuncAttributeMaxDynamicSharedMemorySize,                   \
                                (int)smem_bytes<BN>())) != cudaSuccess)                        \
    return e;
  GAME_MLP_ATTR(64, kEpiL1)
  GAME_MLP_ATTR(128, kEpiL1)
  GAME_MLP_ATTR(64, kEpiL2)
  GAME_MLP_ATTR(128, kEpiL2)
  GAME_MLP_ATTR(256, kEpiL2)
  GAME_MLP_ATTR(64, kEpiB1)
  GAME_MLP_ATTR(128, kEpiB1)
  GAME_MLP_ATTR(128, kEpiGrad)
#undef GAME_MLP_ATTR
  return cudaSuccess;
}

size_t Surrogate::tc_bytes(int max_rows_, int batch) const {
  const size_t dp = (size_t)((D + 7) / 8 * 8);
  const size_t ldt_ = (size_t)((batch + 7) / 8 * 8);
  const size_t b16 = sizeof(__nv_bfloat16);
  return b16 * ((size_t)H * dp + 2 * (size_t)H * H + (size_t)max_rows_ * (dp + H) +
                ((size_t)D + 1 + (size_t)H + 1 + 2 * (size_t)H) * ldt_ + (size_t)batch * H) +
         sizeof(float) * (2 * (size_t)batch * H + (size_t)kGradSplits * n_params() +
                          3 * (size_t)D + 4) +
         16;
}

void Surrogate::tc_carve(void* base, int batch) {
  Dp = (D + 7) / 8 * 8;
  Bt = batch;
  ldt = (batch + 7) / 8 * 8;
  // every block below is a multiple of 16 bytes (Dp, H and ldt are multiples of 8)
  auto* q = reinterpret_cast<__nv_bfloat16*>(base);
  W1b = q;
  q += (size_t)H * Dp;
  W2b = q;
  q += (size_t)H * H;
  W2Tb = q;
  q += (size_t)H * H;
  Xb = q;
  q += (size_t)max_rows * Dp;
  H1b = q;
  q += (size_t)max_rows * H;
  XTb = q;
  q += (size_t)(D + 1) * ldt;
  H1Tb = q;
  q += (size_t)(H + 1) * ldt;
  dZ2Tb = q;
  q += (size_t)H * ldt;
  dZ1Tb = q;
  q += (size_t)H * ldt;
  dZ2b = q;
  q += (size_t)Bt * H;
  auto* f = reinterpret_cast<float*>(q);
  gp1 = f;
  f += (size_t)Bt * H;
  dyh2 = f;
  f += (size_t)Bt * H;
  gws = f;
  f += (size_t)kGradSplits * n_params();
  gnorm = f;
  f += 3 * (size_t)D + 4;
  adam_done = reinterpret_cast<unsigned int*>(f);
  tc = true;
}

cudaError_t Surrogate::tc_prepare(cudaStream_t st) {
  // rows of ones under the transposed batch and hidden activations: the bias
  // gradients come out of the weight-gradient GEMMs as one more column
  fill_bf16_kernel<<<ceil_div(ldt, 256), 256, 0, st>>>(XTb + (size_t)D * ldt, ldt, 1.0f);
  fill_bf16_kernel<<<ceil_div(ldt, 256), 256, 0, st>>>(H1Tb + (size_t)H * ldt, ldt, 1.0f);
  // input standardisation starts as the identity (shift 0, scale 1, count 0)
  fill_f32_tc_kernel<<<ceil_div(D, 256), 256, 0, st>>>(gnorm + D, D, 1.0f);
  return tc_weights(st);
}

cudaError_t Surrogate::tc_weights(cudaStream_t st) {
  const long long n = (long long)H * D + (long long)H * H;
  weights_bf16_kernel<<<ceil_div(n, 256), 256, 0, st>>>(p, D, Dp, H, W1b, W2b, W2Tb);
  return cudaGetLastError();
}

cudaError_t Surrogate::tc_forward(const float* X, long long ldx, int M, float* y, const float* t,
                                  cudaStream_t st) {
  const bool train = t != nullptr;
  if (M < 1 || M > max_rows || (train && M > Bt)) return cudaErrorInvalidValue;
  cast_rows_kernel<<<dim3(ceil_div(D, 32), ceil_div(M, 32)), dim3(32, 8), 0, st>>>(
      X, ldx, M, D, Xb, Dp, train ? XTb : nullptr, ldt, gnorm);
  return tc_layers(M, y, t, st);
}

cudaError_t Surrogate::tc_train_step(int B, const float* t, float lr, cudaStream_t st) {
  cudaError_t e;
  if ((e = tc_layers(B, yb, t, st)) != cudaSuccess) return e;
  // After the forward pass (which leaves dZ2) the output-layer gradients and the W2
  // gradient depend on nothing else: with a second stream they run beside dZ1 and the
  // W1 gradient.  The Adam launch adds the split-K planes itself.
  const bool fork = side && ev_fork && ev_join;
  cudaStream_t s2 = fork ? side : st;
  if (fork) {
    if ((e = cudaEventRecord(ev_fork, st)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(side, ev_fork, 0)) != cudaSuccess) return e;
  }
  if ((e = tc_out_grads(B, s2)) != cudaSuccess) return e;
  if ((e = tc_grad_w2(B, s2)) != cudaSuccess) return e;
  if ((e = tc_backward_b1(B, st)) != cudaSuccess) return e;
  if ((e = tc_grad_w1(B, st)) != cudaSuccess) return e;
  if (fork) {
    if ((e = cudaEventRecord(ev_join, side)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(st, ev_join, 0)) != cudaSuccess) return e;
  }
  return tc_adam(lr, st, true);
}

cudaError_t Surrogate::tc_layers(int M, float* y, const float* t, cudaStream_t st) {
  const bool train = t != nullptr;
  if (M < 1 || M > max_rows || (train && M > Bt)) return cudaErrorInvalidValue;
  float *W1, *b1, *W2, *b2, *w3, *b3;
  views(p, &W1, &b1, &W2, &b2, &w3, &b3);
  const __nv_bfloat16* w3b = ph + ((size_t)H * D + H + (size_t)H * H + H);
  cudaError_t e;
  MlpParams a = {};
  a.state = state;
  a.train = train ? 1 : 0;
  a.ldt = ldt;
  // layer 1: Z1 = Xb W1b^T
  // the B operand's box is one column tile: BN rows (the expected bytes of a stage)
  const int gm = ceil_div(M, 128);
  const int bn1 = hidden_bn(gm, false), bn2 = hidden_bn(gm, true);
  if ((e = map_a(a, Xb, M, D, Dp)) != cudaSuccess) return e;
  if ((e = map_b(a, W1b, H, D, Dp, bn1)) != cudaSuccess) return e;
  a.M = M;
  a.N = H;
  a.kblocks = ceil_div(D, 64);
  a.bias = b1;
  a.out_b = H1b;
  a.out_t = H1Tb;
  a.gp = gp1;
  e = bn1 == 128 ? launch_mlp<128, kEpiL1>(a, gm, H / 128, st)
                 : launch_mlp<64, kEpiL1>(a, gm, H / 64, st);
  if (e != cudaSuccess) return e;
  // layer 2 and the output: Z2 = H1b W2b^T
  MlpParams b = a;
  if ((e = map_a(b, H1b, M, H, H)) != cudaSuccess) return e;
  if ((e = map_b(b, W2b, H, H, H, bn2)) != cudaSuccess) return e;
  b.kblocks = H / 64;
  b.bias = b2;
  b.w3 = w3b;
  b.b3 = b3;
  b.y = y;
  b.t = t;
  b.two_over_b = 2.0f / (float)M;
  b.dy = dy;
  b.sq = sq;
  b.dyh2 = dyh2;
  b.out_b = dZ2b;
  b.out_t = dZ2Tb;
  switch (bn2) {
    case 256: return launch_mlp<256, kEpiL2>(b, gm, 1, st);
    case 128: return launch_mlp<128, kEpiL2>(b, gm, 2, st);
    default: return launch_mlp<64, kEpiL2>(b, gm, 4, st);
  }
}

cudaError_t Surrogate::tc_out_grads(int B, cudaStream_t st) {
  float *gW1, *gb1, *gW2, *gb2, *gw3, *gb3;
  views(g, &gW1, &gb1, &gW2, &gb2, &gw3, &gb3);
  out_grads_kernel<<<H + 1, 256, 0, st>>>(dyh2, dy, sq, B, H, gw3, gb3, loss);
  return cudaGetLastError();
}

cudaError_t Surrogate::tc_adam(float lr, cudaStream_t st, bool from_planes) {
  const long long n = (long long)n_params();
  const long long n12 = (long long)H * D + H + (long long)H * H + H;
  if (from_planes && grad_splits < 1) return cudaErrorInvalidValue;
  adam_tc_kernel<<<ceil_div(n, 256), 256, 0, st>>>(
      p, g, m, v, ph, n, step, adam_done, lr, 0.9f, 0.999f, 1e-8f, D, Dp, H, W1b, W2b, W2Tb,
      from_planes ? gws : nullptr, grad_splits, n12);
  return cudaGetLastError();
}

cudaError_t Surrogate::tc_backward_gemms(int B, cudaStream_t st, bool sum_planes) {
  cudaError_t e;
  if ((e = tc_backward_b1(B, st)) != cudaSuccess) return e;
  if ((e = tc_grad_w2(B, st)) != cudaSuccess) return e;
  if ((e = tc_grad_w1(B, st)) != cudaSuccess) return e;
  if (sum_planes) {
    const long long n12 = (long long)H * D + H + (long long)H * H + H;
    grad_sum_kernel<<<ceil_div(n12, 256), 256, 0, st>>>(gws, grad_splits, n12, g);
  }
  return cudaGetLastError();
}

cudaError_t Surrogate::tc_backward_b1(int B, cudaStream_t st) {
  cudaError_t e;
  MlpParams a = {};
  a.state = state;
  a.ldt = ldt;
  // dZ1^T = ((dZ2 W2) * gelu'(Z1))^T : A = dZ2 [B x H], B operand = W2^T
  const int gm = ceil_div(B, 128);
  const int bn = hidden_bn(gm, false);
  if ((e = map_a(a, dZ2b, B, H, H)) != cudaSuccess) return e;
  if ((e = map_b(a, W2Tb, H, H, H, bn)) != cudaSuccess) return e;
  a.M = B;
  a.N = H;
  a.kblocks = H / 64;
  a.out_t = dZ1Tb;
  a.gp = gp1;
  return bn == 128 ? launch_mlp<128, kEpiB1>(a, gm, H / 128, st)
                   : launch_mlp<64, kEpiB1>(a, gm, H / 64, st);
}

// The weight gradients reduce over the batch (K = B): K is split into up to kGradSplits
// slices, each writing a partial plane laid out like the flat parameters [W1 | b1 | W2 |
// b2] (workspace gws); the planes are added in order later (grad_sum_kernel or Adam).
static void grad_split_plan(int B, int* kblocks, int* kbps, int* splits) {
  *kblocks = ceil_div(B, 64);
  *kbps = ceil_div(*kblocks, kGradSplits);
  *splits = ceil_div(*kblocks, *kbps);
}

cudaError_t Surrogate::tc_grad_w2(int B, cudaStream_t st) {
  cudaError_t e;
  const long long n12 = (long long)H * D + H + (long long)H * H + H;
  int kblocks, kbps, splits;
  grad_split_plan(B, &kblocks, &kbps, &splits);
  grad_splits = splits;
  float *wW1, *wb1, *wW2, *wb2, *ww3, *wb3;
  views(gws, &wW1, &wb1, &wW2, &wb2, &ww3, &wb3);
  // [gW2 | gb2] = dZ2^T [H1 | 1] : A = dZ2^T [H x B], B operand = [H1^T ; 1] [(H + 1) x B]
  MlpParams w = {};
  w.state = state;
  if ((e = map_a(w, dZ2Tb, H, B, ldt)) != cudaSuccess) return e;
  if ((e = map_b(w, H1Tb, H + 1, B, ldt, 128)) != cudaSuccess) return e;
  w.M = H;
  w.N = H + 1;
  w.kblocks = kblocks;
  w.kbps = kbps;
  w.zstride = n12;
  w.g_main = wW2;
  w.g_bias = wb2;
  w.n_main = H;
  w.ld_main = H;
  return launch_mlp<128, kEpiGrad>(w, ceil_div(H, 128), ceil_div(H + 1, 128), st, splits);
}

cudaError_t Surrogate::tc_grad_w1(int B, cudaStream_t st) {
  cudaError_t e;
  const long long n12 = (long long)H * D + H + (long long)H * H + H;
  int kblocks, kbps, splits;
  grad_split_plan(B, &kblocks, &kbps, &splits);
  grad_splits = splits;
  float *wW1, *wb1, *wW2, *wb2, *ww3, *wb3;
  views(gws, &wW1, &wb1, &wW2, &wb2, &ww3, &wb3);
  // [gW1 | gb1] = dZ1^T [X | 1] : A = dZ1^T [H x B], B operand = [X^T ; 1] [(D + 1) x B]
  MlpParams v = {};
  v.state = state;
  v.M = H;
  v.kblocks = kblocks;
  v.kbps = kbps;
  v.zstride = n12;
  if ((e = map_a(v, dZ1Tb, H, B, ldt)) != cudaSuccess) return e;
  if ((e = map_b(v, XTb, D + 1, B, ldt, 128)) != cudaSuccess) return e;
  v.N = D + 1;
  v.g_main = wW1;
  v.g_bias = wb1;
  v.n_main = D;
  v.ld_main = D;
  return launch_mlp<128, kEpiGrad>(v, ceil_div(H, 128), ceil_div(D + 1, 128), st, splits);
}

}  // namespace game
