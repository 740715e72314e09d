// game_fitness_noalloc: population fitness for callers that cannot allocate
// device memory.  It is the SIMT fitness kernel of this library with its
// per-block partial sums kept in one fixed, file-scope device array instead of
// a buffer from cudaMalloc; the caller passes every input and the output.
//
// Who needs it: code that must not call cudaMalloc -- a service whose device
// memory is a fixed arena owned by another allocator (a framework's caching
// allocator, a memory budget set at start-up), a plugin inside a host program
// that owns every device allocation, or a latency-critical path where
// cudaMalloc's implicit device-wide synchronisation would stall other streams.
// This path calls no cudaMalloc, cudaFree or allocating library routine.
//
// Limits and sharing: pop <= 4096 chromosomes; the partial sums use at most
// 32 x 4096 doubles (1 MiB), resident on every device that loads the library
// until the process exits.  All calls share that array and it keeps the last
// call's contents; each call overwrites every entry it reads, so nothing needs
// clearing, but two calls whose kernels overlap on the GPU (different streams,
// or different host threads) race on it.  The first call on a device looks up
// the array's device address (cudaGetSymbolAddress) with that device current;
// make that first call before any stream capture.
#include "game_internal.h"

#include <mutex>

namespace game {

namespace {

constexpr int kMaxPop = 4096;
constexpr int kParts = 32;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_partial[kParts * kMaxPop];

std::mutex g_setup_mu;
double* g_partial_addr[kMaxDevices] = {};   // device address of g_noalloc_partial, per device

__device__ __forceinline__ float pattern_error(float t, float s, int act, int err, float R) {
  const float y = act == GAME_TANH ? tanhf(s) : s;
  const float d = t - y;
  const float e = d * d;
  if (err == GAME_TMSE) return fabsf(d) > R ? e : 0.0f;
  if (err == GAME_TMSE_SQ) return e > R ? e : 0.0f;
  return e;
}

// Same tiling as the context path's SIMT kernel: 64 patterns x 64 chromosomes
// per block, 4 x 4 per thread, blocks stride over pattern tiles and write one
// partial row each.  P is float32 [n x kb] (basis columns), G float32
// [pop x n_genes] with the bias in gene 0.
__global__ void __launch_bounds__(256) noalloc_fitness_kernel(
    const float* __restrict__ P, const float* __restrict__ t, const float* __restrict__ G,
    long long n, int kb, int n_genes, int pop, int act, int err, float R, double* partial,
    int pop_pad) {
  __shared__ float Ps[64][33];
  __shared__ float Gs[64][33];
  __shared__ float red[16][65];
  __shared__ double acc64[64];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int c0 = blockIdx.y * 64;
  if (tid < 64) acc64[tid] = 0.0;
  float bias[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int c = c0 + tx * 4 + j;
    bias[j] = c < pop ? G[(long long)c * n_genes] : 0.0f;
  }
  for (long long m0 = (long long)blockIdx.x * 64; m0 < n; m0 += (long long)gridDim.x * 64) {
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
    for (int k0 = 0; k0 < kb; k0 += 32) {
      for (int i = tid; i < 64 * 32; i += 256) {
        const int r = i >> 5, cc = i & 31;
        const long long row = m0 + r;
        const int col = k0 + cc;
        const int c = c0 + r;
        Ps[r][cc] = (row < n && col < kb) ? P[row * kb + col] : 0.0f;
        Gs[r][cc] = (c < pop && col < kb) ? G[(long long)c * n_genes + 1 + col] : 0.0f;
      }
      __syncthreads();
#pragma unroll 8
      for (int kk = 0; kk < 32; ++kk) {
        float pa[4], gb[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) pa[i] = Ps[ty * 4 + i][kk];
#pragma unroll
        for (int j = 0; j < 4; ++j) gb[j] = Gs[tx * 4 + j][kk];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(pa[i], gb[j], acc[i][j]);
      }
      __syncthreads();
    }
    float cs[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const long long row = m0 + ty * 4 + i;
      if (row < n) {
        const float tt = t[row];
#pragma unroll
        for (int j = 0; j < 4; ++j) cs[j] += pattern_error(tt, acc[i][j] + bias[j], act, err, R);
      }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) red[ty][tx * 4 + j] = cs[j];
    __syncthreads();
    if (tid < 64) {
      double s = 0.0;
      for (int r = 0; r < 16; ++r) s += (double)red[r][tid];
      acc64[tid] += s;
    }
    __syncthreads();
  }
  if (tid < 64) partial[(long long)blockIdx.x * pop_pad + c0 + tid] = acc64[tid];
}

__global__ void noalloc_reduce_kernel(const double* partial, int n_part, int pop, int pop_pad,
                                      double inv_n, int err, double* fitness) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= pop) return;
  const double sse = sum_partials(partial, n_part, pop_pad, c);
  const double mse = sse * inv_n;
  fitness[c] = err == GAME_RMSE ? sqrt(mse) : mse;
}

}  // namespace

void set_global_error(const char* msg);   // api.cu

}  // namespace game

using namespace game;

extern "C" game_status game_fitness_noalloc(const float* P, const float* t, const float* G,
                                            int64_t n_patterns, int32_t n_genes, int32_t pop,
                                            int32_t error, int32_t activation, float tmse_R,
                                            double* fitness, void* stream) {
  if (!P || !t || !G || !fitness) {
    set_global_error("game_fitness_noalloc: P, t, G and fitness must be device pointers");
    return GAME_ERR_INVALID_ARG;
  }
  if (n_patterns < 1 || n_genes < 1 || pop < 1) {
    set_global_error("game_fitness_noalloc: need n_patterns >= 1, n_genes >= 1, pop >= 1");
    return GAME_ERR_INVALID_ARG;
  }
  if (pop > kMaxPop) {
    set_global_error("game_fitness_noalloc: pop exceeds the fixed scratch limit of 4096");
    return GAME_ERR_UNSUPPORTED;
  }
  if (error < GAME_RMSE || error > GAME_TMSE_SQ || (activation != GAME_TANH && activation != GAME_LINEAR) ||
      ((error == GAME_TMSE || error == GAME_TMSE_SQ) && !(tmse_R > 0.0f && tmse_R < 1.0f))) {
    set_global_error("game_fitness_noalloc: bad error / activation / tmse_R");
    return GAME_ERR_INVALID_ARG;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    set_global_error("game_fitness_noalloc: no current CUDA device");
    return GAME_ERR_NO_DEVICE;
  }
  double* partial = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_partial_addr[dev]) {
      void* addr = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&addr, g_noalloc_partial);
      if (e != cudaSuccess || !addr) {
        set_global_error("game_fitness_noalloc: cudaGetSymbolAddress of the scratch array failed");
        return GAME_ERR_CUDA;
      }
      g_partial_addr[dev] = static_cast<double*>(addr);
    }
    partial = g_partial_addr[dev];
  }
  const int pop_pad = (pop + 63) / 64 * 64;
  long long tiles = (n_patterns + 63) / 64;
  const int n_part = (int)(tiles < kParts ? tiles : kParts);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  noalloc_fitness_kernel<<<dim3(n_part, pop_pad / 64), 256, 0, st>>>(
      P, t, G, n_patterns, n_genes - 1, n_genes, pop, activation, error, tmse_R, partial, pop_pad);
  noalloc_reduce_kernel<<<(pop + 127) / 128, 128, 0, st>>>(partial, n_part, pop, pop_pad,
                                                           1.0 / (double)n_patterns, error, fitness);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_global_error(cudaGetErrorString(e));
    return GAME_ERR_CUDA;
  }
  return GAME_OK;
}
