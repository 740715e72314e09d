// Learned surrogate of the fitness (no paper counterpart): an MLP
//   y = w3 . gelu(W2 gelu(W1 g + b1) + b2) + b3,  D -> 256 -> 256 -> 1,
// mapping a chromosome's genes g to its standardised log fitness.  It is
// trained online on the (chromosome, exact fitness) pairs that each generation
// evaluates, and pre-screens an oversized offspring pool: only the children it
// ranks best go on to exact evaluation, which keeps measuring its error
// (Spearman correlation per generation) and is the fallback (plain selection
// when the correlation drops).
//
// Weights live in float32 (master, Adam moments) with bfloat16 copies that the
// forward and backward GEMMs read (float32 accumulation); a float32-weight mode
// exists for gradient checks.  Every reduction over the batch is a fixed-order
// sum, so training is deterministic.
#include "surrogate.h"

#include <math_constants.h>

namespace game {

namespace {

// C[m, n] (=|+=) sum_k A(m, k) * B(k, n), A(m, k) = A[m * am + k * ak],
// B(k, n) = B[k * bk + n * bn].  BW: B is bfloat16.  EPI: 0 plain store,
// 1 store z = acc + bias[n] and h = gelu(z), 2 acc * gelu'(zaux[m, n]).
template <bool BW, int EPI>
__global__ void __launch_bounds__(256) gemm_kernel(const float* __restrict__ A, long long am,
                                                   long long ak, const void* __restrict__ Bv,
                                                   long long bk, long long bn, int M, int N, int K,
                                                   const float* __restrict__ bias,
                                                   float* __restrict__ C, float* __restrict__ H,
                                                   const float* __restrict__ zaux, long long ldc,
                                                   int kc, long long zstride) {
  __shared__ float As[64][17];
  __shared__ float Bs[16][65];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  float acc[4][4] = {};
  // split-K: this CTA covers k in [k_lo, k_hi) and writes its own partial plane
  const int k_lo = blockIdx.z * kc;
  const int k_hi = min(K, k_lo + kc);
  C += blockIdx.z * zstride;
  for (int k0 = k_lo; k0 < k_hi; k0 += 16) {
    for (int i = tid; i < 64 * 16; i += 256) {
      const int r = i >> 4, kk = i & 15;
      const int m = m0 + r, k = k0 + kk;
      As[r][kk] = (m < M && k < k_hi) ? A[m * am + k * ak] : 0.0f;
      const int kb = i >> 6, nn = i & 63;
      const int k2 = k0 + kb, n = n0 + nn;
      float bv = 0.0f;
      if (k2 < k_hi && n < N) {
        const long long o = k2 * bk + n * bn;
        bv = BW ? __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(Bv)[o])
                : reinterpret_cast<const float*>(Bv)[o];
      }
      Bs[kb][nn] = bv;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[ty * 4 + i][kk];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty * 4 + i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx * 4 + j;
      if (n >= N) continue;
      const long long o = m * ldc + n;
      if (EPI == 1) {
        const float z = acc[i][j] + bias[n];
        C[o] = z;
        H[o] = gelu_f(z);
      } else if (EPI == 2) {
        C[o] = acc[i][j] * gelu_grad_f(zaux[o]);
      } else {
        C[o] = acc[i][j];
      }
    }
  }
}

template <bool BW, int EPI>
void gemm(cudaStream_t st, const float* A, long long am, long long ak, const void* B, long long bk,
          long long bn, int M, int N, int K, const float* bias, float* C, float* H,
          const float* zaux, long long ldc) {
  dim3 grid((N + 63) / 64, (M + 63) / 64);
  gemm_kernel<BW, EPI><<<grid, 256, 0, st>>>(A, am, ak, B, bk, bn, M, N, K, bias, C, H, zaux, ldc,
                                             K, 0);
}

// out[i] = sum_z ws[z * n + i], z = 0..splits-1 in order (deterministic).
__global__ void splitk_sum_kernel(const float* __restrict__ ws, int splits, long long n,
                                  float* __restrict__ out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float s = 0.0f;
  for (int z = 0; z < splits; ++z) s += ws[z * n + i];
  out[i] = s;
}

// Weight gradients (output M x N small, K = batch rows): split K over CTAs, then
// add the partial planes in a fixed order.
void gemm_splitk(cudaStream_t st, const float* A, long long am, long long ak, const float* B,
                 long long bk, long long bn, int M, int N, int K, float* C, float* ws, int splits) {
  const int kc = ((K + splits - 1) / splits + 15) / 16 * 16;
  const int z = (K + kc - 1) / kc;
  dim3 grid((N + 63) / 64, (M + 63) / 64, z);
  gemm_kernel<false, 0><<<grid, 256, 0, st>>>(A, am, ak, B, bk, bn, M, N, K, nullptr, ws, nullptr,
                                              nullptr, N, kc, (long long)M * N);
  const long long n = (long long)M * N;
  splitk_sum_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(ws, z, n, C);
}

// Output layer y[m] = sum_n H2[m, n] w3[n] + b3 (one warp per row).
template <bool BW>
__global__ void out_layer_kernel(const float* __restrict__ H2, const void* __restrict__ w3v,
                                 const float* __restrict__ b3, int M, int Hd, float* __restrict__ y) {
  const int row = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= M) return;
  float s = 0.0f;
  for (int n = lane; n < Hd; n += 32) {
    const float w = BW ? __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(w3v)[n])
                       : reinterpret_cast<const float*>(w3v)[n];
    s = fmaf(H2[(long long)row * Hd + n], w, s);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) y[row] = s + b3[0];
}

// dy = 2 (y - t) / B; dZ2 = dy w3 * gelu'(Z2); per-row loss terms.
template <bool BW>
__global__ void out_back_kernel(const float* __restrict__ y, const float* __restrict__ t,
                                const void* __restrict__ w3v, const float* __restrict__ Z2, int B,
                                int Hd, float* __restrict__ dy, float* __restrict__ dZ2,
                                float* __restrict__ sq) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)B * Hd) return;
  const int b = (int)(i / Hd), n = (int)(i % Hd);
  const float e = y[b] - t[b];
  const float d = 2.0f * e / (float)B;
  const float w = BW ? __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(w3v)[n])
                     : reinterpret_cast<const float*>(w3v)[n];
  dZ2[i] = d * w * gelu_grad_f(Z2[i]);
  if (n == 0) {
    dy[b] = d;
    sq[b] = e * e;
  }
}

// out[n] = sum_b X[b * ld + n]: one CTA per column, strided partial sums and a
// fixed tree (deterministic).
__global__ void colsum_kernel(const float* __restrict__ X, int B, int N, long long ld,
                              float* __restrict__ out) {
  __shared__ float red[256];
  const int n = blockIdx.x;
  float s = 0.0f;
  for (int b = threadIdx.x; b < B; b += blockDim.x) s += X[(long long)b * ld + n];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[n] = red[0];
}

// Adam (Kingma & Ba 2015) over the flat parameter vector; refreshes the bf16 copies.
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v,
                            __nv_bfloat16* __restrict__ ph, long long n, const int* __restrict__ step,
                            float lr, float beta1, float beta2, float eps) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int t = *step + 1;
  const float gi = g[i];
  const float mi = beta1 * m[i] + (1.0f - beta1) * gi;
  const float vi = beta2 * v[i] + (1.0f - beta2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float mh = mi / (1.0f - powf(beta1, (float)t));
  const float vh = vi / (1.0f - powf(beta2, (float)t));
  const float pi = p[i] - lr * mh / (sqrtf(vh) + eps);
  p[i] = pi;
  ph[i] = __float2bfloat16_rn(pi);
}

__global__ void step_inc_kernel(int* step) { *step += 1; }

__global__ void refresh_bf16_kernel(const float* __restrict__ p, __nv_bfloat16* __restrict__ ph,
                                    long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) ph[i] = __float2bfloat16_rn(p[i]);
}

__global__ void loss_kernel(const float* __restrict__ sq, int B, float* __restrict__ loss) {
  __shared__ float red[256];
  float s = 0.0f;
  for (int b = threadIdx.x; b < B; b += blockDim.x) s += sq[b];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = red[0] / (float)B;
}

}  // namespace

// ---------------------------------------------------------------------------

size_t Surrogate::n_params() const { return (size_t)H * D + H + (size_t)H * H + H + H + 1; }

void Surrogate::views(float* base, float** W1, float** b1, float** W2, float** b2, float** w3,
                      float** b3) const {
  *W1 = base;
  *b1 = *W1 + (size_t)H * D;
  *W2 = *b1 + H;
  *b2 = *W2 + (size_t)H * H;
  *w3 = *b2 + H;
  *b3 = *w3 + H;
}

cudaError_t Surrogate::forward(const float* X, long long ldx, int M, float* y, cudaStream_t st) {
  if (tc) {
    for (int m0 = 0; m0 < M; m0 += max_rows) {
      const int mm = M - m0 < max_rows ? M - m0 : max_rows;
      cudaError_t e = tc_forward(X + (long long)m0 * ldx, ldx, mm, y + m0, nullptr, st);
      if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
  }
  float *W1, *b1, *W2, *b2, *w3, *b3;
  views(p, &W1, &b1, &W2, &b2, &w3, &b3);
  const void* pw1 = bf16 ? (const void*)(ph) : (const void*)W1;
  const void* pw2 = bf16 ? (const void*)(ph + ((size_t)H * D + H)) : (const void*)W2;
  const void* pw3 = bf16 ? (const void*)(ph + ((size_t)H * D + H + (size_t)H * H + H)) : (const void*)w3;
  for (int m0 = 0; m0 < M; m0 += max_rows) {
    const int mm = M - m0 < max_rows ? M - m0 : max_rows;
    const float* Xm = X + (long long)m0 * ldx;
    // Z1 = X W1^T + b1 : B(k, n) = W1[n * D + k]
    if (bf16)
      gemm<true, 1>(st, Xm, ldx, 1, pw1, 1, D, mm, H, D, b1, Z1, H1, nullptr, H);
    else
      gemm<false, 1>(st, Xm, ldx, 1, pw1, 1, D, mm, H, D, b1, Z1, H1, nullptr, H);
    if (bf16)
      gemm<true, 1>(st, H1, H, 1, pw2, 1, H, mm, H, H, b2, Z2, H2, nullptr, H);
    else
      gemm<false, 1>(st, H1, H, 1, pw2, 1, H, mm, H, H, b2, Z2, H2, nullptr, H);
    if (bf16)
      out_layer_kernel<true><<<(mm * 32 + 255) / 256, 256, 0, st>>>(H2, pw3, b3, mm, H, y + m0);
    else
      out_layer_kernel<false><<<(mm * 32 + 255) / 256, 256, 0, st>>>(H2, pw3, b3, mm, H, y + m0);
  }
  return cudaGetLastError();
}

cudaError_t Surrogate::backward(const float* X, long long ldx, int B, const float* t,
                                cudaStream_t st) {
  if (tc) {
    cudaError_t e = tc_forward(X, ldx, B, yb, t, st);
    if (e != cudaSuccess) return e;
    if ((e = tc_out_grads(B, st)) != cudaSuccess) return e;
    e = tc_backward_gemms(B, st);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
  }
  // forward of the batch keeps Z1, H1, Z2, H2, y (B <= max_rows)
  cudaError_t e = forward(X, ldx, B, yb, st);
  if (e != cudaSuccess) return e;
  float *W1, *b1, *W2, *b2, *w3, *b3;
  views(p, &W1, &b1, &W2, &b2, &w3, &b3);
  float *gW1, *gb1, *gW2, *gb2, *gw3, *gb3;
  views(g, &gW1, &gb1, &gW2, &gb2, &gw3, &gb3);
  const void* pw2 = bf16 ? (const void*)(ph + ((size_t)H * D + H)) : (const void*)W2;
  const void* pw3 = bf16 ? (const void*)(ph + ((size_t)H * D + H + (size_t)H * H + H)) : (const void*)w3;
  const long long n = (long long)B * H;
  if (bf16)
    out_back_kernel<true><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(yb, t, pw3, Z2, B, H, dy, dZ2, sq);
  else
    out_back_kernel<false><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(yb, t, pw3, Z2, B, H, dy, dZ2, sq);
  loss_kernel<<<1, 256, 0, st>>>(sq, B, loss);
  // gw3[n] = sum_b dy[b] H2[b, n];  gb3 = sum_b dy[b]
  gemm_splitk(st, dy, 0, 1, H2, H, 1, 1, H, B, gw3, ws, 16);
  colsum_kernel<<<1, 256, 0, st>>>(dy, B, 1, 1, gb3);
  // gW2[i, j] = sum_b dZ2[b, i] H1[b, j]; gb2 = colsum(dZ2)
  gemm_splitk(st, dZ2, 1, H, H1, H, 1, H, H, B, gW2, ws, 16);
  colsum_kernel<<<H, 256, 0, st>>>(dZ2, B, H, H, gb2);
  // dZ1 = (dZ2 W2) * gelu'(Z1): B(k, n) = W2[k * H + n]
  if (bf16)
    gemm<true, 2>(st, dZ2, H, 1, pw2, H, 1, B, H, H, nullptr, dZ1, nullptr, Z1, H);
  else
    gemm<false, 2>(st, dZ2, H, 1, pw2, H, 1, B, H, H, nullptr, dZ1, nullptr, Z1, H);
  // gW1[i, k] = sum_b dZ1[b, i] X[b, k]; gb1 = colsum(dZ1)
  gemm_splitk(st, dZ1, 1, H, X, ldx, 1, H, D, B, gW1, ws, 16);
  colsum_kernel<<<H, 256, 0, st>>>(dZ1, B, H, H, gb1);
  return cudaGetLastError();
}

cudaError_t Surrogate::adam(float lr, cudaStream_t st) {
  if (tc) return tc_adam(lr, st);
  const long long n = (long long)n_params();
  adam_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(p, g, m, v, ph, n, step, lr, 0.9f,
                                                            0.999f, 1e-8f);
  step_inc_kernel<<<1, 1, 0, st>>>(step);
  return cudaGetLastError();
}

cudaError_t Surrogate::refresh(cudaStream_t st) {
  const long long n = (long long)n_params();
  refresh_bf16_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(p, ph, n);
  if (tc) return tc_weights(st);
  return cudaGetLastError();
}

}  // namespace game
