// Learned fitness surrogate: MLP D -> 256 -> 256 -> 1 with GELU, its online
// training (float32 master weights, bfloat16 GEMM copies, Adam) and the kernels
// that use it to pre-screen an oversized offspring pool.
#pragma once

#include "game_internal.h"

namespace game {

// GELU in the erf form, z Phi(z), and its derivative Phi(z) + z phi(z).
__device__ __forceinline__ float gelu_f(float z) {
  return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f));
}
__device__ __forceinline__ float gelu_grad_f(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) +
         z * expf(-0.5f * z * z) * 0.39894228040143268f;
}
// Both at once with one erf: g = z Phi(z), d = Phi(z) + z phi(z) (the same
// roundings as gelu_f and gelu_grad_f, since halving is exact).
__device__ __forceinline__ void gelu_and_grad_f(float z, float& g, float& d) {
  const float c = 0.5f * (1.0f + erff(z * 0.70710678118654752f));
  g = z * c;
  d = c + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

struct Surrogate {
  int D = 0;                 // input width (genes per chromosome)
  int H = 256;               // hidden width
  bool bf16 = true;          // GEMMs read bfloat16 weight copies
  int max_rows = 0;          // rows of the activation workspaces
  float* p = nullptr;        // flat parameters [W1 (HxD) | b1 | W2 (HxH) | b2 | w3 | b3]
  float* g = nullptr;        // gradients, same layout
  float* m = nullptr;        // Adam first moments
  float* v = nullptr;        // Adam second moments
  __nv_bfloat16* ph = nullptr;   // bfloat16 copy of p
  int* step = nullptr;       // Adam step counter (device)
  float *Z1 = nullptr, *H1 = nullptr, *Z2 = nullptr, *H2 = nullptr;   // [max_rows x H]
  float *dZ1 = nullptr, *dZ2 = nullptr;                              // [max_rows x H]
  float *yb = nullptr, *dy = nullptr, *sq = nullptr;                 // [max_rows]
  float* loss = nullptr;     // last training loss (device scalar)
  float* ws = nullptr;       // split-K partial planes [16 x H x max(D, H)]

  // Tensor-core path (bfloat16 weights; surrogate_tc.cu): bf16 GEMM operands,
  // K-major, with transposed copies for the weight gradients.
  bool tc = false;
  int Dp = 0;                // D rounded up to 8 (16-byte rows)
  int Bt = 0;                // training batch capacity
  long long ldt = 0;         // row stride of the transposed operands (Bt rounded up to 8)
  __nv_bfloat16 *W1b = nullptr, *W2b = nullptr, *W2Tb = nullptr;   // [H x Dp], [H x H], W2^T
  __nv_bfloat16 *Xb = nullptr, *H1b = nullptr;                    // [max_rows x Dp], [max_rows x H]
  __nv_bfloat16 *XTb = nullptr;    // [(D + 1) x ldt], last row ones
  __nv_bfloat16 *H1Tb = nullptr;   // [(H + 1) x ldt], last row ones
  __nv_bfloat16 *dZ2Tb = nullptr, *dZ1Tb = nullptr;   // [H x ldt]
  __nv_bfloat16 *dZ2b = nullptr;   // [Bt x H]
  float *gp1 = nullptr;            // gelu'(Z1) [Bt x H]
  float *dyh2 = nullptr;           // dy * H2 [Bt x H]
  float *gws = nullptr;            // split-K partial gradient planes [4 x n_params]
  unsigned int* adam_done = nullptr;   // blocks finished in the current Adam launch
  float* gnorm = nullptr;          // input standardisation [shift D | scale D | var D]
  DevState* state = nullptr;       // where a timed-out wait records its status

  size_t n_params() const;
  void views(float* base, float** W1, float** b1, float** W2, float** b2, float** w3,
             float** b3) const;
  // y[m] for the M rows of X (row stride ldx floats, first D columns used).
  cudaError_t forward(const float* X, long long ldx, int M, float* y, cudaStream_t st);
  // gradients of mean((y - t)^2) over B <= max_rows rows into g; loss into *loss.
  cudaError_t backward(const float* X, long long ldx, int B, const float* t, cudaStream_t st);
  cudaError_t adam(float lr, cudaStream_t st);
  cudaError_t refresh(cudaStream_t st);     // bfloat16 copy of p

  // bytes of the tensor-core buffers, their layout in one allocation, and the
  // constant parts (rows of ones, weight copies)
  size_t tc_bytes(int max_rows_, int batch) const;
  void tc_carve(void* base, int batch);
  cudaError_t tc_prepare(cudaStream_t st);
  cudaError_t tc_weights(cudaStream_t st);
  // forward of M rows; with targets t (M <= Bt) also the operands of the backward pass
  cudaError_t tc_forward(const float* X, long long ldx, int M, float* y, const float* t,
                         cudaStream_t st);
  // the same from rows already in Xb (and X^T when training)
  cudaError_t tc_layers(int M, float* y, const float* t, cudaStream_t st);
  // one training step on the B rows in Xb / X^T with targets t: gradients, Adam
  cudaError_t tc_train_step(int B, const float* t, float lr, cudaStream_t st);
  // dZ1^T, [gW2 | gb2] and [gW1 | gb1] of the batch just run forward with targets,
  // as split-K planes in gws, added into g when sum_planes
  cudaError_t tc_backward_gemms(int B, cudaStream_t st, bool sum_planes = true);
  // its three GEMMs: dZ1^T (needs dZ2), then [gW1 | gb1]; [gW2 | gb2] (needs dZ2 only)
  cudaError_t tc_backward_b1(int B, cudaStream_t st);
  cudaError_t tc_grad_w1(int B, cudaStream_t st);
  cudaError_t tc_grad_w2(int B, cudaStream_t st);
  // gw3, gb3 and the loss of that batch
  cudaError_t tc_out_grads(int B, cudaStream_t st);
  // Adam step that also refreshes the bf16 GEMM copies and the step counter; with
  // from_planes it adds the split-K planes of the last tc_backward_gemms itself
  cudaError_t tc_adam(float lr, cudaStream_t st, bool from_planes = false);
  int grad_splits = 0;       // split-K planes written by the last tc_backward_gemms
  // Optional second stream and events (owned by the caller): a training step runs the
  // W2 gradient and the output-layer gradients beside dZ1 and the W1 gradient.
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

cudaError_t surrogate_tc_init_attributes();

// Kernels of the surrogate-driven generation (surrogate_ga.cu).
struct PoolArgs {
  const float* g32_0;
  const float* g32_1;
  float* pool;              // [n_pool x kstride] children
  const double* fit;
  const int* rank;
  const unsigned long long* cum;   // roulette / ranking cumulative weights, or nullptr
  DevState* state;
  uint64_t k0, k1;
  int pop, n_genes, kstride, n_pool, tournament_k, clamp;
  float p_c, p_m, sigma;
};
cudaError_t launch_pool_breed(const PoolArgs& a, cudaStream_t st);
// Selects n_sel pool rows with the lowest score (ties: lower index), or the first
// n_sel rows when random_select (or when the monitor switched to the fallback);
// records whether this generation breeds (bred).
cudaError_t launch_select(const float* score, int n_pool, int n_sel, int* sel, DevState* state,
                          const int* fallback, int random_select, cudaStream_t st);
// Next population: elites of the current one, then the selected pool rows; the
// surrogate's score of each selected row goes to pred (NaN for elites).
cudaError_t launch_assemble(const float* pool, const int* sel, const float* score, const PopDev& p,
                            const Shape& s, int elitism, int elite_copies, const int* rank,
                            const DevState* state, float* pred, cudaStream_t st);
// Monitor (Spearman of predicted vs exact over the non-elite rows; dsq [pop]
// holds the squared rank differences), then the
// evaluated population appended to the replay ring with its log fitness
// standardised within the generation (mean / std over that population).
cudaError_t launch_replay_update(const PopDev& p, const Shape& s, int elitism, const double* fit,
                                 const float* pred, DevState* state, float* ring_x,
                                 float* ring_f, int* ring_meta, int ring_cap, float* norm,
                                 double* monitor, int* fallback, float fallback_rho,
                                 long long* dsq, cudaStream_t st);
// Draws a training batch from the ring (Philox) and standardises its targets.
cudaError_t launch_sample_batch(const float* ring_x, const float* ring_f, const int* ring_meta,
                                int kstride, int n_genes, const float* norm, int B, uint64_t k0,
                                uint64_t k1, uint64_t gen_salt, int step, const DevState* state,
                                float* bx, float* bt, cudaStream_t st);
// The same batch written straight into the bf16 operands Xb and X^T of the
// tensor-core path (sg.tc); targets to bt.
// Running per-gene mean / variance of the evaluated populations (exponential
// average) that standardise the network's inputs in the bf16 form.
cudaError_t launch_gene_stats(const PopDev& p, const Shape& s, const DevState* state,
                              const int* ring_meta, Surrogate& sg, cudaStream_t st);
cudaError_t launch_sample_batch_tc(const float* ring_x, const float* ring_f, const int* ring_meta,
                                   int kstride, const Surrogate& sg, int B, uint64_t k0,
                                   uint64_t k1, uint64_t gen_salt, int step, const DevState* state,
                                   float* bt, cudaStream_t st);
cudaError_t surrogate_ga_init_attributes();
cudaError_t launch_surrogate_init(Surrogate& sg, uint64_t seed, cudaStream_t st);

}  // namespace game
