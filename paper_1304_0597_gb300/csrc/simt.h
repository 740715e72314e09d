// Arguments shared by the CUDA-core fitness kernels (fitness_simt.cu, the tiled
// SIMT kernel; fitness_narrow.cu, the stream over P for populations of at most
// 32) and the narrow kernel's host entry points.
#pragma once

#include "game_internal.h"

namespace game {

struct SimtArgs {
  const void* p0;        // P plane(s) of the training rows, row-major [m x kp]:
  const void* p1;        // FP32 = fp16 hi (p0) and lo (p1); BF16 / FP8 = p0 only
  const float* colscale;
  const float* t;
  const float* geval;
  const float* bias;
  const void* ghi;      // FP32 gene planes of prepare_kernel: fp16 hi / lo [pop_pad x kp],
  const void* glo;      // g * s_col / r_c (the narrow warp-MMA kernel's B operand)
  const float* rscale;  // r_c, the per-chromosome power of two of those planes
  double* partial;
  const DevState* state;   // the stop flag, read only inside game_evolve (else null)
  DevState* dev_state;     // where a timed-out wait records GAME_ERR_TIMEOUT
  long long m;          // training rows
  int kb, kp, pop, pop_pad, act, err, in_evolve;
  float R;
};

// The narrow kernel takes pop <= 32 with 16 or 32 stored columns.
bool narrow_shape_ok(int pop, int kp);
int narrow_partials(const Shape& s, int n_sm);   // CTAs = partial-sum rows
cudaError_t launch_narrow(const SimtArgs& a, const Shape& s, int grid, cudaStream_t st);

}  // namespace game
