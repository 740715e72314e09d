// Tensor-core (tcgen05 / TMEM / TMA) fitness engine: plan and launch.
#pragma once

#include <cuda.h>

#include <vector>

#include "game_internal.h"

namespace game {

struct TcPlan {
  CUtensorMap a_map[2];   // gene planes (hi, lo): A operand, chromosomes x genes
  CUtensorMap b_map[2];   // expansion planes (FP32: hi, lo; BF16/FP8: one): B operand
  int n_slices;           // 128-chromosome slices of the population
  int ctas_per_slice;     // CTAs that share one slice (each takes every n-th pattern tile)
  int n_tiles;            // pattern tiles of BN rows over the training rows
  int grid;               // n_slices * ctas_per_slice
  int n_part;             // partial-sum rows written (= ctas_per_slice)
  int bn;                 // patterns per tile (MMA N)
  int kblocks;            // k-blocks of 128 bytes over kp
  int stages;             // B-operand pipeline depth
  int cluster;            // CTAs (one per slice) sharing each B tile by TMA multicast
  size_t smem;            // dynamic shared memory bytes
};

// Requested tile shape; 0 fields are chosen automatically.
struct TileReq {
  int n = 0, stages = 0, cluster = 0;
};

bool tc_supported(const Shape& s);
cudaError_t tc_plan(const Shape& s, const ExpDev& e, const PopDev& p, int n_sm, TcPlan* plan,
                    TileReq req = TileReq{});
// Every valid explicit tile shape for this problem (for the autotuner).
void tc_candidates(const Shape& s, std::vector<TileReq>* out);
cudaError_t tc_launch(const TcPlan& plan, const Shape& s, const Fitness& f, const PopDev& p,
                      const ExpDev& e, double* partial, const DevState* state, cudaStream_t st);
cudaError_t tc_init_attributes();

}  // namespace game
