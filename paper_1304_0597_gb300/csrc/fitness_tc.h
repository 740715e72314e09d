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
  int sp = 1;             // slices per CTA (2: both fed by every 128-pattern tile)
  int n_groups;           // n_slices / sp
  int ctas_per_slice;     // CTAs that share one group (each takes every n-th pattern tile)
  int n_tiles;            // pattern tiles of BN rows over the training rows
  int grid;               // n_groups * ctas_per_slice
  int n_part;             // partial-sum rows written (= ctas_per_slice)
  int bn;                 // patterns per tile (MMA N)
  int kblocks;            // k-blocks of 128 bytes over kp
  int stages;             // B-operand pipeline depth
  int cluster;            // 1, or 2: CTA pairs sharing each MMA (cta_group::2, M = 256)
  int prefetch = 1;       // L2 prefetch of each CTA's next pattern tile
  int kg = 1;             // 128-byte k-blocks per stage (> 1: one 3-D TMA request each)
  int a_rows = 128;       // gene rows per resident A tile (fewer for one small slice)
  size_t smem;            // dynamic shared memory bytes
  int narrow = 0;         // 1: the swapped kernel (patterns on M, <= 32 chromosomes on N)
};

// Requested tile shape; 0 fields are chosen automatically.
struct TileReq {
  int n = 0, stages = 0, cluster = 0, prefetch = -1;   // prefetch: -1 auto (on), 0 off, 1 on
  int sp = 0;                                          // slices per CTA: 0 auto (1), 1, 2
  int kg = 0;                                          // k-blocks per stage: 0 auto (1), 1, 2
};

bool tc_supported(const Shape& s);
cudaError_t tc_plan(const Shape& s, const ExpDev& e, const PopDev& p, int n_sm, TcPlan* plan,
                    TileReq req = TileReq{});
// Every valid explicit tile shape for this problem (for the autotuner).
void tc_candidates(const Shape& s, std::vector<TileReq>* out);
cudaError_t tc_launch(const TcPlan& plan, const Shape& s, const Fitness& f, const PopDev& p,
                      const ExpDev& e, double* partial, const DevState* state, cudaStream_t st);
cudaError_t tc_init_attributes();

// Narrow populations in the FP32 form (at most 32 chromosomes): the swapped
// kernel of fitness_tc_narrow.cu.  tc_narrow_fits: the kernel can take the shape;
// tc_narrow_shape: it fits and the shape is marked for it (Shape::tc_narrow), in
// which case tc_plan / tc_candidates / tc_launch route to it.
bool tc_narrow_fits(const Shape& s);
bool tc_narrow_shape(const Shape& s);
void tc_narrow_candidates(const Shape& s, std::vector<TileReq>* out);
cudaError_t tc_narrow_plan(const Shape& s, const ExpDev& e, const PopDev& p, int n_sm,
                           TcPlan* plan, TileReq req);
cudaError_t tc_narrow_launch(const TcPlan& t, const Shape& s, const Fitness& f, const PopDev& pd,
                             const ExpDev& e, double* partial, const DevState* state,
                             cudaStream_t st);
cudaError_t tc_narrow_init_attributes();
// Tensor map of a K-major operand plane [rows x cols] in the storage type of
// `precision`, 128-byte rows per box, 128-byte swizzle, box of box_rows rows.
cudaError_t tc_timeout_selftest(DevState* st, unsigned long long wait_ns, int* out, cudaStream_t s);
cudaError_t tc_make_map(CUtensorMap* m, const void* base, int precision, long long rows, int cols,
                        int box_rows);

// ---- on-the-fly tensor-core engine (fitness_tc_otf.cu) ------------------------
// The FP32 form with per-feature coefficients: expansion warps form each k-block of P
// in shared memory from X, the MMA warp contracts it with the resident gene planes.
struct OtfTcPlan {
  CUtensorMap a_map[2];   // gene planes (hi, lo)
  int kblocks = 0, stages = 0, cps = 0, grid = 0, n_tiles = 0;
  size_t smem = 0;
};
bool otf_tc_supported(const Shape& s);
cudaError_t otf_tc_plan(const Shape& s, const PopDev& p, int n_sm, OtfTcPlan* plan);
// dev_state: the context's device state (timeouts are recorded there; with in_evolve
// the launch returns at once once the run has stopped); partial rows [plan.cps x pop_pad]
cudaError_t otf_tc_launch(const OtfTcPlan& t, const Shape& s, const Fitness& f, const PopDev& p,
                          const ExpDev& e, const float* X, double* partial, DevState* dev_state,
                          int in_evolve, cudaStream_t st);
cudaError_t otf_tc_init_attributes();

// ---- batched form: many runs in one persistent grouped launch ----------------

// Everything the grouped kernel needs about one run (device-resident; the tensor
// maps must stay 64-byte aligned).
struct alignas(64) BatchRunDev {
  CUtensorMap a[2];       // gene planes (hi, lo)
  CUtensorMap b[2];       // expansion planes
  const float* pk;        // per-pattern epilogue input (2 log2(e) t when fast == 1, else t)
  const float* bias;
  const float* rscale;
  double* partial;        // [n_chunks * 4 x pop_pad]
  const DevState* state;
  long long m;
  int pop_pad, kblocks, ksteps, n_bplanes, n_aplanes, prec;
  int fast;               // 0 general error, 1 exact fast form (FP32), 2 tanh form (BF16 / FP8)
  int act, err;
  float R;
};

// One unit of work: a slice of one run over tiles [tile0, tile1); chunk = its
// index among the slice's items (partial rows chunk*4 .. chunk*4+3).
struct WorkItem {
  int run, slice, tile0, tile1, chunk;
};

cudaError_t batch_init_attributes();
int batch_stages();
size_t batch_smem_bytes();
int batch_tile_rows();
cudaError_t batch_make_run(const Shape& s, const Fitness& f, const PopDev& p, const ExpDev& e,
                           double* partial, const DevState* state, BatchRunDev* out);
cudaError_t batch_fitness_launch(const BatchRunDev* d_runs, const WorkItem* d_items,
                                 const int* d_item_off, int grid, int in_evolve, cudaStream_t st);

}  // namespace game
