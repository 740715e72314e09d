#include "fitness_tc.h"
namespace game {
bool tc_supported(const Shape&) { return false; }
cudaError_t tc_plan(const Shape&, const ExpDev&, const PopDev&, int, TcPlan*) { return cudaErrorNotSupported; }
cudaError_t tc_launch(const TcPlan&, const Shape&, const Fitness&, const PopDev&, const ExpDev&, double*, const DevState*, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t tc_init_attributes() { return cudaSuccess; }
}
