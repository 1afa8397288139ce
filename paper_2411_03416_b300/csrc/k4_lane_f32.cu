// State dimension 4, lane form (sixteen lanes per plan): fused iterations, FP64 recursions.
#include "pgvimp_lane.cuh"

namespace pgv {
template cudaError_t launch_iter_lane<float, double>(const Launch& L, int iters);
}  // namespace pgv
