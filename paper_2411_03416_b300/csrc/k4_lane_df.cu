// State dimension 4, lane form (sixteen lanes per plan): fused iterations, double-float recursions.
#include "pgvimp_lane.cuh"

namespace pgv {
template cudaError_t launch_iter_lane<float, df64>(const Launch& L, int iters);
}  // namespace pgv
