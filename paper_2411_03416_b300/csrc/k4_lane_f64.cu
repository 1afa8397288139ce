// State dimension 4, lane form (sixteen lanes per plan): fused iterations, FP64 throughout.
#include "pgvimp_lane.cuh"

namespace pgv {
template cudaError_t launch_iter_lane<double, double>(const Launch& L, int iters);
}  // namespace pgv
