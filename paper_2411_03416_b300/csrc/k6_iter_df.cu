// State dimension 6: fused iterations, FP32 quadrature, double-float recursions.
#include "pgvimp_kernels.cuh"

namespace pgv {
template cudaError_t launch_iter<6, float, df64>(const Launch& L, int iters);
}  // namespace pgv
