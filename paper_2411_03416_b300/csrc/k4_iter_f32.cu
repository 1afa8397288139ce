// State dimension 4: fused iterations, FP32 quadrature, FP64 recursions.
#include "pgvimp_kernels.cuh"

namespace pgv {
template cudaError_t launch_iter<4, float, double>(const Launch& L, int iters);
}  // namespace pgv
