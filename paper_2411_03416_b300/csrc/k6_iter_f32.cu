// State dimension 6: fused iterations, FP32 quadrature, FP64 recursions.
#include "pgvimp_kernels.cuh"

namespace pgv {
template cudaError_t launch_iter<6, float, double>(const Launch& L, int iters);
}  // namespace pgv
