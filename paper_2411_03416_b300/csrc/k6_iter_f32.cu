// Fused proximal iterations, state dimension 6, FP32 quadrature.
#include "pgvimp_kernels.cuh"

namespace pgv {
template cudaError_t launch_iter<6, float>(const Launch& L, int iters);
}  // namespace pgv
