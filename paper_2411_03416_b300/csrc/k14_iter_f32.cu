// Fused proximal iterations, state dimension 14, FP32 quadrature.
#include "pgvimp_kernels.cuh"

namespace pgv {
template cudaError_t launch_iter<14, float>(const Launch& L, int iters);
}  // namespace pgv
