// Fused proximal iterations, state dimension 4, FP64 quadrature.
#include "pgvimp_kernels.cuh"

namespace pgv {
template cudaError_t launch_iter<4, double>(const Launch& L, int iters);
}  // namespace pgv
