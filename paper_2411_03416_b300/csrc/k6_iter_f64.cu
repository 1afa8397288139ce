// Fused proximal iterations, state dimension 6, FP64 quadrature.
#include "pgvimp_kernels.cuh"

namespace pgv {
template cudaError_t launch_iter<6, double>(const Launch& L, int iters);
}  // namespace pgv
