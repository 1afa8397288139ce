// Fused proximal iterations, state dimension 14, FP64 quadrature.
#include "pgvimp_kernels.cuh"

namespace pgv {
template cudaError_t launch_iter<14, double>(const Launch& L, int iters);
}  // namespace pgv
