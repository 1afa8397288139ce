// State dimension 4: fused iterations, FP64 quadrature and recursions.
#include "pgvimp_kernels.cuh"

namespace pgv {
template cudaError_t launch_iter<4, double, double>(const Launch& L, int iters);
}  // namespace pgv
