// State dimension 14: fused iterations, FP64 quadrature and recursions.
#include "pgvimp_kernels.cuh"

namespace pgv {
template cudaError_t launch_iter<14, double, double>(const Launch& L, int iters);
}  // namespace pgv
