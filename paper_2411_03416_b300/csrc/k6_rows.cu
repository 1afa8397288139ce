// State dimension 6: single-row kernels (marginals, quadrature, one trial).
#include "pgvimp_kernels.cuh"

namespace pgv {
template cudaError_t launch_rows<6>(const Launch& L, int phase, double arg_d, int mixed);
}  // namespace pgv
