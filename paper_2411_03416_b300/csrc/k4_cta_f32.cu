// State dimension 4, block (latency) form: fused iterations by cyclic reduction, FP32 quadrature, FP64 recursions.
#include "pgvimp_cr.cuh"

namespace pgv {
template cudaError_t launch_iter_cta<4, float, double>(const Launch& L, int iters, int tpb);
}  // namespace pgv
