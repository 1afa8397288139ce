// State dimension 14, block (latency) form: fused iterations by cyclic reduction, FP32 quadrature,
// double-float recursions; initial iterate, SLR and LTV prior with double-float storage.
#include "pgvimp_cr.cuh"

namespace pgv {
template cudaError_t launch_iter_cta<14, float, df64>(const Launch& L, int iters, int tpb);
template cudaError_t launch_aux_cta<14, df64>(const Launch& L, int phase, int arg_i, int qt32, int tpb);
}  // namespace pgv
