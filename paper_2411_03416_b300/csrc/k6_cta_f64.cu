// State dimension 6, block (latency) form: fused iterations by cyclic reduction, FP64 throughout.
#include "pgvimp_cr.cuh"

namespace pgv {
template cudaError_t launch_iter_cta<6, double, double>(const Launch& L, int iters, int tpb);
template cudaError_t launch_aux_cta<6, double>(const Launch& L, int phase, int arg_i, int qt32, int tpb);
}  // namespace pgv
