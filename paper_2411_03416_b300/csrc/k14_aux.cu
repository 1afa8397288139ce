// State dimension 14: prior build, initial iterate, SLR and bookkeeping kernels (FP64 recursions).
#include "pgvimp_kernels.cuh"

namespace pgv {
template cudaError_t launch_aux<14, double>(const Launch& L, int phase, int arg_i, int qt32);
}  // namespace pgv
