// State dimension 6: prior build, initial iterate, SLR and bookkeeping kernels (double-float recursions).
#include "pgvimp_kernels.cuh"

namespace pgv {
template cudaError_t launch_aux<6, df64>(const Launch& L, int phase, int arg_i, int qt32);
}  // namespace pgv
