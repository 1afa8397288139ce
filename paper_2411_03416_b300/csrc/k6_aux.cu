// Prior build, initial iterate, SLR and bookkeeping kernels, state dimension 6.
#include "pgvimp_kernels.cuh"

namespace pgv {
template cudaError_t launch_aux<6>(const Launch& L, int phase, int arg_i, int mixed);
}  // namespace pgv
