// pgvimp_internal.h -- entry points shared by the batch API and the server
// inside the library (not part of the C ABI).
#pragma once
#include <stddef.h>

#include "../../include/pgvimp.h"

namespace pgv {

// Device arena and pinned host staging a batch of these problems needs.
// `scan_grids` = false skips the per-cell finiteness scan of the SDF grids
// (requests validated before); every other check still runs.
struct BatchSizes {
  size_t dev, host_in, host_out;
};
pgvimp_status batch_sizes(int count, const pgvimp_problem* problems, const pgvimp_options* options, int precision,
                          BatchSizes* sz, bool scan_grids = true);

// pgvimp_batch_create with caller-owned device arena and pinned host staging
// (sizes from batch_sizes); destroying the batch frees neither.  Creating
// and destroying such a batch makes no CUDA allocation or free call, so it
// does not synchronise the device.
pgvimp_status batch_create_staged(int count, const pgvimp_problem* problems, const pgvimp_options* options,
                                  int precision, void* arena, size_t arena_bytes, void* h_in, void* h_out,
                                  pgvimp_batch** out, bool scan_grids = true);

// Status slot of plan `index` in the staging of the last download (0: ok;
// 1: prior not PD; 2: marginals of the initial iterate not PD; 3: a
// quadrature factor's marginal not PD; 4: SLR linearisation failed).
int batch_plan_status(const pgvimp_batch* b, int index);

}  // namespace pgv
