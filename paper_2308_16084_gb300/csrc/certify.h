// certify.h -- device search used by the host builder.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.h"

namespace p2m {

// Builder certification: for each point x[i] (3 doubles), the nearest
// KD-tree position strictly closer than sqrt(r2[i]) in double precision (the
// lowest position among equal distances), -1 if none, -2 if the traversal
// stack would overflow (search on the host).  Same answers as the host
// search.
cudaError_t launch_nearest_within_f64(const DevView &m, const double *x, const double *r2,
                                      int64_t n, int64_t *out, cudaStream_t stream = 0);

}  // namespace p2m
