// Helpers of the host-array field I/O entry points (device side).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace dgm {

// x[t][q][:] = X0_t + F_t xh_q for element maps [nt][12] (X0, then F row-major)
// and reference points xh [nq][3]
int launch_quad_points(int64_t nt, int nq, const double* maps, const double* xh, double* out, cudaStream_t s);

}  // namespace dgm
