// Physical quadrature points of every element (Sec. 3.2.1: x = Phi_T(xh) =
// X0 + F xh), for host callers that sample initial data there.

#include "fieldio.h"

#include <algorithm>

namespace dgm {

namespace {

__global__ void k_quad_points(int64_t nt, int nq, const double* __restrict__ maps, const double* __restrict__ xh,
                              double* __restrict__ out) {
    const int64_t n = nt * nq;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = i / nq;
        const int q = (int)(i - t * nq);
        const double* M = maps + 12 * t;
        const double* r = xh + 3 * q;
        for (int d = 0; d < 3; ++d)
            out[3 * i + d] = M[d] + M[3 + 3 * d] * r[0] + M[3 + 3 * d + 1] * r[1] + M[3 + 3 * d + 2] * r[2];
    }
}

}  // namespace

int launch_quad_points(int64_t nt, int nq, const double* maps, const double* xh, double* out, cudaStream_t s) {
    const int64_t n = nt * nq;
    if (n <= 0) return 0;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 8192);
    k_quad_points<<<(int)blocks, 256, 0, s>>>(nt, nq, maps, xh, out);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace dgm
