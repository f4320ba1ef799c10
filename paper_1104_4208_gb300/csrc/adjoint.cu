// Kernels of the discrete adjoint (gradient of a field observable with respect
// to the per-element permittivity) and of point observations.
//
// Objective J = sum_{n=1..N} sum_o |E^n(x_o)|^2, E^n of the leapfrog of Sec. 3.
// With e = M_eps e^, g = M_mu g^ the adjoint recursion runs the same kicks with
// a negative step (see adjoint_grad in capi.cpp); these kernels add the point
// sources M_eps^{-1} 2 P^T P E^m, accumulate -e^_T . (G (x) I)(E^m - E^{m-1})_T
// (= dJ/d eps_T, since d M_eps^{-1} / d eps_T = -M_eps^{-1}|_T / eps_T), and
// evaluate E at the observation points.  Every state layout is supported:
// element-major [t][m][a] and both tensor-core tile layouts.

#include <cuda_runtime.h>

#include <cstdint>

#include "adjoint.h"
#include "kernels.h"

namespace dgm {

namespace {

struct Lay {
    int N, K, tiled;
    __device__ __forceinline__ int64_t at(int64_t t, int m, int a) const {
        if (!tiled) return (t * 3 + m) * N + a;
        // tensor-core tiles, row length K: interleaved (k = 3 a + m) or component-major (k = m K/3 + a)
        const int k = tiled == 2 ? m * (K / 3) + a : 3 * a + m;
        return (((t >> 7) * (K >> 2) + (k >> 2)) * 128 + (t & 127)) * 4 + (k & 3);
    }
};

// E at observation point o, v = F^{-T} sum_a c[:, a] phi'_a, summed by the 32 lanes
// of one warp: lane-strided partial sums, a fixed shuffle tree, then lane 0's value
// broadcast (every lane returns the same bits)
template <typename real>
__device__ void eval_point_warp(const ObsDev& O, const real* E, Lay L, int o, int lane, double v[3]) {
    const int64_t t = O.elem[o];
    const double* ph = O.phi + (size_t)o * L.N;
    double c[3] = {0, 0, 0};
    for (int a = lane; a < L.N; a += 32)
        for (int m = 0; m < 3; ++m) c[m] += ph[a] * (double)E[L.at(t, m, a)];
    for (int m = 0; m < 3; ++m) {
        for (int off = 16; off > 0; off >>= 1) c[m] += __shfl_down_sync(0xffffffffu, c[m], off);
        c[m] = __shfl_sync(0xffffffffu, c[m], 0);
    }
    const double* Fi = O.Finv + 9 * o;   // F^{-1} row-major
    for (int i = 0; i < 3; ++i) v[i] = Fi[0 * 3 + i] * c[0] + Fi[1 * 3 + i] * c[1] + Fi[2 * 3 + i] * c[2];
}

constexpr int kObsWarps = 8;
constexpr int kMaxObs = 1024;

// J += sum_o |E(x_o)|^2: one warp per point, then the points summed in order
template <typename real>
__global__ void k_observe(ObsDev O, const real* E, Lay L, double* J) {
    __shared__ double val[kMaxObs];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = warp; o < O.nobs; o += kObsWarps) {
        double v[3];
        eval_point_warp(O, E, L, o, lane, v);
        if (lane == 0) val[o] = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int o = 0; o < O.nobs; ++o) s += val[o];
        *J += s;
    }
}

// e^ += M_eps^{-1} 2 P^T P E: all points evaluated first (one warp per point; E is
// not changed by this kernel), then their contributions added in point order
// (several points may share an element)
template <typename real>
__global__ void k_obs_source(ObsDev O, const real* E, real* adj, Lay L) {
    __shared__ double wo[kMaxObs][3];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = warp; o < O.nobs; o += kObsWarps) {
        double v[3];
        eval_point_warp(O, E, L, o, lane, v);
        if (lane == 0) {
            const double* Fi = O.Finv + 9 * o;
            for (int m = 0; m < 3; ++m)
                wo[o][m] = 2.0 * (Fi[m * 3 + 0] * v[0] + Fi[m * 3 + 1] * v[1] + Fi[m * 3 + 2] * v[2]);
        }
    }
    __syncthreads();
    for (int o = 0; o < O.nobs; ++o) {
        const double* w = wo[o];
        const int64_t t = O.elem[o];
        const double* gi = O.ginv_eps + 6 * o;   // G^{-1} / eps
        const double* ph = O.phi + (size_t)o * L.N;
        for (int a = threadIdx.x; a < L.N; a += blockDim.x) {
            const double u0 = ph[a] * w[0], u1 = ph[a] * w[1], u2 = ph[a] * w[2];
            adj[L.at(t, 0, a)] += (real)(gi[0] * u0 + gi[1] * u1 + gi[2] * u2);
            adj[L.at(t, 1, a)] += (real)(gi[1] * u0 + gi[3] * u1 + gi[4] * u2);
            adj[L.at(t, 2, a)] += (real)(gi[2] * u0 + gi[4] * u1 + gi[5] * u2);
        }
        __syncthreads();
    }
}

// grad[t] -= sum_a e^[:, a] . G (E1 - E0)[:, a]; one warp per element, lanes over a,
// fixed shuffle tree
template <typename real>
__global__ void k_grad_accum(int64_t nt, const double* geo, const real* adj, const real* E1, const real* E0, Lay L,
                             double* grad) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t t = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < nt; t += nwarps) {
        const double* g = geo + t * kGeoStride + 6;
        double s = 0.0;
        for (int a = lane; a < L.N; a += 32) {
            double d[3], e[3];
            for (int m = 0; m < 3; ++m) {
                const int64_t i = L.at(t, m, a);
                d[m] = (double)E1[i] - (double)E0[i];
                e[m] = (double)adj[i];
            }
            s += e[0] * (g[0] * d[0] + g[1] * d[1] + g[2] * d[2]) + e[1] * (g[1] * d[0] + g[3] * d[1] + g[4] * d[2]) +
                 e[2] * (g[2] * d[0] + g[4] * d[1] + g[5] * d[2]);
        }
        for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
        if (lane == 0) grad[t] -= s;
    }
}

// point dipole source: E[t_s][m][a] += coef * v[m] * phi[a], coef = -dt f(t_{n+1/2}) from fvals[n]
template <typename real>
__global__ void k_point_source(real* E, Lay L, int64_t ts, const double* phi, const double* v, const double* fvals,
                               int64_t n, double dt) {
    const double c = -dt * fvals[n];
    for (int a = threadIdx.x; a < L.N; a += blockDim.x)
        for (int m = 0; m < 3; ++m) E[L.at(ts, m, a)] += (real)(c * v[m] * phi[a]);
}

}  // namespace

template <typename real>
int add_point_source(real* E, int N, int K, int tiled, int64_t ts, const double* phi, const double* v,
                     const double* fvals, int64_t n, double dt, cudaStream_t s) {
    k_point_source<real><<<1, 128, 0, s>>>(E, Lay{N, K, tiled}, ts, phi, v, fvals, n, dt);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}
template int add_point_source<double>(double*, int, int, int, int64_t, const double*, const double*, const double*,
                                      int64_t, double, cudaStream_t);
template int add_point_source<float>(float*, int, int, int, int64_t, const double*, const double*, const double*,
                                     int64_t, double, cudaStream_t);

template <typename real>
int adj_observe(const ObsDev& O, const real* E, int N, int K, int tiled, double* J, cudaStream_t s) {
    if (O.nobs > kMaxObs) return -1;
    k_observe<real><<<1, kObsWarps * 32, 0, s>>>(O, E, Lay{N, K, tiled}, J);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

template <typename real>
int adj_source(const ObsDev& O, const real* E, real* adj, int N, int K, int tiled, cudaStream_t s) {
    if (O.nobs > kMaxObs) return -1;
    k_obs_source<real><<<1, kObsWarps * 32, 0, s>>>(O, E, adj, Lay{N, K, tiled});
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

template <typename real>
int adj_grad(int64_t nt, const double* geo, const real* adj, const real* E1, const real* E0, int N, int K, int tiled,
             double* grad, cudaStream_t s) {
    const int64_t blocks = (nt + 7) / 8;   // 8 warps of 32 per block, one warp per element
    k_grad_accum<real><<<(int)(blocks < 8192 ? blocks : 8192), 256, 0, s>>>(nt, geo, adj, E1, E0, Lay{N, K, tiled},
                                                                           grad);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

template int adj_observe<double>(const ObsDev&, const double*, int, int, int, double*, cudaStream_t);
template int adj_observe<float>(const ObsDev&, const float*, int, int, int, double*, cudaStream_t);
template int adj_source<double>(const ObsDev&, const double*, double*, int, int, int, cudaStream_t);
template int adj_source<float>(const ObsDev&, const float*, float*, int, int, int, cudaStream_t);
template int adj_grad<double>(int64_t, const double*, const double*, const double*, const double*, int, int, int,
                              double*, cudaStream_t);
template int adj_grad<float>(int64_t, const double*, const float*, const float*, const float*, int, int, int, double*,
                             cudaStream_t);

}  // namespace dgm
