// Point observations and adjoint helpers (device side).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace dgm {

struct ObsDev {
    int nobs;
    const int32_t* elem;       // [nobs] element containing the point
    const double* phi;         // [nobs][N3(p)] orthonormalised basis at the reference point
    const double* Finv;        // [nobs][9] F^{-1} of that element, row-major
    const double* ginv_eps;    // [nobs][6] G^{-1} / eps of that element
};

template <typename real>
int adj_observe(const ObsDev& O, const real* E, int N, int K, int tiled, double* J, cudaStream_t s);
template <typename real>
int adj_source(const ObsDev& O, const real* E, real* adj, int N, int K, int tiled, cudaStream_t s);
template <typename real>
int adj_grad(int64_t nt, const double* geo, const real* adj, const real* E1, const real* E0, int N, int K, int tiled,
             double* grad, cudaStream_t s);

template <typename real>
int add_point_source(real* E, int N, int K, int tiled, int64_t ts, const double* phi, const double* v,
                     const double* fvals, int64_t n, double dt, cudaStream_t s);

}  // namespace dgm
