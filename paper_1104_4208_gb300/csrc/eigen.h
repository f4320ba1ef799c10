// Lanczos building blocks for the cavity resonance frequencies (device side)
// and the symmetric tridiagonal eigen-solver they feed (host side).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

namespace dgm {

// z = M_eps x for an FP64 E-field in the element-major orthonormalised layout
// [t][3][N]: per element z[:, a] = eps_t G_t x[:, a], G = |det F| F^{-1} F^{-T}
int eig_mass_apply(int64_t nt, int N, const double* geo, const double* x, double* z, cudaStream_t s);
// y = a x (y is only written, never read: it may hold stale bits)
int eig_scale(int64_t n, double a, const double* x, double* y, cudaStream_t s);
// out[j] = V[j] . z for j < k (rows of V ld apart), fixed-order sums
int eig_dots(const double* V, int64_t ld, int k, const double* z, int64_t n, double* out, cudaStream_t s);
// w -= sum_{j<k} h[j] V[j]
int eig_sub_combination(double* w, const double* V, int64_t ld, int k, const double* h, int64_t n, cudaStream_t s);

// Eigenvalues of the symmetric tridiagonal matrix (diagonal d[0..k), off-diagonal
// e[0..k-1)) with indices [i0, i1) in ascending order, by bisection on Sturm counts.
std::vector<double> tridiag_eigenvalues(const std::vector<double>& d, const std::vector<double>& e, int i0, int i1);
// number of eigenvalues of the same matrix below x
int tridiag_count_below(const std::vector<double>& d, const std::vector<double>& e, double x);
// unit eigenvector for the eigenvalue theta, by inverse iteration
std::vector<double> tridiag_eigenvector(const std::vector<double>& d, const std::vector<double>& e, double theta);

}  // namespace dgm
