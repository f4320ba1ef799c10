// Lanczos building blocks for the cavity resonance frequencies.
//
// The frequency-domain problem (Sec. 2.2: i omega eps E = curl H,
// i omega mu H = -curl E, PEC) discretised by the DG operator of Sec. 2.1 is
// the generalized symmetric eigenproblem omega^2 M_eps e = K e with
// K = C_H^T M_mu^{-1} C_H (+ the face-unknown term of the stabilized flux).
// A = M_eps^{-1} K is self-adjoint in the M_eps inner product, so the Lanczos
// recursion runs in that inner product; the device kernels here provide it
// (mass application, dot products, combinations) for FP64 E-fields in the
// element-major orthonormalised layout [t][3][N], where
// M_eps|_T = eps_T G_T (x) I with G = |det F| F^{-1} F^{-T}.
//
// The host part solves the Lanczos tridiagonal matrix: eigenvalues by
// bisection on Sturm sequence counts (the number of negative pivots of
// T - x I in its LDL^T factorisation equals the number of eigenvalues below
// x), eigenvectors by inverse iteration with a pivoted tridiagonal LU.

#include "eigen.h"

#include <algorithm>
#include <cfloat>
#include <cmath>

#include "kernels.h"

namespace dgm {

namespace {

constexpr int kThreads = 256;

__global__ void k_mass_apply(int64_t nt, int N, const double* __restrict__ geo, const double* __restrict__ x,
                             double* __restrict__ z) {
    const int64_t n = nt * N;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = i / N;
        const int a = (int)(i - t * N);
        const double* g = geo + t * kGeoStride;
        const double e = g[kGeoEps];
        const double* G = g + 6;   // xx, xy, xz, yy, yz, zz
        const int64_t b = t * 3 * N + a;
        const double x0 = x[b], x1 = x[b + N], x2 = x[b + 2 * N];
        z[b] = e * (G[0] * x0 + G[1] * x1 + G[2] * x2);
        z[b + N] = e * (G[1] * x0 + G[3] * x1 + G[4] * x2);
        z[b + 2 * N] = e * (G[2] * x0 + G[4] * x1 + G[5] * x2);
    }
}

// one block per row j: fixed-order strided partial sums, then a tree
__global__ void k_dots(const double* __restrict__ V, int64_t ld, const double* __restrict__ z, int64_t n,
                       double* __restrict__ out) {
    __shared__ double red[kThreads];
    const double* v = V + (int64_t)blockIdx.x * ld;
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += kThreads) s += v[i] * z[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = red[0];
}

__global__ void k_sub_combination(double* __restrict__ w, const double* __restrict__ V, int64_t ld, int k,
                                  const double* __restrict__ h, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int j = 0; j < k; ++j) s += h[j] * V[(int64_t)j * ld + i];
        w[i] -= s;
    }
}

__global__ void k_scale(int64_t n, double a, const double* __restrict__ x, double* __restrict__ y) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = a * x[i];
}

int grid_for(int64_t n) {
    const int64_t b = (n + kThreads - 1) / kThreads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, 8192));
}

}  // namespace

int eig_mass_apply(int64_t nt, int N, const double* geo, const double* x, double* z, cudaStream_t s) {
    if (nt <= 0) return 0;
    k_mass_apply<<<grid_for(nt * N), kThreads, 0, s>>>(nt, N, geo, x, z);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

int eig_scale(int64_t n, double a, const double* x, double* y, cudaStream_t s) {
    if (n <= 0) return 0;
    k_scale<<<grid_for(n), kThreads, 0, s>>>(n, a, x, y);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

int eig_dots(const double* V, int64_t ld, int k, const double* z, int64_t n, double* out, cudaStream_t s) {
    if (k <= 0) return 0;
    k_dots<<<k, kThreads, 0, s>>>(V, ld, z, n, out);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

int eig_sub_combination(double* w, const double* V, int64_t ld, int k, const double* h, int64_t n, cudaStream_t s) {
    if (k <= 0 || n <= 0) return 0;
    k_sub_combination<<<grid_for(n), kThreads, 0, s>>>(w, V, ld, k, h, n);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

// ------------------------------------------------------------------ host side

int tridiag_count_below(const std::vector<double>& d, const std::vector<double>& e, double x) {
    const int k = (int)d.size();
    double emax2 = 0.0;
    for (double v : e) emax2 = std::max(emax2, v * v);
    const double pivmin = DBL_MIN * std::max(1.0, emax2);
    int c = 0;
    double q = 1.0;
    for (int i = 0; i < k; ++i) {
        q = d[i] - x - (i > 0 ? e[i - 1] * e[i - 1] / q : 0.0);
        if (std::fabs(q) < pivmin) q = -pivmin;
        if (q < 0.0) ++c;
    }
    return c;
}

std::vector<double> tridiag_eigenvalues(const std::vector<double>& d, const std::vector<double>& e, int i0, int i1) {
    const int k = (int)d.size();
    double lo = INFINITY, hi = -INFINITY;
    for (int i = 0; i < k; ++i) {
        const double r = (i > 0 ? std::fabs(e[i - 1]) : 0.0) + (i < k - 1 ? std::fabs(e[i]) : 0.0);
        lo = std::min(lo, d[i] - r);
        hi = std::max(hi, d[i] + r);
    }
    const double tol = 4.0 * DBL_EPSILON * std::max(std::fabs(lo), std::fabs(hi));
    std::vector<double> out;
    for (int idx = std::max(0, i0); idx < std::min(k, i1); ++idx) {
        double a = lo, b = hi;
        for (int it = 0; it < 200 && b - a > tol; ++it) {
            const double mid = 0.5 * (a + b);
            if (tridiag_count_below(d, e, mid) > idx)
                b = mid;
            else
                a = mid;
        }
        out.push_back(0.5 * (a + b));
    }
    return out;
}

std::vector<double> tridiag_eigenvector(const std::vector<double>& d, const std::vector<double>& e, double theta) {
    const int k = (int)d.size();
    double scale = 0.0;
    for (int i = 0; i < k; ++i) scale = std::max(scale, std::fabs(d[i]) + (i < k - 1 ? std::fabs(e[i]) : 0.0));
    const double tiny = std::max(DBL_EPSILON * scale, DBL_MIN);
    // LU of T - theta I with partial pivoting: U has diagonal dd, superdiagonals du, du2;
    // dl holds the multipliers, piv[i] whether rows i, i+1 were exchanged
    std::vector<double> dl(std::max(k - 1, 0)), dd(k), du(std::max(k - 1, 0)), du2(std::max(k - 2, 0), 0.0);
    std::vector<char> piv(std::max(k - 1, 0), 0);
    for (int i = 0; i < k; ++i) dd[i] = d[i] - theta;
    for (int i = 0; i + 1 < k; ++i) {
        dl[i] = e[i];
        du[i] = e[i];
    }
    for (int i = 0; i + 1 < k; ++i) {
        if (std::fabs(dd[i]) >= std::fabs(dl[i])) {
            if (dd[i] == 0.0) dd[i] = tiny;
            const double f = dl[i] / dd[i];
            dl[i] = f;
            dd[i + 1] -= f * du[i];
        } else {
            const double f = dd[i] / dl[i];
            dd[i] = dl[i];
            dl[i] = f;
            const double t = du[i];
            du[i] = dd[i + 1];
            dd[i + 1] = t - f * dd[i + 1];
            if (i + 2 < k) {
                du2[i] = du[i + 1];
                du[i + 1] = -f * du[i + 1];
            }
            piv[i] = 1;
        }
    }
    if (dd[k - 1] == 0.0) dd[k - 1] = tiny;
    auto solve = [&](std::vector<double>& b) {
        for (int i = 0; i + 1 < k; ++i) {
            if (piv[i]) {
                const double t = b[i];
                b[i] = b[i + 1];
                b[i + 1] = t - dl[i] * b[i];
            } else {
                b[i + 1] -= dl[i] * b[i];
            }
        }
        // near-singular pivots (clustered Ritz values) can grow the solution past the
        // double range: the system is linear, so rescale the whole vector (solved part
        // and remaining right-hand side alike) when an entry gets large
        auto guard = [&](int i) {
            if (std::fabs(b[i]) > 1e100)
                for (double& v : b) v *= 1e-100;
        };
        b[k - 1] /= dd[k - 1];
        guard(k - 1);
        if (k > 1) {
            b[k - 2] = (b[k - 2] - du[k - 2] * b[k - 1]) / dd[k - 2];
            guard(k - 2);
        }
        for (int i = k - 3; i >= 0; --i) {
            b[i] = (b[i] - du[i] * b[i + 1] - du2[i] * b[i + 2]) / dd[i];
            guard(i);
        }
    };
    auto normalise = [&](std::vector<double>& b) {
        double s = 0.0;
        for (double v : b) s += v * v;
        s = std::sqrt(s);
        if (s > 0.0 && std::isfinite(s))
            for (double& v : b) v /= s;
    };
    // start: a fixed sequence without structure (golden-ratio fractional parts)
    std::vector<double> y(k);
    for (int i = 0; i < k; ++i) {
        const double g = std::fmod(0.6180339887498949 * (i + 1), 1.0);
        y[i] = 0.5 + g;
    }
    normalise(y);
    for (int it = 0; it < 3; ++it) {
        solve(y);
        normalise(y);
    }
    return y;
}

}  // namespace dgm
