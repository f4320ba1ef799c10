// CUDA kernels of the DG Maxwell time step (sm_103a).
//
// One time step of the symplectic Euler / leapfrog scheme (Sec. 3) is two
// phase kernels:
//   H-phase: H += dt M_mu^{-1} C_h E       (volume curl + facet jump + lift)
//   E-phase: E -= dt M_eps^{-1} C_h^T H    (volume curl^T + facet average + lift)
// Both work on the orthonormalised covariant coefficients of each element,
// with the geometry-free reference operators of Sec. 3.2.1:
//   r_H[m,b] = -s_T (curl E)[m,b]
//              + sum_f sigma_f sum_g Tr_f[g,b] (t2_m a1_g - t1_m a2_g),  a = [[E]]/2
//   r_E[m,a] =  s_T (curl^T H)[m,a]
//              + sum_f sigma_f sum_g Tr_f[g,a] (t2_m b1_g - t1_m b2_g),  b = {{H}}
// where a_i, b_i are tangential covariant face coefficients in the shared face
// frame (both sides order the face's vertices by key), sigma_f = s_T * sign of
// the reference face orientation, s_T = sign det F.  The inverse mass is the
// 3x3 block (F^T F)/(|det F| eps) per coefficient (Sec. 3.3.1).
//
// Mapping: one warp per element, the element's coefficients staged in shared
// memory, lanes over output coefficients, reference tables read through the
// read-only cache.  The neighbour's trace on a shared face is recomputed from
// the neighbour's coefficients (read from L2), so no per-step face buffer is
// written.  Energy partials are accumulated in FP64 per warp in a fixed
// order and reduced per block in a fixed order (bitwise reproducible).

#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.h"

namespace dgm {

__constant__ double c_that[4][2][3];
__constant__ double c_sigma_hat[4];

int upload_face_frames(const double that[4][2][3], const double sigma_hat[4]) {
    if (cudaMemcpyToSymbol(c_that, that, sizeof(double) * 24) != cudaSuccess) return -1;
    if (cudaMemcpyToSymbol(c_sigma_hat, sigma_hat, sizeof(double) * 4) != cudaSuccess) return -1;
    return 0;
}

namespace {

constexpr int kWarps = 4;   // warps per block

template <typename real>
__device__ __forceinline__ real ld(const real* p) {
    return __ldg(p);
}

// fixed-order block reduction of one double per warp
__device__ void block_energy_store(double v, double* out) {
    __shared__ double red[kWarps];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) red[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < kWarps; ++i) s += red[i];
        out[blockIdx.x] = s;
    }
}

template <typename real>
__global__ void __launch_bounds__(kWarps * 32)
k_phase_H(KParams<real> P, double dt, double a_lo, double c_out, double* __restrict__ partials) {
    extern __shared__ unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    real* sE = reinterpret_cast<real*>(smem_raw) + (size_t)wib * P.warp_smem;
    real* sN = sE + 3 * P.NE;
    real* sA = sN + 3 * P.NE;
    const int NE = P.NE, NH = P.NH, N2H = P.N2H;
    double eacc = 0.0;
    const int64_t nwarps = (int64_t)gridDim.x * kWarps;
    for (int64_t t = (int64_t)blockIdx.x * kWarps + wib; t < P.nt; t += nwarps) {
        const real* Et = P.E + t * 3 * NE;
        for (int k = lane; k < 3 * NE; k += 32) sE[k] = Et[k];
        const double* g = P.geo + t * kGeoStride;
        const double sT = g[kGeoSign];
        __syncwarp();
        for (int f = 0; f < 4; ++f) {
            const int32_t nb = P.nbr[t * 4 + f];
            const double sig = sT * c_sigma_hat[f];
            if (nb >= 0) {
                const real* En = P.E + (int64_t)(nb >> 2) * 3 * NE;
                for (int k = lane; k < 3 * NE; k += 32) sN[k] = En[k];
            }
            __syncwarp();
            for (int gm = lane; gm < N2H; gm += 32) {
                const real* T = P.TrEqT + (size_t)f * NE * N2H + gm;
                real t0 = 0, t1 = 0, t2 = 0;
                for (int a = 0; a < NE; ++a) {
                    const real w = ld(T + (size_t)a * N2H);
                    t0 += w * sE[a];
                    t1 += w * sE[NE + a];
                    t2 += w * sE[2 * NE + a];
                }
                real J0 = (real)c_that[f][0][0] * t0 + (real)c_that[f][0][1] * t1 + (real)c_that[f][0][2] * t2;
                real J1 = (real)c_that[f][1][0] * t0 + (real)c_that[f][1][1] * t1 + (real)c_that[f][1][2] * t2;
                real a0, a1;
                if (nb >= 0) {
                    const int nf = nb & 3;
                    const real* Tn = P.TrEqT + (size_t)nf * NE * N2H + gm;
                    real n0 = 0, n1 = 0, n2 = 0;
                    for (int a = 0; a < NE; ++a) {
                        const real w = ld(Tn + (size_t)a * N2H);
                        n0 += w * sN[a];
                        n1 += w * sN[NE + a];
                        n2 += w * sN[2 * NE + a];
                    }
                    const real K0 = (real)c_that[nf][0][0] * n0 + (real)c_that[nf][0][1] * n1 + (real)c_that[nf][0][2] * n2;
                    const real K1 = (real)c_that[nf][1][0] * n0 + (real)c_that[nf][1][1] * n1 + (real)c_that[nf][1][2] * n2;
                    a0 = (real)(0.5 * sig) * (J0 - K0);
                    a1 = (real)(0.5 * sig) * (J1 - K1);
                } else {
                    a0 = (real)sig * J0;
                    a1 = (real)sig * J1;
                }
                sA[(2 * f) * N2H + gm] = a0;
                sA[(2 * f + 1) * N2H + gm] = a1;
            }
            if (P.K) {
                // stabilized flux: the owning side advances H^F of this face,
                // (h_F/alpha) (dH^F/dt, h^F)_F = ([[E]] x nu_F, h^F)_F
                const int32_t fe = P.fid[t * 4 + f];
                if (fe & 1) {
                    const int64_t F = fe >> 1;
                    const double* fg = P.fgeo + F * kFaceGeoStride;
                    const int N2E = P.N2E;
                    real* KF = P.K + F * 2 * N2E;
                    for (int gm = lane; gm < N2E; gm += 32) {
                        const real* T = P.TrEfT + (size_t)f * NE * N2E + gm;
                        real t0 = 0, t1 = 0, t2 = 0;
                        for (int a = 0; a < NE; ++a) {
                            const real w = ld(T + (size_t)a * N2E);
                            t0 += w * sE[a];
                            t1 += w * sE[NE + a];
                            t2 += w * sE[2 * NE + a];
                        }
                        real j0 = (real)c_that[f][0][0] * t0 + (real)c_that[f][0][1] * t1 + (real)c_that[f][0][2] * t2;
                        real j1 = (real)c_that[f][1][0] * t0 + (real)c_that[f][1][1] * t1 + (real)c_that[f][1][2] * t2;
                        if (nb >= 0) {
                            const int nf = nb & 3;
                            const real* Tn = P.TrEfT + (size_t)nf * NE * N2E + gm;
                            real n0 = 0, n1 = 0, n2 = 0;
                            for (int a = 0; a < NE; ++a) {
                                const real w = ld(Tn + (size_t)a * N2E);
                                n0 += w * sN[a];
                                n1 += w * sN[NE + a];
                                n2 += w * sN[2 * NE + a];
                            }
                            j0 -= (real)c_that[nf][0][0] * n0 + (real)c_that[nf][0][1] * n1 + (real)c_that[nf][0][2] * n2;
                            j1 -= (real)c_that[nf][1][0] * n0 + (real)c_that[nf][1][1] * n1 + (real)c_that[nf][1][2] * n2;
                        } else {
                            j0 = (real)2 * j0;
                            j1 = (real)2 * j1;
                        }
                        // [[E]]_F = sigma_f (E_T - E_nbr); dK = dt c g (J_2, -J_1)
                        const real c = (real)(dt * fg[0] * sig);
                        const real dk0 = c * ((real)fg[1] * j1 - (real)fg[2] * j0);
                        const real dk1 = c * ((real)fg[2] * j1 - (real)fg[3] * j0);
                        const real k0 = KF[gm], k1 = KF[N2E + gm];
                        if (partials) {
                            const double l0 = (double)k0 - a_lo * (double)dk0, l1 = (double)k1 - a_lo * (double)dk1;
                            const double u0 = l0 + (double)dk0, u1 = l1 + (double)dk1;
                            eacc += 0.5 * fg[4] * (l0 * (fg[5] * u0 + fg[6] * u1) + l1 * (fg[6] * u0 + fg[7] * u1));
                        }
                        KF[gm] = k0 + (real)c_out * dk0;
                        KF[N2E + gm] = k1 + (real)c_out * dk1;
                    }
                }
            }
            __syncwarp();
        }
        const double ginv[6] = {g[0], g[1], g[2], g[3], g[4], g[5]};
        const double gm6[6] = {g[6], g[7], g[8], g[9], g[10], g[11]};
        const double inv_mu = g[kGeoInvMu], mu = g[kGeoMu];
        real* Ht = P.H + t * 3 * NH;
        for (int b = lane; b < NH; b += 32) {
            real cx = 0, cy = 0, cz = 0;
            const real* Dx = P.DT + b;
            const real* Dy = Dx + (size_t)NE * NH;
            const real* Dz = Dy + (size_t)NE * NH;
            for (int a = 0; a < NE; ++a) {
                const real dx = ld(Dx + (size_t)a * NH), dy = ld(Dy + (size_t)a * NH), dz = ld(Dz + (size_t)a * NH);
                const real ex = sE[a], ey = sE[NE + a], ez = sE[2 * NE + a];
                cx += dy * ez - dz * ey;
                cy += dz * ex - dx * ez;
                cz += dx * ey - dy * ex;
            }
            real r0 = -(real)sT * cx, r1 = -(real)sT * cy, r2 = -(real)sT * cz;
            for (int f = 0; f < 4; ++f) {
                const real* L = P.TrH + (size_t)f * N2H * NH + b;
                const real* A0 = sA + (2 * f) * N2H;
                const real* A1 = A0 + N2H;
                real u0 = 0, u1 = 0;
                for (int gm = 0; gm < N2H; ++gm) {
                    const real l = ld(L + (size_t)gm * NH);
                    u0 += l * A0[gm];
                    u1 += l * A1[gm];
                }
                r0 += (real)c_that[f][1][0] * u0 - (real)c_that[f][0][0] * u1;
                r1 += (real)c_that[f][1][1] * u0 - (real)c_that[f][0][1] * u1;
                r2 += (real)c_that[f][1][2] * u0 - (real)c_that[f][0][2] * u1;
            }
            const real s = (real)(dt * inv_mu);
            const real d0 = s * ((real)ginv[0] * r0 + (real)ginv[1] * r1 + (real)ginv[2] * r2);
            const real d1 = s * ((real)ginv[1] * r0 + (real)ginv[3] * r1 + (real)ginv[4] * r2);
            const real d2 = s * ((real)ginv[2] * r0 + (real)ginv[4] * r1 + (real)ginv[5] * r2);
            const real h0 = Ht[b], h1 = Ht[NH + b], h2 = Ht[2 * NH + b];
            if (partials) {
                const double l0 = (double)h0 - a_lo * (double)d0, l1 = (double)h1 - a_lo * (double)d1,
                             l2 = (double)h2 - a_lo * (double)d2;
                const double u0 = l0 + (double)d0, u1 = l1 + (double)d1, u2 = l2 + (double)d2;
                eacc += 0.5 * mu *
                        (l0 * (gm6[0] * u0 + gm6[1] * u1 + gm6[2] * u2) + l1 * (gm6[1] * u0 + gm6[3] * u1 + gm6[4] * u2) +
                         l2 * (gm6[2] * u0 + gm6[4] * u1 + gm6[5] * u2));
            }
            Ht[b] = h0 + (real)c_out * d0;
            Ht[NH + b] = h1 + (real)c_out * d1;
            Ht[2 * NH + b] = h2 + (real)c_out * d2;
        }
        if (partials) {
            const double eps = g[kGeoEps];
            for (int a = lane; a < NE; a += 32) {
                const double e0 = sE[a], e1 = sE[NE + a], e2 = sE[2 * NE + a];
                eacc += 0.5 * eps *
                        (e0 * (gm6[0] * e0 + gm6[1] * e1 + gm6[2] * e2) + e1 * (gm6[1] * e0 + gm6[3] * e1 + gm6[4] * e2) +
                         e2 * (gm6[2] * e0 + gm6[4] * e1 + gm6[5] * e2));
            }
        }
        __syncwarp();
    }
    if (partials) block_energy_store(eacc, partials);
}

template <typename real>
__global__ void __launch_bounds__(kWarps * 32)
k_phase_E(KParams<real> P, double dt) {
    extern __shared__ unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    real* sH = reinterpret_cast<real*>(smem_raw) + (size_t)wib * P.warp_smem;
    real* sN = sH + 3 * P.NH;
    real* sB = sN + 3 * P.NH;
    real* sKf = sB + 8 * P.N2H;     // [4][2][N2E] (stabilized flux only)
    const int NE = P.NE, NH = P.NH, N2H = P.N2H;
    const int64_t nwarps = (int64_t)gridDim.x * kWarps;
    for (int64_t t = (int64_t)blockIdx.x * kWarps + wib; t < P.nt; t += nwarps) {
        const real* Ht = P.H + t * 3 * NH;
        for (int k = lane; k < 3 * NH; k += 32) sH[k] = Ht[k];
        const double* g = P.geo + t * kGeoStride;
        const double sT = g[kGeoSign];
        __syncwarp();
        for (int f = 0; f < 4; ++f) {
            const int32_t nb = P.nbr[t * 4 + f];
            const double sig = sT * c_sigma_hat[f];
            if (nb >= 0) {
                const real* Hn = P.H + (int64_t)(nb >> 2) * 3 * NH;
                for (int k = lane; k < 3 * NH; k += 32) sN[k] = Hn[k];
            }
            __syncwarp();
            for (int gm = lane; gm < N2H; gm += 32) {
                const real* T = P.TrHT + (size_t)f * NH * N2H + gm;
                real t0 = 0, t1 = 0, t2 = 0;
                for (int b = 0; b < NH; ++b) {
                    const real w = ld(T + (size_t)b * N2H);
                    t0 += w * sH[b];
                    t1 += w * sH[NH + b];
                    t2 += w * sH[2 * NH + b];
                }
                real J0 = (real)c_that[f][0][0] * t0 + (real)c_that[f][0][1] * t1 + (real)c_that[f][0][2] * t2;
                real J1 = (real)c_that[f][1][0] * t0 + (real)c_that[f][1][1] * t1 + (real)c_that[f][1][2] * t2;
                real b0, b1;
                if (nb >= 0) {
                    const int nf = nb & 3;
                    const real* Tn = P.TrHT + (size_t)nf * NH * N2H + gm;
                    real n0 = 0, n1 = 0, n2 = 0;
                    for (int b = 0; b < NH; ++b) {
                        const real w = ld(Tn + (size_t)b * N2H);
                        n0 += w * sN[b];
                        n1 += w * sN[NH + b];
                        n2 += w * sN[2 * NH + b];
                    }
                    const real K0 = (real)c_that[nf][0][0] * n0 + (real)c_that[nf][0][1] * n1 + (real)c_that[nf][0][2] * n2;
                    const real K1 = (real)c_that[nf][1][0] * n0 + (real)c_that[nf][1][1] * n1 + (real)c_that[nf][1][2] * n2;
                    b0 = (real)(0.5 * sig) * (J0 + K0);
                    b1 = (real)(0.5 * sig) * (J1 + K1);
                } else {
                    b0 = (real)sig * J0;
                    b1 = (real)sig * J1;
                }
                sB[(2 * f) * N2H + gm] = b0;
                sB[(2 * f + 1) * N2H + gm] = b1;
            }
            if (P.K) {
                // (H^F x nu_F, [[e]])_F with [[e]] = sigma_f e_T (2 sigma_f e_T on PEC faces)
                const int64_t F = P.fid[t * 4 + f] >> 1;
                const real* KF = P.K + F * 2 * P.N2E;
                const real s = (real)(nb >= 0 ? sig : 2.0 * sig);
                for (int gm = lane; gm < 2 * P.N2E; gm += 32) sKf[f * 2 * P.N2E + gm] = s * KF[gm];
            }
            __syncwarp();
        }
        const double ginv[6] = {g[0], g[1], g[2], g[3], g[4], g[5]};
        const double inv_eps = g[kGeoInvEps];
        real* Et = P.E + t * 3 * NE;
        for (int a = lane; a < NE; a += 32) {
            real rx = 0, ry = 0, rz = 0;
            const real* Dx = P.D + a;
            const real* Dy = Dx + (size_t)NH * NE;
            const real* Dz = Dy + (size_t)NH * NE;
            for (int b = 0; b < NH; ++b) {
                const real dx = ld(Dx + (size_t)b * NE), dy = ld(Dy + (size_t)b * NE), dz = ld(Dz + (size_t)b * NE);
                const real hx = sH[b], hy = sH[NH + b], hz = sH[2 * NH + b];
                rx += dz * hy - dy * hz;
                ry += dx * hz - dz * hx;
                rz += dy * hx - dx * hy;
            }
            real r0 = (real)sT * rx, r1 = (real)sT * ry, r2 = (real)sT * rz;
            for (int f = 0; f < 4; ++f) {
                const real* L = P.TrEq + (size_t)f * N2H * NE + a;
                const real* B0 = sB + (2 * f) * N2H;
                const real* B1 = B0 + N2H;
                real u0 = 0, u1 = 0;
                for (int gm = 0; gm < N2H; ++gm) {
                    const real l = ld(L + (size_t)gm * NE);
                    u0 += l * B0[gm];
                    u1 += l * B1[gm];
                }
                r0 += (real)c_that[f][1][0] * u0 - (real)c_that[f][0][0] * u1;
                r1 += (real)c_that[f][1][1] * u0 - (real)c_that[f][0][1] * u1;
                r2 += (real)c_that[f][1][2] * u0 - (real)c_that[f][0][2] * u1;
            }
            if (P.K) {
                const int N2E = P.N2E;
                for (int f = 0; f < 4; ++f) {
                    const real* L = P.TrEf + (size_t)f * N2E * NE + a;
                    const real* K0 = sKf + f * 2 * N2E;
                    const real* K1 = K0 + N2E;
                    real u0 = 0, u1 = 0;
                    for (int gm = 0; gm < N2E; ++gm) {
                        const real l = ld(L + (size_t)gm * NE);
                        u0 += l * K0[gm];
                        u1 += l * K1[gm];
                    }
                    // K_2 t1_m - K_1 t2_m
                    r0 += (real)c_that[f][0][0] * u1 - (real)c_that[f][1][0] * u0;
                    r1 += (real)c_that[f][0][1] * u1 - (real)c_that[f][1][1] * u0;
                    r2 += (real)c_that[f][0][2] * u1 - (real)c_that[f][1][2] * u0;
                }
            }
            const real s = (real)(dt * inv_eps);
            Et[a] += s * ((real)ginv[0] * r0 + (real)ginv[1] * r1 + (real)ginv[2] * r2);
            Et[NE + a] += s * ((real)ginv[1] * r0 + (real)ginv[3] * r1 + (real)ginv[4] * r2);
            Et[2 * NE + a] += s * ((real)ginv[2] * r0 + (real)ginv[4] * r1 + (real)ginv[5] * r2);
        }
        __syncwarp();
    }
}

// canonical FP64 (unnormalised basis) <-> internal (orthonormalised, real)
template <typename real>
__global__ void k_import(const double* __restrict__ src, real* __restrict__ dst, const double* __restrict__ nrm,
                         int64_t n, int ncoef) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (real)(src[i] * nrm[i % ncoef]);
}

template <typename real>
__global__ void k_export(const real* __restrict__ src, double* __restrict__ dst, const double* __restrict__ nrm,
                         int64_t n, int ncoef) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (double)src[i] / nrm[i % ncoef];
}

// y = a x + b y (power iteration of the stability estimate)
template <typename real>
__global__ void k_axpby(int64_t n, double a, const real* __restrict__ x, double b, real* __restrict__ y) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = (real)(a * (double)x[i] + b * (double)y[i]);
}

__global__ void k_energy_reduce(const double* __restrict__ partials, int n, double* __restrict__ out) {
    __shared__ double red[256];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += partials[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

// covariant L2 projection of point values (setup): c'_{m,a} = (F^T sum_q w_q phi'_a(q) u_q)_m
template <typename real>
__global__ void k_project(int64_t nt, int N, int nq, const double* __restrict__ maps,
                          const double* __restrict__ wphi, const double* __restrict__ pts, real* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t t = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < nt; t += nw) {
        const double* F = maps + t * 12 + 3;
        const double* u = pts + t * (int64_t)nq * 3;
        for (int a = lane; a < N; a += 32) {
            double s0 = 0, s1 = 0, s2 = 0;
            for (int q = 0; q < nq; ++q) {
                const double w = wphi[(size_t)q * N + a];
                s0 += w * u[3 * q];
                s1 += w * u[3 * q + 1];
                s2 += w * u[3 * q + 2];
            }
            real* o = out + t * 3 * N;
            o[a] = (real)(F[0] * s0 + F[3] * s1 + F[6] * s2);
            o[N + a] = (real)(F[1] * s0 + F[4] * s1 + F[7] * s2);
            o[2 * N + a] = (real)(F[2] * s0 + F[5] * s1 + F[8] * s2);
        }
    }
}

// physical values u(x_q) = F^{-T} sum_a c'_a phi'_a(q) of the current field (setup / diagnostics)
template <typename real>
__global__ void k_eval(int64_t nt, int N, int nq, const double* __restrict__ maps, const double* __restrict__ phi,
                       const real* __restrict__ c, double* __restrict__ pts) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t t = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < nt; t += nw) {
        const double* F = maps + t * 12 + 3;
        const double det = F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) +
                           F[2] * (F[3] * F[7] - F[4] * F[6]);
        // rows of F^{-T} = columns of F^{-1}
        double Fi[9];
        Fi[0] = (F[4] * F[8] - F[5] * F[7]) / det;
        Fi[1] = (F[2] * F[7] - F[1] * F[8]) / det;
        Fi[2] = (F[1] * F[5] - F[2] * F[4]) / det;
        Fi[3] = (F[5] * F[6] - F[3] * F[8]) / det;
        Fi[4] = (F[0] * F[8] - F[2] * F[6]) / det;
        Fi[5] = (F[2] * F[3] - F[0] * F[5]) / det;
        Fi[6] = (F[3] * F[7] - F[4] * F[6]) / det;
        Fi[7] = (F[1] * F[6] - F[0] * F[7]) / det;
        Fi[8] = (F[0] * F[4] - F[1] * F[3]) / det;
        const real* ct = c + t * 3 * N;
        for (int q = lane; q < nq; q += 32) {
            double v0 = 0, v1 = 0, v2 = 0;
            for (int a = 0; a < N; ++a) {
                const double f = phi[(size_t)q * N + a];
                v0 += f * (double)ct[a];
                v1 += f * (double)ct[N + a];
                v2 += f * (double)ct[2 * N + a];
            }
            double* o = pts + (t * nq + q) * 3;
            // (F^{-T} v)_i = sum_j Finv[j][i] v_j
            o[0] = Fi[0] * v0 + Fi[3] * v1 + Fi[6] * v2;
            o[1] = Fi[1] * v0 + Fi[4] * v1 + Fi[7] * v2;
            o[2] = Fi[2] * v0 + Fi[5] * v1 + Fi[8] * v2;
        }
    }
}

}  // namespace

template <typename real>
int launch_project(int64_t nt, int N, int nq, const double* maps, const double* wphi, const double* pts, real* out,
                   cudaStream_t s) {
    const int64_t blocks = (nt + 3) / 4;
    k_project<real><<<(int)(blocks < 65535 ? blocks : 65535), 128, 0, s>>>(nt, N, nq, maps, wphi, pts, out);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

template <typename real>
int launch_eval(int64_t nt, int N, int nq, const double* maps, const double* phi, const real* c, double* pts,
                cudaStream_t s) {
    const int64_t blocks = (nt + 3) / 4;
    k_eval<real><<<(int)(blocks < 65535 ? blocks : 65535), 128, 0, s>>>(nt, N, nq, maps, phi, c, pts);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

template int launch_project<double>(int64_t, int, int, const double*, const double*, const double*, double*, cudaStream_t);
template int launch_project<float>(int64_t, int, int, const double*, const double*, const double*, float*, cudaStream_t);
template int launch_eval<double>(int64_t, int, int, const double*, const double*, const double*, double*, cudaStream_t);
template int launch_eval<float>(int64_t, int, int, const double*, const double*, const float*, double*, cudaStream_t);

template <typename real>
size_t phase_smem_bytes(const KParams<real>& P) {
    return (size_t)kWarps * P.warp_smem * sizeof(real);
}

template <typename real>
int launch_phase_H(const KParams<real>& P, int grid, double dt, double a_lo, double c_out, double* partials,
                   cudaStream_t s) {
    const size_t smem = phase_smem_bytes(P);
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_phase_H<real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_phase_H<real><<<grid, kWarps * 32, smem, s>>>(P, dt, a_lo, c_out, partials);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

template <typename real>
int launch_phase_E(const KParams<real>& P, int grid, double dt, cudaStream_t s) {
    const size_t smem = phase_smem_bytes(P);
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_phase_E<real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_phase_E<real><<<grid, kWarps * 32, smem, s>>>(P, dt);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

template <typename real>
int launch_import(const double* src, real* dst, const double* nrm, int64_t n, int ncoef, cudaStream_t s) {
    if (n == 0) return 0;
    const int64_t blocks = (n + 255) / 256;
    k_import<real><<<(int)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(src, dst, nrm, n, ncoef);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

template <typename real>
int launch_export(const real* src, double* dst, const double* nrm, int64_t n, int ncoef, cudaStream_t s) {
    if (n == 0) return 0;
    const int64_t blocks = (n + 255) / 256;
    k_export<real><<<(int)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(src, dst, nrm, n, ncoef);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

template <typename real>
int launch_axpby(int64_t n, double a, const real* x, double b, real* y, cudaStream_t s) {
    if (n == 0) return 0;
    const int64_t blocks = (n + 255) / 256;
    k_axpby<real><<<(int)(blocks < 8192 ? blocks : 8192), 256, 0, s>>>(n, a, x, b, y);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}
template int launch_axpby<double>(int64_t, double, const double*, double, double*, cudaStream_t);
template int launch_axpby<float>(int64_t, double, const float*, double, float*, cudaStream_t);

int launch_energy_reduce(const double* partials, int n, double* out, cudaStream_t s) {
    k_energy_reduce<<<1, 256, 0, s>>>(partials, n, out);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

// ---------------------------------------------------------------------------
// Trace-buffer phase kernels (central flux).  The kernels above recompute, per
// element and face, the neighbour's trace from the neighbour's coefficients:
// every face trace is computed twice per phase.  Here the phase that updates a
// field also writes that field's tangential face traces (degree <= p-1 face
// modes, the only ones the central flux needs, Sec. 3.2.3) once per element
// into a buffer, and the other phase reads its own and its neighbours' traces
// from there.  Lanes run over (face, face mode) pairs -- 4 N2(p-1) of them --
// for the flux and the traces, and over coefficients for curl, lift and update.
// The traces are the same sums in the same order as above.

namespace {

// tangential traces J_i = sum_m t_{f,i,m} sum_a Tr_f[g, a] X_m[a] of the field
// staged in sX [3][N] (one warp), TT = [4][N][N2H] -> row [4][2][N2H]
template <typename real>
__device__ void warp_traces(const real* sX, int N, const real* __restrict__ TT, int N2H, real* row, int lane) {
    for (int item = lane; item < 4 * N2H; item += 32) {
        const int f = item / N2H, gm = item - f * N2H;
        const real* T = TT + (size_t)f * N * N2H + gm;
        real t0 = 0, t1 = 0, t2 = 0;
        for (int a = 0; a < N; ++a) {
            const real w = ld(T + (size_t)a * N2H);
            t0 += w * sX[a];
            t1 += w * sX[N + a];
            t2 += w * sX[2 * N + a];
        }
        row[(2 * f) * N2H + gm] = (real)c_that[f][0][0] * t0 + (real)c_that[f][0][1] * t1 + (real)c_that[f][0][2] * t2;
        row[(2 * f + 1) * N2H + gm] =
            (real)c_that[f][1][0] * t0 + (real)c_that[f][1][1] * t1 + (real)c_that[f][1][2] * t2;
    }
}

// flux values of the element's four faces from the trace buffer tr: jump
// (1/2) sigma_f (J - K) for the H-phase, average (1/2) sigma_f (J + K) for the
// E-phase; PEC faces use the ghost state (sigma_f J)
template <typename real, bool JUMP>
__device__ void warp_flux(const real* __restrict__ tr, const int32_t* __restrict__ nbr, int64_t t, double sT, int N2H,
                          real* sF, int lane) {
    for (int item = lane; item < 4 * N2H; item += 32) {
        const int f = item / N2H, gm = item - f * N2H;
        const int32_t nb = nbr[t * 4 + f];
        const double sig = sT * c_sigma_hat[f];
        const real* own = tr + (t * 4 + f) * 2 * N2H;
        const real J0 = own[gm], J1 = own[N2H + gm];
        real a0, a1;
        if (nb >= 0) {
            const real* nbt = tr + ((int64_t)(nb >> 2) * 4 + (nb & 3)) * 2 * N2H;
            const real K0 = nbt[gm], K1 = nbt[N2H + gm];
            a0 = (real)(0.5 * sig) * (JUMP ? J0 - K0 : J0 + K0);
            a1 = (real)(0.5 * sig) * (JUMP ? J1 - K1 : J1 + K1);
        } else {
            a0 = (real)sig * J0;
            a1 = (real)sig * J1;
        }
        sF[(2 * f) * N2H + gm] = a0;
        sF[(2 * f + 1) * N2H + gm] = a1;
    }
}

template <typename real, bool SPARSE>
__global__ void __launch_bounds__(kWarps * 32)
k_phase_H2(KParams<real> P, double dt, double a_lo, double c_out, double* __restrict__ partials) {
    extern __shared__ unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int NE = P.NE, NH = P.NH, N2H = P.N2H;
    real* sE = reinterpret_cast<real*>(smem_raw) + (size_t)wib * P.warp_smem;
    real* sA = sE + 3 * NE;
    real* sHn = sA + 8 * N2H;
    double eacc = 0.0;
    const int64_t nwarps = (int64_t)gridDim.x * kWarps;
    for (int64_t t = (int64_t)blockIdx.x * kWarps + wib; t < P.nt; t += nwarps) {
        const real* Et = P.E + t * 3 * NE;
        for (int k = lane; k < 3 * NE; k += 32) sE[k] = Et[k];
        const double* g = P.geo + t * kGeoStride;
        const double sT = g[kGeoSign];
        warp_flux<real, true>(P.trE, P.nbr, t, sT, N2H, sA, lane);
        __syncwarp();
        const double ginv[6] = {g[0], g[1], g[2], g[3], g[4], g[5]};
        const double gm6[6] = {g[6], g[7], g[8], g[9], g[10], g[11]};
        const double inv_mu = g[kGeoInvMu], mu = g[kGeoMu];
        real* Ht = P.H + t * 3 * NH;
        for (int b = lane; b < NH; b += 32) {
            real cx = 0, cy = 0, cz = 0;
            if (SPARSE) {
                // the nonzeros of row b of D_x, D_y, D_z (Sec. 4.2.2: each derivative of
                // a Dubiner function has few components): curl = (D_y e_z - D_z e_y, ...)
                for (int k = ld(P.ptrH + b), k1 = ld(P.ptrH + b + 1); k < k1; ++k) {
                    const int a = ld(P.idxH + k);
                    const real v = ld(P.valH + k);
                    cy -= v * sE[2 * NE + a];
                    cz += v * sE[NE + a];
                }
                for (int k = ld(P.ptrH + (NH + 1) + b), k1 = ld(P.ptrH + (NH + 1) + b + 1); k < k1; ++k) {
                    const int a = ld(P.idxH + k);
                    const real v = ld(P.valH + k);
                    cx += v * sE[2 * NE + a];
                    cz -= v * sE[a];
                }
                for (int k = ld(P.ptrH + 2 * (NH + 1) + b), k1 = ld(P.ptrH + 2 * (NH + 1) + b + 1); k < k1; ++k) {
                    const int a = ld(P.idxH + k);
                    const real v = ld(P.valH + k);
                    cx -= v * sE[NE + a];
                    cy += v * sE[a];
                }
            } else {
                const real* Dx = P.DT + b;
                const real* Dy = Dx + (size_t)NE * NH;
                const real* Dz = Dy + (size_t)NE * NH;
                for (int a = 0; a < NE; ++a) {
                    const real dx = ld(Dx + (size_t)a * NH), dy = ld(Dy + (size_t)a * NH), dz = ld(Dz + (size_t)a * NH);
                    const real ex = sE[a], ey = sE[NE + a], ez = sE[2 * NE + a];
                    cx += dy * ez - dz * ey;
                    cy += dz * ex - dx * ez;
                    cz += dx * ey - dy * ex;
                }
            }
            real r0 = -(real)sT * cx, r1 = -(real)sT * cy, r2 = -(real)sT * cz;
            for (int f = 0; f < 4; ++f) {
                const real* L = P.TrH + (size_t)f * N2H * NH + b;
                const real* A0 = sA + (2 * f) * N2H;
                const real* A1 = A0 + N2H;
                real u0 = 0, u1 = 0;
                for (int gm = 0; gm < N2H; ++gm) {
                    const real l = ld(L + (size_t)gm * NH);
                    u0 += l * A0[gm];
                    u1 += l * A1[gm];
                }
                r0 += (real)c_that[f][1][0] * u0 - (real)c_that[f][0][0] * u1;
                r1 += (real)c_that[f][1][1] * u0 - (real)c_that[f][0][1] * u1;
                r2 += (real)c_that[f][1][2] * u0 - (real)c_that[f][0][2] * u1;
            }
            const real s = (real)(dt * inv_mu);
            const real d0 = s * ((real)ginv[0] * r0 + (real)ginv[1] * r1 + (real)ginv[2] * r2);
            const real d1 = s * ((real)ginv[1] * r0 + (real)ginv[3] * r1 + (real)ginv[4] * r2);
            const real d2 = s * ((real)ginv[2] * r0 + (real)ginv[4] * r1 + (real)ginv[5] * r2);
            const real h0 = Ht[b], h1 = Ht[NH + b], h2 = Ht[2 * NH + b];
            if (partials) {
                const double l0 = (double)h0 - a_lo * (double)d0, l1 = (double)h1 - a_lo * (double)d1,
                             l2 = (double)h2 - a_lo * (double)d2;
                const double u0 = l0 + (double)d0, u1 = l1 + (double)d1, u2 = l2 + (double)d2;
                eacc += 0.5 * mu *
                        (l0 * (gm6[0] * u0 + gm6[1] * u1 + gm6[2] * u2) + l1 * (gm6[1] * u0 + gm6[3] * u1 + gm6[4] * u2) +
                         l2 * (gm6[2] * u0 + gm6[4] * u1 + gm6[5] * u2));
            }
            real n0, n1, n2;
            if (P.cH) {
                // Kahan: the last update's rounding error re-enters this one
                real* c = P.cH + t * 3 * NH + b;
                const real y0 = (real)c_out * d0 - c[0], y1 = (real)c_out * d1 - c[NH], y2 = (real)c_out * d2 - c[2 * NH];
                n0 = h0 + y0;
                n1 = h1 + y1;
                n2 = h2 + y2;
                c[0] = (n0 - h0) - y0;
                c[NH] = (n1 - h1) - y1;
                c[2 * NH] = (n2 - h2) - y2;
            } else {
                n0 = h0 + (real)c_out * d0;
                n1 = h1 + (real)c_out * d1;
                n2 = h2 + (real)c_out * d2;
            }
            Ht[b] = n0;
            Ht[NH + b] = n1;
            Ht[2 * NH + b] = n2;
            sHn[b] = n0;
            sHn[NH + b] = n1;
            sHn[2 * NH + b] = n2;
        }
        if (partials) {
            const double eps = g[kGeoEps];
            for (int a = lane; a < NE; a += 32) {
                const double e0 = sE[a], e1 = sE[NE + a], e2 = sE[2 * NE + a];
                eacc += 0.5 * eps *
                        (e0 * (gm6[0] * e0 + gm6[1] * e1 + gm6[2] * e2) + e1 * (gm6[1] * e0 + gm6[3] * e1 + gm6[4] * e2) +
                         e2 * (gm6[2] * e0 + gm6[4] * e1 + gm6[5] * e2));
            }
        }
        __syncwarp();
        warp_traces(sHn, NH, P.TrHT, N2H, P.trH + t * 8 * N2H, lane);
        __syncwarp();
    }
    if (partials) block_energy_store(eacc, partials);
}

template <typename real, bool SPARSE>
__global__ void __launch_bounds__(kWarps * 32)
k_phase_E2(KParams<real> P, double dt) {
    extern __shared__ unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int NE = P.NE, NH = P.NH, N2H = P.N2H;
    real* sH = reinterpret_cast<real*>(smem_raw) + (size_t)wib * P.warp_smem;
    real* sB = sH + 3 * NH;
    real* sEn = sB + 8 * N2H;
    const int64_t nwarps = (int64_t)gridDim.x * kWarps;
    for (int64_t t = (int64_t)blockIdx.x * kWarps + wib; t < P.nt; t += nwarps) {
        const real* Ht = P.H + t * 3 * NH;
        for (int k = lane; k < 3 * NH; k += 32) sH[k] = Ht[k];
        const double* g = P.geo + t * kGeoStride;
        const double sT = g[kGeoSign];
        warp_flux<real, false>(P.trH, P.nbr, t, sT, N2H, sB, lane);
        __syncwarp();
        const double ginv[6] = {g[0], g[1], g[2], g[3], g[4], g[5]};
        const double inv_eps = g[kGeoInvEps];
        real* Et = P.E + t * 3 * NE;
        for (int a = lane; a < NE; a += 32) {
            real rx = 0, ry = 0, rz = 0;
            if (SPARSE) {
                // the nonzeros of column a of D_x, D_y, D_z: curl^T = (D_z^T h_y - D_y^T h_z, ...)
                for (int k = ld(P.ptrE + a), k1 = ld(P.ptrE + a + 1); k < k1; ++k) {
                    const int b = ld(P.idxE + k);
                    const real v = ld(P.valE + k);
                    ry += v * sH[2 * NH + b];
                    rz -= v * sH[NH + b];
                }
                for (int k = ld(P.ptrE + (NE + 1) + a), k1 = ld(P.ptrE + (NE + 1) + a + 1); k < k1; ++k) {
                    const int b = ld(P.idxE + k);
                    const real v = ld(P.valE + k);
                    rx -= v * sH[2 * NH + b];
                    rz += v * sH[b];
                }
                for (int k = ld(P.ptrE + 2 * (NE + 1) + a), k1 = ld(P.ptrE + 2 * (NE + 1) + a + 1); k < k1; ++k) {
                    const int b = ld(P.idxE + k);
                    const real v = ld(P.valE + k);
                    rx += v * sH[NH + b];
                    ry -= v * sH[b];
                }
            } else {
                const real* Dx = P.D + a;
                const real* Dy = Dx + (size_t)NH * NE;
                const real* Dz = Dy + (size_t)NH * NE;
                for (int b = 0; b < NH; ++b) {
                    const real dx = ld(Dx + (size_t)b * NE), dy = ld(Dy + (size_t)b * NE), dz = ld(Dz + (size_t)b * NE);
                    const real hx = sH[b], hy = sH[NH + b], hz = sH[2 * NH + b];
                    rx += dz * hy - dy * hz;
                    ry += dx * hz - dz * hx;
                    rz += dy * hx - dx * hy;
                }
            }
            real r0 = (real)sT * rx, r1 = (real)sT * ry, r2 = (real)sT * rz;
            for (int f = 0; f < 4; ++f) {
                const real* L = P.TrEq + (size_t)f * N2H * NE + a;
                const real* B0 = sB + (2 * f) * N2H;
                const real* B1 = B0 + N2H;
                real u0 = 0, u1 = 0;
                for (int gm = 0; gm < N2H; ++gm) {
                    const real l = ld(L + (size_t)gm * NE);
                    u0 += l * B0[gm];
                    u1 += l * B1[gm];
                }
                r0 += (real)c_that[f][1][0] * u0 - (real)c_that[f][0][0] * u1;
                r1 += (real)c_that[f][1][1] * u0 - (real)c_that[f][0][1] * u1;
                r2 += (real)c_that[f][1][2] * u0 - (real)c_that[f][0][2] * u1;
            }
            const real s = (real)(dt * inv_eps);
            const real d0 = s * ((real)ginv[0] * r0 + (real)ginv[1] * r1 + (real)ginv[2] * r2);
            const real d1 = s * ((real)ginv[1] * r0 + (real)ginv[3] * r1 + (real)ginv[4] * r2);
            const real d2 = s * ((real)ginv[2] * r0 + (real)ginv[4] * r1 + (real)ginv[5] * r2);
            const real e0 = Et[a], e1 = Et[NE + a], e2 = Et[2 * NE + a];
            real n0, n1, n2;
            if (P.cE) {
                // Kahan: the last update's rounding error re-enters this one
                real* c = P.cE + t * 3 * NE + a;
                const real y0 = d0 - c[0], y1 = d1 - c[NE], y2 = d2 - c[2 * NE];
                n0 = e0 + y0;
                n1 = e1 + y1;
                n2 = e2 + y2;
                c[0] = (n0 - e0) - y0;
                c[NE] = (n1 - e1) - y1;
                c[2 * NE] = (n2 - e2) - y2;
            } else {
                n0 = e0 + d0;
                n1 = e1 + d1;
                n2 = e2 + d2;
            }
            Et[a] = n0;
            Et[NE + a] = n1;
            Et[2 * NE + a] = n2;
            sEn[a] = n0;
            sEn[NE + a] = n1;
            sEn[2 * NE + a] = n2;
        }
        __syncwarp();
        warp_traces(sEn, NE, P.TrEqT, N2H, P.trE + t * 8 * N2H, lane);
        __syncwarp();
    }
}

// traces of the current E (which = 0) or H (which = 1) of elements [e0, e1)
template <typename real>
__global__ void __launch_bounds__(kWarps * 32) k_traces2(KParams<real> P, int which, int64_t e0, int64_t e1) {
    extern __shared__ unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int N = which == 0 ? P.NE : P.NH, N2H = P.N2H;
    real* sX = reinterpret_cast<real*>(smem_raw) + (size_t)wib * P.warp_smem;
    const real* X = which == 0 ? P.E : P.H;
    real* tr = which == 0 ? P.trE : P.trH;
    const real* TT = which == 0 ? P.TrEqT : P.TrHT;
    const int64_t nwarps = (int64_t)gridDim.x * kWarps;
    for (int64_t t = e0 + (int64_t)blockIdx.x * kWarps + wib; t < e1; t += nwarps) {
        const real* Xt = X + t * 3 * N;
        for (int k = lane; k < 3 * N; k += 32) sX[k] = Xt[k];
        __syncwarp();
        warp_traces(sX, N, TT, N2H, tr + t * 8 * N2H, lane);
        __syncwarp();
    }
}

}  // namespace

int phase_warps_per_block() { return kWarps; }

template <typename real>
int launch_phase_H2(const KParams<real>& P, int grid, double dt, double a_lo, double c_out, double* partials,
                    cudaStream_t s) {
    const size_t smem = phase_smem_bytes(P);
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(P.sparse ? k_phase_H2<real, true> : k_phase_H2<real, false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (P.sparse)
        k_phase_H2<real, true><<<grid, kWarps * 32, smem, s>>>(P, dt, a_lo, c_out, partials);
    else
        k_phase_H2<real, false><<<grid, kWarps * 32, smem, s>>>(P, dt, a_lo, c_out, partials);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

template <typename real>
int launch_phase_E2(const KParams<real>& P, int grid, double dt, cudaStream_t s) {
    const size_t smem = phase_smem_bytes(P);
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(P.sparse ? k_phase_E2<real, true> : k_phase_E2<real, false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (P.sparse)
        k_phase_E2<real, true><<<grid, kWarps * 32, smem, s>>>(P, dt);
    else
        k_phase_E2<real, false><<<grid, kWarps * 32, smem, s>>>(P, dt);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

template <typename real>
int launch_traces2(const KParams<real>& P, int grid, int which, int64_t e0, int64_t e1, cudaStream_t s) {
    if (e1 <= e0) return 0;
    const int64_t need = (e1 - e0 + kWarps - 1) / kWarps;
    const int g = (int)(need < grid ? need : grid);
    const size_t smem = phase_smem_bytes(P);
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_traces2<real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_traces2<real><<<g, kWarps * 32, smem, s>>>(P, which, e0, e1);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

template int launch_phase_H2<double>(const KParams<double>&, int, double, double, double, double*, cudaStream_t);
template int launch_phase_H2<float>(const KParams<float>&, int, double, double, double, double*, cudaStream_t);
template int launch_phase_E2<double>(const KParams<double>&, int, double, cudaStream_t);
template int launch_phase_E2<float>(const KParams<float>&, int, double, cudaStream_t);
template int launch_traces2<double>(const KParams<double>&, int, int, int64_t, int64_t, cudaStream_t);
template int launch_traces2<float>(const KParams<float>&, int, int, int64_t, int64_t, cudaStream_t);

template int launch_phase_H<double>(const KParams<double>&, int, double, double, double, double*, cudaStream_t);
template int launch_phase_H<float>(const KParams<float>&, int, double, double, double, double*, cudaStream_t);
template int launch_phase_E<double>(const KParams<double>&, int, double, cudaStream_t);
template int launch_phase_E<float>(const KParams<float>&, int, double, cudaStream_t);
template int launch_import<double>(const double*, double*, const double*, int64_t, int, cudaStream_t);
template int launch_import<float>(const double*, float*, const double*, int64_t, int, cudaStream_t);
template int launch_export<double>(const double*, double*, const double*, int64_t, int, cudaStream_t);
template int launch_export<float>(const float*, double*, const double*, int64_t, int, cudaStream_t);

// ---------------------------------------------------------------------------
// Element-group phase kernels (central flux, trace buffers, sparse curl).
// The kernels above give one warp one element and spread its coefficients and
// (face, mode) pairs over the lanes; the counts at p = 6 (56, 84 and 84) leave a
// last pass with 20 to 24 of 32 lanes, and the sparse rows of D_x, D_y, D_z
// differ in length, so lanes wait for the longest row of their warp.  Here a
// block takes 32 elements at a time and lane e of every warp works on element e:
// warps split the rows (and the (face, mode) pairs), and every lane of a warp
// runs the same row, so each multiply-add instruction has all 32 lanes busy and
// the table entries it reads are the same for the whole warp.  Fields, flux and
// traces of the group are staged in shared memory (per-element strides odd, so
// the 32 lanes hit distinct banks), and read from and written to global memory
// in whole contiguous rows.  The sums are those of the kernels above, in the
// same order.

namespace {

constexpr int kEG = 32;        // elements per group: one per lane
constexpr int kEGMaxWarps = 16;   // warps per block: chosen per degree, 8 to 16

struct EGLayout {
    int sIn, sF, sOut;         // per-element strides (reals)
    int oF, oOut, total;       // offsets and size of the block's region (reals)
};

__host__ __device__ inline EGLayout eg_layout(int Nin, int Nout, int G) {
    EGLayout L;
    L.sIn = (3 * Nin) | 1;
    L.sF = (8 * G) | 1;
    L.sOut = (3 * Nout) | 1;
    L.oF = kEG * L.sIn;
    L.oOut = L.oF + kEG * L.sF;
    L.total = L.oOut + kEG * L.sOut;
    return L;
}

__device__ void block_energy_store_w(double v, double* out) {
    __shared__ double red[kEGMaxWarps];
    const int W = blockDim.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) red[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < W; ++i) s += red[i];
        out[blockIdx.x] = s;
    }
}

// contiguous rows [t0, t0 + ne) of X ([nt][n] reals) <-> padded shared rows
template <typename real>
__device__ void eg_stage_in(const real* __restrict__ X, int64_t t0, int ne, int n, real* s, int stride) {
    const real* src = X + t0 * n;
    for (int i = threadIdx.x; i < ne * n; i += blockDim.x) {
        const int e = i / n;
        s[e * stride + (i - e * n)] = src[i];
    }
}

template <typename real>
__device__ void eg_stage_out(real* X, int64_t t0, int ne, int n, const real* s, int stride) {
    real* dst = X + t0 * n;
    for (int i = threadIdx.x; i < ne * n; i += blockDim.x) {
        const int e = i / n;
        dst[i] = s[e * stride + (i - e * n)];
    }
}

// flux values of the group's faces from the trace buffer tr (jump for the
// H-phase, average for the E-phase, PEC ghost state on boundary faces) into
// sF [e][f][2][G]; warps over (element, face) pairs, lanes over the 2G values
template <typename real, bool JUMP>
__device__ void eg_flux(const KParams<real>& P, const real* __restrict__ tr, int64_t t0, int ne, real* sF,
                        int stride) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, W = blockDim.x >> 5, G2 = 2 * P.N2H;
    for (int pair = w; pair < 4 * ne; pair += W) {
        const int e = pair >> 2, f = pair & 3;
        const int64_t t = t0 + e;
        const int32_t nb = P.nbr[t * 4 + f];
        const double sig = P.geo[t * kGeoStride + kGeoSign] * c_sigma_hat[f];
        const real* own = tr + (t * 4 + f) * G2;
        const real* nbt = nb >= 0 ? tr + ((int64_t)(nb >> 2) * 4 + (nb & 3)) * G2 : own;
        for (int k = lane; k < G2; k += 32) {
            const real J = own[k];
            real a;
            if (nb >= 0) {
                const real K = nbt[k];
                a = (real)(0.5 * sig) * (JUMP ? J - K : J + K);
            } else {
                a = (real)sig * J;
            }
            sF[e * stride + f * G2 + k] = a;
        }
    }
}

// tangential traces of the staged field sX [e][3][N] into sT [e][f][2][G];
// warps over (face, mode) pairs, lane = element
template <typename real>
__device__ void eg_traces(const real* sX, int N, int sx, const real* __restrict__ TT, int G, real* sT, int st) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, W = blockDim.x >> 5;
    const real* x = sX + lane * sx;
    for (int item = w; item < 4 * G; item += W) {
        const int f = item / G, gm = item - f * G;
        const real* T = TT + (size_t)f * N * G + gm;
        real t0 = 0, t1 = 0, t2 = 0;
        for (int a = 0; a < N; ++a) {
            const real v = ld(T + (size_t)a * G);
            t0 += v * x[a];
            t1 += v * x[N + a];
            t2 += v * x[2 * N + a];
        }
        real* o = sT + lane * st + f * 2 * G + gm;
        o[0] = (real)c_that[f][0][0] * t0 + (real)c_that[f][0][1] * t1 + (real)c_that[f][0][2] * t2;
        o[G] = (real)c_that[f][1][0] * t0 + (real)c_that[f][1][1] * t1 + (real)c_that[f][1][2] * t2;
    }
}

template <typename real>
__global__ void __launch_bounds__(kEGMaxWarps * 32, 1)
k_phase_H3(KParams<real> P, double dt, double a_lo, double c_out, double* __restrict__ partials) {
    extern __shared__ unsigned char smem_raw[];
    real* s = reinterpret_cast<real*>(smem_raw);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, W = blockDim.x >> 5;
    const int NE = P.NE, NH = P.NH, G = P.N2H;
    const EGLayout L = eg_layout(NE, NH, G);
    real* sE = s;
    real* sF = s + L.oF;
    real* sH = s + L.oOut;
    double eacc = 0.0;
    const int64_t ngroups = (P.nt + kEG - 1) / kEG;
    for (int64_t grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
        const int64_t t0 = grp * kEG;
        const int ne = (int)(P.nt - t0 < kEG ? P.nt - t0 : kEG);
        eg_stage_in(P.E, t0, ne, 3 * NE, sE, L.sIn);
        eg_stage_in(P.H, t0, ne, 3 * NH, sH, L.sOut);
        eg_flux<real, true>(P, P.trE, t0, ne, sF, L.sF);
        __syncthreads();
        const bool valid = lane < ne;
        const double* g = P.geo + (t0 + (valid ? lane : 0)) * kGeoStride;
        const double ginv[6] = {g[0], g[1], g[2], g[3], g[4], g[5]};
        const double gm6[6] = {g[6], g[7], g[8], g[9], g[10], g[11]};
        const double sT = g[kGeoSign], inv_mu = g[kGeoInvMu], mu = g[kGeoMu];
        const real* ex = sE + lane * L.sIn;
        const real* fl = sF + lane * L.sF;
        real* hx = sH + lane * L.sOut;
        for (int b = w; b < NH; b += W) {
            real cx = 0, cy = 0, cz = 0;
            for (int k = ld(P.ptrH + b), k1 = ld(P.ptrH + b + 1); k < k1; ++k) {
                const int a = ld(P.idxH + k);
                const real v = ld(P.valH + k);
                cy -= v * ex[2 * NE + a];
                cz += v * ex[NE + a];
            }
            for (int k = ld(P.ptrH + (NH + 1) + b), k1 = ld(P.ptrH + (NH + 1) + b + 1); k < k1; ++k) {
                const int a = ld(P.idxH + k);
                const real v = ld(P.valH + k);
                cx += v * ex[2 * NE + a];
                cz -= v * ex[a];
            }
            for (int k = ld(P.ptrH + 2 * (NH + 1) + b), k1 = ld(P.ptrH + 2 * (NH + 1) + b + 1); k < k1; ++k) {
                const int a = ld(P.idxH + k);
                const real v = ld(P.valH + k);
                cx -= v * ex[NE + a];
                cy += v * ex[a];
            }
            real r0 = -(real)sT * cx, r1 = -(real)sT * cy, r2 = -(real)sT * cz;
            for (int f = 0; f < 4; ++f) {
                const real* Lf = P.TrH + (size_t)f * G * NH + b;
                const real* A0 = fl + f * 2 * G;
                const real* A1 = A0 + G;
                real u0 = 0, u1 = 0;
                for (int gm = 0; gm < G; ++gm) {
                    const real l = ld(Lf + (size_t)gm * NH);
                    u0 += l * A0[gm];
                    u1 += l * A1[gm];
                }
                r0 += (real)c_that[f][1][0] * u0 - (real)c_that[f][0][0] * u1;
                r1 += (real)c_that[f][1][1] * u0 - (real)c_that[f][0][1] * u1;
                r2 += (real)c_that[f][1][2] * u0 - (real)c_that[f][0][2] * u1;
            }
            const real sc = (real)(dt * inv_mu);
            const real d0 = sc * ((real)ginv[0] * r0 + (real)ginv[1] * r1 + (real)ginv[2] * r2);
            const real d1 = sc * ((real)ginv[1] * r0 + (real)ginv[3] * r1 + (real)ginv[4] * r2);
            const real d2 = sc * ((real)ginv[2] * r0 + (real)ginv[4] * r1 + (real)ginv[5] * r2);
            const real h0 = hx[b], h1 = hx[NH + b], h2 = hx[2 * NH + b];
            if (partials && valid) {
                const double l0 = (double)h0 - a_lo * (double)d0, l1 = (double)h1 - a_lo * (double)d1,
                             l2 = (double)h2 - a_lo * (double)d2;
                const double u0 = l0 + (double)d0, u1 = l1 + (double)d1, u2 = l2 + (double)d2;
                eacc += 0.5 * mu *
                        (l0 * (gm6[0] * u0 + gm6[1] * u1 + gm6[2] * u2) + l1 * (gm6[1] * u0 + gm6[3] * u1 + gm6[4] * u2) +
                         l2 * (gm6[2] * u0 + gm6[4] * u1 + gm6[5] * u2));
            }
            hx[b] = h0 + (real)c_out * d0;
            hx[NH + b] = h1 + (real)c_out * d1;
            hx[2 * NH + b] = h2 + (real)c_out * d2;
        }
        if (partials && valid) {
            const double eps = g[kGeoEps];
            for (int a = w; a < NE; a += W) {
                const double e0 = ex[a], e1 = ex[NE + a], e2 = ex[2 * NE + a];
                eacc += 0.5 * eps *
                        (e0 * (gm6[0] * e0 + gm6[1] * e1 + gm6[2] * e2) + e1 * (gm6[1] * e0 + gm6[3] * e1 + gm6[4] * e2) +
                         e2 * (gm6[2] * e0 + gm6[4] * e1 + gm6[5] * e2));
            }
        }
        __syncthreads();
        eg_stage_out(P.H, t0, ne, 3 * NH, sH, L.sOut);
        eg_traces(sH, NH, L.sOut, P.TrHT, G, sF, L.sF);
        __syncthreads();
        eg_stage_out(P.trH, t0, ne, 8 * G, sF, L.sF);
        __syncthreads();
    }
    if (partials) block_energy_store_w(eacc, partials);
}

template <typename real>
__global__ void __launch_bounds__(kEGMaxWarps * 32, 1) k_phase_E3(KParams<real> P, double dt) {
    extern __shared__ unsigned char smem_raw[];
    real* s = reinterpret_cast<real*>(smem_raw);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, W = blockDim.x >> 5;
    const int NE = P.NE, NH = P.NH, G = P.N2H;
    const EGLayout L = eg_layout(NH, NE, G);
    real* sH = s;
    real* sF = s + L.oF;
    real* sE = s + L.oOut;
    const int64_t ngroups = (P.nt + kEG - 1) / kEG;
    for (int64_t grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
        const int64_t t0 = grp * kEG;
        const int ne = (int)(P.nt - t0 < kEG ? P.nt - t0 : kEG);
        eg_stage_in(P.H, t0, ne, 3 * NH, sH, L.sIn);
        eg_stage_in(P.E, t0, ne, 3 * NE, sE, L.sOut);
        eg_flux<real, false>(P, P.trH, t0, ne, sF, L.sF);
        __syncthreads();
        const bool valid = lane < ne;
        const double* g = P.geo + (t0 + (valid ? lane : 0)) * kGeoStride;
        const double ginv[6] = {g[0], g[1], g[2], g[3], g[4], g[5]};
        const double sT = g[kGeoSign], inv_eps = g[kGeoInvEps];
        const real* hx = sH + lane * L.sIn;
        const real* fl = sF + lane * L.sF;
        real* ex = sE + lane * L.sOut;
        for (int a = w; a < NE; a += W) {
            real rx = 0, ry = 0, rz = 0;
            for (int k = ld(P.ptrE + a), k1 = ld(P.ptrE + a + 1); k < k1; ++k) {
                const int b = ld(P.idxE + k);
                const real v = ld(P.valE + k);
                ry += v * hx[2 * NH + b];
                rz -= v * hx[NH + b];
            }
            for (int k = ld(P.ptrE + (NE + 1) + a), k1 = ld(P.ptrE + (NE + 1) + a + 1); k < k1; ++k) {
                const int b = ld(P.idxE + k);
                const real v = ld(P.valE + k);
                rx -= v * hx[2 * NH + b];
                rz += v * hx[b];
            }
            for (int k = ld(P.ptrE + 2 * (NE + 1) + a), k1 = ld(P.ptrE + 2 * (NE + 1) + a + 1); k < k1; ++k) {
                const int b = ld(P.idxE + k);
                const real v = ld(P.valE + k);
                rx += v * hx[NH + b];
                ry -= v * hx[b];
            }
            real r0 = (real)sT * rx, r1 = (real)sT * ry, r2 = (real)sT * rz;
            for (int f = 0; f < 4; ++f) {
                const real* Lf = P.TrEq + (size_t)f * G * NE + a;
                const real* B0 = fl + f * 2 * G;
                const real* B1 = B0 + G;
                real u0 = 0, u1 = 0;
                for (int gm = 0; gm < G; ++gm) {
                    const real l = ld(Lf + (size_t)gm * NE);
                    u0 += l * B0[gm];
                    u1 += l * B1[gm];
                }
                r0 += (real)c_that[f][1][0] * u0 - (real)c_that[f][0][0] * u1;
                r1 += (real)c_that[f][1][1] * u0 - (real)c_that[f][0][1] * u1;
                r2 += (real)c_that[f][1][2] * u0 - (real)c_that[f][0][2] * u1;
            }
            const real sc = (real)(dt * inv_eps);
            const real d0 = sc * ((real)ginv[0] * r0 + (real)ginv[1] * r1 + (real)ginv[2] * r2);
            const real d1 = sc * ((real)ginv[1] * r0 + (real)ginv[3] * r1 + (real)ginv[4] * r2);
            const real d2 = sc * ((real)ginv[2] * r0 + (real)ginv[4] * r1 + (real)ginv[5] * r2);
            ex[a] += d0;
            ex[NE + a] += d1;
            ex[2 * NE + a] += d2;
        }
        __syncthreads();
        eg_stage_out(P.E, t0, ne, 3 * NE, sE, L.sOut);
        eg_traces(sE, NE, L.sOut, P.TrEqT, G, sF, L.sF);
        __syncthreads();
        eg_stage_out(P.trE, t0, ne, 8 * G, sF, L.sF);
        __syncthreads();
    }
}

}  // namespace

template <typename real>
size_t phase_eg_smem_bytes(const KParams<real>& P) {
    const EGLayout a = eg_layout(P.NE, P.NH, P.N2H), b = eg_layout(P.NH, P.NE, P.N2H);
    return (size_t)(a.total > b.total ? a.total : b.total) * sizeof(real);
}

// warps per block: the one from 8 to wmax (<= 16) that leaves the fewest idle
// warps over the rows of H, the rows of E and the (face, mode) pairs (ties: more
// warps); wmax = 8 when two blocks share an SM, whose registers hold 16 warps
int phase_eg_warps(int NE, int NH, int G, int wmax) {
    if (wmax > kEGMaxWarps) wmax = kEGMaxWarps;
    if (wmax < 8) wmax = 8;
    int best = 8;
    double best_eff = 0.0;
    for (int W = 8; W <= wmax; ++W) {
        const int c[3] = {NH, NE, 4 * G};
        double used = 0.0, slots = 0.0;
        for (int n : c) {
            used += n;
            slots += (double)W * ((n + W - 1) / W);
        }
        const double eff = used / slots;
        if (eff >= best_eff - 1e-12) {
            best_eff = eff;
            best = W;
        }
    }
    return best;
}

template <typename real>
int launch_phase_H3(const KParams<real>& P, int grid, double dt, double a_lo, double c_out, double* partials,
                    cudaStream_t s) {
    const size_t smem = phase_eg_smem_bytes(P);
    if (P.eg_warps < 1 || P.eg_warps > kEGMaxWarps) return -1;
    if (cudaFuncSetAttribute(k_phase_H3<real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return -1;
    k_phase_H3<real><<<grid, P.eg_warps * 32, smem, s>>>(P, dt, a_lo, c_out, partials);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

template <typename real>
int launch_phase_E3(const KParams<real>& P, int grid, double dt, cudaStream_t s) {
    const size_t smem = phase_eg_smem_bytes(P);
    if (P.eg_warps < 1 || P.eg_warps > kEGMaxWarps) return -1;
    if (cudaFuncSetAttribute(k_phase_E3<real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return -1;
    k_phase_E3<real><<<grid, P.eg_warps * 32, smem, s>>>(P, dt);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

template size_t phase_eg_smem_bytes<double>(const KParams<double>&);
template size_t phase_eg_smem_bytes<float>(const KParams<float>&);
template int launch_phase_H3<double>(const KParams<double>&, int, double, double, double, double*, cudaStream_t);
template int launch_phase_H3<float>(const KParams<float>&, int, double, double, double, double*, cudaStream_t);
template int launch_phase_E3<double>(const KParams<double>&, int, double, cudaStream_t);
template int launch_phase_E3<float>(const KParams<float>&, int, double, cudaStream_t);

}  // namespace dgm
