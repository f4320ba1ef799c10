// 2D triangle solver (TE fields): the two phases of the leapfrog of Sec. 3 with
// the central flux of Sec. 2.1 (the operator is written out in tri2d.h).
//
// One warp per element: the element's field and, edge by edge, its
// neighbour's field are staged in the warp's shared memory; lanes run over
// edge modes for the traces and over coefficients for the volume curl, the
// lift and the update.  The reference vectors of the three edges are
// constants: edge f joins the two vertices other than f, lower one first.

#include <cuda_runtime.h>

#include "tri2d.h"

namespace dgm {
namespace {

constexpr int kW2 = 4;   // warps per block

__constant__ double c_tau2[3][2] = {{-1.0, 1.0}, {0.0, 1.0}, {1.0, 0.0}};

template <typename real>
__device__ __forceinline__ real ld2(const real* p) {
    return __ldg(p);
}

// reals of shared memory per warp: own field, neighbour field, edge values [3][p]
__host__ __device__ inline int warp2_smem(int NE, int NH, int p) {
    const int n = 2 * NE > NH ? 2 * NE : NH;
    return 2 * n + 3 * p;
}

template <typename real>
__device__ void stage(const real* src, int n, real* dst, int lane) {
    for (int k = lane; k < n; k += 32) dst[k] = src[k];
}

template <typename real>
__global__ void __launch_bounds__(kW2 * 32)
k2d_phase_H(KParams2D<real> P, double dt, double a_lo, double c_out, double* __restrict__ partials) {
    extern __shared__ unsigned char smem2[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int NE = P.NE, NH = P.NH, p = P.p;
    real* sE = reinterpret_cast<real*>(smem2) + (size_t)wib * warp2_smem(NE, NH, p);
    const int n1 = 2 * NE > NH ? 2 * NE : NH;
    real* sN = sE + n1;
    real* sQ = sN + n1;
    double eacc = 0.0;
    const int64_t nwarps = (int64_t)gridDim.x * kW2;
    for (int64_t t = (int64_t)blockIdx.x * kW2 + wib; t < P.nt; t += nwarps) {
        stage(P.E + t * 2 * NE, 2 * NE, sE, lane);
        __syncwarp();
        for (int f = 0; f < 3; ++f) {
            const int32_t nb = P.nbr[t * 3 + f];
            const double sg = (double)P.sig[t * 3 + f];
            if (nb >= 0) {
                stage(P.E + (int64_t)(nb / 3) * 2 * NE, 2 * NE, sN, lane);
                __syncwarp();
            }
            for (int g = lane; g < p; g += 32) {
                const real* T = P.TrE + ((size_t)f * (p + 1) + g) * NE;
                const real t0 = (real)c_tau2[f][0], t1 = (real)c_tau2[f][1];
                real J = 0;
                for (int a = 0; a < NE; ++a) J += ld2(T + a) * (t0 * sE[a] + t1 * sE[NE + a]);
                real q;
                if (nb >= 0) {
                    const int f2 = nb % 3;
                    const real* T2 = P.TrE + ((size_t)f2 * (p + 1) + g) * NE;
                    const real u0 = (real)c_tau2[f2][0], u1 = (real)c_tau2[f2][1];
                    real K = 0;
                    for (int a = 0; a < NE; ++a) K += ld2(T2 + a) * (u0 * sN[a] + u1 * sN[NE + a]);
                    q = (real)(0.5 * sg) * (J - K);
                } else {
                    q = (real)sg * J;
                }
                sQ[f * p + g] = q;
            }
            __syncwarp();
        }
        const double* gm = P.geo + t * kGeo2Stride;
        const double sT = gm[7], vol = gm[6], mu = gm[9];
        const double sc = dt / (mu * vol);
        real* Ht = P.H + t * NH;
        for (int b = lane; b < NH; b += 32) {
            real c = 0;
            for (int a = 0; a < NE; ++a)
                c += ld2(P.Dx + (size_t)b * NE + a) * sE[NE + a] - ld2(P.Dy + (size_t)b * NE + a) * sE[a];
            real r = -(real)sT * c;
            for (int f = 0; f < 3; ++f)
                for (int g = 0; g < p; ++g) r += ld2(P.TrH + ((size_t)f * p + g) * NH + b) * sQ[f * p + g];
            const real d = (real)sc * r;
            const real h = Ht[b];
            if (partials) {
                const double lo = (double)h - a_lo * (double)d, hi = lo + (double)d;
                eacc += 0.5 * mu * vol * lo * hi;
            }
            Ht[b] = h + (real)c_out * d;
        }
        if (partials) {
            const double eps = gm[8], g00 = gm[3], g01 = gm[4], g11 = gm[5];
            for (int a = lane; a < NE; a += 32) {
                const double e0 = sE[a], e1 = sE[NE + a];
                eacc += 0.5 * eps * vol * (e0 * (g00 * e0 + g01 * e1) + e1 * (g01 * e0 + g11 * e1));
            }
        }
        __syncwarp();
    }
    if (partials) {
        __shared__ double red[kW2];
        for (int o = 16; o > 0; o >>= 1) eacc += __shfl_down_sync(0xffffffffu, eacc, o);
        if (lane == 0) red[wib] = eacc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int w = 0; w < kW2; ++w) s += red[w];
            partials[blockIdx.x] = s;
        }
    }
}

template <typename real>
__global__ void __launch_bounds__(kW2 * 32) k2d_phase_E(KParams2D<real> P, double dt) {
    extern __shared__ unsigned char smem2[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int NE = P.NE, NH = P.NH, p = P.p;
    real* sH = reinterpret_cast<real*>(smem2) + (size_t)wib * warp2_smem(NE, NH, p);
    const int n1 = 2 * NE > NH ? 2 * NE : NH;
    real* sN = sH + n1;
    real* sK = sN + n1;
    const int64_t nwarps = (int64_t)gridDim.x * kW2;
    for (int64_t t = (int64_t)blockIdx.x * kW2 + wib; t < P.nt; t += nwarps) {
        stage(P.H + t * NH, NH, sH, lane);
        __syncwarp();
        for (int f = 0; f < 3; ++f) {
            const int32_t nb = P.nbr[t * 3 + f];
            if (nb >= 0) {
                stage(P.H + (int64_t)(nb / 3) * NH, NH, sN, lane);
                __syncwarp();
            }
            for (int g = lane; g < p; g += 32) {
                const real* T = P.TrH + ((size_t)f * p + g) * NH;
                real J = 0;
                for (int b = 0; b < NH; ++b) J += ld2(T + b) * sH[b];
                real avg = J;
                if (nb >= 0) {
                    const real* T2 = P.TrH + ((size_t)(nb % 3) * p + g) * NH;
                    real K = 0;
                    for (int b = 0; b < NH; ++b) K += ld2(T2 + b) * sN[b];
                    avg = (real)0.5 * (J + K);
                }
                sK[f * p + g] = avg;
            }
            __syncwarp();
        }
        const double* gm = P.geo + t * kGeo2Stride;
        const double sT = gm[7], vol = gm[6], eps = gm[8];
        const double sc = dt / (eps * vol);
        const double gi00 = gm[0], gi01 = gm[1], gi11 = gm[2];
        real* Et = P.E + t * 2 * NE;
        for (int a = lane; a < NE; a += 32) {
            real cy = 0, cx = 0;
            for (int b = 0; b < NH; ++b) {
                const real h = sH[b];
                cy += ld2(P.Dy + (size_t)b * NE + a) * h;
                cx += ld2(P.Dx + (size_t)b * NE + a) * h;
            }
            real r0 = -(real)sT * cy, r1 = (real)sT * cx;
            for (int f = 0; f < 3; ++f) {
                real u = 0;
                for (int g = 0; g < p; ++g) u += ld2(P.TrE + ((size_t)f * (p + 1) + g) * NE + a) * sK[f * p + g];
                const real sg = (real)P.sig[t * 3 + f];
                r0 -= sg * (real)c_tau2[f][0] * u;
                r1 -= sg * (real)c_tau2[f][1] * u;
            }
            Et[a] += (real)(sc * (gi00 * (double)r0 + gi01 * (double)r1));
            Et[NE + a] += (real)(sc * (gi01 * (double)r0 + gi11 * (double)r1));
        }
        __syncwarp();
    }
}

}  // namespace

int phase2d_warps_per_block() { return kW2; }

template <typename real>
int launch2d_phase_H(const KParams2D<real>& P, double dt, double a_lo, double c_out, double* partials, int grid,
                     cudaStream_t s) {
    const size_t smem = (size_t)kW2 * warp2_smem(P.NE, P.NH, P.p) * sizeof(real);
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k2d_phase_H<real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return -1;
    k2d_phase_H<real><<<grid, kW2 * 32, smem, s>>>(P, dt, a_lo, c_out, partials);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

template <typename real>
int launch2d_phase_E(const KParams2D<real>& P, double dt, int grid, cudaStream_t s) {
    const size_t smem = (size_t)kW2 * warp2_smem(P.NE, P.NH, P.p) * sizeof(real);
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k2d_phase_E<real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return -1;
    k2d_phase_E<real><<<grid, kW2 * 32, smem, s>>>(P, dt);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

template int launch2d_phase_H<double>(const KParams2D<double>&, double, double, double, double*, int, cudaStream_t);
template int launch2d_phase_H<float>(const KParams2D<float>&, double, double, double, double*, int, cudaStream_t);
template int launch2d_phase_E<double>(const KParams2D<double>&, double, int, cudaStream_t);
template int launch2d_phase_E<float>(const KParams2D<float>&, double, int, cudaStream_t);

}  // namespace dgm
