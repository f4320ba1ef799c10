// 2D triangle solver (TE fields): kernel parameters and launchers.
//
// Per element, in the orthonormalised basis psi'_a = psi_a / ||psi_a|| of
// Eq. (4) (the central-flux system of Sec. 2.1 for E in the plane, H along z):
//   E-phase:  E_a += dt/(eps |det F|) G^{-1} r_a,  G^{-1} = F^T F,
//     r_{0,a} = -s_T sum_b D_y[b][a] H_b - sum_f sigma_f tau_f,0 sum_g TrE_f[g][a] K_{f,g}
//     r_{1,a} =  s_T sum_b D_x[b][a] H_b - sum_f sigma_f tau_f,1 sum_g TrE_f[g][a] K_{f,g}
//     K_{f,g} = {{H}} on edge f in edge mode g (g < p)
//   H-phase:  H_b += dt/(mu |det F|) r_b,
//     r_b = -s_T sum_a (D_x[b][a] E_{1,a} - D_y[b][a] E_{0,a}) + sum_f sum_g TrH_f[g][b] Q_{f,g}
//     Q_{f,g} = sigma_f (J_own - J_nbr)_g / 2 (PEC: sigma_f J_own,g),
//     J_g = sum_a TrE_f[g][a] (tau_f . E_a), the tangential trace in edge mode g < p
// s_T = sign det F; tau_f the reference vector of edge f (from its lower vertex
// to its higher one; both sides of an edge run it the same way, because
// vertices are ordered by key); sigma_f = +-1 the orientation of the physical
// edge vector against the outward normal turned counter-clockwise (so that
// n x E = sigma_f E . tau / |tau|, and |tau| cancels against the edge length).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace dgm {

constexpr int kGeo2Stride = 12;   // doubles per element
// [0..2] G^{-1} = F^T F (00, 01, 11); [3..5] G = F^{-1} F^{-T} (00, 01, 11);
// [6] |det F|; [7] s_T; [8] eps; [9] mu; [10] unused; [11] unused

template <typename real>
struct KParams2D {
    int64_t nt;
    int p, NE, NH;               // NE = N2(p), NH = N2(p-1); edge modes used: p
    real* E;                     // [nt][2][NE] orthonormalised coefficients
    real* H;                     // [nt][NH]
    const double* geo;           // [nt][kGeo2Stride]
    const int32_t* nbr;          // [nt][3] = 3*neighbour + its local edge, or -1 (PEC)
    const int8_t* sig;           // [nt][3] sigma_f
    const real* Dx;              // [NH][NE]
    const real* Dy;              // [NH][NE]
    const real* TrE;             // [3][p+1][NE]
    const real* TrH;             // [3][p][NH]
};

template <typename real>
int launch2d_phase_H(const KParams2D<real>& P, double dt, double a_lo, double c_out, double* partials, int grid,
                     cudaStream_t s);
template <typename real>
int launch2d_phase_E(const KParams2D<real>& P, double dt, int grid, cudaStream_t s);
int phase2d_warps_per_block();

}  // namespace dgm
