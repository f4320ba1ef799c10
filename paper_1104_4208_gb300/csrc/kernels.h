// Launch interface of the CUDA kernels (host side, no torch types).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace dgm {

// Per-element geometry record (FP64), kGeoStride doubles per element:
//   [0..5]  G^{-1} = F^T F / |det F|         (xx, xy, xz, yy, yz, zz)
//   [6..11] G      = |det F| F^{-1} F^{-T}   (same order)
//   [12] eps  [13] 1/eps  [14] mu  [15] 1/mu  [16] sign(det F)
constexpr int kGeoStride = 20;
constexpr int kGeoEps = 12, kGeoInvEps = 13, kGeoMu = 14, kGeoInvMu = 15, kGeoSign = 16;

template <typename real>
struct KParams {
    int64_t nt;
    int NE, NH, N2E, N2H;
    int warp_smem;              // reals of shared memory per warp
    real* E;                    // [nt][3][NE] orthonormalised coefficients
    real* H;                    // [nt][3][NH]
    const double* geo;          // [nt][kGeoStride]
    const int32_t* nbr;         // [nt][4] = 4*neighbour + neighbour's local face, or -1 (PEC)
    const real* DT;             // [3][NE][NH]   D_d transposed
    const real* D;              // [3][NH][NE]
    const real* TrEqT;          // [4][NE][N2H]  E trace onto the face modes up to H's degree, transposed
    const real* TrEq;           // [4][N2H][NE]
    const real* TrHT;           // [4][NH][N2H]  H trace, transposed
    const real* TrH;            // [4][N2H][NH]
    // stabilized central flux (K == nullptr: central flux)
    real* K;                    // [nfaces][2][N2E] face unknown H^F, covariant tangential, orthonormal
    const double* fgeo;         // [nfaces][kFaceGeoStride]
    const int32_t* fid;         // [nt][4] = 2*face + (1 if this element side updates the face)
    const real* TrEfT;          // [4][NE][N2E]  E trace onto all degree <= p face modes, transposed
    const real* TrEf;           // [4][N2E][NE]
    // central flux, trace-buffer kernels: tangential face traces of E and H on the
    // face modes up to H's degree, [nt][4 faces][2 tangents][N2H], written by the phase
    // that updates the field and read (own and neighbour side) by the other phase
    real* trE;
    real* trH;
    // sparse form of the derivative tables (their exact zeros skipped): per direction d,
    // H-phase rows b: entries [ptrH[d][b], ptrH[d][b+1]) of (a, D_d[b][a]);
    // E-phase columns a: entries [ptrE[d][a], ptrE[d][a+1]) of (b, D_d[b][a])
    // compensated update (FP32 option): the rounding error of each coefficient's last
    // update, [nt][3][N] like the fields (nullptr: plain update)
    real* cE;
    real* cH;
    int sparse;                 // 1: the trace-buffer kernels apply the curl in sparse form
    int eg;                     // 1: element-group kernels (32 elements per block, lane = element)
    int eg_warps;               // their warps per block (phase_eg_warps)
    const int32_t* ptrH;        // [3][NH+1]
    const int32_t* idxH;
    const real* valH;
    const int32_t* ptrE;        // [3][NE+1]
    const int32_t* idxE;
    const real* valE;
};

// Per-face record of the stabilized flux (FP64), kFaceGeoStride doubles:
//   [0] alpha / (h_F |t1 x t2|)     rate of H^F
//   [1..3] g = (t_i . t_j): g11, g12, g22
//   [4] (h_F / alpha) |t1 x t2|     energy weight
//   [5..7] g^{-1}: 11, 12, 22
constexpr int kFaceGeoStride = 8;

int upload_face_frames(const double that[4][2][3], const double sigma_hat[4]);

template <typename real>
int launch_phase_H(const KParams<real>& P, int grid, double dt, double a_lo, double c_out, double* partials,
                   cudaStream_t s);
template <typename real>
int launch_phase_E(const KParams<real>& P, int grid, double dt, cudaStream_t s);
template <typename real>
int launch_import(const double* src, real* dst, const double* nrm, int64_t n, int ncoef, cudaStream_t s);
template <typename real>
int launch_export(const real* src, double* dst, const double* nrm, int64_t n, int ncoef, cudaStream_t s);
template <typename real>
int launch_project(int64_t nt, int N, int nq, const double* maps, const double* wphi, const double* pts, real* out,
                   cudaStream_t s);
template <typename real>
int launch_eval(int64_t nt, int N, int nq, const double* maps, const double* phi, const real* c, double* pts,
                cudaStream_t s);
int launch_energy_reduce(const double* partials, int n, double* out, cudaStream_t s);
// trace-buffer phase kernels (central flux): as launch_phase_H / _E, reading the other
// field's traces from its buffer and writing the traces of the updated field
template <typename real>
int launch_phase_H2(const KParams<real>& P, int grid, double dt, double a_lo, double c_out, double* partials,
                    cudaStream_t s);
template <typename real>
int launch_phase_E2(const KParams<real>& P, int grid, double dt, cudaStream_t s);
// traces of the current E (which = 0) or H (which = 1) of elements [e0, e1) into the buffer
template <typename real>
int launch_traces2(const KParams<real>& P, int grid, int which, int64_t e0, int64_t e1, cudaStream_t s);
// element-group phase kernels (central flux, trace buffers, sparse curl): `grid`
// blocks of 32 P.eg_warps threads and phase_eg_smem_bytes(P) bytes of shared
// memory, each taking groups of 32 elements in turn; the H-phase writes one
// energy partial per block
template <typename real>
size_t phase_eg_smem_bytes(const KParams<real>& P);
int phase_eg_warps(int NE, int NH, int G, int wmax);
template <typename real>
int launch_phase_H3(const KParams<real>& P, int grid, double dt, double a_lo, double c_out, double* partials,
                    cudaStream_t s);
template <typename real>
int launch_phase_E3(const KParams<real>& P, int grid, double dt, cudaStream_t s);
template <typename real>
int launch_axpby(int64_t n, double a, const real* x, double b, real* y, cudaStream_t s);
int phase_warps_per_block();

}  // namespace dgm
