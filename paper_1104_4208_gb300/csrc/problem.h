// Handle structures behind the opaque C types of include/dgm.h (internal).
#pragma once

#include <cstdint>
#include <vector>

#include "dgm_internal.h"
#include "kernels.h"
#include "tc_kernels.h"

struct dgm_ctx {
    int device = 0;
    int num_sms = 0;
};

struct dgm_mesh {
    dgm_ctx* ctx = nullptr;
    dgm::MeshData m;
};

struct dgm_problem {
    dgm_ctx* ctx = nullptr;
    int p = 0;
    dgm_options opt{};
    dgm::RefTables tab;
    int64_t nt = 0, nfaces = 0;
    int NE = 0, NH = 0, N2E = 0, N2H = 0;
    bool fp32 = false;
    int grid = 0;                        // blocks of the CUDA-core phase kernels (autotuned)
    int grid_cap = 0;                    // largest grid the partial sums are sized for
    void* dE = nullptr;
    void* dH = nullptr;
    void* dTables = nullptr;
    double* dGeo = nullptr;
    int32_t* dNbr = nullptr;
    double* dNrmE = nullptr;
    double* dNrmH = nullptr;
    double* dPartials = nullptr;
    double* dEnergy = nullptr;
    int64_t energy_cap = 0;
    double* dStage = nullptr;
    dgm::KParams<double> kd{};
    dgm::KParams<float> kf{};
    std::vector<double> eps, mu;
    double* dMaps = nullptr;             // [nt][12] X0, F (setup and diagnostics only)
    int rule_q1d = 0;                    // cached projection rule
    double* dWphiE = nullptr;            // [nq][NE] w_q phi'_a
    double* dWphiH = nullptr;
    double* dPhiE = nullptr;             // [nq][NE] phi'_a
    double* dPhiH = nullptr;
    void* dK = nullptr;                  // stabilized flux: H^F [nfaces][2][N2E]
    double* dFaceGeo = nullptr;          // [nfaces][kFaceGeoStride]
    int32_t* dFid = nullptr;             // [nt][4]
    double* dNrmF = nullptr;             // [N2E] ||psi_g||
    // CUDA-core precisions, central flux: tangential face-trace buffers of E and H
    // ([nt][4][2][N2(p-1)]), valid per the trE_valid / trH_valid flags below
    void* dTrE = nullptr;
    void* dTrH = nullptr;
    void* dComp = nullptr;               // compensated update: [nE + nH] floats (E terms, then H)
    // tensor-core path (precisions TC32, TC16)
    bool tc = false;
    int tc_grid = 0;                     // CTAs of the tensor-core kernels (autotuned)
    int tc_grid_cap = 0;                 // largest tc_grid the partial sums are sized for
    // with trE_valid: tiles (blocks of 128 elements) whose E traces are stale (point
    // sources, adjoint observation sources); more than kMaxDirtyTiles of them clear
    // trE_valid instead (one-tile
    // refreshes are separate launches: beyond two, one pass over all tiles was faster
    // on a 192-tile mesh)
    static constexpr int kMaxDirtyTiles = 2;
    int trE_dirty[kMaxDirtyTiles] = {};
    int trE_ndirty = 0;
    dgm::TCArgs tca{};
    void* dTc = nullptr;                 // one allocation: tiled state, traces, tables, partials
    double* dTcGeo = nullptr;
    int32_t* dTcNbr = nullptr;
    int* dErr = nullptr;
    int tc_stall_tests = 0;              // phase launches still to run as failure injections
    bool trE_valid = false, trH_valid = false;
    std::vector<double> hmaps;           // [nt][12] X0, F (host copy, point location)
    double time = 0.0;                   // time of the state (advanced by dgm_run)
    // point dipole source (dgm_set_source)
    bool src_on = false;
    int64_t src_elem = -1;
    double src_t0 = 0.0, src_tau = 1.0, src_amp = 0.0;
    double* dSrc = nullptr;              // [3 + NE]: v = G^{-1} F^{-1} dir / eps, phi'(xh_s)
    double* dSrcF = nullptr;             // [src_cap] f(t_{n+1/2}) of the current run
    int64_t src_cap = 0;
    std::vector<double> hgeo;            // [nt][kGeoStride] (host copy)
};

struct dgm_batch {
    dgm_ctx* ctx = nullptr;
    std::vector<dgm_problem*> probs;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> joins;
    cudaEvent_t fork = nullptr;
    cudaStream_t cap = nullptr;          // capture stream (the legacy default stream cannot be captured)
    cudaGraphExec_t exec = nullptr;
    int64_t g_nsteps = -1;
    std::vector<double> g_dt;
    bool g_energy = false;
    cudaStream_t g_stream = nullptr;
};

namespace dgm {
int tc_problem_init(dgm_problem* P, const MeshData& m, const std::vector<double>& geo,
                    const std::vector<int32_t>& nbr);
void tc_problem_free(dgm_problem* P);
int tc_import(dgm_problem* P, const double* dE, const double* dH, const double* nrmE, const double* nrmH,
              cudaStream_t s);
int tc_export(dgm_problem* P, double* dE, double* dH, const double* nrmE, const double* nrmH, cudaStream_t s);
// the problem's kernel arguments for one phase launch (a pending failure
// injection of dgm_inject_wait_timeout is consumed here)
TCArgs tc_launch_args(dgm_problem* P);
int tc_phase_H(dgm_problem* P, double dt, double a_lo, double c_out, double* energy_slot, cudaStream_t s);
int tc_phase_E(dgm_problem* P, double dt, bool energy, cudaStream_t s);
int tc_traces(dgm_problem* P, int which, cudaStream_t s);
// make the E traces current before an H-phase: all tiles if they are invalid
// (or if the H-phase needs E's energy partials), else the tiles that point
// sources changed
int tc_ensure_traces_E(dgm_problem* P, bool energy, cudaStream_t s);
// record that E changed inside one tile only (its traces are stale)
void tc_mark_tile_dirty(dgm_problem* P, int64_t tile);
int tc_state_energy(dgm_problem* P, double* slot, cudaStream_t s);
int tc_check_error(dgm_problem* P);
}  // namespace dgm
