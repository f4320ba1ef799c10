// Handle structures behind the opaque C types of include/dgm.h (internal).
#pragma once

#include <cstdint>
#include <vector>

#include "dgm_internal.h"
#include "kernels.h"

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
    int grid = 0;
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
};
