// C ABI implementation (host).  See include/dgm.h for the contract.

#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "dgm_internal.h"
#include "kernels.h"
#include "problem.h"
#include "adjoint.h"
#include "eigen.h"
#include "fieldio.h"

namespace dgm {

static thread_local std::string g_err;

void set_error(const std::string& msg) { g_err = msg; }

}  // namespace dgm

using dgm::set_error;

namespace {

// largest blocks per SM the autotuner tries for the CUDA-core kernels (the
// allocation-free energy entry point holds at most 4096 block partial sums)
constexpr int kAutotuneMaxBlocksPerSm = 24;

int cuda_fail(cudaError_t e, const char* what) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? DGM_ERR_OOM : DGM_ERR_CUDA;
}

int prepare_source(dgm_problem* P, double t0, double dt, int64_t nsteps);
int apply_source(dgm_problem* P, void* E, int64_t n, double dt, cudaStream_t s);
void* current_E(dgm_problem* P);

#define DGM_CUDA(call)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

template <typename real>
int upload_tables(dgm_problem* P, dgm::KParams<real>& K) {
    const dgm::RefTables& t = P->tab;
    const int NE = t.NE, NH = t.NH, N2H = t.N2H, N2E = t.N2E;
    const size_t nD = (size_t)3 * NE * NH, nT = (size_t)4 * NE * N2H, nTH = (size_t)4 * NH * N2H;
    const bool stab = P->opt.flux == DGM_FLUX_STABILIZED;
    const size_t nTF = stab ? (size_t)4 * NE * N2E : 0;
    std::vector<real> buf(2 * nD + 2 * nT + 2 * nTH + 2 * nTF);
    real* DT = buf.data();
    real* D = DT + nD;
    real* TrEqT = D + nD;
    real* TrEq = TrEqT + nT;
    real* TrHT = TrEq + nT;
    real* TrH = TrHT + nTH;
    for (int d = 0; d < 3; ++d)
        for (int b = 0; b < NH; ++b)
            for (int a = 0; a < NE; ++a) {
                const real v = (real)t.D[d][(size_t)b * NE + a];
                DT[(size_t)d * NE * NH + (size_t)a * NH + b] = v;
                D[(size_t)d * NH * NE + (size_t)b * NE + a] = v;
            }
    for (int f = 0; f < 4; ++f) {
        for (int g = 0; g < N2H; ++g) {
            const int gE = t.pos2H[g];
            for (int a = 0; a < NE; ++a) {
                const real v = (real)t.TrE[f][(size_t)gE * NE + a];
                TrEqT[(size_t)f * NE * N2H + (size_t)a * N2H + g] = v;
                TrEq[(size_t)f * N2H * NE + (size_t)g * NE + a] = v;
            }
            for (int b = 0; b < NH; ++b) {
                const real v = (real)t.TrH[f][(size_t)g * NH + b];
                TrHT[(size_t)f * NH * N2H + (size_t)b * N2H + g] = v;
                TrH[(size_t)f * N2H * NH + (size_t)g * NH + b] = v;
            }
        }
    }
    if (stab) {
        real* TrEfT = TrH + nTH;
        real* TrEf = TrEfT + nTF;
        for (int f = 0; f < 4; ++f)
            for (int g = 0; g < N2E; ++g)
                for (int a = 0; a < NE; ++a) {
                    const real v = (real)t.TrE[f][(size_t)g * NE + a];
                    TrEfT[(size_t)f * NE * N2E + (size_t)a * N2E + g] = v;
                    TrEf[(size_t)f * N2E * NE + (size_t)g * NE + a] = v;
                }
    }
    // sparse form of D_x, D_y, D_z (exact zeros skipped) for the sparse-curl kernels:
    // rows b for the H-phase, columns a for the E-phase
    std::vector<int32_t> ptrH(3 * (NH + 1)), ptrE(3 * (NE + 1)), idxH, idxE;
    std::vector<real> valH, valE;
    for (int d = 0; d < 3; ++d) {
        for (int b = 0; b < NH; ++b) {
            ptrH[d * (NH + 1) + b] = (int32_t)idxH.size();
            for (int a = 0; a < NE; ++a)
                if (t.D[d][(size_t)b * NE + a] != 0.0) {
                    idxH.push_back(a);
                    valH.push_back((real)t.D[d][(size_t)b * NE + a]);
                }
        }
        ptrH[d * (NH + 1) + NH] = (int32_t)idxH.size();
        for (int a = 0; a < NE; ++a) {
            ptrE[d * (NE + 1) + a] = (int32_t)idxE.size();
            for (int b = 0; b < NH; ++b)
                if (t.D[d][(size_t)b * NE + a] != 0.0) {
                    idxE.push_back(b);
                    valE.push_back((real)t.D[d][(size_t)b * NE + a]);
                }
        }
        ptrE[d * (NE + 1) + NE] = (int32_t)idxE.size();
    }
    const size_t nI = ptrH.size() + ptrE.size() + idxH.size() + idxE.size();
    const size_t nIr = (nI * sizeof(int32_t) + sizeof(real) - 1) / sizeof(real);   // ints, in reals
    const size_t o_sp = buf.size();
    buf.resize(o_sp + nIr + valH.size() + valE.size());
    {
        int32_t* ip = reinterpret_cast<int32_t*>(buf.data() + o_sp);
        for (auto* v : {&ptrH, &ptrE, &idxH, &idxE}) {
            std::copy(v->begin(), v->end(), ip);
            ip += v->size();
        }
        std::copy(valH.begin(), valH.end(), buf.begin() + (o_sp + nIr));
        std::copy(valE.begin(), valE.end(), buf.begin() + (o_sp + nIr + valH.size()));
    }
    DGM_CUDA(cudaMalloc(&P->dTables, buf.size() * sizeof(real)));
    DGM_CUDA(cudaMemcpy(P->dTables, buf.data(), buf.size() * sizeof(real), cudaMemcpyHostToDevice));
    {
        const int32_t* ib = reinterpret_cast<const int32_t*>((real*)P->dTables + o_sp);
        K.ptrH = ib;
        K.ptrE = ib + ptrH.size();
        K.idxH = ib + ptrH.size() + ptrE.size();
        K.idxE = K.idxH + idxH.size();
        K.valH = (real*)P->dTables + o_sp + nIr;
        K.valE = K.valH + valH.size();
        K.sparse = P->opt.variant == 2 || P->opt.variant == 3 ? 1 : 0;
        K.eg = P->opt.variant == 3 ? 1 : 0;
    }
    real* base = (real*)P->dTables;
    K.DT = base;
    K.D = base + nD;
    K.TrEqT = base + 2 * nD;
    K.TrEq = base + 2 * nD + nT;
    K.TrHT = base + 2 * nD + 2 * nT;
    K.TrH = base + 2 * nD + 2 * nT + nTH;
    K.TrEfT = stab ? base + 2 * nD + 2 * nT + 2 * nTH : nullptr;
    K.TrEf = stab ? base + 2 * nD + 2 * nT + 2 * nTH + nTF : nullptr;
    return DGM_OK;
}

template <typename real>
void fill_params(dgm_problem* P, dgm::KParams<real>& K) {
    K.nt = P->nt;
    K.NE = P->NE;
    K.NH = P->NH;
    K.N2E = P->N2E;
    K.N2H = P->N2H;
    const bool stab = P->opt.flux == DGM_FLUX_STABILIZED;
    K.warp_smem = std::max(2 * 3 * P->NE, 2 * 3 * P->NH + (stab ? 8 * P->N2E : 0)) + 8 * P->N2H;
    K.E = (real*)P->dE;
    K.H = (real*)P->dH;
    K.geo = P->dGeo;
    K.nbr = P->dNbr;
    K.K = stab ? (real*)P->dK : nullptr;
    K.fgeo = P->dFaceGeo;
    K.fid = P->dFid;
    K.trE = (real*)P->dTrE;
    K.trH = (real*)P->dTrH;
    K.cE = P->dComp ? (real*)P->dComp : nullptr;
    K.cH = P->dComp ? (real*)P->dComp + P->nt * 3 * P->NE : nullptr;
}

// the compensation terms restart at zero whenever the state is replaced from outside
void reset_comp(dgm_problem* P) {
    if (P->dComp) cudaMemset(P->dComp, 0, (size_t)P->nt * 3 * (P->NE + P->NH) * sizeof(float));
}

int ensure_energy(dgm_problem* P, int64_t n) {
    if (n <= P->energy_cap) return DGM_OK;
    if (P->dEnergy) cudaFree(P->dEnergy);
    P->dEnergy = nullptr;
    P->energy_cap = 0;
    DGM_CUDA(cudaMalloc(&P->dEnergy, n * sizeof(double)));
    P->energy_cap = n;
    return DGM_OK;
}

// CUDA-core precisions with the central flux keep face-trace buffers: the phase
// that updates a field writes its traces, the other phase reads them
bool cc_buffered(const dgm_problem* P) { return !P->tc && P->dTrE != nullptr; }

// element-group kernels: do `blocks` resident blocks fit in an SM's shared memory?
bool eg_fits(const dgm_problem* P, int blocks) {
    const size_t need = P->fp32 ? dgm::phase_eg_smem_bytes<float>(P->kf) : dgm::phase_eg_smem_bytes<double>(P->kd);
    int per_block = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&per_block, cudaDevAttrMaxSharedMemoryPerBlockOptin, P->ctx->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, P->ctx->device) != cudaSuccess)
        return false;
    return need + 1024 <= (size_t)per_block && (size_t)blocks * (need + 1024) <= (size_t)per_sm;
}

int cc_traces(dgm_problem* P, int which, int64_t e0, int64_t e1, cudaStream_t s) {
    const int r = P->fp32 ? dgm::launch_traces2<float>(P->kf, P->grid, which, e0, e1, s)
                          : dgm::launch_traces2<double>(P->kd, P->grid, which, e0, e1, s);
    return r ? cuda_fail(cudaGetLastError(), "traces launch") : DGM_OK;
}

// E traces current before an H-phase: all elements if invalid, else the blocks of
// 128 elements that point sources changed
int cc_ensure_traces_E(dgm_problem* P, cudaStream_t s) {
    int rc = DGM_OK;
    if (!P->trE_valid) {
        rc = cc_traces(P, 0, 0, P->nt, s);
    } else {
        for (int i = 0; i < P->trE_ndirty && !rc; ++i) {
            const int64_t e0 = (int64_t)P->trE_dirty[i] * dgm::kTcRows;
            rc = cc_traces(P, 0, e0, std::min<int64_t>(P->nt, e0 + dgm::kTcRows), s);
        }
    }
    if (rc) return rc;
    P->trE_valid = true;
    P->trE_ndirty = 0;
    return DGM_OK;
}

int cc_phase_H(dgm_problem* P, double dt, double a_lo, double c_out, double* partials, cudaStream_t s) {
    if (!cc_buffered(P)) {
        const int r = P->fp32 ? dgm::launch_phase_H<float>(P->kf, P->grid, dt, a_lo, c_out, partials, s)
                              : dgm::launch_phase_H<double>(P->kd, P->grid, dt, a_lo, c_out, partials, s);
        return r ? cuda_fail(cudaGetLastError(), "H-phase launch") : DGM_OK;
    }
    int rc = cc_ensure_traces_E(P, s);
    if (rc) return rc;
    const bool eg = P->fp32 ? P->kf.eg != 0 : P->kd.eg != 0;
    const int r = eg ? (P->fp32 ? dgm::launch_phase_H3<float>(P->kf, P->grid, dt, a_lo, c_out, partials, s)
                                : dgm::launch_phase_H3<double>(P->kd, P->grid, dt, a_lo, c_out, partials, s))
                     : (P->fp32 ? dgm::launch_phase_H2<float>(P->kf, P->grid, dt, a_lo, c_out, partials, s)
                                : dgm::launch_phase_H2<double>(P->kd, P->grid, dt, a_lo, c_out, partials, s));
    if (r) return cuda_fail(cudaGetLastError(), "H-phase launch");
    P->trH_valid = true;
    return DGM_OK;
}

int cc_phase_E(dgm_problem* P, double dt, cudaStream_t s) {
    if (!cc_buffered(P)) {
        const int r = P->fp32 ? dgm::launch_phase_E<float>(P->kf, P->grid, dt, s)
                              : dgm::launch_phase_E<double>(P->kd, P->grid, dt, s);
        return r ? cuda_fail(cudaGetLastError(), "E-phase launch") : DGM_OK;
    }
    if (!P->trH_valid) {
        int rc = cc_traces(P, 1, 0, P->nt, s);
        if (rc) return rc;
        P->trH_valid = true;
    }
    const bool eg = P->fp32 ? P->kf.eg != 0 : P->kd.eg != 0;
    const int r = eg ? (P->fp32 ? dgm::launch_phase_E3<float>(P->kf, P->grid, dt, s)
                                : dgm::launch_phase_E3<double>(P->kd, P->grid, dt, s))
                     : (P->fp32 ? dgm::launch_phase_E2<float>(P->kf, P->grid, dt, s)
                                : dgm::launch_phase_E2<double>(P->kd, P->grid, dt, s));
    if (r) return cuda_fail(cudaGetLastError(), "E-phase launch");
    P->trE_valid = true;
    P->trE_ndirty = 0;
    return DGM_OK;
}

int phase_H(dgm_problem* P, double dt, double a_lo, double c_out, double* energy_slot, cudaStream_t s) {
    if (P->tc) return dgm::tc_phase_H(P, dt, a_lo, c_out, energy_slot, s);
    double* partials = energy_slot ? P->dPartials : nullptr;
    int rc = cc_phase_H(P, dt, a_lo, c_out, partials, s);
    if (rc) return rc;
    if (energy_slot && dgm::launch_energy_reduce(P->dPartials, P->grid, energy_slot, s))
        return cuda_fail(cudaGetLastError(), "energy reduce launch");
    return DGM_OK;
}

int phase_E(dgm_problem* P, double dt, cudaStream_t s, bool energy = false) {
    if (P->tc) return dgm::tc_phase_E(P, dt, energy, s);
    return cc_phase_E(P, dt, s);
}

int import_fields(dgm_problem* P, const double* dEsrc, const double* dHsrc, cudaStream_t s) {
    if (P->tc) return dgm::tc_import(P, dEsrc, dHsrc, P->dNrmE, P->dNrmH, s);
    if (dEsrc) P->trE_valid = false;
    if (dHsrc) P->trH_valid = false;
    reset_comp(P);
    const int64_t nE = P->nt * 3 * P->NE, nH = P->nt * 3 * P->NH;
    int rc = 0;
    if (P->fp32) {
        if (dEsrc) rc |= dgm::launch_import<float>(dEsrc, (float*)P->dE, P->dNrmE, nE, P->NE, s);
        if (dHsrc) rc |= dgm::launch_import<float>(dHsrc, (float*)P->dH, P->dNrmH, nH, P->NH, s);
    } else {
        if (dEsrc) rc |= dgm::launch_import<double>(dEsrc, (double*)P->dE, P->dNrmE, nE, P->NE, s);
        if (dHsrc) rc |= dgm::launch_import<double>(dHsrc, (double*)P->dH, P->dNrmH, nH, P->NH, s);
    }
    return rc ? cuda_fail(cudaGetLastError(), "import launch") : DGM_OK;
}

int import_faces(dgm_problem* P, const double* src, cudaStream_t s) {
    const int64_t n = P->nfaces * 2 * P->N2E;
    int rc = P->fp32 ? dgm::launch_import<float>(src, (float*)P->dK, P->dNrmF, n, P->N2E, s)
                     : dgm::launch_import<double>(src, (double*)P->dK, P->dNrmF, n, P->N2E, s);
    return rc ? cuda_fail(cudaGetLastError(), "import launch") : DGM_OK;
}

int export_faces(dgm_problem* P, double* dst, cudaStream_t s) {
    const int64_t n = P->nfaces * 2 * P->N2E;
    int rc = P->fp32 ? dgm::launch_export<float>((const float*)P->dK, dst, P->dNrmF, n, P->N2E, s)
                     : dgm::launch_export<double>((const double*)P->dK, dst, P->dNrmF, n, P->N2E, s);
    return rc ? cuda_fail(cudaGetLastError(), "export launch") : DGM_OK;
}

int export_fields(dgm_problem* P, double* dEdst, double* dHdst, cudaStream_t s) {
    if (P->tc) return dgm::tc_export(P, dEdst, dHdst, P->dNrmE, P->dNrmH, s);
    const int64_t nE = P->nt * 3 * P->NE, nH = P->nt * 3 * P->NH;
    int rc = 0;
    if (P->fp32) {
        if (dEdst) rc |= dgm::launch_export<float>((const float*)P->dE, dEdst, P->dNrmE, nE, P->NE, s);
        if (dHdst) rc |= dgm::launch_export<float>((const float*)P->dH, dHdst, P->dNrmH, nH, P->NH, s);
    } else {
        if (dEdst) rc |= dgm::launch_export<double>((const double*)P->dE, dEdst, P->dNrmE, nE, P->NE, s);
        if (dHdst) rc |= dgm::launch_export<double>((const double*)P->dH, dHdst, P->dNrmH, nH, P->NH, s);
    }
    return rc ? cuda_fail(cudaGetLastError(), "export launch") : DGM_OK;
}

void free_problem(dgm_problem* P) {
    void* ptrs[] = {P->dE, P->dH, P->dTables, P->dGeo, P->dNbr, P->dNrmE, P->dNrmH,
                    P->dPartials, P->dEnergy, P->dStage, P->dMaps, P->dWphiE, P->dWphiH, P->dPhiE, P->dPhiH,
                    P->dK, P->dFaceGeo, P->dFid, P->dNrmF, P->dSrc, P->dSrcF, P->dTrE, P->dTrH, P->dComp};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    if (P->tc) dgm::tc_problem_free(P);
}

}  // namespace

extern "C" {

int dgm_version(void) { return 100; }

const char* dgm_last_error(void) { return dgm::g_err.c_str(); }

void dgm_default_options(dgm_options* opt) {
    if (!opt) return;
    opt->flux = DGM_FLUX_CENTRAL;
    opt->alpha0 = 1.0;
    opt->precision = DGM_PREC_FP64;
    opt->variant = 0;
    opt->checks = 1;
    opt->compensated = 0;
    opt->equal_order = 0;
}

int dgm_create(dgm_ctx** ctx, int device) {
    if (!ctx) {
        set_error("dgm_create: null output");
        return DGM_ERR_INVALID_ARG;
    }
    *ctx = nullptr;
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || device < 0 || device >= n) {
        set_error(std::string("dgm_create: CUDA device unavailable: ") +
                  (e != cudaSuccess ? cudaGetErrorString(e) : "index out of range"));
        return DGM_ERR_CUDA;
    }
    DGM_CUDA(cudaSetDevice(device));
    dgm_ctx* c = new (std::nothrow) dgm_ctx;
    if (!c) return DGM_ERR_OOM;
    c->device = device;
    DGM_CUDA(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device));
    *ctx = c;
    return DGM_OK;
}

int dgm_destroy(dgm_ctx* ctx) {
    delete ctx;
    return DGM_OK;
}

int dgm_mesh_create(dgm_ctx* ctx, int64_t nv, const double* xyz, int64_t nt, const int32_t* tets,
                    const int32_t* vertex_key, dgm_mesh** out) {
    if (!out) {
        set_error("dgm_mesh_create: null output");
        return DGM_ERR_INVALID_ARG;
    }
    *out = nullptr;
    dgm_mesh* M = new (std::nothrow) dgm_mesh;
    if (!M) return DGM_ERR_OOM;
    M->ctx = ctx;
    int rc = dgm::build_mesh(nv, xyz, nt, tets, vertex_key, M->m);
    if (rc) {
        delete M;
        return rc;
    }
    *out = M;
    return DGM_OK;
}

int dgm_mesh_destroy(dgm_mesh* mesh) {
    delete mesh;
    return DGM_OK;
}

int dgm_mesh_info(const dgm_mesh* mesh, int64_t* nt, int64_t* nfaces, int64_t* nboundary) {
    if (!mesh) {
        set_error("dgm_mesh_info: null mesh");
        return DGM_ERR_INVALID_ARG;
    }
    if (nt) *nt = mesh->m.nt;
    if (nfaces) *nfaces = mesh->m.nfaces;
    if (nboundary) *nboundary = mesh->m.nboundary;
    return DGM_OK;
}

int dgm_problem_create(dgm_ctx* ctx, const dgm_mesh* mesh, int p, const double* eps, const double* mu,
                       const dgm_options* opt, dgm_problem** out) {
    if (!ctx || !mesh || !eps || !mu || !out) {
        set_error("dgm_problem_create: null argument");
        return DGM_ERR_INVALID_ARG;
    }
    *out = nullptr;
    dgm_options o;
    dgm_default_options(&o);
    if (opt) o = *opt;
    if (o.flux != DGM_FLUX_CENTRAL && o.flux != DGM_FLUX_STABILIZED) {
        set_error("dgm_problem_create: unknown flux");
        return DGM_ERR_INVALID_ARG;
    }
    if (o.flux == DGM_FLUX_STABILIZED && !(o.alpha0 > 0.0 && std::isfinite(o.alpha0))) {
        set_error("dgm_problem_create: alpha0 must be positive");
        return DGM_ERR_INVALID_ARG;
    }
    if (o.precision != DGM_PREC_FP64 && o.precision != DGM_PREC_FP32 && o.precision != DGM_PREC_TC32 &&
        o.precision != DGM_PREC_TC16 && o.precision != DGM_PREC_TCBF16 && o.precision != DGM_PREC_TC16X2) {
        set_error("dgm_problem_create: unknown precision");
        return DGM_ERR_INVALID_ARG;
    }
    {
        const bool cc_central = (o.precision == DGM_PREC_FP64 || o.precision == DGM_PREC_FP32) &&
                                o.flux == DGM_FLUX_CENTRAL;
        const bool ok = o.variant == 0 || (o.variant == 1 && (o.precision == DGM_PREC_TC16 || cc_central)) ||
                        ((o.variant == 2 || o.variant == 3) && cc_central);
        if (!ok) {
            set_error("dgm_problem_create: variant 1 exists for TC16 and for FP64/FP32 with the central flux, "
                      "variants 2 and 3 for FP64/FP32 with the central flux; else use 0");
            return DGM_ERR_INVALID_ARG;
        }
        if (o.variant == 3 && o.compensated) {
            set_error("dgm_problem_create: the element-group kernels (variant 3) have no compensated update");
            return DGM_ERR_UNSUPPORTED;
        }
    }
    if (o.equal_order && o.precision != DGM_PREC_FP64 && o.precision != DGM_PREC_FP32) {
        set_error("dgm_problem_create: the equal-order pair exists for FP64 and FP32");
        return DGM_ERR_UNSUPPORTED;
    }
    if (o.compensated && !(o.precision == DGM_PREC_FP32 && o.flux == DGM_FLUX_CENTRAL)) {
        set_error("dgm_problem_create: the compensated update exists for FP32 with the central flux");
        return DGM_ERR_UNSUPPORTED;
    }
    const dgm::MeshData& m = mesh->m;
    for (int64_t t = 0; t < m.nt; ++t)
        if (!(eps[t] > 0.0) || !(mu[t] > 0.0) || !std::isfinite(eps[t]) || !std::isfinite(mu[t])) {
            set_error("dgm_problem_create: eps and mu must be positive and finite");
            return DGM_ERR_INVALID_ARG;
        }
    dgm_problem* P = new (std::nothrow) dgm_problem;
    if (!P) return DGM_ERR_OOM;
    P->ctx = ctx;
    P->p = p;
    P->opt = o;
    int rc = dgm::build_ref_tables(p, P->tab, o.equal_order != 0);
    if (rc) {
        delete P;
        return rc;
    }
    P->nt = m.nt;
    P->nfaces = m.nfaces;
    P->NE = P->tab.NE;
    P->NH = P->tab.NH;
    P->N2E = P->tab.N2E;
    P->N2H = P->tab.N2H;
    P->fp32 = o.precision == DGM_PREC_FP32;
    P->eps.assign(eps, eps + m.nt);
    P->mu.assign(mu, mu + m.nt);
    const int wpb = dgm::phase_warps_per_block();
    const int64_t want = (m.nt + wpb - 1) / wpb;
    P->grid = (int)std::min<int64_t>(want, (int64_t)ctx->num_sms * 16);
    // partial sums sized for the largest grid the autotuner may choose
    P->grid_cap = (int)std::min<int64_t>(want, (int64_t)ctx->num_sms * kAutotuneMaxBlocksPerSm);

    auto fail = [&](int code) {
        free_problem(P);
        delete P;
        return code;
    };
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(cuda_fail(cudaGetLastError(), "cudaSetDevice"));
    const size_t rs = P->fp32 ? sizeof(float) : sizeof(double);
    const int64_t nE = m.nt * 3 * P->NE, nH = m.nt * 3 * P->NH;
    const bool tc = o.precision == DGM_PREC_TC32 || o.precision == DGM_PREC_TC16 || o.precision == DGM_PREC_TCBF16 ||
                    o.precision == DGM_PREC_TC16X2;
    cudaError_t e;
    if (!tc) {
        if ((e = cudaMalloc(&P->dE, nE * rs)) != cudaSuccess) return fail(cuda_fail(e, "alloc E"));
        if ((e = cudaMalloc(&P->dH, nH * rs)) != cudaSuccess) return fail(cuda_fail(e, "alloc H"));
        if ((e = cudaMemset(P->dE, 0, nE * rs)) != cudaSuccess) return fail(cuda_fail(e, "memset E"));
        if ((e = cudaMemset(P->dH, 0, nH * rs)) != cudaSuccess) return fail(cuda_fail(e, "memset H"));
    }
    const bool stab = o.flux == DGM_FLUX_STABILIZED;
    const int64_t nK = stab ? m.nfaces * 2 * P->N2E : 0;
    if (stab) {
        if ((e = cudaMalloc(&P->dK, nK * rs)) != cudaSuccess) return fail(cuda_fail(e, "alloc HF"));
        if ((e = cudaMemset(P->dK, 0, nK * rs)) != cudaSuccess) return fail(cuda_fail(e, "memset HF"));
        // face records: frame of the first side, h_F = min over sides of |det F| / |t1 x t2|
        const double alpha = o.alpha0 * p * p;
        std::vector<double> fg((size_t)m.nfaces * dgm::kFaceGeoStride);
        std::vector<int32_t> fid(4 * m.nt);
        for (int64_t F = 0; F < m.nfaces; ++F) {
            const int32_t s0 = m.face_elem[2 * F], s1 = m.face_elem[2 * F + 1];
            const int64_t t = s0 / 4;
            const int f = s0 % 4;
            int v[3], q = 0;
            for (int r = 0; r < 4; ++r)
                if (r != f) v[q++] = r;
            const double* Xa = &m.xyz[3 * (int64_t)m.tets[4 * t + v[0]]];
            const double* Xb = &m.xyz[3 * (int64_t)m.tets[4 * t + v[1]]];
            const double* Xc = &m.xyz[3 * (int64_t)m.tets[4 * t + v[2]]];
            double t1[3], t2[3];
            for (int d = 0; d < 3; ++d) {
                t1[d] = Xb[d] - Xa[d];
                t2[d] = Xc[d] - Xa[d];
            }
            const double cr[3] = {t1[1] * t2[2] - t1[2] * t2[1], t1[2] * t2[0] - t1[0] * t2[2],
                                  t1[0] * t2[1] - t1[1] * t2[0]};
            const double J = std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
            double hF = std::fabs(m.detF[t]) / J;
            if (s1 >= 0) hF = std::min(hF, std::fabs(m.detF[s1 / 4]) / J);
            const double g11 = t1[0] * t1[0] + t1[1] * t1[1] + t1[2] * t1[2];
            const double g12 = t1[0] * t2[0] + t1[1] * t2[1] + t1[2] * t2[2];
            const double g22 = t2[0] * t2[0] + t2[1] * t2[1] + t2[2] * t2[2];
            const double dg = g11 * g22 - g12 * g12;
            double* r = &fg[(size_t)F * dgm::kFaceGeoStride];
            r[0] = alpha / (hF * J);
            r[1] = g11;
            r[2] = g12;
            r[3] = g22;
            r[4] = hF / alpha * J;
            r[5] = g22 / dg;
            r[6] = -g12 / dg;
            r[7] = g11 / dg;
            fid[s0] = (int32_t)(2 * F + 1);
            if (s1 >= 0) fid[s1] = (int32_t)(2 * F);
        }
        if ((e = cudaMalloc(&P->dFaceGeo, fg.size() * sizeof(double))) != cudaSuccess)
            return fail(cuda_fail(e, "alloc face geo"));
        if ((e = cudaMalloc(&P->dFid, fid.size() * sizeof(int32_t))) != cudaSuccess)
            return fail(cuda_fail(e, "alloc face ids"));
        cudaMemcpy(P->dFaceGeo, fg.data(), fg.size() * sizeof(double), cudaMemcpyHostToDevice);
        cudaMemcpy(P->dFid, fid.data(), fid.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
        std::vector<int> i2;
        dgm::index2(p, i2);
        std::vector<double> nrmF(P->N2E);
        for (int g = 0; g < P->N2E; ++g) nrmF[g] = std::sqrt(dgm::dubiner2_norm2(i2[2 * g], i2[2 * g + 1]));
        if ((e = cudaMalloc(&P->dNrmF, P->N2E * sizeof(double))) != cudaSuccess) return fail(cuda_fail(e, "alloc nrm"));
        cudaMemcpy(P->dNrmF, nrmF.data(), P->N2E * sizeof(double), cudaMemcpyHostToDevice);
    }
    if (o.compensated) {
        const size_t nC = (size_t)m.nt * 3 * (P->NE + P->NH);
        if ((e = cudaMalloc(&P->dComp, nC * sizeof(float))) != cudaSuccess) return fail(cuda_fail(e, "alloc comp"));
        cudaMemset(P->dComp, 0, nC * sizeof(float));
    }
    if (!tc && !stab) {
        // tangential face-trace buffers of the trace-buffer phase kernels
        const size_t nTr = (size_t)m.nt * 8 * P->N2H;
        if ((e = cudaMalloc(&P->dTrE, nTr * rs)) != cudaSuccess) return fail(cuda_fail(e, "alloc traces"));
        if ((e = cudaMalloc(&P->dTrH, nTr * rs)) != cudaSuccess) return fail(cuda_fail(e, "alloc traces"));
        cudaMemset(P->dTrE, 0, nTr * rs);
        cudaMemset(P->dTrH, 0, nTr * rs);
        P->trE_valid = P->trH_valid = false;
    }
    if ((e = cudaMalloc(&P->dStage, std::max(std::max(nE, nH), nK) * sizeof(double))) != cudaSuccess)
        return fail(cuda_fail(e, "alloc staging"));
    if ((e = cudaMalloc(&P->dPartials, (size_t)std::max(P->grid, P->grid_cap) * sizeof(double))) != cudaSuccess)
        return fail(cuda_fail(e, "alloc partials"));

    // geometry records
    std::vector<double> geo((size_t)m.nt * dgm::kGeoStride, 0.0);
    std::vector<int32_t> nbr(4 * m.nt);
    for (int64_t t = 0; t < m.nt; ++t) {
        const double* F = &m.F[9 * t];
        const double det = m.detF[t], ad = std::fabs(det);
        // F^T F
        double FtF[3][3], Finv[3][3], G[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double s = 0.0;
                for (int k = 0; k < 3; ++k) s += F[3 * k + i] * F[3 * k + j];
                FtF[i][j] = s;
            }
        Finv[0][0] = (F[4] * F[8] - F[5] * F[7]) / det;
        Finv[0][1] = (F[2] * F[7] - F[1] * F[8]) / det;
        Finv[0][2] = (F[1] * F[5] - F[2] * F[4]) / det;
        Finv[1][0] = (F[5] * F[6] - F[3] * F[8]) / det;
        Finv[1][1] = (F[0] * F[8] - F[2] * F[6]) / det;
        Finv[1][2] = (F[2] * F[3] - F[0] * F[5]) / det;
        Finv[2][0] = (F[3] * F[7] - F[4] * F[6]) / det;
        Finv[2][1] = (F[1] * F[6] - F[0] * F[7]) / det;
        Finv[2][2] = (F[0] * F[4] - F[1] * F[3]) / det;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double s = 0.0;
                for (int k = 0; k < 3; ++k) s += Finv[i][k] * Finv[j][k];
                G[i][j] = ad * s;
            }
        double* g = &geo[(size_t)t * dgm::kGeoStride];
        const int iu[6] = {0, 0, 0, 1, 1, 2}, ju[6] = {0, 1, 2, 1, 2, 2};
        for (int q = 0; q < 6; ++q) {
            g[q] = FtF[iu[q]][ju[q]] / ad;
            g[6 + q] = G[iu[q]][ju[q]];
        }
        g[dgm::kGeoEps] = eps[t];
        g[dgm::kGeoInvEps] = 1.0 / eps[t];
        g[dgm::kGeoMu] = mu[t];
        g[dgm::kGeoInvMu] = 1.0 / mu[t];
        g[dgm::kGeoSign] = det > 0 ? 1.0 : -1.0;
        for (int f = 0; f < 4; ++f) {
            const int32_t nb = m.nbr[4 * t + f];
            nbr[4 * t + f] = nb >= 0 ? 4 * nb + m.nbr_face[4 * t + f] : -1;
        }
    }
    {
        std::vector<double> maps((size_t)m.nt * 12);
        for (int64_t t = 0; t < m.nt; ++t) {
            const double* X0 = &m.xyz[3 * (int64_t)m.tets[4 * t]];
            for (int d = 0; d < 3; ++d) maps[12 * t + d] = X0[d];
            for (int q = 0; q < 9; ++q) maps[12 * t + 3 + q] = m.F[9 * t + q];
        }
        if ((e = cudaMalloc(&P->dMaps, maps.size() * sizeof(double))) != cudaSuccess)
            return fail(cuda_fail(e, "alloc maps"));
        cudaMemcpy(P->dMaps, maps.data(), maps.size() * sizeof(double), cudaMemcpyHostToDevice);
        P->hmaps = maps;
        P->hgeo = geo;
    }
    if ((e = cudaMalloc(&P->dGeo, geo.size() * sizeof(double))) != cudaSuccess) return fail(cuda_fail(e, "alloc geo"));
    if ((e = cudaMalloc(&P->dNbr, nbr.size() * sizeof(int32_t))) != cudaSuccess) return fail(cuda_fail(e, "alloc nbr"));
    cudaMemcpy(P->dGeo, geo.data(), geo.size() * sizeof(double), cudaMemcpyHostToDevice);
    cudaMemcpy(P->dNbr, nbr.data(), nbr.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
    {
        std::vector<double> nrmE(P->NE), nrmH(P->NH);
        std::vector<int> iH;
        dgm::index3(P->tab.ph, iH);
        for (int a = 0; a < P->NE; ++a) nrmE[a] = std::sqrt(P->tab.norm2E[a]);
        for (int b = 0; b < P->NH; ++b) nrmH[b] = std::sqrt(dgm::dubiner3_norm2(iH[3 * b], iH[3 * b + 1], iH[3 * b + 2]));
        if ((e = cudaMalloc(&P->dNrmE, P->NE * sizeof(double))) != cudaSuccess) return fail(cuda_fail(e, "alloc nrm"));
        if ((e = cudaMalloc(&P->dNrmH, P->NH * sizeof(double))) != cudaSuccess) return fail(cuda_fail(e, "alloc nrm"));
        cudaMemcpy(P->dNrmE, nrmE.data(), P->NE * sizeof(double), cudaMemcpyHostToDevice);
        cudaMemcpy(P->dNrmH, nrmH.data(), P->NH * sizeof(double), cudaMemcpyHostToDevice);
    }
    if (dgm::upload_face_frames(P->tab.that, P->tab.sigma_hat)) return fail(cuda_fail(cudaGetLastError(), "frames"));
    if (tc) {
        rc = dgm::tc_problem_init(P, m, geo, nbr);
    } else if (P->fp32) {
        fill_params(P, P->kf);
        rc = upload_tables<float>(P, P->kf);
    } else {
        fill_params(P, P->kd);
        rc = upload_tables<double>(P, P->kd);
    }
    if (rc) return fail(rc);
    if (!tc && o.variant == 3) {
        if (!eg_fits(P, 1)) {
            set_error("dgm_problem_create: the element-group kernels (variant 3) need more shared memory than a "
                      "block may have at this degree");
            return fail(DGM_ERR_UNSUPPORTED);
        }
        P->grid = std::min(P->grid_cap, ctx->num_sms);
        P->kd.eg_warps = P->kf.eg_warps = dgm::phase_eg_warps(P->NE, P->NH, P->N2H, 16);
    }
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return fail(cuda_fail(e, "setup"));
    *out = P;
    return DGM_OK;
}

int dgm_problem_destroy(dgm_problem* prob) {
    if (!prob) return DGM_OK;
    free_problem(prob);
    delete prob;
    return DGM_OK;
}

int dgm_problem_sizes(const dgm_problem* P, int64_t* nE, int64_t* nH, int64_t* nHF) {
    if (!P) {
        set_error("dgm_problem_sizes: null problem");
        return DGM_ERR_INVALID_ARG;
    }
    if (nE) *nE = P->nt * 3 * P->NE;
    if (nH) *nH = P->nt * 3 * P->NH;
    if (nHF) *nHF = P->opt.flux == DGM_FLUX_STABILIZED ? P->nfaces * 2 * P->N2E : 0;
    return DGM_OK;
}

int dgm_set_fields_device(dgm_problem* P, const double* E, const double* H, const double* HF, void* stream) {
    if (!P) {
        set_error("dgm_set_fields_device: null problem");
        return DGM_ERR_INVALID_ARG;
    }
    if (HF && P->opt.flux != DGM_FLUX_STABILIZED) {
        set_error("dgm_set_fields_device: HF given for the central flux");
        return DGM_ERR_INVALID_ARG;
    }
    int rc = import_fields(P, E, H, (cudaStream_t)stream);
    if (!rc && HF) rc = import_faces(P, HF, (cudaStream_t)stream);
    return rc;
}

int dgm_get_fields_device(dgm_problem* P, double* E, double* H, double* HF, void* stream) {
    if (!P) {
        set_error("dgm_get_fields_device: null problem");
        return DGM_ERR_INVALID_ARG;
    }
    int rc = export_fields(P, E, H, (cudaStream_t)stream);
    if (!rc && HF && P->opt.flux == DGM_FLUX_STABILIZED) rc = export_faces(P, HF, (cudaStream_t)stream);
    return rc;
}

int dgm_set_fields(dgm_problem* P, const double* E, const double* H, const double* HF) {
    if (!P) {
        set_error("dgm_set_fields: null problem");
        return DGM_ERR_INVALID_ARG;
    }
    if (HF && P->opt.flux != DGM_FLUX_STABILIZED) {
        set_error("dgm_set_fields: HF given for the central flux");
        return DGM_ERR_INVALID_ARG;
    }
    const int64_t nE = P->nt * 3 * P->NE, nH = P->nt * 3 * P->NH;
    if (E) {
        DGM_CUDA(cudaMemcpy(P->dStage, E, nE * sizeof(double), cudaMemcpyHostToDevice));
        int rc = import_fields(P, P->dStage, nullptr, 0);
        if (rc) return rc;
    }
    if (H) {
        DGM_CUDA(cudaMemcpy(P->dStage, H, nH * sizeof(double), cudaMemcpyHostToDevice));
        int rc = import_fields(P, nullptr, P->dStage, 0);
        if (rc) return rc;
    }
    if (HF) {
        DGM_CUDA(cudaMemcpy(P->dStage, HF, P->nfaces * 2 * P->N2E * sizeof(double), cudaMemcpyHostToDevice));
        int rc = import_faces(P, P->dStage, 0);
        if (rc) return rc;
    }
    DGM_CUDA(cudaDeviceSynchronize());
    return DGM_OK;
}

int dgm_get_fields(dgm_problem* P, double* E, double* H, double* HF) {
    if (!P) {
        set_error("dgm_get_fields: null problem");
        return DGM_ERR_INVALID_ARG;
    }
    const int64_t nE = P->nt * 3 * P->NE, nH = P->nt * 3 * P->NH;
    DGM_CUDA(cudaDeviceSynchronize());
    if (P->tc) {
        int rc = dgm::tc_check_error(P);
        if (rc) return rc;
    }
    if (HF && P->opt.flux == DGM_FLUX_STABILIZED) {
        int rc = export_faces(P, P->dStage, 0);
        if (rc) return rc;
        DGM_CUDA(cudaMemcpy(HF, P->dStage, P->nfaces * 2 * P->N2E * sizeof(double), cudaMemcpyDeviceToHost));
    }
    if (E) {
        int rc = export_fields(P, P->dStage, nullptr, 0);
        if (rc) return rc;
        DGM_CUDA(cudaMemcpy(E, P->dStage, nE * sizeof(double), cudaMemcpyDeviceToHost));
    }
    if (H) {
        int rc = export_fields(P, nullptr, P->dStage, 0);
        if (rc) return rc;
        DGM_CUDA(cudaMemcpy(H, P->dStage, nH * sizeof(double), cudaMemcpyDeviceToHost));
    }
    return DGM_OK;
}

int dgm_kick(dgm_problem* P, int which, double dt, void* stream) {
    if (!P || (which != 0 && which != 1) || !std::isfinite(dt)) {
        set_error("dgm_kick: bad argument");
        return DGM_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    return which == 0 ? phase_H(P, dt, 0.0, 1.0, nullptr, s) : phase_E(P, dt, s);
}

int dgm_run(dgm_problem* P, double dt, int64_t nsteps, void* stream, double* energy_out) {
    return dgm_run_timed(P, dt, nsteps, stream, energy_out, nullptr);
}

int dgm_run_timed(dgm_problem* P, double dt, int64_t nsteps, void* stream, double* energy_out,
                  dgm_run_stats* stats) {
    if (!P || nsteps < 0 || !std::isfinite(dt)) {
        set_error("dgm_run: bad argument");
        return DGM_ERR_INVALID_ARG;
    }
    if (stats) *stats = dgm_run_stats{};
    if (nsteps == 0) {
        if (energy_out) return dgm_energy(P, energy_out);
        return DGM_OK;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int rc = ensure_energy(P, nsteps + 1);
    if (rc) return rc;
    double* W = P->dEnergy;
    const bool want = energy_out != nullptr;
    // optional event timing: one (start, stop) pair per phase launch
    std::vector<cudaEvent_t> ev;
    std::vector<int> kind;
    auto mark = [&](int k) -> int {
        if (!stats) return DGM_OK;
        cudaEvent_t a, b;
        DGM_CUDA(cudaEventCreate(&a));
        DGM_CUDA(cudaEventCreate(&b));
        DGM_CUDA(cudaEventRecord(a, s));
        ev.push_back(a);
        ev.push_back(b);
        kind.push_back(k);
        return DGM_OK;
    };
    auto done = [&]() -> int {
        if (!stats) return DGM_OK;
        DGM_CUDA(cudaEventRecord(ev.back(), s));
        return DGM_OK;
    };
    auto run_H = [&](double a_lo, double c_out, double* slot) -> int {
        int r = mark(0);
        if (r) return r;
        if (P->tc) {
            // the tensor-core H-phase writes its partials; the reduction is timed separately below
            r = dgm::tc_ensure_traces_E(P, slot != nullptr, s);
            if (r) return r;
            r = dgm::tc_launch_phase_H(dgm::tc_launch_args(P), P->tc_grid, dt, a_lo, c_out, slot ? 1 : 0, s);
            if (r) return cuda_fail(cudaGetLastError(), "H-phase launch");
            P->trH_valid = true;
            if ((r = done())) return r;
            if (slot) {
                if ((r = mark(2))) return r;
                if (dgm::launch_energy_reduce(P->tca.partE, 2 * P->tc_grid, slot, s))
                    return cuda_fail(cudaGetLastError(), "energy reduce launch");
                if ((r = done())) return r;
            }
            return DGM_OK;
        }
        if ((r = cc_phase_H(P, dt, a_lo, c_out, slot ? P->dPartials : nullptr, s))) return r;
        if ((r = done())) return r;
        if (slot) {
            if ((r = mark(2))) return r;
            if (dgm::launch_energy_reduce(P->dPartials, P->grid, slot, s))
                return cuda_fail(cudaGetLastError(), "energy reduce launch");
            if ((r = done())) return r;
        }
        return DGM_OK;
    };
    int64_t step = 0;
    auto run_E = [&]() -> int {
        int r = mark(1);
        if (r) return r;
        r = phase_E(P, dt, s, want);
        if (r) return r;
        if ((r = apply_source(P, current_E(P), step, dt, s))) return r;
        return done();
    };
    rc = prepare_source(P, P->time, dt, nsteps);
    if (!rc && P->tc && want) {
        rc = mark(2);
        if (!rc) rc = dgm::tc_traces(P, 0, s);
        if (!rc) rc = done();
    }
    if (!rc) rc = run_H(0.5, 0.5, want ? W : nullptr);
    for (int64_t n = 0; n < nsteps && !rc; ++n) {
        step = n;
        rc = run_E();
        if (rc) break;
        const bool last = n == nsteps - 1;
        rc = run_H(0.0, last ? 0.5 : 1.0, want ? W + n + 1 : nullptr);
    }
    if (!rc && want) {
        cudaError_t e = cudaMemcpyAsync(energy_out, W, (nsteps + 1) * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) rc = cuda_fail(e, "energy copy");
    }
    if (!rc && (want || stats)) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_fail(e, "run");
        if (!rc && P->tc) rc = dgm::tc_check_error(P);
    }
    if (stats) {
        for (size_t i = 0; i < kind.size() && !rc; ++i) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]);
            if (kind[i] == 0) { stats->h_phase_ms += ms; stats->h_launches++; }
            else if (kind[i] == 1) { stats->e_phase_ms += ms; stats->e_launches++; }
            else { stats->other_ms += ms; stats->other_launches++; }
        }
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
    }
    if (rc) return rc;
    P->time += nsteps * dt;
    if (want) {
        // a point source feeds energy in, so only a non-finite energy is a blow-up then
        for (int64_t n = 0; n <= nsteps; ++n)
            if (!std::isfinite(energy_out[n]) ||
                (!P->src_on && energy_out[n] > 10.0 * std::fabs(energy_out[0]) + 1e-300)) {
                set_error("dgm_run: energy blew up (time step above the stability bound?)");
                return DGM_ERR_UNSTABLE;
            }
    }
    return DGM_OK;
}

int dgm_run_composed(dgm_problem* P, double dt, int64_t nsteps, int order, void* stream) {
    if (!P || nsteps < 0 || !std::isfinite(dt) || (order != 2 && order != 4)) {
        set_error("dgm_run_composed: bad argument (order must be 2 or 4)");
        return DGM_ERR_INVALID_ARG;
    }
    if (P->src_on) {
        set_error("dgm_run_composed: point sources are evaluated at leapfrog midpoints; use dgm_run");
        return DGM_ERR_UNSUPPORTED;
    }
    if (nsteps == 0) return DGM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    // substep weights: one leapfrog step (order 2), or the symmetric triple jump
    // w1, w0, w1 with w1 = 1 / (2 - 2^{1/3}), w0 = 1 - 2 w1 (order 4)
    double w[3] = {1.0, 0.0, 0.0};
    int nw = 1;
    if (order == 4) {
        const double c = std::cbrt(2.0);
        w[0] = w[2] = 1.0 / (2.0 - c);
        w[1] = 1.0 - 2.0 * w[0];
        nw = 3;
    }
    // each substep is kick-drift-kick; adjacent H half kicks are merged
    int rc = phase_H(P, 0.5 * w[0] * dt, 0.0, 1.0, nullptr, s);
    for (int64_t n = 0; n < nsteps && !rc; ++n) {
        for (int k = 0; k < nw && !rc; ++k) {
            rc = phase_E(P, w[k] * dt, s);
            if (rc) break;
            const bool last = n == nsteps - 1 && k == nw - 1;
            const double h = last ? 0.5 * w[k] * dt : 0.5 * (w[k] + w[(k + 1) % nw]) * dt;
            rc = phase_H(P, h, 0.0, 1.0, nullptr, s);
        }
    }
    if (rc) return rc;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "dgm_run_composed");
    if (P->tc && (rc = dgm::tc_check_error(P))) return rc;
    P->time += nsteps * dt;
    return DGM_OK;
}

int dgm_inject_wait_timeout(dgm_problem* P, int nlaunches) {
    if (!P || nlaunches < 0) {
        set_error("dgm_inject_wait_timeout: bad argument");
        return DGM_ERR_INVALID_ARG;
    }
    if (!P->tc) {
        set_error("dgm_inject_wait_timeout: only the tensor-core precisions have bounded waits");
        return DGM_ERR_UNSUPPORTED;
    }
    P->tc_stall_tests = nlaunches;
    return DGM_OK;
}

int dgm_energy(dgm_problem* P, double* W) {
    if (!P || !W) {
        set_error("dgm_energy: null argument");
        return DGM_ERR_INVALID_ARG;
    }
    int rc = ensure_energy(P, 1);
    if (rc) return rc;
    rc = P->tc ? dgm::tc_state_energy(P, P->dEnergy, 0) : phase_H(P, 0.0, 0.0, 0.0, P->dEnergy, 0);
    if (rc) return rc;
    DGM_CUDA(cudaMemcpy(W, P->dEnergy, sizeof(double), cudaMemcpyDeviceToHost));
    return DGM_OK;
}

}  // extern "C"

namespace {

// Element of the mesh containing x (largest minimum barycentric coordinate),
// its reference coordinates and F^{-1} (row-major).  Returns the element or -1.
int64_t locate_point(const dgm_problem* P, const double* x, double* xh_out, double* Fi_out) {
    int64_t best = -1;
    double bestmin = -1e300;
    for (int64_t t = 0; t < P->nt; ++t) {
        const double* M = &P->hmaps[12 * t];
        const double* F = M + 3;
        const double det = F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) +
                           F[2] * (F[3] * F[7] - F[4] * F[6]);
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
        double xh[3];
        for (int i = 0; i < 3; ++i)
            xh[i] = Fi[3 * i] * (x[0] - M[0]) + Fi[3 * i + 1] * (x[1] - M[1]) + Fi[3 * i + 2] * (x[2] - M[2]);
        const double mn = std::min(std::min(xh[0], xh[1]), std::min(xh[2], 1.0 - xh[0] - xh[1] - xh[2]));
        if (mn > bestmin) {
            bestmin = mn;
            best = t;
            std::memcpy(xh_out, xh, sizeof(xh));
            std::memcpy(Fi_out, Fi, sizeof(Fi));
        }
    }
    return bestmin < -1e-10 ? -1 : best;
}

double dipole_waveform(const dgm_problem* P, double t) {
    const double s = (t - P->src_t0) / P->src_tau;
    return -P->src_amp * s * std::exp(-s * s);
}

// f(t0 + (n + 1/2) dt), n = 0..nsteps-1, into the device array of the source
int prepare_source(dgm_problem* P, double t0, double dt, int64_t nsteps) {
    if (!P->src_on) return DGM_OK;
    if (P->src_cap < nsteps) {
        if (P->dSrcF) cudaFree(P->dSrcF);
        P->dSrcF = nullptr;
        P->src_cap = 0;
        DGM_CUDA(cudaMalloc(&P->dSrcF, nsteps * sizeof(double)));
        P->src_cap = nsteps;
    }
    std::vector<double> f(nsteps);
    for (int64_t n = 0; n < nsteps; ++n) f[n] = dipole_waveform(P, t0 + (n + 0.5) * dt);
    DGM_CUDA(cudaMemcpy(P->dSrcF, f.data(), nsteps * sizeof(double), cudaMemcpyHostToDevice));
    return DGM_OK;
}

// E += -dt f(t_{n+1/2}) M_eps^{-1} (dir . e(x_s)) on the source element
int apply_source(dgm_problem* P, void* E, int64_t n, double dt, cudaStream_t s) {
    if (!P->src_on) return DGM_OK;
    const int K = P->tc ? P->tca.d.KE : 0, tiled = P->tc ? P->tca.d.layout : 0;
    const bool f32 = P->tc || P->fp32;
    const int r = f32 ? dgm::add_point_source<float>((float*)E, P->NE, K, tiled, P->src_elem, P->dSrc + 3, P->dSrc,
                                                     P->dSrcF, n, dt, s)
                      : dgm::add_point_source<double>((double*)E, P->NE, K, tiled, P->src_elem, P->dSrc + 3, P->dSrc,
                                                      P->dSrcF, n, dt, s);
    // the source changes E in one element: only its block's E traces are stale
    dgm::tc_mark_tile_dirty(P, P->src_elem / dgm::kTcRows);
    return r ? cuda_fail(cudaGetLastError(), "source launch") : DGM_OK;
}

void* current_E(dgm_problem* P) {
    if (P->tc) return P->tca.E;
    return P->fp32 ? (void*)P->kf.E : (void*)P->kd.E;
}

}  // namespace

extern "C" {

int dgm_set_source(dgm_problem* P, const double* xs, const double* dir, double t0, double tau, double amp) {
    if (!P || !xs || !dir || !(tau > 0.0) || !std::isfinite(t0) || !std::isfinite(amp)) {
        set_error("dgm_set_source: bad argument");
        return DGM_ERR_INVALID_ARG;
    }
    if (amp == 0.0) {
        P->src_on = false;
        return DGM_OK;
    }
    double xh[3], Fi[9];
    const int64_t t = locate_point(P, xs, xh, Fi);
    if (t < 0) {
        set_error("dgm_set_source: point outside the mesh");
        return DGM_ERR_INVALID_ARG;
    }
    std::vector<double> phi;
    dgm::phi_at_points(P->p, xh, 1, phi);
    const double* g = &P->hgeo[(size_t)t * dgm::kGeoStride];
    double w[3];
    for (int m = 0; m < 3; ++m) w[m] = Fi[3 * m] * dir[0] + Fi[3 * m + 1] * dir[1] + Fi[3 * m + 2] * dir[2];
    std::vector<double> rec(3 + P->NE);
    const double ie = g[dgm::kGeoInvEps];
    rec[0] = ie * (g[0] * w[0] + g[1] * w[1] + g[2] * w[2]);
    rec[1] = ie * (g[1] * w[0] + g[3] * w[1] + g[4] * w[2]);
    rec[2] = ie * (g[2] * w[0] + g[4] * w[1] + g[5] * w[2]);
    for (int a = 0; a < P->NE; ++a) rec[3 + a] = phi[a];
    if (!P->dSrc) DGM_CUDA(cudaMalloc(&P->dSrc, rec.size() * sizeof(double)));
    DGM_CUDA(cudaMemcpy(P->dSrc, rec.data(), rec.size() * sizeof(double), cudaMemcpyHostToDevice));
    P->src_elem = t;
    P->src_t0 = t0;
    P->src_tau = tau;
    P->src_amp = amp;
    P->src_on = true;
    return DGM_OK;
}

int dgm_set_time(dgm_problem* P, double t) {
    if (!P || !std::isfinite(t)) {
        set_error("dgm_set_time: bad argument");
        return DGM_ERR_INVALID_ARG;
    }
    P->time = t;
    return DGM_OK;
}

int dgm_get_time(const dgm_problem* P, double* t) {
    if (!P || !t) {
        set_error("dgm_get_time: null argument");
        return DGM_ERR_INVALID_ARG;
    }
    *t = P->time;
    return DGM_OK;
}

namespace {

struct StateView {
    void* E;
    int64_t nE;
    void* H;
    int64_t nH;
    void* K;
    int64_t nK;
    bool f32;
};

StateView state_view(dgm_problem* P) {
    StateView v{};
    if (P->tc) {
        v.E = P->tca.E;
        v.nE = (int64_t)P->tca.ntiles * dgm::kTcRows * P->tca.d.KE;
        v.H = P->tca.H;
        v.nH = (int64_t)P->tca.ntiles * dgm::kTcRows * P->tca.d.KH;
        v.f32 = true;
    } else {
        v.E = P->dE;
        v.nE = P->nt * 3 * P->NE;
        v.H = P->dH;
        v.nH = P->nt * 3 * P->NH;
        v.f32 = P->fp32;
    }
    v.K = P->dK;
    v.nK = P->dK ? P->nfaces * 2 * P->N2E : 0;
    return v;
}

int axpby(const StateView& v, int64_t n, double a, const void* x, double b, void* y) {
    if (!n) return 0;
    return v.f32 ? dgm::launch_axpby<float>(n, a, (const float*)x, b, (float*)y, 0)
                 : dgm::launch_axpby<double>(n, a, (const double*)x, b, (double*)y, 0);
}

}  // namespace

int dgm_autotune(dgm_problem* P, int steps, int* ncand_out, int* cand_config, double* cand_ms, int* chosen_out) {
    if (!P || steps < 1) {
        set_error("dgm_autotune: bad argument");
        return DGM_ERR_INVALID_ARG;
    }
    const int sms = P->ctx->num_sms;
    std::vector<int> cand;
    const bool resident = P->tc && P->tca.d.layout == 2;
    if (resident) {
        cand.push_back(1);   // resident-table kernels: one CTA per SM, nothing to choose
    } else if (P->tc) {
        cand.push_back(1);
        if (P->tc_grid_cap > sms) cand.push_back(2);   // two CTAs per SM allowed
    } else {
        // trace-buffer kernels: the dense and the sparse curl (configuration + 1000)
        // are timed unless the variant option fixed one
        const bool both = cc_buffered(P) && P->opt.variant == 0;
        const int fixed = cc_buffered(P) && P->opt.variant == 2 ? 1000 : 0;
        if (P->opt.variant != 3)
            for (int v : {0, 1000})
                if (both || v == fixed)
                    for (int b : {4, 8, 16, kAutotuneMaxBlocksPerSm}) cand.push_back(b + v);
        // element-group kernels (configuration 2000 + blocks per SM), which have no
        // compensated update
        const bool comp = P->fp32 && P->kf.cE != nullptr;
        if (cc_buffered(P) && !comp && (P->opt.variant == 0 || P->opt.variant == 3))
            for (int b : {1, 2})
                if (eg_fits(P, b)) cand.push_back(2000 + b);
    }
    if (cand.size() > DGM_AUTOTUNE_MAX) cand.resize(DGM_AUTOTUNE_MAX);
    auto apply = [&](int c) {
        if (resident) {
            (void)c;
        } else if (P->tc) {
            P->tc_grid = std::min(P->tc_grid_cap, sms * c);
            P->tca.partH = P->tca.partE + P->tc_grid;   // the reduction sums 2 tc_grid contiguous partials
        } else {
            P->grid = std::min(P->grid_cap, sms * (c % 1000));
            P->kd.sparse = P->kf.sparse = c >= 1000 ? 1 : 0;
            P->kd.eg = P->kf.eg = c >= 2000 ? 1 : 0;
            if (c >= 2000)   // one block per SM: up to 16 warps; two: 8 each (the SM's registers)
                P->kd.eg_warps = P->kf.eg_warps = dgm::phase_eg_warps(P->NE, P->NH, P->N2H, 16 / (c - 2000));
        }
    };
    const int keep_grid = P->grid, keep_tc = P->tc_grid, keep_sparse = P->kd.sparse | P->kf.sparse,
              keep_eg = P->kd.eg | P->kf.eg, keep_egw = P->kd.eg_warps | P->kf.eg_warps;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    DGM_CUDA(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(cudaGetLastError(), "dgm_autotune events");
    }
    std::vector<double> ms(cand.size(), 0.0);
    int rc = DGM_OK;
    for (size_t i = 0; i < cand.size() && !rc; ++i) {
        apply(cand[i]);
        // one warm-up step, then `steps` timed steps, dt = 0 (fields unchanged)
        for (int n = 0; n <= steps && !rc; ++n) {
            if (n == 1 && cudaEventRecord(e0, 0) != cudaSuccess) rc = cuda_fail(cudaGetLastError(), "event");
            if (!rc) rc = phase_E(P, 0.0, 0);
            if (!rc) rc = phase_H(P, 0.0, 0.0, 1.0, nullptr, 0);
        }
        if (!rc && cudaEventRecord(e1, 0) != cudaSuccess) rc = cuda_fail(cudaGetLastError(), "event");
        if (!rc && cudaEventSynchronize(e1) != cudaSuccess) rc = cuda_fail(cudaGetLastError(), "autotune run");
        float t = 0.f;
        if (!rc) cudaEventElapsedTime(&t, e0, e1);
        ms[i] = t / steps;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!rc && P->tc) rc = dgm::tc_check_error(P);
    if (rc) {
        P->grid = keep_grid;
        P->tc_grid = keep_tc;
        P->kd.sparse = P->kf.sparse = keep_sparse;
        P->kd.eg = P->kf.eg = keep_eg;
        P->kd.eg_warps = P->kf.eg_warps = keep_egw;
        if (P->tc) P->tca.partH = P->tca.partE + P->tc_grid;
        return rc;
    }
    const int best = (int)(std::min_element(ms.begin(), ms.end()) - ms.begin());
    apply(cand[best]);
    if (ncand_out) *ncand_out = (int)cand.size();
    for (size_t i = 0; i < cand.size(); ++i) {
        if (cand_config) cand_config[i] = cand[i];
        if (cand_ms) cand_ms[i] = ms[i];
    }
    if (chosen_out) *chosen_out = best;
    return DGM_OK;
}

int dgm_estimate_dt(dgm_problem* P, int iters, double* rho_out, double* dt_out) {
    if (!P || iters < 1) {
        set_error("dgm_estimate_dt: bad argument");
        return DGM_ERR_INVALID_ARG;
    }
    const StateView v = state_view(P);
    const size_t es = v.f32 ? sizeof(float) : sizeof(double);
    const size_t bytes = (size_t)(v.nE + 2 * v.nH + 2 * v.nK) * es;
    void* tmp = nullptr;
    DGM_CUDA(cudaMalloc(&tmp, bytes));
    char* saveE = (char*)tmp;
    char* saveH = saveE + v.nE * es;
    char* saveK = saveH + v.nH * es;
    char* xH = saveK + v.nK * es;
    char* xK = xH + v.nH * es;
    int rc = DGM_OK;
    double rho = 0.0;
    auto fin = [&](int code) {
        cudaFree(tmp);
        P->trE_valid = P->trH_valid = false;
        reset_comp(P);
        return code;
    };
    if (cudaMemcpy(saveE, v.E, v.nE * es, cudaMemcpyDeviceToDevice) != cudaSuccess ||
        cudaMemcpy(saveH, v.H, v.nH * es, cudaMemcpyDeviceToDevice) != cudaSuccess ||
        (v.nK && cudaMemcpy(saveK, v.K, v.nK * es, cudaMemcpyDeviceToDevice) != cudaSuccess))
        return fin(cuda_fail(cudaGetLastError(), "dgm_estimate_dt save"));
    // start vector: fixed pseudo-random canonical H (and H^F), through the normal import
    {
        const int64_t nHc = P->nt * 3 * P->NH, nKc = v.nK ? P->nfaces * 2 * P->N2E : 0;
        std::vector<double> h(std::max(nHc, nKc));
        uint64_t st = 0x9E3779B97F4A7C15ull;
        auto rnd = [&]() {
            st ^= st << 13;
            st ^= st >> 7;
            st ^= st << 17;
            return (double)(st >> 11) * (1.0 / 9007199254740992.0) - 0.5;
        };
        for (int64_t i = 0; i < nHc; ++i) h[i] = rnd();
        if (cudaMemcpy(P->dStage, h.data(), nHc * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
            return fin(cuda_fail(cudaGetLastError(), "dgm_estimate_dt init"));
        if ((rc = import_fields(P, nullptr, P->dStage, 0))) return fin(rc);
        if (v.nK) {
            for (int64_t i = 0; i < nKc; ++i) h[i] = rnd();
            cudaMemcpy(P->dStage, h.data(), nKc * sizeof(double), cudaMemcpyHostToDevice);
            if ((rc = import_faces(P, P->dStage, 0))) return fin(rc);
        }
    }
    double nx = 0.0;
    cudaMemset(v.E, 0, v.nE * es);
    P->trE_valid = P->trH_valid = false;
    if ((rc = dgm_energy(P, &nx))) return fin(rc);
    for (int it = 0; it < iters; ++it) {
        // x := H (and K) / ||.||;  H <- x - dt=1 kicks (E=0) = x - B x;  y = x - H = B x
        const double sc = 1.0 / std::sqrt(2.0 * nx);
        if (axpby(v, v.nH, 0.0, v.H, sc, v.H) || axpby(v, v.nK, 0.0, v.K, sc, v.K))
            return fin(cuda_fail(cudaGetLastError(), "axpby"));
        cudaMemcpy(xH, v.H, v.nH * es, cudaMemcpyDeviceToDevice);
        if (v.nK) cudaMemcpy(xK, v.K, v.nK * es, cudaMemcpyDeviceToDevice);
        cudaMemset(v.E, 0, v.nE * es);
        P->trE_valid = P->trH_valid = false;
        if ((rc = phase_E(P, 1.0, 0)) || (rc = phase_H(P, 1.0, 0.0, 1.0, nullptr, 0))) return fin(rc);
        if (axpby(v, v.nH, 1.0, xH, -1.0, v.H) || axpby(v, v.nK, 1.0, xK, -1.0, v.K))
            return fin(cuda_fail(cudaGetLastError(), "axpby"));
        cudaMemset(v.E, 0, v.nE * es);
        P->trE_valid = P->trH_valid = false;
        double ny = 0.0;
        if ((rc = dgm_energy(P, &ny))) return fin(rc);
        rho = std::sqrt(ny / 0.5);   // ||B x||_M with ||x||_M = 1
        nx = ny;
        if (!(nx > 0.0) || !std::isfinite(nx)) break;
    }
    if (cudaMemcpy(v.E, saveE, v.nE * es, cudaMemcpyDeviceToDevice) != cudaSuccess ||
        cudaMemcpy(v.H, saveH, v.nH * es, cudaMemcpyDeviceToDevice) != cudaSuccess ||
        (v.nK && cudaMemcpy(v.K, saveK, v.nK * es, cudaMemcpyDeviceToDevice) != cudaSuccess))
        return fin(cuda_fail(cudaGetLastError(), "dgm_estimate_dt restore"));
    if (rho_out) *rho_out = rho;
    if (dt_out) *dt_out = rho > 0.0 ? 2.0 / std::sqrt(rho) : INFINITY;
    return fin(DGM_OK);
}

namespace {

void set_state_ptrs(dgm_problem* P, void* E, void* H) {
    if (P->tc) {
        P->tca.E = (float*)E;
        P->tca.H = (float*)H;
        if (!P->tca.d.f16) {   // TF32: the operand is the state itself; fp16 copies follow via the refresh
            P->tca.Eop = E;
            P->tca.Hop = H;
        }
    } else if (P->fp32) {
        P->kf.E = (float*)E;
        P->kf.H = (float*)H;
    } else {
        P->kd.E = (double*)E;
        P->kd.H = (double*)H;
    }
    P->trE_valid = P->trH_valid = false;
    reset_comp(P);
}

struct DevBuf {
    void* p = nullptr;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
};

}  // namespace

int dgm_adjoint_grad(dgm_problem* P, double dt, int64_t nsteps, int nobs, const double* xobs, int ckpt_every,
                     double* J_out, double* dJdeps, double* dJdmu) {
    if (!P || !xobs || nobs < 1 || nobs > 1024 || nsteps < 1 || ckpt_every < 1 || !std::isfinite(dt)) {
        set_error("dgm_adjoint_grad: bad argument");
        return DGM_ERR_INVALID_ARG;
    }
    if (P->opt.flux != DGM_FLUX_CENTRAL) {
        set_error("dgm_adjoint_grad: central flux only");
        return DGM_ERR_UNSUPPORTED;
    }
    // observation points: containing element, reference coordinates, basis values
    std::vector<int32_t> oe(nobs);
    std::vector<double> oxh(3 * nobs), oFi(9 * nobs), ogi(6 * nobs);
    for (int o = 0; o < nobs; ++o) {
        const double* x = xobs + 3 * o;
        int64_t best = -1;
        double bestmin = -1e300, bxh[3] = {0, 0, 0}, bFi[9] = {0};
        for (int64_t t = 0; t < P->nt; ++t) {
            const double* M = &P->hmaps[12 * t];
            const double* F = M + 3;
            const double det = F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) +
                               F[2] * (F[3] * F[7] - F[4] * F[6]);
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
            double xh[3];
            for (int i = 0; i < 3; ++i)
                xh[i] = Fi[3 * i] * (x[0] - M[0]) + Fi[3 * i + 1] * (x[1] - M[1]) + Fi[3 * i + 2] * (x[2] - M[2]);
            const double mn = std::min(std::min(xh[0], xh[1]), std::min(xh[2], 1.0 - xh[0] - xh[1] - xh[2]));
            if (mn > bestmin) {
                bestmin = mn;
                best = t;
                std::memcpy(bxh, xh, sizeof(bxh));
                std::memcpy(bFi, Fi, sizeof(bFi));
            }
        }
        if (bestmin < -1e-10) {
            set_error("dgm_adjoint_grad: observation point outside the mesh");
            return DGM_ERR_INVALID_ARG;
        }
        oe[o] = (int32_t)best;
        std::memcpy(&oxh[3 * o], bxh, sizeof(bxh));
        std::memcpy(&oFi[9 * o], bFi, sizeof(bFi));
        const double* g = &P->hgeo[(size_t)best * dgm::kGeoStride];
        for (int q = 0; q < 6; ++q) ogi[6 * o + q] = g[q] * g[dgm::kGeoInvEps];
    }
    std::vector<double> ophi;
    dgm::phi_at_points(P->p, oxh.data(), nobs, ophi);
    const StateView v = state_view(P);
    const size_t es = v.f32 ? sizeof(float) : sizeof(double);
    const int64_t nck = (nsteps + ckpt_every - 1) / ckpt_every;
    const int N = P->NE, K = P->tc ? P->tca.d.KE : 0, tiled = P->tc ? P->tca.d.layout : 0;
    const size_t sE = v.nE * es, sH = v.nH * es;
    // one allocation: obs data, J, grad, saved state, checkpoints, segment, adjoint state
    const size_t obs_bytes = ((nobs * sizeof(int32_t) + 255) / 256) * 256 + (ophi.size() + oFi.size() + ogi.size()) * 8;
    const size_t total = obs_bytes + 256 + 2 * ((size_t)P->nt * 8 + 256) + (sE + sH) * (1 + nck) +
                         (sE + sH) * (ckpt_every + 1) + sE + sH + 2048;
    DevBuf buf;
    DGM_CUDA(cudaMalloc(&buf.p, total));
    char* q = (char*)buf.p;
    auto take = [&](size_t bytes) {
        char* r = q;
        q += (bytes + 255) / 256 * 256;
        return r;
    };
    int32_t* dElem = (int32_t*)take(nobs * sizeof(int32_t));
    double* dPhi = (double*)take(ophi.size() * 8);
    double* dFi = (double*)take(oFi.size() * 8);
    double* dGi = (double*)take(ogi.size() * 8);
    double* dJ = (double*)take(8);
    double* dGrad = (double*)take((size_t)P->nt * 8);
    double* dGradMu = (double*)take((size_t)P->nt * 8);
    char* save = take(sE + sH);
    char* ck = take((sE + sH) * nck);
    char* seg = take(sE * (ckpt_every + 1));
    char* segG = take(sH * (ckpt_every + 1));   // G^n = H^{n+1/2} of the segment (dJ/d mu)
    char* aE = take(sE);
    char* aH = take(sH);
    cudaMemcpy(dElem, oe.data(), nobs * sizeof(int32_t), cudaMemcpyHostToDevice);
    cudaMemcpy(dPhi, ophi.data(), ophi.size() * 8, cudaMemcpyHostToDevice);
    cudaMemcpy(dFi, oFi.data(), oFi.size() * 8, cudaMemcpyHostToDevice);
    cudaMemcpy(dGi, ogi.data(), ogi.size() * 8, cudaMemcpyHostToDevice);
    cudaMemset(dJ, 0, 8);
    cudaMemset(dGrad, 0, (size_t)P->nt * 8);
    cudaMemset(dGradMu, 0, (size_t)P->nt * 8);
    cudaMemset(aE, 0, sE);
    cudaMemset(aH, 0, sH);
    const dgm::ObsDev O{nobs, dElem, dPhi, dFi, dGi};
    const double* geo = P->tc ? P->dTcGeo : P->dGeo;
    auto observe = [&](const void* E) {
        return v.f32 ? dgm::adj_observe<float>(O, (const float*)E, N, K, tiled, dJ, 0)
                     : dgm::adj_observe<double>(O, (const double*)E, N, K, tiled, dJ, 0);
    };
    int rc = DGM_OK;
    void* E0p = v.E;
    void* H0p = v.H;
    cudaMemcpy(save, v.E, sE, cudaMemcpyDeviceToDevice);
    cudaMemcpy(save + sE, v.H, sH, cudaMemcpyDeviceToDevice);
    P->trE_valid = P->trH_valid = false;
    // forward: G^0 = H^0 + dt/2 A E^0; per step E-kick, observe, H-kick; checkpoints (E^n, G^n)
    rc = prepare_source(P, P->time, dt, nsteps);
    if (!rc) rc = phase_H(P, 0.5 * dt, 0.0, 1.0, nullptr, 0);
    for (int64_t n = 0; n < nsteps && !rc; ++n) {
        if (n % ckpt_every == 0) {
            cudaMemcpy(ck + (n / ckpt_every) * (sE + sH), v.E, sE, cudaMemcpyDeviceToDevice);
            cudaMemcpy(ck + (n / ckpt_every) * (sE + sH) + sE, v.H, sH, cudaMemcpyDeviceToDevice);
        }
        rc = phase_E(P, dt, 0);
        if (!rc) rc = apply_source(P, v.E, n, dt, 0);
        if (!rc && observe(v.E)) rc = cuda_fail(cudaGetLastError(), "observe");
        if (!rc) rc = phase_H(P, dt, 0.0, 1.0, nullptr, 0);
    }
    // backward over segments, recomputing each segment's E from its checkpoint
    for (int64_t s = nck - 1; s >= 0 && !rc; --s) {
        const int64_t n0 = s * ckpt_every, n1 = std::min<int64_t>(nsteps, n0 + ckpt_every);
        set_state_ptrs(P, E0p, H0p);
        cudaMemcpy(v.E, ck + s * (sE + sH), sE, cudaMemcpyDeviceToDevice);
        cudaMemcpy(v.H, ck + s * (sE + sH) + sE, sH, cudaMemcpyDeviceToDevice);
        cudaMemcpy(seg, v.E, sE, cudaMemcpyDeviceToDevice);
        cudaMemcpy(segG, v.H, sH, cudaMemcpyDeviceToDevice);
        for (int64_t n = n0; n < n1 && !rc; ++n) {
            rc = phase_E(P, dt, 0);
            if (!rc) rc = apply_source(P, v.E, n, dt, 0);
            cudaMemcpyAsync(seg + (n - n0 + 1) * sE, v.E, sE, cudaMemcpyDeviceToDevice, 0);
            if (!rc && n < n1 - 1) {
                rc = phase_H(P, dt, 0.0, 1.0, nullptr, 0);
                cudaMemcpyAsync(segG + (n - n0 + 1) * sH, v.H, sH, cudaMemcpyDeviceToDevice, 0);
            }
        }
        // G^{n1}: the next segment's checkpoint (not needed at n1 = N, where g^ = 0)
        if (n1 < nsteps)
            cudaMemcpy(segG + (n1 - n0) * sH, ck + (s + 1) * (sE + sH) + sE, sH, cudaMemcpyDeviceToDevice);
        set_state_ptrs(P, aE, aH);
        for (int64_t m = n1; m > n0 && !rc; --m) {
            const char* Em = seg + (m - n0) * sE;
            const char* Emm = seg + (m - n0 - 1) * sE;
            rc = phase_E(P, -dt, 0);   // e^ += dt M_eps^{-1} C^T g^
            if (rc) break;
            int r = v.f32 ? dgm::adj_source<float>(O, (const float*)Em, (float*)aE, N, K, tiled, 0)
                          : dgm::adj_source<double>(O, (const double*)Em, (double*)aE, N, K, tiled, 0);
            // the observation sources change e^ only in the observed elements' tiles
            for (int o = 0; o < nobs; ++o) dgm::tc_mark_tile_dirty(P, oe[o] / dgm::kTcRows);
            r |= v.f32 ? dgm::adj_grad<float>(P->nt, geo, (const float*)aE, (const float*)Em, (const float*)Emm, N,
                                              K, tiled, dGrad, 0)
                       : dgm::adj_grad<double>(P->nt, geo, (const double*)aE, (const double*)Em, (const double*)Emm,
                                               N, K, tiled, dGrad, 0);
            if (r) {
                rc = cuda_fail(cudaGetLastError(), "adjoint kernels");
                break;
            }
            // dJ/d mu_T -= g^m . (G (x) I)(G^m - G^{m-1})_T  (g^N = 0: nothing at m = N)
            if (dJdmu && m < nsteps) {
                const char* Gm = segG + (m - n0) * sH;
                const char* Gmm = segG + (m - n0 - 1) * sH;
                const int KH = P->tc ? P->tca.d.KH : 0;
                const int rr = v.f32 ? dgm::adj_grad<float>(P->nt, geo, (const float*)aH, (const float*)Gm,
                                                             (const float*)Gmm, P->NH, KH, tiled, dGradMu, 0)
                                     : dgm::adj_grad<double>(P->nt, geo, (const double*)aH, (const double*)Gm,
                                                              (const double*)Gmm, P->NH, KH, tiled, dGradMu, 0);
                if (rr) {
                    rc = cuda_fail(cudaGetLastError(), "adjoint kernels");
                    break;
                }
            }
            rc = phase_H(P, -dt, 0.0, 1.0, nullptr, 0);   // g^ -= dt M_mu^{-1} C e^
        }
    }
    // opening half kick: dJ/d mu_T -= g^0 . (G (x) I)(G^0 - H^0)_T
    if (!rc && dJdmu) {
        const int KH = P->tc ? P->tca.d.KH : 0;
        const char* G0 = ck + sE;          // checkpoint 0: (E^0, G^0)
        const char* H0 = save + sE;        // the state before the run
        const int rr = v.f32 ? dgm::adj_grad<float>(P->nt, geo, (const float*)aH, (const float*)G0, (const float*)H0,
                                                     P->NH, KH, tiled, dGradMu, 0)
                             : dgm::adj_grad<double>(P->nt, geo, (const double*)aH, (const double*)G0,
                                                      (const double*)H0, P->NH, KH, tiled, dGradMu, 0);
        if (rr) rc = cuda_fail(cudaGetLastError(), "adjoint kernels");
    }
    set_state_ptrs(P, E0p, H0p);
    cudaMemcpy(v.E, save, sE, cudaMemcpyDeviceToDevice);
    cudaMemcpy(v.H, save + sE, sH, cudaMemcpyDeviceToDevice);
    P->trE_valid = P->trH_valid = false;
    if (rc) return rc;
    DGM_CUDA(cudaDeviceSynchronize());
    if (P->tc && (rc = dgm::tc_check_error(P))) return rc;
    if (J_out) DGM_CUDA(cudaMemcpy(J_out, dJ, 8, cudaMemcpyDeviceToHost));
    if (dJdeps) DGM_CUDA(cudaMemcpy(dJdeps, dGrad, (size_t)P->nt * 8, cudaMemcpyDeviceToHost));
    if (dJdmu) DGM_CUDA(cudaMemcpy(dJdmu, dGradMu, (size_t)P->nt * 8, cudaMemcpyDeviceToHost));
    return DGM_OK;
}

int dgm_tridiag_eig(int k, const double* d, const double* e, int i0, int i1, double* vals, double* vecs) {
    if (k < 1 || !d || (k > 1 && !e) || i0 < 0 || i1 > k || i0 >= i1 || !vals) {
        set_error("dgm_tridiag_eig: bad argument");
        return DGM_ERR_INVALID_ARG;
    }
    const std::vector<double> dv(d, d + k), ev(e ? e : d, e ? e + (k - 1) : d);
    const std::vector<double> th = dgm::tridiag_eigenvalues(dv, ev, i0, i1);
    for (int i = 0; i < i1 - i0; ++i) {
        vals[i] = th[i];
        if (vecs) {
            const std::vector<double> y = dgm::tridiag_eigenvector(dv, ev, th[i]);
            std::copy(y.begin(), y.end(), vecs + (size_t)i * k);
        }
    }
    return DGM_OK;
}

int dgm_resonances(dgm_problem* P, int m, int nev, double zero_rel, double* omega_out, double* resid_out,
                   int* nfound_out) {
    if (!P || m < 2 || nev < 1 || !omega_out || !nfound_out || !(zero_rel >= 0.0 && zero_rel < 1.0)) {
        set_error("dgm_resonances: bad argument");
        return DGM_ERR_INVALID_ARG;
    }
    *nfound_out = 0;
    if (P->tc || P->fp32) {
        set_error("dgm_resonances: FP64 precision only");
        return DGM_ERR_UNSUPPORTED;
    }
    const StateView v = state_view(P);
    const int64_t n = v.nE;
    m = (int)std::min<int64_t>(m, n);
    // one allocation: saved state (E, H, K), Lanczos basis V[m+1][n], two work vectors,
    // coefficient vector, scalars
    const size_t sE = n * 8, sH = v.nH * 8, sK = v.nK * 8;
    const size_t total = sE + sH + sK + (size_t)(m + 1) * sE + 2 * sE + (size_t)(m + 1) * 8 + 64 + 8 * 256;
    DevBuf buf;
    DGM_CUDA(cudaMalloc(&buf.p, total));
    char* q = (char*)buf.p;
    auto take = [&](size_t bytes) {
        char* r = q;
        q += (bytes + 255) / 256 * 256;
        return r;
    };
    char* saveE = take(sE);
    char* saveH = take(sH);
    char* saveK = take(sK);
    double* V = (double*)take((size_t)(m + 1) * sE);
    double* Z = (double*)take(sE);
    double* U = (double*)take(sE);
    double* dh = (double*)take((size_t)(m + 1) * 8);
    double* dsc = (double*)take(64);
    double* E = (double*)v.E;
    const double* geo = P->dGeo;
    const int N = P->NE;
    cudaMemcpy(saveE, v.E, sE, cudaMemcpyDeviceToDevice);
    cudaMemcpy(saveH, v.H, sH, cudaMemcpyDeviceToDevice);
    if (sK) cudaMemcpy(saveK, v.K, sK, cudaMemcpyDeviceToDevice);
    int rc = DGM_OK;
    auto fin = [&](int code) {
        cudaMemcpy(v.E, saveE, sE, cudaMemcpyDeviceToDevice);
        cudaMemcpy(v.H, saveH, sH, cudaMemcpyDeviceToDevice);
        if (sK) cudaMemcpy(v.K, saveK, sK, cudaMemcpyDeviceToDevice);
        P->trE_valid = P->trH_valid = false;
        return code;
    };
    auto fail = [&](const char* what) { return fin(cuda_fail(cudaGetLastError(), what)); };
    // y = A x = M_eps^{-1} K x: E = x, H = 0 (H^F = 0), one H-kick and one E-kick with
    // dt = 1 leave E = x - A x
    auto apply = [&](const double* x, double* y) -> int {
        cudaMemcpy(E, x, sE, cudaMemcpyDeviceToDevice);
        cudaMemset(v.H, 0, sH);
        if (sK) cudaMemset(v.K, 0, sK);
        P->trE_valid = P->trH_valid = false;
        int r = phase_H(P, 1.0, 0.0, 1.0, nullptr, 0);
        if (!r) r = phase_E(P, 1.0, 0);
        if (r) return r;
        if (dgm::launch_axpby<double>(n, 1.0, x, -1.0, E, 0)) return cuda_fail(cudaGetLastError(), "axpby");
        if (y != E) cudaMemcpy(y, E, sE, cudaMemcpyDeviceToDevice);
        return DGM_OK;
    };
    auto mnorm2 = [&](const double* x, double* out) -> int {
        if (dgm::eig_mass_apply(P->nt, N, geo, x, Z, 0) || dgm::eig_dots(x, 0, 1, Z, n, dsc, 0)) return -1;
        return cudaMemcpy(out, dsc, 8, cudaMemcpyDeviceToHost) == cudaSuccess ? 0 : -1;
    };
    // start vector: fixed pseudo-random canonical E through the normal import
    {
        std::vector<double> h(n);
        uint64_t st = 0xD1B54A32D192ED03ull;
        for (int64_t i = 0; i < n; ++i) {
            st ^= st << 13;
            st ^= st >> 7;
            st ^= st << 17;
            h[i] = (double)(st >> 11) * (1.0 / 9007199254740992.0) - 0.5;
        }
        if (cudaMemcpy(P->dStage, h.data(), sE, cudaMemcpyHostToDevice) != cudaSuccess) return fail("resonances init");
        if ((rc = import_fields(P, P->dStage, nullptr, 0))) return fin(rc);
        double nx = 0.0;
        if (mnorm2(E, &nx) || !(nx > 0.0)) return fail("resonances start");
        if (dgm::eig_scale(n, 1.0 / std::sqrt(nx), E, V, 0)) return fail("scale");
    }
    // Lanczos with full reorthogonalisation (classical Gram-Schmidt, twice) in <.,.>_M
    std::vector<double> alpha, beta;
    std::vector<double> hh(m + 1);
    int k = 0;
    for (int j = 0; j < m; ++j) {
        double* vj = V + (size_t)j * n;
        double* w = U;
        if ((rc = apply(vj, w))) return fin(rc);
        double a = 0.0;
        for (int pass = 0; pass < 2; ++pass) {
            if (dgm::eig_mass_apply(P->nt, N, geo, w, Z, 0) || dgm::eig_dots(V, n, j + 1, Z, n, dh, 0) ||
                dgm::eig_sub_combination(w, V, n, j + 1, dh, n, 0))
                return fail("reorthogonalisation");
            if (cudaMemcpy(hh.data(), dh, (j + 1) * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
                return fail("reorthogonalisation");
            a += hh[j];
        }
        alpha.push_back(a);
        k = j + 1;
        double b2 = 0.0;
        if (mnorm2(w, &b2)) return fail("norm");
        const double b = std::sqrt(std::max(b2, 0.0));
        // invariant subspace found (or the basis is complete)
        if (!(b > 1e-13 * std::max(std::fabs(a), 1.0)) || j == m - 1) {
            beta.push_back(b);
            break;
        }
        beta.push_back(b);
        if (dgm::eig_scale(n, 1.0 / b, w, V + (size_t)(j + 1) * n, 0)) return fail("scale");
    }
    // Ritz values: skip the discrete null space (at or below zero_rel * the largest)
    const std::vector<double> ev(beta.begin(), beta.begin() + (k - 1));
    const double top = dgm::tridiag_eigenvalues(alpha, ev, k - 1, k)[0];
    const int c0 = dgm::tridiag_count_below(alpha, ev, zero_rel * top * (1.0 + 1e-12) + DBL_MIN);
    const int c1 = std::min(k, c0 + nev);
    const std::vector<double> th = dgm::tridiag_eigenvalues(alpha, ev, c0, c1);
    int found = 0;
    for (size_t i = 0; i < th.size(); ++i) {
        if (!(th[i] > zero_rel * top)) continue;
        omega_out[found] = std::sqrt(th[i]);
        if (resid_out) {
            // Ritz vector u = V y; relative residual ||A u - theta u||_M / (theta ||u||_M)
            const std::vector<double> y = dgm::tridiag_eigenvector(alpha, ev, th[i]);
            for (int j = 0; j < k; ++j) hh[j] = -y[j];
            cudaMemset(U, 0, sE);
            if (cudaMemcpy(dh, hh.data(), k * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
                dgm::eig_sub_combination(U, V, n, k, dh, n, 0))
                return fail("Ritz vector");
            double uu = 0.0, rr = 0.0;
            if (mnorm2(U, &uu)) return fail("norm");
            if ((rc = apply(U, E))) return fin(rc);
            if (dgm::launch_axpby<double>(n, -th[i], U, 1.0, E, 0)) return fail("axpby");
            if (mnorm2(E, &rr)) return fail("norm");
            resid_out[found] = std::sqrt(std::max(rr, 0.0)) / (th[i] * std::sqrt(uu));
        }
        ++found;
    }
    *nfound_out = found;
    return fin(DGM_OK);
}

int dgm_set_materials(dgm_problem* P, const double* eps, const double* mu) {
    if (!P || !eps || !mu) {
        set_error("dgm_set_materials: null argument");
        return DGM_ERR_INVALID_ARG;
    }
    for (int64_t t = 0; t < P->nt; ++t)
        if (!(eps[t] > 0.0) || !(mu[t] > 0.0) || !std::isfinite(eps[t]) || !std::isfinite(mu[t])) {
            set_error("dgm_set_materials: eps and mu must be positive and finite");
            return DGM_ERR_INVALID_ARG;
        }
    for (int64_t t = 0; t < P->nt; ++t) {
        double* g = &P->hgeo[(size_t)t * dgm::kGeoStride];
        g[dgm::kGeoEps] = eps[t];
        g[dgm::kGeoInvEps] = 1.0 / eps[t];
        g[dgm::kGeoMu] = mu[t];
        g[dgm::kGeoInvMu] = 1.0 / mu[t];
    }
    P->eps.assign(eps, eps + P->nt);
    P->mu.assign(mu, mu + P->nt);
    DGM_CUDA(cudaDeviceSynchronize());
    DGM_CUDA(cudaMemcpy(P->dGeo, P->hgeo.data(), P->hgeo.size() * sizeof(double), cudaMemcpyHostToDevice));
    if (P->tc) DGM_CUDA(cudaMemcpy(P->dTcGeo, P->hgeo.data(), P->hgeo.size() * sizeof(double), cudaMemcpyHostToDevice));
    return DGM_OK;
}

}  // extern "C"

namespace {

// Enqueue the kernels of nsteps leapfrog steps on stream s, no host
// synchronisation or copies (usable inside stream capture); the source values
// must have been prepared.  Energies (optional) go to the problem's device array.
int enqueue_run(dgm_problem* P, double dt, int64_t nsteps, cudaStream_t s, bool want) {
    double* W = P->dEnergy;
    P->trE_valid = false;   // the first H-phase recomputes E traces (tensor cores: and E^0's energy)
    int rc = phase_H(P, dt, 0.5, 0.5, want ? W : nullptr, s);
    for (int64_t n = 0; n < nsteps && !rc; ++n) {
        rc = phase_E(P, dt, s, want);
        if (!rc) rc = apply_source(P, current_E(P), n, dt, s);
        if (!rc) rc = phase_H(P, dt, 0.0, n == nsteps - 1 ? 0.5 : 1.0, want ? W + n + 1 : nullptr, s);
    }
    return rc;
}

void batch_release_graph(dgm_batch* B) {
    if (B->exec) cudaGraphExecDestroy(B->exec);
    B->exec = nullptr;
    B->g_nsteps = -1;
}

}  // namespace

extern "C" {

int dgm_batch_create(dgm_ctx* ctx, dgm_problem** probs, int nruns, dgm_batch** out) {
    if (!ctx || !probs || nruns < 1 || !out) {
        set_error("dgm_batch_create: bad argument");
        return DGM_ERR_INVALID_ARG;
    }
    *out = nullptr;
    dgm_batch* B = new (std::nothrow) dgm_batch;
    if (!B) return DGM_ERR_OOM;
    B->ctx = ctx;
    for (int r = 0; r < nruns; ++r) {
        if (!probs[r] || probs[r]->ctx->device != ctx->device) {
            delete B;
            set_error("dgm_batch_create: null problem or problem on another device");
            return DGM_ERR_INVALID_ARG;
        }
        for (int q = 0; q < r; ++q)
            if (probs[q] == probs[r]) {
                delete B;
                set_error("dgm_batch_create: a problem appears twice");
                return DGM_ERR_INVALID_ARG;
            }
        B->probs.push_back(probs[r]);
    }
    B->streams.resize(nruns);
    B->joins.resize(nruns);
    for (int r = 0; r < nruns; ++r) {
        if (cudaStreamCreateWithFlags(&B->streams[r], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&B->joins[r], cudaEventDisableTiming) != cudaSuccess) {
            dgm_batch_destroy(B);
            return cuda_fail(cudaGetLastError(), "dgm_batch_create");
        }
    }
    if (cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking) != cudaSuccess) {
        dgm_batch_destroy(B);
        return cuda_fail(cudaGetLastError(), "dgm_batch_create");
    }
    *out = B;
    return DGM_OK;
}

int dgm_batch_destroy(dgm_batch* B) {
    if (!B) return DGM_OK;
    batch_release_graph(B);
    for (cudaStream_t s : B->streams)
        if (s) cudaStreamDestroy(s);
    for (cudaEvent_t e : B->joins)
        if (e) cudaEventDestroy(e);
    if (B->fork) cudaEventDestroy(B->fork);
    if (B->cap) cudaStreamDestroy(B->cap);
    delete B;
    return DGM_OK;
}

int dgm_batch_run(dgm_batch* B, const double* dt, int64_t nsteps, void* stream, double* energy_out) {
    if (!B || !dt || nsteps < 1) {
        set_error("dgm_batch_run: bad argument");
        return DGM_ERR_INVALID_ARG;
    }
    const int nr = (int)B->probs.size();
    for (int r = 0; r < nr; ++r)
        if (!std::isfinite(dt[r])) {
            set_error("dgm_batch_run: non-finite time step");
            return DGM_ERR_INVALID_ARG;
        }
    cudaStream_t s = (cudaStream_t)stream;
    const bool want = energy_out != nullptr;
    int rc = DGM_OK;
    for (int r = 0; r < nr && !rc; ++r) {
        dgm_problem* P = B->probs[r];
        rc = ensure_energy(P, nsteps + 1);
        if (!rc) rc = prepare_source(P, P->time, dt[r], nsteps);   // values refreshed before every launch
    }
    if (rc) return rc;
    const bool same = B->exec && B->g_nsteps == nsteps && B->g_energy == want &&
                      std::equal(B->g_dt.begin(), B->g_dt.end(), dt);
    if (!same) {
        batch_release_graph(B);
        // one graph: fork from the capture stream, every run's loop on its own
        // stream, join back; launched afterwards on the caller's stream
        cudaStream_t c = B->cap;
        DGM_CUDA(cudaStreamBeginCapture(c, cudaStreamCaptureModeRelaxed));
        int crc = cudaEventRecord(B->fork, c) == cudaSuccess ? DGM_OK : DGM_ERR_CUDA;
        for (int r = 0; r < nr && !crc; ++r) {
            if (cudaStreamWaitEvent(B->streams[r], B->fork, 0) != cudaSuccess) crc = DGM_ERR_CUDA;
            if (!crc) crc = enqueue_run(B->probs[r], dt[r], nsteps, B->streams[r], want);
            if (!crc && cudaEventRecord(B->joins[r], B->streams[r]) != cudaSuccess) crc = DGM_ERR_CUDA;
            if (!crc && cudaStreamWaitEvent(c, B->joins[r], 0) != cudaSuccess) crc = DGM_ERR_CUDA;
        }
        cudaGraph_t graph = nullptr;
        const cudaError_t ee = cudaStreamEndCapture(c, &graph);
        if (crc || ee != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return crc ? crc : cuda_fail(ee, "dgm_batch_run capture");
        }
        const cudaError_t ie = cudaGraphInstantiate(&B->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) {
            B->exec = nullptr;
            return cuda_fail(ie, "dgm_batch_run instantiate");
        }
        B->g_nsteps = nsteps;
        B->g_dt.assign(dt, dt + nr);
        B->g_energy = want;
    }
    DGM_CUDA(cudaGraphLaunch(B->exec, s));
    for (int r = 0; r < nr; ++r) B->probs[r]->time += nsteps * dt[r];
    if (want) {
        DGM_CUDA(cudaStreamSynchronize(s));
        for (int r = 0; r < nr; ++r) {
            double* Wr = energy_out + (size_t)r * (nsteps + 1);
            DGM_CUDA(cudaMemcpy(Wr, B->probs[r]->dEnergy, (nsteps + 1) * sizeof(double), cudaMemcpyDeviceToHost));
            if (B->probs[r]->tc && (rc = dgm::tc_check_error(B->probs[r]))) return rc;
            for (int64_t n = 0; n <= nsteps; ++n)
                if (!std::isfinite(Wr[n]) ||
                    (!B->probs[r]->src_on && Wr[n] > 10.0 * std::fabs(Wr[0]) + 1e-300)) {
                    set_error("dgm_batch_run: energy blew up in run " + std::to_string(r));
                    return DGM_ERR_UNSTABLE;
                }
        }
    }
    return DGM_OK;
}

int dgm_quad_rule(int q1d, int* nq, double* xh, double* w) {
    if (q1d < 1 || q1d > 32) {
        set_error("dgm_quad_rule: q1d must be in [1, 32]");
        return DGM_ERR_INVALID_ARG;
    }
    std::vector<double> x, ww, col;
    dgm::collapsed_rule(q1d, x, ww, col);
    if (nq) *nq = (int)ww.size();
    if (xh) std::memcpy(xh, x.data(), x.size() * sizeof(double));
    if (w) std::memcpy(w, ww.data(), ww.size() * sizeof(double));
    return DGM_OK;
}

int dgm_element_maps(const dgm_mesh* mesh, double* out) {
    if (!mesh || !out) {
        set_error("dgm_element_maps: null argument");
        return DGM_ERR_INVALID_ARG;
    }
    const dgm::MeshData& m = mesh->m;
    for (int64_t t = 0; t < m.nt; ++t) {
        const double* X0 = &m.xyz[3 * (int64_t)m.tets[4 * t]];
        for (int d = 0; d < 3; ++d) out[12 * t + d] = X0[d];
        for (int q = 0; q < 9; ++q) out[12 * t + 3 + q] = m.F[9 * t + q];
    }
    return DGM_OK;
}

static int ensure_rule(dgm_problem* P, int q1d) {
    if (q1d < 1 || q1d > 32) {
        set_error("projection rule: q1d must be in [1, 32]");
        return DGM_ERR_INVALID_ARG;
    }
    if (P->rule_q1d == q1d) return DGM_OK;
    double* old[] = {P->dWphiE, P->dWphiH, P->dPhiE, P->dPhiH};
    for (double* q : old)
        if (q) cudaFree(q);
    P->dWphiE = P->dWphiH = P->dPhiE = P->dPhiH = nullptr;
    P->rule_q1d = 0;
    std::vector<double> x, w, col, phE, phH;
    dgm::collapsed_rule(q1d, x, w, col);
    dgm::phi_table(P->p, q1d, phE);
    dgm::phi_table(P->tab.ph, q1d, phH);
    const int nq = (int)w.size();
    std::vector<double> wE(phE.size()), wH(phH.size());
    for (int q = 0; q < nq; ++q) {
        for (int a = 0; a < P->NE; ++a) wE[(size_t)q * P->NE + a] = w[q] * phE[(size_t)q * P->NE + a];
        for (int b = 0; b < P->NH; ++b) wH[(size_t)q * P->NH + b] = w[q] * phH[(size_t)q * P->NH + b];
    }
    DGM_CUDA(cudaMalloc(&P->dWphiE, wE.size() * sizeof(double)));
    DGM_CUDA(cudaMalloc(&P->dWphiH, wH.size() * sizeof(double)));
    DGM_CUDA(cudaMalloc(&P->dPhiE, phE.size() * sizeof(double)));
    DGM_CUDA(cudaMalloc(&P->dPhiH, phH.size() * sizeof(double)));
    DGM_CUDA(cudaMemcpy(P->dWphiE, wE.data(), wE.size() * sizeof(double), cudaMemcpyHostToDevice));
    DGM_CUDA(cudaMemcpy(P->dWphiH, wH.data(), wH.size() * sizeof(double), cudaMemcpyHostToDevice));
    DGM_CUDA(cudaMemcpy(P->dPhiE, phE.data(), phE.size() * sizeof(double), cudaMemcpyHostToDevice));
    DGM_CUDA(cudaMemcpy(P->dPhiH, phH.data(), phH.size() * sizeof(double), cudaMemcpyHostToDevice));
    P->rule_q1d = q1d;
    return DGM_OK;
}

int dgm_project_device(dgm_problem* P, int q1d, const double* E_pts, const double* H_pts, void* stream) {
    if (!P) {
        set_error("dgm_project_device: null problem");
        return DGM_ERR_INVALID_ARG;
    }
    int rc = ensure_rule(P, q1d);
    if (rc) return rc;
    const int nq = q1d * q1d * q1d;
    cudaStream_t s = (cudaStream_t)stream;
    int r = 0;
    if (P->tc) {
        // project into the FP64 staging buffer (orthonormal coefficients), then pack
        if (E_pts) {
            r |= dgm::launch_project<double>(P->nt, P->NE, nq, P->dMaps, P->dWphiE, E_pts, P->dStage, s);
            if (!r) r = dgm::tc_import(P, P->dStage, nullptr, nullptr, nullptr, s);
        }
        if (H_pts && !r) {
            r |= dgm::launch_project<double>(P->nt, P->NH, nq, P->dMaps, P->dWphiH, H_pts, P->dStage, s);
            if (!r) r = dgm::tc_import(P, nullptr, P->dStage, nullptr, nullptr, s);
        }
        return r ? cuda_fail(cudaGetLastError(), "project") : DGM_OK;
    }
    if (E_pts) P->trE_valid = false;
    if (H_pts) P->trH_valid = false;
    reset_comp(P);
    if (P->fp32) {
        if (E_pts) r |= dgm::launch_project<float>(P->nt, P->NE, nq, P->dMaps, P->dWphiE, E_pts, (float*)P->dE, s);
        if (H_pts) r |= dgm::launch_project<float>(P->nt, P->NH, nq, P->dMaps, P->dWphiH, H_pts, (float*)P->dH, s);
    } else {
        if (E_pts) r |= dgm::launch_project<double>(P->nt, P->NE, nq, P->dMaps, P->dWphiE, E_pts, (double*)P->dE, s);
        if (H_pts) r |= dgm::launch_project<double>(P->nt, P->NH, nq, P->dMaps, P->dWphiH, H_pts, (double*)P->dH, s);
    }
    return r ? cuda_fail(cudaGetLastError(), "project launch") : DGM_OK;
}

int dgm_eval_device(dgm_problem* P, int q1d, double* E_pts, double* H_pts, void* stream) {
    if (!P) {
        set_error("dgm_eval_device: null problem");
        return DGM_ERR_INVALID_ARG;
    }
    int rc = ensure_rule(P, q1d);
    if (rc) return rc;
    const int nq = q1d * q1d * q1d;
    cudaStream_t s = (cudaStream_t)stream;
    int r = 0;
    if (P->tc) {
        if (E_pts) {
            r = dgm::tc_export(P, P->dStage, nullptr, nullptr, nullptr, s);
            if (!r) r = dgm::launch_eval<double>(P->nt, P->NE, nq, P->dMaps, P->dPhiE, P->dStage, E_pts, s);
        }
        if (H_pts && !r) {
            r = dgm::tc_export(P, nullptr, P->dStage, nullptr, nullptr, s);
            if (!r) r = dgm::launch_eval<double>(P->nt, P->NH, nq, P->dMaps, P->dPhiH, P->dStage, H_pts, s);
        }
        return r ? cuda_fail(cudaGetLastError(), "eval") : DGM_OK;
    }
    if (P->fp32) {
        if (E_pts) r |= dgm::launch_eval<float>(P->nt, P->NE, nq, P->dMaps, P->dPhiE, (const float*)P->dE, E_pts, s);
        if (H_pts) r |= dgm::launch_eval<float>(P->nt, P->NH, nq, P->dMaps, P->dPhiH, (const float*)P->dH, H_pts, s);
    } else {
        if (E_pts) r |= dgm::launch_eval<double>(P->nt, P->NE, nq, P->dMaps, P->dPhiE, (const double*)P->dE, E_pts, s);
        if (H_pts) r |= dgm::launch_eval<double>(P->nt, P->NH, nq, P->dMaps, P->dPhiH, (const double*)P->dH, H_pts, s);
    }
    return r ? cuda_fail(cudaGetLastError(), "eval launch") : DGM_OK;
}

int dgm_reference_table(int p, int which, double* out, int64_t count, int64_t* needed) {
    dgm::RefTables t;
    int rc = dgm::build_ref_tables(p, t);
    if (rc) return rc;
    const std::vector<double>* v = nullptr;
    if (which >= 0 && which <= 2) v = &t.D[which];
    else if (which >= 3 && which <= 6) v = &t.TrE[which - 3];
    else if (which == 7) v = &t.norm2E;
    else {
        set_error("dgm_reference_table: which out of range");
        return DGM_ERR_INVALID_ARG;
    }
    if (needed) *needed = (int64_t)v->size();
    if (out) {
        if (count < (int64_t)v->size()) {
            set_error("dgm_reference_table: output too small");
            return DGM_ERR_INVALID_ARG;
        }
        std::memcpy(out, v->data(), v->size() * sizeof(double));
    }
    return DGM_OK;
}

int dgm_reference_table_2d(int p, int which, double* out, int64_t count, int64_t* needed) {
    dgm::RefTables2D t;
    int rc = dgm::build_ref_tables_2d(p, t);
    if (rc) return rc;
    const std::vector<double>* v = nullptr;
    if (which >= 0 && which <= 1) v = &t.D[which];
    else if (which >= 2 && which <= 4) v = &t.TrE[which - 2];
    else if (which >= 5 && which <= 7) v = &t.TrH[which - 5];
    else if (which == 8) v = &t.norm2E;
    else {
        set_error("dgm_reference_table_2d: which out of range");
        return DGM_ERR_INVALID_ARG;
    }
    if (needed) *needed = (int64_t)v->size();
    if (out) {
        if (count < (int64_t)v->size()) {
            set_error("dgm_reference_table_2d: output too small");
            return DGM_ERR_INVALID_ARG;
        }
        std::memcpy(out, v->data(), v->size() * sizeof(double));
    }
    return DGM_OK;
}

int dgm_quad_points(dgm_problem* P, int q1d, int64_t* count, double* xyz) {
    if (!P || !count || q1d < 1 || q1d > 32) {
        set_error("dgm_quad_points: bad argument");
        return DGM_ERR_INVALID_ARG;
    }
    const int nq = q1d * q1d * q1d;
    *count = P->nt * nq * 3;
    if (!xyz) return DGM_OK;
    std::vector<double> x, w, col;
    dgm::collapsed_rule(q1d, x, w, col);
    DevBuf buf;
    DGM_CUDA(cudaMalloc(&buf.p, (x.size() + (size_t)*count) * sizeof(double)));
    double* dxh = (double*)buf.p;
    double* dout = dxh + x.size();
    DGM_CUDA(cudaMemcpy(dxh, x.data(), x.size() * sizeof(double), cudaMemcpyHostToDevice));
    if (dgm::launch_quad_points(P->nt, nq, P->dMaps, dxh, dout, 0))
        return cuda_fail(cudaGetLastError(), "quad points launch");
    DGM_CUDA(cudaMemcpy(xyz, dout, (size_t)*count * sizeof(double), cudaMemcpyDeviceToHost));
    return DGM_OK;
}

int dgm_project(dgm_problem* P, int q1d, const double* E_pts, const double* H_pts) {
    if (!P || (!E_pts && !H_pts) || q1d < 1 || q1d > 32) {
        set_error("dgm_project: bad argument");
        return DGM_ERR_INVALID_ARG;
    }
    const size_t n = (size_t)P->nt * q1d * q1d * q1d * 3;
    DevBuf buf;
    DGM_CUDA(cudaMalloc(&buf.p, ((E_pts ? n : 0) + (H_pts ? n : 0)) * sizeof(double)));
    double* dE = E_pts ? (double*)buf.p : nullptr;
    double* dH = H_pts ? (double*)buf.p + (E_pts ? n : 0) : nullptr;
    if (dE) DGM_CUDA(cudaMemcpy(dE, E_pts, n * sizeof(double), cudaMemcpyHostToDevice));
    if (dH) DGM_CUDA(cudaMemcpy(dH, H_pts, n * sizeof(double), cudaMemcpyHostToDevice));
    int rc = dgm_project_device(P, q1d, dE, dH, nullptr);
    if (rc) return rc;
    DGM_CUDA(cudaDeviceSynchronize());
    return DGM_OK;
}

int dgm_eval(dgm_problem* P, int q1d, double* E_pts, double* H_pts) {
    if (!P || (!E_pts && !H_pts) || q1d < 1 || q1d > 32) {
        set_error("dgm_eval: bad argument");
        return DGM_ERR_INVALID_ARG;
    }
    const size_t n = (size_t)P->nt * q1d * q1d * q1d * 3;
    DevBuf buf;
    DGM_CUDA(cudaMalloc(&buf.p, ((E_pts ? n : 0) + (H_pts ? n : 0)) * sizeof(double)));
    double* dE = E_pts ? (double*)buf.p : nullptr;
    double* dH = H_pts ? (double*)buf.p + (E_pts ? n : 0) : nullptr;
    int rc = dgm_eval_device(P, q1d, dE, dH, nullptr);
    if (rc) return rc;
    if (dE) DGM_CUDA(cudaMemcpy(E_pts, dE, n * sizeof(double), cudaMemcpyDeviceToHost));
    if (dH) DGM_CUDA(cudaMemcpy(H_pts, dH, n * sizeof(double), cudaMemcpyDeviceToHost));
    return DGM_OK;
}

int dgm_grad_support(int dir, int* nterms, int32_t* shifts, int* lead) {
    if (dir < 0 || dir > 2 || !nterms) {
        set_error("dgm_grad_support: bad argument");
        return DGM_ERR_INVALID_ARG;
    }
    int sh[80];
    dgm::grad_support(dir, nterms, sh, lead);
    if (shifts) std::copy(sh, sh + 4 * (*nterms), shifts);
    return DGM_OK;
}

int dgm_grad_recurrence(int p, int dir, int* count, int32_t* ijk, double* coef) {
    if (p < 1 || p > DGM_PMAX || dir < 0 || dir > 2 || !count) {
        set_error("dgm_grad_recurrence: bad argument");
        return DGM_ERR_INVALID_ARG;
    }
    std::vector<int> r_ijk;
    std::vector<double> r_c;
    *count = dgm::grad_relations(p, dir, r_ijk, r_c);
    if (ijk) std::copy(r_ijk.begin(), r_ijk.end(), ijk);
    if (coef) std::copy(r_c.begin(), r_c.end(), coef);
    return DGM_OK;
}

int dgm_grad_sweep(int p, int dir, const double* a, double* b, int* swept) {
    if (p < 1 || p > DGM_PMAX || dir < 0 || dir > 2 || !a || !b) {
        set_error("dgm_grad_sweep: bad argument");
        return DGM_ERR_INVALID_ARG;
    }
    const int n = dgm::grad_sweep(p, dir, a, b);
    if (swept) *swept = n;
    return DGM_OK;
}

}  // extern "C"
