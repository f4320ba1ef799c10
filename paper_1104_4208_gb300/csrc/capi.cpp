// C ABI implementation (host).  See include/dgm.h for the contract.

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "dgm_internal.h"
#include "kernels.h"
#include "problem.h"

namespace dgm {

static thread_local std::string g_err;

void set_error(const std::string& msg) { g_err = msg; }

}  // namespace dgm

using dgm::set_error;

namespace {

int cuda_fail(cudaError_t e, const char* what) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? DGM_ERR_OOM : DGM_ERR_CUDA;
}

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
    DGM_CUDA(cudaMalloc(&P->dTables, buf.size() * sizeof(real)));
    DGM_CUDA(cudaMemcpy(P->dTables, buf.data(), buf.size() * sizeof(real), cudaMemcpyHostToDevice));
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

int phase_H(dgm_problem* P, double dt, double a_lo, double c_out, double* energy_slot, cudaStream_t s) {
    if (P->tc) return dgm::tc_phase_H(P, dt, a_lo, c_out, energy_slot, s);
    double* partials = energy_slot ? P->dPartials : nullptr;
    int rc = P->fp32 ? dgm::launch_phase_H<float>(P->kf, P->grid, dt, a_lo, c_out, partials, s)
                     : dgm::launch_phase_H<double>(P->kd, P->grid, dt, a_lo, c_out, partials, s);
    if (rc) return cuda_fail(cudaGetLastError(), "H-phase launch");
    if (energy_slot && dgm::launch_energy_reduce(P->dPartials, P->grid, energy_slot, s))
        return cuda_fail(cudaGetLastError(), "energy reduce launch");
    return DGM_OK;
}

int phase_E(dgm_problem* P, double dt, cudaStream_t s, bool energy = false) {
    if (P->tc) return dgm::tc_phase_E(P, dt, energy, s);
    int rc = P->fp32 ? dgm::launch_phase_E<float>(P->kf, P->grid, dt, s)
                     : dgm::launch_phase_E<double>(P->kd, P->grid, dt, s);
    if (rc) return cuda_fail(cudaGetLastError(), "E-phase launch");
    return DGM_OK;
}

int import_fields(dgm_problem* P, const double* dEsrc, const double* dHsrc, cudaStream_t s) {
    if (P->tc) return dgm::tc_import(P, dEsrc, dHsrc, P->dNrmE, P->dNrmH, s);
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
                    P->dK, P->dFaceGeo, P->dFid, P->dNrmF};
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
    if (o.precision != DGM_PREC_FP64 && o.precision != DGM_PREC_FP32 && o.precision != DGM_PREC_TC32) {
        set_error("dgm_problem_create: unknown precision");
        return DGM_ERR_INVALID_ARG;
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
    int rc = dgm::build_ref_tables(p, P->tab);
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

    auto fail = [&](int code) {
        free_problem(P);
        delete P;
        return code;
    };
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(cuda_fail(cudaGetLastError(), "cudaSetDevice"));
    const size_t rs = P->fp32 ? sizeof(float) : sizeof(double);
    const int64_t nE = m.nt * 3 * P->NE, nH = m.nt * 3 * P->NH;
    const bool tc = o.precision == DGM_PREC_TC32;
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
    if ((e = cudaMalloc(&P->dStage, std::max(std::max(nE, nH), nK) * sizeof(double))) != cudaSuccess)
        return fail(cuda_fail(e, "alloc staging"));
    if ((e = cudaMalloc(&P->dPartials, (size_t)P->grid * sizeof(double))) != cudaSuccess)
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
    }
    if ((e = cudaMalloc(&P->dGeo, geo.size() * sizeof(double))) != cudaSuccess) return fail(cuda_fail(e, "alloc geo"));
    if ((e = cudaMalloc(&P->dNbr, nbr.size() * sizeof(int32_t))) != cudaSuccess) return fail(cuda_fail(e, "alloc nbr"));
    cudaMemcpy(P->dGeo, geo.data(), geo.size() * sizeof(double), cudaMemcpyHostToDevice);
    cudaMemcpy(P->dNbr, nbr.data(), nbr.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
    {
        std::vector<double> nrmE(P->NE), nrmH(P->NH);
        std::vector<int> iH;
        dgm::index3(p - 1, iH);
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
            if (!P->trE_valid) {
                r = dgm::tc_traces(P, 0, s);
                if (r) return r;
            }
            r = dgm::tc_launch_phase_H(P->tca, P->tc_grid, dt, a_lo, c_out, slot ? 1 : 0, s);
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
        r = P->fp32 ? dgm::launch_phase_H<float>(P->kf, P->grid, dt, a_lo, c_out, slot ? P->dPartials : nullptr, s)
                    : dgm::launch_phase_H<double>(P->kd, P->grid, dt, a_lo, c_out, slot ? P->dPartials : nullptr, s);
        if (r) return cuda_fail(cudaGetLastError(), "H-phase launch");
        if ((r = done())) return r;
        if (slot) {
            if ((r = mark(2))) return r;
            if (dgm::launch_energy_reduce(P->dPartials, P->grid, slot, s))
                return cuda_fail(cudaGetLastError(), "energy reduce launch");
            if ((r = done())) return r;
        }
        return DGM_OK;
    };
    auto run_E = [&]() -> int {
        int r = mark(1);
        if (r) return r;
        r = phase_E(P, dt, s, want);
        if (r) return r;
        return done();
    };
    if (P->tc && want) {
        rc = mark(2);
        if (!rc) rc = dgm::tc_traces(P, 0, s);
        if (!rc) rc = done();
    }
    if (!rc) rc = run_H(0.5, 0.5, want ? W : nullptr);
    for (int64_t n = 0; n < nsteps && !rc; ++n) {
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
    if (want) {
        for (int64_t n = 0; n <= nsteps; ++n)
            if (!std::isfinite(energy_out[n]) || energy_out[n] > 10.0 * std::fabs(energy_out[0]) + 1e-300) {
                set_error("dgm_run: energy blew up (time step above the stability bound?)");
                return DGM_ERR_UNSTABLE;
            }
    }
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
    dgm::phi_table(P->p - 1, q1d, phH);
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

}  // extern "C"
