// 2D triangle solver (TE fields): mesh adjacency, element geometry, tables and
// the C-ABI entry points (include/dgm.h).  The operator is the central-flux
// system of Sec. 2.1 for E in the plane and H along z (tri2d.h); the time loop
// is the leapfrog of Sec. 3 with opening and closing half kicks of H.

#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "dgm.h"
#include "dgm_internal.h"
#include "kernels.h"
#include "problem.h"
#include "tri2d.h"

using dgm::set_error;

struct dgm_problem2d {
    dgm_ctx* ctx = nullptr;
    int p = 0, NE = 0, NH = 0;
    int64_t nt = 0;
    bool fp32 = false;
    int grid = 1;
    dgm::RefTables2D tab;
    void* dE = nullptr;
    void* dH = nullptr;
    void* dTables = nullptr;
    double* dGeo = nullptr;
    int32_t* dNbr = nullptr;
    int8_t* dSig = nullptr;
    double* dNrmE = nullptr;
    double* dNrmH = nullptr;
    double* dStage = nullptr;      // host-copy staging, max(nE, nH) doubles
    double* dPartials = nullptr;
    double* dEnergy = nullptr;     // energies of a run, device
    int64_t nEnergy = 0;
    dgm::KParams2D<double> kd{};
    dgm::KParams2D<float> kf{};
};

namespace {

int fail2(cudaError_t e, const char* what) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? DGM_ERR_OOM : DGM_ERR_CUDA;
}

#define DGM2_CUDA(call)                                  \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return fail2(e_, #call);  \
    } while (0)

void free2(dgm_problem2d* P) {
    void* ptrs[] = {P->dE, P->dH, P->dTables, P->dGeo, P->dNbr, P->dSig, P->dNrmE, P->dNrmH, P->dStage,
                    P->dPartials, P->dEnergy};
    for (void* q : ptrs)
        if (q) cudaFree(q);
}

struct Mesh2 {
    std::vector<std::array<int32_t, 3>> tri;   // vertices by ascending key
    std::vector<double> geo;                   // [nt][kGeo2Stride]
    std::vector<int32_t> nbr;                  // [nt][3]
    std::vector<int8_t> sig;                   // [nt][3]
};

int build_mesh2(int64_t nv, const double* xy, int64_t nt, const int32_t* tris, const int32_t* key_in,
                const double* eps, const double* mu, Mesh2& M) {
    M.tri.resize(nt);
    M.geo.assign((size_t)nt * dgm::kGeo2Stride, 0.0);
    M.nbr.assign((size_t)nt * 3, -1);
    M.sig.assign((size_t)nt * 3, 0);
    auto key = [&](int32_t v) { return key_in ? (int64_t)key_in[v] : (int64_t)v; };
    std::map<std::pair<int64_t, int64_t>, std::vector<std::pair<int64_t, int>>> edges;
    for (int64_t t = 0; t < nt; ++t) {
        std::array<int32_t, 3> v = {tris[3 * t], tris[3 * t + 1], tris[3 * t + 2]};
        for (int32_t x : v)
            if (x < 0 || x >= nv) {
                set_error("dgm_problem2d_create: vertex id out of range");
                return DGM_ERR_INVALID_ARG;
            }
        std::stable_sort(v.begin(), v.end(), [&](int32_t a, int32_t b) { return key(a) < key(b); });
        if (key(v[0]) == key(v[1]) || key(v[1]) == key(v[2])) {
            set_error("dgm_problem2d_create: triangle with repeated vertex keys");
            return DGM_ERR_INVALID_ARG;
        }
        M.tri[t] = v;
        const double* X0 = xy + 2 * v[0];
        const double* X1 = xy + 2 * v[1];
        const double* X2 = xy + 2 * v[2];
        const double F00 = X1[0] - X0[0], F10 = X1[1] - X0[1], F01 = X2[0] - X0[0], F11 = X2[1] - X0[1];
        const double det = F00 * F11 - F01 * F10;
        const double scale = std::max({std::fabs(F00), std::fabs(F01), std::fabs(F10), std::fabs(F11)});
        if (!(std::fabs(det) > 1e-12 * scale * scale)) {
            set_error("dgm_problem2d_create: degenerate triangle");
            return DGM_ERR_INVALID_ARG;
        }
        if (!(eps[t] > 0.0) || !(mu[t] > 0.0)) {
            set_error("dgm_problem2d_create: eps and mu must be positive");
            return DGM_ERR_INVALID_ARG;
        }
        // F^{-1} = [[F11, -F01], [-F10, F00]] / det
        const double I00 = F11 / det, I01 = -F01 / det, I10 = -F10 / det, I11 = F00 / det;
        double* g = &M.geo[(size_t)t * dgm::kGeo2Stride];
        g[0] = F00 * F00 + F10 * F10;   // F^T F
        g[1] = F00 * F01 + F10 * F11;
        g[2] = F01 * F01 + F11 * F11;
        g[3] = I00 * I00 + I01 * I01;   // F^{-1} F^{-T}
        g[4] = I00 * I10 + I01 * I11;
        g[5] = I10 * I10 + I11 * I11;
        g[6] = std::fabs(det);
        g[7] = det > 0.0 ? 1.0 : -1.0;
        g[8] = eps[t];
        g[9] = mu[t];
        for (int f = 0; f < 3; ++f) {
            const int a = f == 0 ? 1 : 0, b = f == 2 ? 1 : 2;   // the two local vertices other than f
            const double* Xa = xy + 2 * v[a];
            const double* Xb = xy + 2 * v[b];
            const double* Xo = xy + 2 * v[f];
            const double dx = Xb[0] - Xa[0], dy = Xb[1] - Xa[1];
            double nx = dy, ny = -dx;   // a normal; point it away from the opposite vertex
            if (nx * (Xo[0] - Xa[0]) + ny * (Xo[1] - Xa[1]) > 0.0) {
                nx = -nx;
                ny = -ny;
            }
            // sigma: the edge vector against the outward normal turned counter-clockwise
            M.sig[(size_t)t * 3 + f] = (int8_t)((-ny) * dx + nx * dy > 0.0 ? 1 : -1);
            edges[{key(v[a]), key(v[b])}].push_back({t, f});
        }
    }
    for (auto& kv : edges) {
        auto& lst = kv.second;
        if (lst.size() > 2) {
            set_error("dgm_problem2d_create: edge shared by more than two triangles");
            return DGM_ERR_INVALID_ARG;
        }
        if (lst.size() == 2) {
            if (lst[0].first == lst[1].first) {
                set_error("dgm_problem2d_create: triangle glued to itself");
                return DGM_ERR_INVALID_ARG;
            }
            M.nbr[(size_t)lst[0].first * 3 + lst[0].second] = (int32_t)(3 * lst[1].first + lst[1].second);
            M.nbr[(size_t)lst[1].first * 3 + lst[1].second] = (int32_t)(3 * lst[0].first + lst[0].second);
        }
    }
    return DGM_OK;
}

template <typename real>
int upload2(dgm_problem2d* P, dgm::KParams2D<real>& K) {
    const dgm::RefTables2D& t = P->tab;
    const int NE = t.NE, NH = t.NH, p = t.p;
    const size_t nD = (size_t)NH * NE, nTE = (size_t)3 * (p + 1) * NE, nTH = (size_t)3 * p * NH;
    std::vector<real> buf(2 * nD + nTE + nTH);
    for (size_t i = 0; i < nD; ++i) {
        buf[i] = (real)t.D[0][i];
        buf[nD + i] = (real)t.D[1][i];
    }
    for (int f = 0; f < 3; ++f) {
        std::copy(t.TrE[f].begin(), t.TrE[f].end(), buf.begin() + (2 * nD + (size_t)f * (p + 1) * NE));
        std::copy(t.TrH[f].begin(), t.TrH[f].end(), buf.begin() + (2 * nD + nTE + (size_t)f * p * NH));
    }
    DGM2_CUDA(cudaMalloc(&P->dTables, buf.size() * sizeof(real)));
    DGM2_CUDA(cudaMemcpy(P->dTables, buf.data(), buf.size() * sizeof(real), cudaMemcpyHostToDevice));
    real* base = (real*)P->dTables;
    K.nt = P->nt;
    K.p = p;
    K.NE = NE;
    K.NH = NH;
    K.E = (real*)P->dE;
    K.H = (real*)P->dH;
    K.geo = P->dGeo;
    K.nbr = P->dNbr;
    K.sig = P->dSig;
    K.Dx = base;
    K.Dy = base + nD;
    K.TrE = base + 2 * nD;
    K.TrH = base + 2 * nD + nTE;
    return DGM_OK;
}

int phase_H2d(dgm_problem2d* P, double dt, double a_lo, double c_out, double* partials, cudaStream_t s) {
    const int r = P->fp32 ? dgm::launch2d_phase_H<float>(P->kf, dt, a_lo, c_out, partials, P->grid, s)
                          : dgm::launch2d_phase_H<double>(P->kd, dt, a_lo, c_out, partials, P->grid, s);
    return r ? fail2(cudaGetLastError(), "2D H-phase launch") : DGM_OK;
}

int phase_E2d(dgm_problem2d* P, double dt, cudaStream_t s) {
    const int r = P->fp32 ? dgm::launch2d_phase_E<float>(P->kf, dt, P->grid, s)
                          : dgm::launch2d_phase_E<double>(P->kd, dt, P->grid, s);
    return r ? fail2(cudaGetLastError(), "2D E-phase launch") : DGM_OK;
}

}  // namespace

int dgm_mesh2d_info(int64_t nv, const double* xy, int64_t nt, const int32_t* tris, const int32_t* vertex_key,
                    int64_t* nedges, int64_t* nboundary) {
    if (!xy || !tris || nv < 3 || nt < 1) {
        set_error("dgm_mesh2d_info: bad argument");
        return DGM_ERR_INVALID_ARG;
    }
    std::vector<double> one((size_t)nt, 1.0);
    Mesh2 M;
    const int rc = build_mesh2(nv, xy, nt, tris, vertex_key, one.data(), one.data(), M);
    if (rc) return rc;
    int64_t interior_sides = 0, boundary = 0;
    for (int32_t nb : M.nbr) (nb >= 0 ? interior_sides : boundary) += 1;
    if (nedges) *nedges = interior_sides / 2 + boundary;
    if (nboundary) *nboundary = boundary;
    return DGM_OK;
}

int dgm_problem2d_create(dgm_ctx* ctx, int64_t nv, const double* xy, int64_t nt, const int32_t* tris,
                         const int32_t* vertex_key, int p, const double* eps, const double* mu, int precision,
                         dgm_problem2d** out) {
    if (!out) {
        set_error("dgm_problem2d_create: null output");
        return DGM_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (!ctx || !xy || !tris || !eps || !mu || nv < 3 || nt < 1) {
        set_error("dgm_problem2d_create: bad argument");
        return DGM_ERR_INVALID_ARG;
    }
    if (precision != DGM_PREC_FP64 && precision != DGM_PREC_FP32) {
        set_error("dgm_problem2d_create: the 2D solver runs in FP64 or FP32");
        return DGM_ERR_UNSUPPORTED;
    }
    Mesh2 M;
    int rc = build_mesh2(nv, xy, nt, tris, vertex_key, eps, mu, M);
    if (rc) return rc;
    dgm_problem2d* P = new (std::nothrow) dgm_problem2d;
    if (!P) return DGM_ERR_OOM;
    auto fail = [&](int code) {
        free2(P);
        delete P;
        return code;
    };
    rc = dgm::build_ref_tables_2d(p, P->tab);
    if (rc) return fail(rc);
    P->ctx = ctx;
    P->p = p;
    P->NE = P->tab.NE;
    P->NH = P->tab.NH;
    P->nt = nt;
    P->fp32 = precision == DGM_PREC_FP32;
    const int wpb = dgm::phase2d_warps_per_block();
    P->grid = (int)std::min<int64_t>((nt + wpb - 1) / wpb, (int64_t)ctx->num_sms * 16);
    cudaError_t e;
    if ((e = cudaSetDevice(ctx->device)) != cudaSuccess) return fail(fail2(e, "cudaSetDevice"));
    const size_t rs = P->fp32 ? sizeof(float) : sizeof(double);
    const int64_t nE = nt * 2 * P->NE, nH = nt * P->NH;
    if ((e = cudaMalloc(&P->dE, nE * rs)) != cudaSuccess) return fail(fail2(e, "alloc E"));
    if ((e = cudaMalloc(&P->dH, nH * rs)) != cudaSuccess) return fail(fail2(e, "alloc H"));
    if ((e = cudaMemset(P->dE, 0, nE * rs)) != cudaSuccess || (e = cudaMemset(P->dH, 0, nH * rs)) != cudaSuccess)
        return fail(fail2(e, "clear fields"));
    if ((e = cudaMalloc(&P->dGeo, M.geo.size() * sizeof(double))) != cudaSuccess) return fail(fail2(e, "alloc geo"));
    if ((e = cudaMalloc(&P->dNbr, M.nbr.size() * sizeof(int32_t))) != cudaSuccess) return fail(fail2(e, "alloc nbr"));
    if ((e = cudaMalloc(&P->dSig, M.sig.size())) != cudaSuccess) return fail(fail2(e, "alloc sig"));
    if ((e = cudaMemcpy(P->dGeo, M.geo.data(), M.geo.size() * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(P->dNbr, M.nbr.data(), M.nbr.size() * sizeof(int32_t), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(P->dSig, M.sig.data(), M.sig.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
        return fail(fail2(e, "upload geometry"));
    {
        std::vector<int> iE, iH;
        dgm::index2(p, iE);
        dgm::index2(p - 1, iH);
        std::vector<double> nrmE(P->NE), nrmH(P->NH);
        for (int a = 0; a < P->NE; ++a) nrmE[a] = std::sqrt(dgm::dubiner2_norm2(iE[2 * a], iE[2 * a + 1]));
        for (int b = 0; b < P->NH; ++b) nrmH[b] = std::sqrt(dgm::dubiner2_norm2(iH[2 * b], iH[2 * b + 1]));
        if ((e = cudaMalloc(&P->dNrmE, P->NE * sizeof(double))) != cudaSuccess) return fail(fail2(e, "alloc nrm"));
        if ((e = cudaMalloc(&P->dNrmH, P->NH * sizeof(double))) != cudaSuccess) return fail(fail2(e, "alloc nrm"));
        if ((e = cudaMemcpy(P->dNrmE, nrmE.data(), P->NE * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess ||
            (e = cudaMemcpy(P->dNrmH, nrmH.data(), P->NH * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess)
            return fail(fail2(e, "upload norms"));
    }
    if ((e = cudaMalloc(&P->dStage, std::max(nE, nH) * sizeof(double))) != cudaSuccess)
        return fail(fail2(e, "alloc stage"));
    if ((e = cudaMalloc(&P->dPartials, (size_t)P->grid * sizeof(double))) != cudaSuccess)
        return fail(fail2(e, "alloc partials"));
    rc = P->fp32 ? upload2<float>(P, P->kf) : upload2<double>(P, P->kd);
    if (rc) return fail(rc);
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return fail(fail2(e, "2D setup"));
    *out = P;
    return DGM_OK;
}

int dgm_problem2d_destroy(dgm_problem2d* P) {
    if (!P) return DGM_OK;
    free2(P);
    delete P;
    return DGM_OK;
}

int dgm_problem2d_sizes(const dgm_problem2d* P, int64_t* nE, int64_t* nH) {
    if (!P) {
        set_error("dgm_problem2d_sizes: null problem");
        return DGM_ERR_INVALID_ARG;
    }
    if (nE) *nE = P->nt * 2 * P->NE;
    if (nH) *nH = P->nt * P->NH;
    return DGM_OK;
}

int dgm_set_fields2d(dgm_problem2d* P, const double* E, const double* H) {
    if (!P) {
        set_error("dgm_set_fields2d: null problem");
        return DGM_ERR_INVALID_ARG;
    }
    DGM2_CUDA(cudaSetDevice(P->ctx->device));
    const int64_t nE = P->nt * 2 * P->NE, nH = P->nt * P->NH;
    int r = 0;
    if (E) {
        DGM2_CUDA(cudaMemcpy(P->dStage, E, nE * sizeof(double), cudaMemcpyHostToDevice));
        r = P->fp32 ? dgm::launch_import<float>(P->dStage, (float*)P->dE, P->dNrmE, nE, P->NE, 0)
                    : dgm::launch_import<double>(P->dStage, (double*)P->dE, P->dNrmE, nE, P->NE, 0);
        if (r) return fail2(cudaGetLastError(), "2D import E");
        DGM2_CUDA(cudaDeviceSynchronize());
    }
    if (H) {
        DGM2_CUDA(cudaMemcpy(P->dStage, H, nH * sizeof(double), cudaMemcpyHostToDevice));
        r = P->fp32 ? dgm::launch_import<float>(P->dStage, (float*)P->dH, P->dNrmH, nH, P->NH, 0)
                    : dgm::launch_import<double>(P->dStage, (double*)P->dH, P->dNrmH, nH, P->NH, 0);
        if (r) return fail2(cudaGetLastError(), "2D import H");
        DGM2_CUDA(cudaDeviceSynchronize());
    }
    return DGM_OK;
}

int dgm_get_fields2d(dgm_problem2d* P, double* E, double* H) {
    if (!P) {
        set_error("dgm_get_fields2d: null problem");
        return DGM_ERR_INVALID_ARG;
    }
    DGM2_CUDA(cudaSetDevice(P->ctx->device));
    const int64_t nE = P->nt * 2 * P->NE, nH = P->nt * P->NH;
    int r = 0;
    if (E) {
        r = P->fp32 ? dgm::launch_export<float>((const float*)P->dE, P->dStage, P->dNrmE, nE, P->NE, 0)
                    : dgm::launch_export<double>((const double*)P->dE, P->dStage, P->dNrmE, nE, P->NE, 0);
        if (r) return fail2(cudaGetLastError(), "2D export E");
        DGM2_CUDA(cudaMemcpy(E, P->dStage, nE * sizeof(double), cudaMemcpyDeviceToHost));
    }
    if (H) {
        r = P->fp32 ? dgm::launch_export<float>((const float*)P->dH, P->dStage, P->dNrmH, nH, P->NH, 0)
                    : dgm::launch_export<double>((const double*)P->dH, P->dStage, P->dNrmH, nH, P->NH, 0);
        if (r) return fail2(cudaGetLastError(), "2D export H");
        DGM2_CUDA(cudaMemcpy(H, P->dStage, nH * sizeof(double), cudaMemcpyDeviceToHost));
    }
    return DGM_OK;
}

int dgm_kick2d(dgm_problem2d* P, int which, double dt) {
    if (!P || (which != 0 && which != 1) || !std::isfinite(dt)) {
        set_error("dgm_kick2d: bad argument");
        return DGM_ERR_INVALID_ARG;
    }
    DGM2_CUDA(cudaSetDevice(P->ctx->device));
    const int rc = which == 0 ? phase_H2d(P, dt, 0.0, 1.0, nullptr, 0) : phase_E2d(P, dt, 0);
    if (rc) return rc;
    DGM2_CUDA(cudaDeviceSynchronize());
    return DGM_OK;
}

int dgm_run2d(dgm_problem2d* P, double dt, int64_t nsteps, void* stream, double* energy_out) {
    if (!P || nsteps < 0 || !std::isfinite(dt)) {
        set_error("dgm_run2d: bad argument");
        return DGM_ERR_INVALID_ARG;
    }
    DGM2_CUDA(cudaSetDevice(P->ctx->device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (energy_out && P->nEnergy < nsteps + 1) {
        if (P->dEnergy) cudaFree(P->dEnergy);
        P->dEnergy = nullptr;
        P->nEnergy = 0;
        DGM2_CUDA(cudaMalloc(&P->dEnergy, (size_t)(nsteps + 1) * sizeof(double)));
        P->nEnergy = nsteps + 1;
    }
    auto energy_slot = [&](int64_t n) { return energy_out ? P->dEnergy + n : nullptr; };
    auto H_phase = [&](double a_lo, double c_out, int64_t n) {
        double* slot = energy_slot(n);
        int rc = phase_H2d(P, dt, a_lo, c_out, slot ? P->dPartials : nullptr, s);
        if (rc) return rc;
        if (slot && dgm::launch_energy_reduce(P->dPartials, P->grid, slot, s))
            return fail2(cudaGetLastError(), "2D energy reduce launch");
        return (int)DGM_OK;
    };
    // opening half kick: W^0 pairs H^{-1/2} and H^{+1/2} around H^0
    int rc = H_phase(0.5, 0.5, 0);
    for (int64_t n = 0; n < nsteps && !rc; ++n) {
        rc = phase_E2d(P, dt, s);
        if (!rc) rc = H_phase(0.0, 1.0, n + 1);
    }
    // closing half kick back to H^N
    if (!rc) rc = phase_H2d(P, dt, 0.0, -0.5, nullptr, s);
    if (rc) return rc;
    if (energy_out)
        DGM2_CUDA(cudaMemcpyAsync(energy_out, P->dEnergy, (size_t)(nsteps + 1) * sizeof(double),
                                  cudaMemcpyDeviceToHost, s));
    DGM2_CUDA(cudaStreamSynchronize(s));
    return DGM_OK;
}
