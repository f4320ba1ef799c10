// Host side of the tensor-core path: reference operators laid out in the
// MMA's shared-memory order ([K/4][rows][4], TF32-rounded), the tiled state,
// face-trace buffers, and the launch sequence of one time step.
//
// Internal coefficient order of one element: k = 3 a + m (coefficient a,
// component m), so the 3x3 inverse-mass block of a coefficient acts on three
// consecutive values.  Face-trace columns: j = f FB + i N2(p-1) + g (face f,
// tangential component i, face mode g of degree <= p-1; FB = 2 N2(p-1) padded
// to a multiple of 4 so that each face's block is 16-byte aligned).

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include <cstring>

#include "problem.h"

namespace dgm {

namespace {

// Round to the nearest TF32 value (10-bit mantissa), ties away from zero.
float round_tf32(float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    if ((u & 0x7f800000u) != 0x7f800000u) u = (u + 0x1000u) & 0xffffe000u;
    float r;
    std::memcpy(&r, &u, 4);
    return r;
}

// One table in the MMA operand layout [K/VPC][rows][VPC].  TF32 values are
// rounded here; fp16 values are rounded on the device when the fp32 staging
// copy is converted.
struct TableWriter {
    std::vector<float>& buf;
    size_t base;
    int rows;
    int vpc;
    void put(int row, int k, double v) {
        const float x = (float)v;
        buf[base + ((size_t)(k / vpc) * rows + row) * vpc + (k % vpc)] = vpc == 4 ? round_tf32(x) : x;
    }
};

size_t round_up(size_t n, size_t a) { return (n + a - 1) / a * a; }

// (curl E)_m[b] = sum_{a, m'} curl_entry(b, m, a, m') E_{m'}[a]  (Sec. 3.2.2: curl from gradients)
double curl_entry(const RefTables& t, int b, int m, int a, int mp) {
    const size_t i = (size_t)b * t.NE + a;
    switch (m) {
        case 0: return mp == 2 ? t.D[1][i] : (mp == 1 ? -t.D[2][i] : 0.0);
        case 1: return mp == 0 ? t.D[2][i] : (mp == 2 ? -t.D[0][i] : 0.0);
        default: return mp == 1 ? t.D[0][i] : (mp == 0 ? -t.D[1][i] : 0.0);
    }
}

int cuda_err(cudaError_t e, const char* what) {
    set_error(std::string("tensor-core path: ") + what + ": " + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? DGM_ERR_OOM : DGM_ERR_CUDA;
}

}  // namespace

namespace {
int tc2_problem_init(dgm_problem* P, const MeshData& m, const std::vector<double>& geo,
                     const std::vector<int32_t>& nbr);
}

int tc_problem_init(dgm_problem* P, const MeshData& m, const std::vector<double>& geo,
                    const std::vector<int32_t>& nbr) {
    if ((P->opt.precision == DGM_PREC_TC16 && P->opt.variant != 1) || P->opt.precision == DGM_PREC_TCBF16)
        return tc2_problem_init(P, m, geo, nbr);
    const RefTables& T = P->tab;
    const bool split = P->opt.precision == DGM_PREC_TC16X2;
    const bool f16 = P->opt.precision == DGM_PREC_TC16 || split;
    const char* name = split ? "TC16X2" : f16 ? "TC16" : "TC32";
    const TCDims d = tc_dims(T.NE, T.NH, T.N2H, f16, split);
    uint32_t stage = 0, r2 = 0;
    const size_t smem = tc_smem_bytes(d, &stage, &r2);
    if (P->p > 6 || smem + 1024 > 227 * 1024 || tc_tmem_cols(d) > 512) {
        set_error(std::string("precision ") + name + " supports p <= 6");
        return DGM_ERR_UNSUPPORTED;
    }
    if (tc_tmem_reach(d) > tc_tmem_cols(d)) {
        set_error(std::string(name) + " epilogue would read past its TMEM allocation");
        return DGM_ERR_UNSUPPORTED;
    }
    if (P->opt.flux != DGM_FLUX_CENTRAL) {
        set_error(std::string("precision ") + name + " supports the central flux only");
        return DGM_ERR_UNSUPPORTED;
    }
    const int64_t ntiles = (m.nt + kTcRows - 1) / kTcRows;
    const int64_t nrow = ntiles * kTcRows;
    const size_t esz = f16 ? 2 : 4;   // bytes per operand value
    // one allocation, regions 1 KB aligned: fp32 state E, H; (fp16) operand
    // copies of E, H; trace buffers; tables
    const size_t bE = round_up((size_t)nrow * d.KE * 4, 1024), bH = round_up((size_t)nrow * d.KH * 4, 1024);
    const size_t bEo = f16 ? round_up((size_t)nrow * d.KEo * esz, 1024) : 0;
    const size_t bHo = f16 ? round_up((size_t)nrow * d.KHo * esz, 1024) : 0;
    const size_t bTr = round_up((size_t)nrow * d.NT * esz, 1024);
    // table sizes in values
    const size_t b1h = (size_t)d.KEo * d.NC, blh = (size_t)d.NT * d.NC, bth = (size_t)d.KHo * d.NT;
    const size_t b1e = (size_t)d.KHo * d.NCE, ble = (size_t)d.NT * d.NCE, bte = (size_t)d.KEo * d.NT;
    const size_t ntab = b1h + blh + bth + b1e + ble + bte;
    const size_t o_state = 0, o_Eo = bE + bH, o_Ho = o_Eo + bEo, o_tr = o_Ho + bHo, o_tab = o_tr + 2 * bTr;
    // two-term tables: the lo terms follow the hi terms, at one offset for all tables
    const size_t lo_off = split ? round_up(ntab * esz, 1024) : 0;
    const size_t total = o_tab + (split ? 2 * lo_off : ntab * esz);
    cudaError_t e;
    if ((e = cudaMalloc(&P->dTc, total)) != cudaSuccess) return cuda_err(e, "alloc");
    if ((e = cudaMemset(P->dTc, 0, o_tab)) != cudaSuccess) return cuda_err(e, "memset");
    uint8_t* base8 = static_cast<uint8_t*>(P->dTc);

    std::vector<float> tab(ntab, 0.0f);
    const size_t o_b1h = 0, o_blh = o_b1h + b1h, o_bth = o_blh + blh, o_b1e = o_bth + bth, o_ble = o_b1e + b1e,
                 o_bte = o_ble + ble;
    const int V = d.VPC;
    TableWriter B1H{tab, o_b1h, d.NC, V}, BLH{tab, o_blh, d.NC, V}, BTH{tab, o_bth, d.NT, V};
    TableWriter B1E{tab, o_b1e, d.NCE, V}, BLE{tab, o_ble, d.NCE, V}, BTE{tab, o_bte, d.NT, V};
    const int NE = T.NE, NH = T.NH, N2H = T.N2H;
    for (int b = 0; b < NH; ++b)
        for (int mo = 0; mo < 3; ++mo)
            for (int a = 0; a < NE; ++a)
                for (int mi = 0; mi < 3; ++mi) {
                    const double v = curl_entry(T, b, mo, a, mi);
                    if (v == 0.0) continue;
                    B1H.put(3 * b + mo, 3 * a + mi, v);   // H-phase: curl of E
                    B1E.put(3 * a + mi, 3 * b + mo, v);   // E-phase: the same numbers transposed
                }
    for (int f = 0; f < 4; ++f)
        for (int i = 0; i < 2; ++i)
            for (int gm = 0; gm < N2H; ++gm) {
                const int j = f * d.FB + i * N2H + gm;
                const int gE = T.pos2H[gm];
                for (int a = 0; a < NE; ++a) {
                    const double tr = T.TrE[f][(size_t)gE * NE + a];
                    for (int mm = 0; mm < 3; ++mm) {
                        const double v = T.that[f][i][mm] * tr;
                        if (v == 0.0) continue;
                        BTE.put(j, 3 * a + mm, v);
                        // lift of the face average into E: (t2_m b1 - t1_m b2)
                        BLE.put(3 * a + mm, f * d.FB + (1 - i) * N2H + gm, i == 1 ? v : -v);
                    }
                }
                for (int b = 0; b < NH; ++b) {
                    const double tr = T.TrH[f][(size_t)gm * NH + b];
                    for (int mm = 0; mm < 3; ++mm) {
                        const double v = T.that[f][i][mm] * tr;
                        if (v == 0.0) continue;
                        BTH.put(j, 3 * b + mm, v);
                        BLH.put(3 * b + mm, f * d.FB + (1 - i) * N2H + gm, i == 1 ? v : -v);
                    }
                }
            }
    uint8_t* dtab = base8 + o_tab;
    if (!f16) {
        if ((e = cudaMemcpy(dtab, tab.data(), ntab * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess)
            return cuda_err(e, "tables");
    } else {
        // fp32 staging copy, rounded to fp16 (or split into two fp16 terms) on the device
        float* stage32 = nullptr;
        if ((e = cudaMalloc(&stage32, ntab * sizeof(float))) != cudaSuccess) return cuda_err(e, "alloc tables");
        e = cudaMemcpy(stage32, tab.data(), ntab * sizeof(float), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) {
            const int r = split ? tc_launch_split_half(stage32, dtab, dtab + lo_off, ntab, 0)
                                : tc_launch_to_half(stage32, dtab, ntab, 0);
            if (r) e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        cudaFree(stage32);
        if (e != cudaSuccess) return cuda_err(e, "tables");
    }

    // padded geometry and topology (padding elements: identity metric, PEC faces, zero fields)
    std::vector<double> g2((size_t)nrow * kGeoStride, 0.0);
    std::copy(geo.begin(), geo.end(), g2.begin());
    for (int64_t t = m.nt; t < nrow; ++t) {
        double* r = &g2[(size_t)t * kGeoStride];
        r[0] = r[3] = r[5] = r[6] = r[9] = r[11] = 1.0;
        r[kGeoEps] = r[kGeoInvEps] = r[kGeoMu] = r[kGeoInvMu] = r[kGeoSign] = 1.0;
    }
    std::vector<int32_t> n2((size_t)nrow * 4, -1);
    std::copy(nbr.begin(), nbr.end(), n2.begin());
    if ((e = cudaMalloc(&P->dTcGeo, g2.size() * sizeof(double))) != cudaSuccess) return cuda_err(e, "alloc geo");
    if ((e = cudaMalloc(&P->dTcNbr, n2.size() * sizeof(int32_t))) != cudaSuccess) return cuda_err(e, "alloc nbr");
    cudaMemcpy(P->dTcGeo, g2.data(), g2.size() * sizeof(double), cudaMemcpyHostToDevice);
    cudaMemcpy(P->dTcNbr, n2.data(), n2.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
    if ((e = cudaMalloc(&P->dErr, sizeof(int))) != cudaSuccess) return cuda_err(e, "alloc err");
    cudaMemset(P->dErr, 0, sizeof(int));

    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, P->ctx->device);
    // CTAs resident per SM: two when their TMEM columns and shared memory allow it
    const uint32_t tcols = tc_tmem_cols(d);
    const int per_sm = (tcols <= 256 && 2 * (smem + 1024) <= 227 * 1024) ? 2 : 1;
    P->tc_grid = (int)std::min<int64_t>(ntiles, (int64_t)sms * per_sm);
    P->tc_grid_cap = P->tc_grid;   // the autotuner may lower it to one CTA per SM
    double* part = nullptr;
    if ((e = cudaMalloc(&part, 2 * (size_t)P->tc_grid_cap * sizeof(double))) != cudaSuccess)
        return cuda_err(e, "alloc partials");
    cudaMemset(part, 0, 2 * (size_t)P->tc_grid_cap * sizeof(double));

    TCArgs& A = P->tca;
    A.nt = m.nt;
    A.ntiles = (int)ntiles;
    A.d = d;
    A.E = reinterpret_cast<float*>(base8 + o_state);
    A.H = reinterpret_cast<float*>(base8 + bE);
    A.Eop = f16 ? static_cast<void*>(base8 + o_Eo) : static_cast<void*>(A.E);
    A.Hop = f16 ? static_cast<void*>(base8 + o_Ho) : static_cast<void*>(A.H);
    A.trE = base8 + o_tr;
    A.trH = base8 + o_tr + bTr;
    A.geo = P->dTcGeo;
    A.nbr = P->dTcNbr;
    A.B1H = dtab + o_b1h * esz;
    A.BliftH = dtab + o_blh * esz;
    A.BtrH = dtab + o_bth * esz;
    A.B1E = dtab + o_b1e * esz;
    A.BliftE = dtab + o_ble * esz;
    A.BtrE = dtab + o_bte * esz;
    A.partE = part;
    A.partH = part + P->tc_grid;   // contiguous with partE for the reduction; moves with tc_grid
    A.tab_lo = (int64_t)lo_off;
    A.err = P->dErr;
    for (int f = 0; f < 4; ++f) A.sigma_hat[f] = (float)T.sigma_hat[f];
    A.stage_bytes = stage;
    A.tmem_cols = tcols;
    A.r2_offset = r2;
    P->tc = true;
    P->trE_valid = P->trH_valid = false;
    return DGM_OK;
}

namespace {

int pad_to(int x, int m) { return (x + m - 1) / m * m; }

// Layout 2 (resident-table kernels, 2-byte operands): component-separated
// tables, component-major state, trace blocks per (face, tangent).
int tc2_problem_init(dgm_problem* P, const MeshData& m, const std::vector<double>& geo,
                     const std::vector<int32_t>& nbr) {
    const RefTables& T = P->tab;
    const bool bf = P->opt.precision == DGM_PREC_TCBF16;
    const char* name = bf ? "TCBF16" : "TC16";
    TCDims d{};
    d.NE = T.NE;
    d.NH = T.NH;
    d.N2H = T.N2H;
    d.layout = 2;
    d.f16 = 1;
    d.bf16 = bf ? 1 : 0;
    d.VPC = 8;
    d.NEp = pad_to(T.NE, 16);
    d.NHp = pad_to(T.NH, 16);
    d.G8 = pad_to(T.N2H, 8);
    d.G = pad_to(T.N2H, 16);
    d.KE = d.KEo = 3 * d.NEp;
    d.KH = d.KHo = 3 * d.NHp;
    d.FB = 2 * d.G8;
    d.NT = 8 * d.G8;
    const TC2Smem LH = tc2_smem(d, true), LE = tc2_smem(d, false);
    if (P->p > 6 || LH.total > 227 * 1024 || LE.total > 227 * 1024 || 8 * d.G > 512 || 3 * d.NEp > 512) {
        set_error(std::string("precision ") + name + " supports p <= 6");
        return DGM_ERR_UNSUPPORTED;
    }
    if (P->opt.flux != DGM_FLUX_CENTRAL) {
        set_error(std::string("precision ") + name + " supports the central flux only");
        return DGM_ERR_UNSUPPORTED;
    }
    TCArgs& A = P->tca;
    for (int f = 0; f < 4; ++f)
        for (int i = 0; i < 2; ++i)
            for (int c = 0; c < 3; ++c) {
                const double v = T.that[f][i][c];
                if (v != 0.0 && v != 1.0 && v != -1.0) {
                    set_error("reference face tangent with an entry other than -1, 0, 1");
                    return DGM_ERR_UNSUPPORTED;
                }
                A.tsgn[f][i][c] = (int8_t)v;
            }
    const int64_t ntiles = (m.nt + kTcRows - 1) / kTcRows;
    const int64_t nrow = ntiles * kTcRows;
    // one allocation: fp32 state E, H; 2-byte operand copies; trace buffers; tables; float geometry
    const size_t bE = round_up((size_t)nrow * d.KE * 4, 1024), bH = round_up((size_t)nrow * d.KH * 4, 1024);
    const size_t bEo = round_up((size_t)nrow * d.KE * 2, 1024), bHo = round_up((size_t)nrow * d.KH * 2, 1024);
    const size_t bTr = round_up((size_t)nrow * d.NT * 2, 1024);
    const size_t nTabH = LH.tab / 2, nTabE = LE.tab / 2;   // values
    const size_t bTab = round_up((nTabH + nTabE) * 2, 1024);
    const size_t bGeo = (size_t)nrow * 16 * sizeof(float);
    const size_t o_E = 0, o_H = bE, o_Eo = o_H + bH, o_Ho = o_Eo + bEo, o_trE = o_Ho + bHo, o_trH = o_trE + bTr,
                 o_tab = o_trH + bTr, o_geo = o_tab + bTab;
    const size_t total = o_geo + bGeo;
    cudaError_t e;
    if ((e = cudaMalloc(&P->dTc, total)) != cudaSuccess) return cuda_err(e, "alloc");
    if ((e = cudaMemset(P->dTc, 0, o_tab)) != cudaSuccess) return cuda_err(e, "memset");
    uint8_t* base8 = static_cast<uint8_t*>(P->dTc);

    // tables (fp32 staging, rounded to the operand type on the device)
    std::vector<float> tab(nTabH + nTabE, 0.0f);
    const int NE = T.NE, NH = T.NH, N2H = T.N2H, G = d.G;
    for (int ph = 0; ph < 2; ++ph) {
        const bool is_h = ph == 0;
        const TC2Smem& L = is_h ? LH : LE;
        float* base = tab.data() + (is_h ? 0 : nTabH);
        const int npin = is_h ? d.NEp : d.NHp, npout = is_h ? d.NHp : d.NEp;
        const int nout = is_h ? NH : NE;
        // curl tables d = x, y, z: [npin/8][npout][8], row = output coefficient, k = input coefficient
        for (int dd = 0; dd < 3; ++dd) {
            float* tb = base + (size_t)dd * npin * npout;
            for (int b = 0; b < NH; ++b)
                for (int a = 0; a < NE; ++a) {
                    const float v = (float)T.D[dd][(size_t)b * NE + a];
                    const int row = is_h ? b : a, k = is_h ? a : b;
                    tb[((size_t)(k / 8) * npout + row) * 8 + (k % 8)] = v;
                }
        }
        // per face: lift [G/8][npout][8] (row = output coefficient, k = face mode) and
        // trace [npout/8][G][8] (row = face mode, k = coefficient), the same numbers
        float* lift = base + L.curl / 2;
        float* trace = base + (L.curl + L.lift) / 2;
        for (int f = 0; f < 4; ++f)
            for (int g = 0; g < N2H; ++g)
                for (int a = 0; a < nout; ++a) {
                    const double v = is_h ? T.TrH[f][(size_t)g * NH + a] : T.TrE[f][(size_t)T.pos2H[g] * NE + a];
                    float* lf = lift + (size_t)f * npout * G;
                    float* tf = trace + (size_t)f * G * npout;
                    lf[((size_t)(g / 8) * npout + a) * 8 + (g % 8)] = (float)v;
                    tf[((size_t)(a / 8) * G + g) * 8 + (a % 8)] = (float)v;
                }
    }
    uint8_t* dtab = base8 + o_tab;
    {
        float* stage32 = nullptr;
        if ((e = cudaMalloc(&stage32, tab.size() * sizeof(float))) != cudaSuccess) return cuda_err(e, "alloc tables");
        e = cudaMemcpy(stage32, tab.data(), tab.size() * sizeof(float), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) {
            const int r = bf ? tc_launch_to_bf16(stage32, dtab, tab.size(), 0)
                             : tc_launch_to_half(stage32, dtab, tab.size(), 0);
            if (r) e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        cudaFree(stage32);
        if (e != cudaSuccess) return cuda_err(e, "tables");
    }
    // geometry: double records (energy of the state) and the kernels' float records
    std::vector<double> g2((size_t)nrow * kGeoStride, 0.0);
    std::copy(geo.begin(), geo.end(), g2.begin());
    std::vector<float> gf((size_t)nrow * 16, 0.0f);
    for (int64_t t = 0; t < nrow; ++t) {
        double* r = &g2[(size_t)t * kGeoStride];
        if (t >= m.nt) {   // padding elements: identity metric, unit materials, PEC faces, zero fields
            r[0] = r[3] = r[5] = r[6] = r[9] = r[11] = 1.0;
            r[kGeoEps] = r[kGeoInvEps] = r[kGeoMu] = r[kGeoInvMu] = r[kGeoSign] = 1.0;
        }
        float* o = &gf[(size_t)t * 16];
        for (int q = 0; q < 12; ++q) o[q] = (float)r[q];
        o[12] = (float)r[kGeoEps];
        o[13] = (float)r[kGeoMu];
        o[14] = (float)r[kGeoSign];
    }
    std::vector<int32_t> n2((size_t)nrow * 4, -1);
    std::copy(nbr.begin(), nbr.end(), n2.begin());
    if ((e = cudaMalloc(&P->dTcGeo, g2.size() * sizeof(double))) != cudaSuccess) return cuda_err(e, "alloc geo");
    if ((e = cudaMalloc(&P->dTcNbr, n2.size() * sizeof(int32_t))) != cudaSuccess) return cuda_err(e, "alloc nbr");
    cudaMemcpy(P->dTcGeo, g2.data(), g2.size() * sizeof(double), cudaMemcpyHostToDevice);
    cudaMemcpy(P->dTcNbr, n2.data(), n2.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
    cudaMemcpy(base8 + o_geo, gf.data(), bGeo, cudaMemcpyHostToDevice);
    if ((e = cudaMalloc(&P->dErr, sizeof(int))) != cudaSuccess) return cuda_err(e, "alloc err");
    cudaMemset(P->dErr, 0, sizeof(int));

    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, P->ctx->device);
    P->tc_grid = (int)std::min<int64_t>(ntiles, (int64_t)sms);   // one CTA per SM
    P->tc_grid_cap = P->tc_grid;
    double* part = nullptr;
    if ((e = cudaMalloc(&part, 2 * (size_t)P->tc_grid_cap * sizeof(double))) != cudaSuccess)
        return cuda_err(e, "alloc partials");
    cudaMemset(part, 0, 2 * (size_t)P->tc_grid_cap * sizeof(double));

    A.nt = m.nt;
    A.ntiles = (int)ntiles;
    A.d = d;
    A.E = reinterpret_cast<float*>(base8 + o_E);
    A.H = reinterpret_cast<float*>(base8 + o_H);
    A.Eop = base8 + o_Eo;
    A.Hop = base8 + o_Ho;
    A.trE = base8 + o_trE;
    A.trH = base8 + o_trH;
    A.geo = P->dTcGeo;
    A.geoF = reinterpret_cast<const float*>(base8 + o_geo);
    A.nbr = P->dTcNbr;
    A.T2H = dtab;
    A.T2E = dtab + nTabH * 2;
    A.partE = part;
    A.partH = part + P->tc_grid;
    A.err = P->dErr;
    for (int f = 0; f < 4; ++f) A.sigma_hat[f] = (float)T.sigma_hat[f];
    P->tc = true;
    P->trE_valid = P->trH_valid = false;
    return DGM_OK;
}

}  // namespace

void tc_problem_free(dgm_problem* P) {
    void* ptrs[] = {P->dTc, P->dTcGeo, P->dTcNbr, P->dErr, P->tca.partE};
    for (void* q : ptrs)
        if (q) cudaFree(q);
}

int tc_import(dgm_problem* P, const double* dE, const double* dH, const double* nrmE, const double* nrmH,
              cudaStream_t s) {
    const TCArgs& A = P->tca;
    int r = 0;
    if (A.d.layout == 2) {
        if (dE) r |= tc2_launch_pack(dE, A.E, nrmE, A.nt, A.d.NE, A.d.NEp, s);
        if (dH) r |= tc2_launch_pack(dH, A.H, nrmH, A.nt, A.d.NH, A.d.NHp, s);
    } else {
        if (dE) r |= tc_launch_pack(dE, A.E, nrmE, A.nt, A.d.NE, A.d.KE, s);
        if (dH) r |= tc_launch_pack(dH, A.H, nrmH, A.nt, A.d.NH, A.d.KH, s);
    }
    if (dE) P->trE_valid = false;
    if (dH) P->trH_valid = false;
    return r ? cuda_err(cudaGetLastError(), "pack") : DGM_OK;
}

int tc_export(dgm_problem* P, double* dE, double* dH, const double* nrmE, const double* nrmH, cudaStream_t s) {
    const TCArgs& A = P->tca;
    int r = 0;
    if (A.d.layout == 2) {
        if (dE) r |= tc2_launch_unpack(A.E, dE, nrmE, A.nt, A.d.NE, A.d.NEp, s);
        if (dH) r |= tc2_launch_unpack(A.H, dH, nrmH, A.nt, A.d.NH, A.d.NHp, s);
    } else {
        if (dE) r |= tc_launch_unpack(A.E, dE, nrmE, A.nt, A.d.NE, A.d.KE, s);
        if (dH) r |= tc_launch_unpack(A.H, dH, nrmH, A.nt, A.d.NH, A.d.KH, s);
    }
    return r ? cuda_err(cudaGetLastError(), "unpack") : DGM_OK;
}

int tc_traces(dgm_problem* P, int which, cudaStream_t s) {
    if (tc_launch_traces(P->tca, P->tc_grid, which, s)) return cuda_err(cudaGetLastError(), "traces launch");
    (which == 0 ? P->trE_valid : P->trH_valid) = true;
    if (which == 0) P->trE_ndirty = 0;
    return DGM_OK;
}

void tc_mark_tile_dirty(dgm_problem* P, int64_t tile) {
    if (!P->trE_valid) return;   // a full refresh is pending anyway
    for (int i = 0; i < P->trE_ndirty; ++i)
        if (P->trE_dirty[i] == tile) return;
    if (P->trE_ndirty < dgm_problem::kMaxDirtyTiles)
        P->trE_dirty[P->trE_ndirty++] = (int)tile;
    else
        P->trE_valid = false;
}

int tc_ensure_traces_E(dgm_problem* P, bool energy, cudaStream_t s) {
    if (!P->trE_valid || (P->trE_ndirty > 0 && energy)) return tc_traces(P, 0, s);
    for (int i = 0; i < P->trE_ndirty; ++i)
        if (tc_launch_traces_tile(P->tca, 0, P->trE_dirty[i], s)) return cuda_err(cudaGetLastError(), "traces launch");
    P->trE_ndirty = 0;
    return DGM_OK;
}

TCArgs tc_launch_args(dgm_problem* P) {
    TCArgs a = P->tca;
    a.stall_test = 0;
    if (P->tc_stall_tests > 0) {
        a.stall_test = 1;
        --P->tc_stall_tests;
    }
    return a;
}

int tc_phase_H(dgm_problem* P, double dt, double a_lo, double c_out, double* energy_slot, cudaStream_t s) {
    {
        int rc = tc_ensure_traces_E(P, energy_slot != nullptr, s);
        if (rc) return rc;
    }
    if (tc_launch_phase_H(tc_launch_args(P), P->tc_grid, dt, a_lo, c_out, energy_slot ? 1 : 0, s))
        return cuda_err(cudaGetLastError(), "H-phase launch");
    P->trH_valid = true;
    if (energy_slot && launch_energy_reduce(P->tca.partE, 2 * P->tc_grid, energy_slot, s))
        return cuda_err(cudaGetLastError(), "energy reduce launch");
    return DGM_OK;
}

int tc_phase_E(dgm_problem* P, double dt, bool energy, cudaStream_t s) {
    if (!P->trH_valid) {
        int rc = tc_traces(P, 1, s);
        if (rc) return rc;
    }
    if (tc_launch_phase_E(tc_launch_args(P), P->tc_grid, dt, energy ? 1 : 0, s))
        return cuda_err(cudaGetLastError(), "E-phase launch");
    P->trE_valid = true;
    P->trE_ndirty = 0;
    return DGM_OK;
}

int tc_state_energy(dgm_problem* P, double* slot, cudaStream_t s) {
    if (tc_launch_state_energy(P->tca, P->tc_grid, s)) return cuda_err(cudaGetLastError(), "energy launch");
    if (launch_energy_reduce(P->tca.partE, 2 * P->tc_grid, slot, s))
        return cuda_err(cudaGetLastError(), "energy reduce launch");
    return DGM_OK;
}

int tc_check_error(dgm_problem* P) {
    int h = 0;
    cudaError_t e = cudaMemcpy(&h, P->dErr, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_err(e, "error word");
    if (h != 0) {
        set_error("tensor-core kernel gave up waiting (error word set); results are invalid");
        cudaMemset(P->dErr, 0, sizeof(int));
        return DGM_ERR_TIMEOUT;
    }
    return DGM_OK;
}

}  // namespace dgm
