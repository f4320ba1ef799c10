// Tensor-core (tcgen05) phase kernels: TF32 or FP16 operands, FP32 accumulation.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace dgm {

constexpr int kTcRows = 128;   // elements per tile = MMA M

// Dimensions of the tensor-core path for one p and operand type.  State
// values are fp32; operand values are fp32 (TF32, 4 per 16-byte chunk) or
// fp16 (8 per chunk).
struct TCDims {
    int NE, NH, N2H;
    int layout;      // 1: interleaved element rows (k = 3 a + m; TC32 kernels)
                     // 2: component-major element rows (k = m Np + a; the resident-table kernels)
    int f16;         // operands are 2-byte (fp16, or bf16 when bf16 = 1); else TF32
    int bf16;        // 2-byte operands are bf16 (8-bit mantissa, fp32 range)
    int NEp, NHp;    // layout 2: per-component padded lengths (multiples of 16)
    int G8, G;       // layout 2: face modes per tangent block, padded to 8 (trace buffer) and 16 (MMA)
    int split;       // layout 1, fp16: two-term tables (hi + lo), two MMAs per table K-step
    int VPC;         // operand values per 16-byte chunk: 4 (TF32) or 8 (fp16)
    int KE, KH;      // padded fp32 state row lengths (multiples of 24): E, H
    int KEo, KHo;    // padded operand row lengths (whole MMA K-steps of 2 VPC): E, H
    int FB;          // trace columns per face: 2 N2(p-1) padded to VPC
    int NT;          // face-trace columns 4 FB
    int NC;          // H-output columns (12 ceil(NH/4) padded to 16)
    int NCE;         // E-output columns (12 ceil(NE/4) padded to 16)
};

TCDims tc_dims(int NE, int NH, int N2H, bool f16, bool split = false);

struct TCArgs {
    int64_t nt;
    int ntiles;
    TCDims d;
    float* E;                  // fp32 state [ntiles][KE/4][128][4]
    float* H;                  // fp32 state [ntiles][KH/4][128][4]
    void* Eop;                 // MMA operand copy of E [ntiles][KEo/VPC][128][VPC] (TF32: E itself)
    void* Hop;                 // MMA operand copy of H (TF32: H itself)
    void* trE;                 // [ntiles*128][NT] tangential E traces (degree <= p-1 face modes),
                               // column f FB + i N2(p-1) + g, operand type
    void* trH;                 // [ntiles*128][NT]
    const double* geo;         // [ntiles*128][kGeoStride] (padding rows benign)
    const int32_t* nbr;        // [ntiles*128][4]
    const void* B1H;           // [KEo/VPC][NC][VPC]    curl
    const void* BliftH;        // [NT/VPC][NC][VPC]
    const void* BtrH;          // [KHo/VPC][NT][VPC]
    const void* B1E;           // [KHo/VPC][NCE][VPC]   curl^T
    const void* BliftE;        // [NT/VPC][NCE][VPC]
    const void* BtrE;          // [KEo/VPC][NT][VPC]
    double* partE;             // [grid] energy partials, E part
    double* partH;             // [grid] energy partials, H part
    int* err;                  // device error word (0 = ok)
    float sigma_hat[4];        // reference face orientation signs
    uint32_t stage_bytes;      // bytes of one ring stage
    uint32_t tmem_cols;        // TMEM columns allocated per CTA (power of two)
    uint32_t r2_offset;        // offset of the resident tile region
    int64_t tab_lo;            // two-term tables: byte offset from each hi table to its lo table
    int stall_test;            // nonzero: the phase kernel waits on a barrier nothing arrives at,
                               // gives up after a short limit, records a timeout and does no work
    // layout 2 (resident-table kernels)
    const float* geoF;         // [ntiles*128][16] floats: G^{-1} (6), G (6), eps, mu, sign det F, 0
    const void* T2H;           // H-phase tables: curl D_d (3), lift (4 faces), trace (4 faces)
    const void* T2E;           // E-phase tables: curl^T, lift, trace
    int8_t tsgn[4][2][3];      // reference face tangents t_{f,i} (entries -1, 0, 1)
};

// Byte sizes and shared-memory offsets of one layout-2 kernel instance.
struct TC2Smem {
    uint32_t curl, lift, trace;   // table bytes (curl: 3 tables; lift, trace: 4 faces each)
    uint32_t tab;                 // all tables of the phase
    uint32_t o_tab, o_sa, o_sf;   // offsets
    uint32_t sa, sf;              // operand tile region (input, then updated field), flux blocks
    uint32_t total;               // dynamic shared memory of the kernel
};
__host__ __device__ TC2Smem tc2_smem(const TCDims& d, bool is_h);
// TMEM columns of the accumulator (3 Np_out) and the first trace column of a phase
uint32_t tc2_tr0(const TCDims& d, bool is_h);
int tc2_launch_phase(const TCArgs& a, bool is_h, int grid, double dt, double a_lo, double c_out, int energy,
                     cudaStream_t s);
// refresh the 2-byte operand copy of a field from its fp32 state, then its traces;
// with energy (which = 0) also the energy partials of E; tiles [tile0, tile1)
int tc2_launch_traces(const TCArgs& a, int which, int grid, int tile0, int tile1, int energy, cudaStream_t s);
int tc2_launch_state_energy(const TCArgs& a, int grid, cudaStream_t s);
int tc2_launch_pack(const double* src, float* dst, const double* nrm, int64_t nt, int N, int Np, cudaStream_t s);
int tc2_launch_unpack(const float* src, double* dst, const double* nrm, int64_t nt, int N, int Np, cudaStream_t s);
int tc_launch_to_bf16(const float* src, void* dst, size_t n, cudaStream_t s);

size_t tc_smem_bytes(const TCDims& d, uint32_t* stage_bytes, uint32_t* r2_offset);
uint32_t tc_tmem_cols(const TCDims& d);
// one past the highest TMEM column any GEMM or epilogue of the phase kernels touches
uint32_t tc_tmem_reach(const TCDims& d);

int tc_launch_phase_H(const TCArgs& a, int grid, double dt, double a_lo, double c_out, int energy, cudaStream_t s);
int tc_launch_phase_E(const TCArgs& a, int grid, double dt, int energy, cudaStream_t s);
// traces (and, for E, the energy partials of E) of the current field: which = 0 E, 1 H;
// with fp16 operands the operand copy of the field is refreshed from the state first
int tc_launch_traces(const TCArgs& a, int grid, int which, cudaStream_t s);
// the same for one tile, without energy partials (one CTA)
int tc_launch_traces_tile(const TCArgs& a, int which, int tile, cudaStream_t s);
// energy partials of the state (no staggering)
int tc_launch_state_energy(const TCArgs& a, int grid, cudaStream_t s);
// canonical (or orthonormal) [t][3][N] doubles <-> tiled floats, scaled by nrm[a] (import) / 1/nrm[a] (export)
int tc_launch_pack(const double* src, float* dst, const double* nrm, int64_t nt, int N, int K, cudaStream_t s);
int tc_launch_unpack(const float* src, double* dst, const double* nrm, int64_t nt, int N, int K, cudaStream_t s);
// fp32 -> fp16, round to nearest even (tables of the fp16 operand path)
int tc_launch_to_half(const float* src, void* dst, size_t n, cudaStream_t s);
// fp32 -> two fp16 terms: hi = fp16(x), lo = fp16(x - hi), both round to nearest even
int tc_launch_split_half(const float* src, void* hi, void* lo, size_t n, cudaStream_t s);

}  // namespace dgm
