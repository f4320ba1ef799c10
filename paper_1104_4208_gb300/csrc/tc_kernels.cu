// Tensor-core phase kernels of the DG Maxwell time step (sm_103a, tcgen05).
//
// The same operator as kernels.cu (Sec. 2.1 fluxes, Sec. 3.2 reference curl
// and traces, Sec. 3.3.1 block inverse mass, Sec. 3 symplectic Euler), but
// every dense reference operator is applied to a tile of 128 elements at once
// as a GEMM on the 5th-generation tensor cores:
//
//   H-phase (tile of E, H):
//     GEMM1  D = E * Curl^T                                (K = 3 N3(p))
//     flux   a~ = -sigma_hat (J - J_nbr)/2   (PEC: -sigma_hat J), J and
//            J_nbr from the trace buffer the previous E-phase wrote
//     GEMM2  D += a~ * LiftH^T                             (K = 8 N2(p-1))
//     update H += dt/mu G^{-1} (-s_T D), energy partial
//     GEMM3  D = H_new * TrH^T -> H trace buffer (for the E-phase)
//   E-phase: the transposed operators with {{H}}, the same rounded numbers, so
//   the discrete operator stays exactly skew.
//
// Two operand types share the code (template parameter OP): TF32 (the fp32
// state itself is the operand; the multiplier uses 10 mantissa bits, K = 8
// per MMA) and FP16 (an fp16 copy of each field, written by the update
// epilogue next to the fp32 state, fp16 tables and trace buffers; K = 16 per
// MMA, so a ring slot of the same bytes carries twice the K range).  The
// state, the update and the energy stay fp32 in both.  The accumulators are
// FP32 in tensor memory (TMEM), one thread per element in the epilogues
// (element = TMEM lane).  State tiles and reference tables are
// stored in global memory in the MMA's shared-memory layout, so each K slice
// arrives with one bulk asynchronous copy into a 4-stage ring; one thread
// issues copies and MMAs, mbarriers track both.  Every wait is bounded: on
// timeout the kernel records an error code, lets its copies drain, frees its
// tensor memory and returns.

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "kernels.h"
#include "tc_kernels.h"
#include "tc_ptx.h"

namespace dgm {

namespace {

constexpr int kStages = 4;
constexpr uint32_t kHead = 256;             // control block at the start of shared memory
constexpr long long kLimit = 4000000000LL;  // cycles before a wait gives up (~2 s)
constexpr long long kDrain = 200000000LL;
constexpr long long kStallTestLimit = 2000000LL;   // ~1 ms: the injected wait's limit
constexpr int kErrTimeout = 1;

int padto(int x, int m) { return (x + m - 1) / m * m; }

// Operand types: values per 16-byte chunk, the MMA, and chunk <-> floats.
struct OpTf32 {
    using T = float;
    static constexpr int VPC = 4;
    static constexpr int MAXC = 11;   // 16-byte chunks of a face block for p <= 6 (FB = 44)
    static __device__ __forceinline__ void unpack(const uint4& c, float* v) {
        v[0] = __uint_as_float(c.x);
        v[1] = __uint_as_float(c.y);
        v[2] = __uint_as_float(c.z);
        v[3] = __uint_as_float(c.w);
    }
    static __device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, int n, uint32_t acc) {
        tc::mma_tf32(d, a, b, tc::idesc_tf32(kTcRows, n), acc);
    }
    static __device__ __forceinline__ uint4 pack(const float* v) {
        return make_uint4(__float_as_uint(v[0]), __float_as_uint(v[1]), __float_as_uint(v[2]), __float_as_uint(v[3]));
    }
};

struct OpF16 {
    using T = __half;
    static constexpr int VPC = 8;
    static constexpr int MAXC = 6;    // FB = 48
    static __device__ __forceinline__ void unpack(const uint4& c, float* v) {
        const uint32_t w[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            __half2 h;
            memcpy(&h, &w[i], 4);
            const float2 f = __half22float2(h);
            v[2 * i] = f.x;
            v[2 * i + 1] = f.y;
        }
    }
    static __device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, int n, uint32_t acc) {
        tc::mma_f16(d, a, b, tc::idesc_f16(kTcRows, n), acc);
    }
    static __device__ __forceinline__ uint4 pack(const float* v) {
        uint32_t w[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const __half2 h = __floats2half2_rn(v[2 * i], v[2 * i + 1]);
            memcpy(&w[i], &h, 4);
        }
        return make_uint4(w[0], w[1], w[2], w[3]);
    }
};

struct Ctl {
    uint64_t full[kStages];
    uint64_t empty[kStages];
    uint64_t done;
    uint64_t load;
    uint32_t tmem;
    volatile int abort;
};

struct GemmDesc {
    const uint8_t* gA;   // A K-slices in global memory (tile base) or nullptr: A resident in shared memory
    uint32_t sA;         // shared address of the resident A tile
    const uint8_t* gB;   // B K-slices in global memory, [K/VPC][brows][VPC]
    int brows;
    int nk;            // number of MMA K-steps (32 bytes of every row each)
    int nmma;          // MMAs per K step (B row ranges)
    int row0[3];
    int n[3];
    uint32_t dcol[3];
    int acc_first;     // accumulate onto D from the first step
    int64_t lo_off;    // two-term tables: byte offset of B's lo term (0: one term)
};

// Producer + MMA issuer (thread 0).  g counts ring uses across GEMMs.  A
// K-step is 32 bytes of every row of A (4 KB) and of B, whatever the type.
template <typename OP>
__device__ bool ring_gemm(Ctl* ctl, uint8_t* ring, uint32_t stage_bytes, uint32_t& g, const GemmDesc& G,
                          uint32_t tmem) {
    const uint32_t a_bytes = G.gA ? (uint32_t)(kTcRows * 32) : 0u;
    const uint32_t b_bytes = (uint32_t)G.brows * 32u;
    const uint32_t lo_bytes = G.lo_off ? b_bytes : 0u;   // the lo slice follows the hi slice
    int produced = 0, consumed = 0;
    bool ok = true;
    auto produce = [&](int c) -> bool {
        const uint32_t gg = g + (uint32_t)c;
        const int st = (int)(gg % kStages);
        const uint32_t use = gg / kStages;
        if (use > 0 && !tc::mbar_wait(&ctl->empty[st], (use - 1) & 1u, kLimit)) return false;
        uint8_t* sp = ring + (size_t)st * stage_bytes;
        tc::mbar_expect_tx(&ctl->full[st], a_bytes + b_bytes + lo_bytes);
        if (G.gA) tc::bulk_g2s(sp, G.gA + (size_t)c * kTcRows * 32, a_bytes, &ctl->full[st]);
        tc::bulk_g2s(sp + a_bytes, G.gB + (size_t)c * G.brows * 32, b_bytes, &ctl->full[st]);
        if (lo_bytes)
            tc::bulk_g2s(sp + a_bytes + b_bytes, G.gB + G.lo_off + (size_t)c * G.brows * 32, lo_bytes, &ctl->full[st]);
        ++produced;
        return true;
    };
    auto consume = [&](int c) -> bool {
        const uint32_t gg = g + (uint32_t)c;
        const int st = (int)(gg % kStages);
        const uint32_t use = gg / kStages;
        if (!tc::mbar_wait(&ctl->full[st], use & 1u, kLimit)) return false;
        uint8_t* sp = ring + (size_t)st * stage_bytes;
        const uint32_t aaddr = G.gA ? tc::smem_u32(sp) : G.sA + (uint32_t)c * 2u * kTcRows * 16u;
        const uint64_t ad = tc::sdesc(aaddr, kTcRows * 16u, 128u);
        const uint32_t baddr = tc::smem_u32(sp + a_bytes);
        for (int j = 0; j < G.nmma; ++j) {
            const uint64_t bd = tc::sdesc(baddr + (uint32_t)G.row0[j] * 16u, (uint32_t)G.brows * 16u, 128u);
            OP::mma(tmem + G.dcol[j], ad, bd, G.n[j], (c > 0 || G.acc_first) ? 1u : 0u);
            if (lo_bytes) {   // the table's lo term into the same accumulator
                const uint64_t bl = tc::sdesc(baddr + b_bytes + (uint32_t)G.row0[j] * 16u, (uint32_t)G.brows * 16u, 128u);
                OP::mma(tmem + G.dcol[j], ad, bl, G.n[j], 1u);
            }
        }
        tc::mma_commit(&ctl->empty[st]);
        ++consumed;
        return true;
    };
    tc::tc_fence_after();
    const int pre = G.nk < kStages ? G.nk : kStages;
    for (int c = 0; c < pre && ok; ++c) ok = produce(c);
    for (int c = 0; c < G.nk && ok; ++c) {
        ok = consume(c);
        const int p = c - 1 + kStages;
        if (ok && c >= 1 && p < G.nk) ok = produce(p);
    }
    if (!ok) {
        // let the copies already issued land before the shared memory is given up
        for (int c = consumed; c < produced; ++c) {
            const uint32_t gg = g + (uint32_t)c;
            tc::mbar_wait(&ctl->full[gg % kStages], (gg / kStages) & 1u, kDrain);
        }
    }
    tc::mma_commit(&ctl->done);
    g += (uint32_t)G.nk;
    return ok;
}

__device__ void record_error(int* err) { atomicCAS(err, 0, kErrTimeout); }

// all threads: wait for the GEMM's completion; false on timeout
__device__ bool wait_done(Ctl* ctl, uint32_t& done_cnt) {
    const bool ok = tc::mbar_wait(&ctl->done, done_cnt & 1u, kLimit);
    ++done_cnt;
    tc::tc_fence_after();
    return ok;
}

__device__ void setup(Ctl* ctl, int warp, uint32_t tmem_cols) {
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            tc::mbar_init(&ctl->full[s], 1);
            tc::mbar_init(&ctl->empty[s], 1);
        }
        tc::mbar_init(&ctl->done, 1);
        tc::mbar_init(&ctl->load, 1);
        ctl->abort = 0;
        tc::fence_mbar_init();
        tc::fence_proxy_async();
    }
    if (warp == 0) {
        tc::tmem_alloc(&ctl->tmem, tmem_cols);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
}

__device__ void teardown(Ctl* ctl, int warp, uint32_t tmem_cols) {
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    if (warp == 0) tc::tmem_dealloc(ctl->tmem, tmem_cols);
}

// make shared-memory writes of the epilogue visible to the tensor cores and
// hand TMEM back to the MMA issuer
__device__ void epilogue_barrier() {
    tc::fence_proxy_async();
    tc::tc_fence_before();
    __syncthreads();
}

__device__ void block_sum_store(double v, double* out) {
    __shared__ double red[4];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) out[blockIdx.x] = ((red[0] + red[1]) + red[2]) + red[3];
}

// flux of a tile's faces [f0, f0+2) into the resident region: thread =
// element; the element's own trace block and its neighbour's (FB values each,
// 16-B aligned, written by the previous phase in the operand type) are loaded
// with 16-byte loads issued together.  Jump (H-phase, avg = false) or average
// (E-phase) formed in fp32 and rounded to the operand type; PEC faces use the
// ghost state.  A2 column = (f - f0) FB + r.
template <typename OP>
__device__ void epi_flux(const TCArgs& A, int f0, const typename OP::T* tr, int64_t t, bool avg,
                         typename OP::T* a2) {
    constexpr int V = OP::VPC, kMaxFaceChunks = OP::MAXC;
    const TCDims& d = A.d;
    const int tid = threadIdx.x;
    const int FB = d.FB, nvalid = 2 * d.N2H, nchunk = FB / V;
    const int4 nb4 = *reinterpret_cast<const int4*>(A.nbr + t * 4);
    const int32_t nbf[4] = {nb4.x, nb4.y, nb4.z, nb4.w};
    uint4* A2 = reinterpret_cast<uint4*>(a2);
#pragma unroll 1
    for (int f = f0; f < f0 + 2; ++f) {
        const int32_t nb = nbf[f];
        const float sh = A.sigma_hat[f];
        const uint4* own = reinterpret_cast<const uint4*>(tr + (size_t)t * d.NT + f * FB);
        const uint4* src = reinterpret_cast<const uint4*>(tr + (size_t)(nb >= 0 ? nb >> 2 : t) * d.NT +
                                                          (nb >= 0 ? (nb & 3) : f) * FB);
        uint4 ov[kMaxFaceChunks], nv[kMaxFaceChunks];
#pragma unroll
        for (int c = 0; c < kMaxFaceChunks; ++c)
            if (c < nchunk) {
                ov[c] = own[c];
                nv[c] = src[c];
            }
#pragma unroll
        for (int c = 0; c < kMaxFaceChunks; ++c) {
            if (c >= nchunk) break;
            float v[V], n4[V], o[V];
            OP::unpack(ov[c], v);
            OP::unpack(nv[c], n4);
#pragma unroll
            for (int q = 0; q < V; ++q) {
                const int r = V * c + q;
                if (r >= nvalid) {
                    o[q] = 0.f;
                } else if (nb >= 0) {
                    o[q] = avg ? sh * 0.5f * (v[q] + n4[q]) : -sh * 0.5f * (v[q] - n4[q]);
                } else {
                    o[q] = avg ? sh * v[q] : -sh * v[q];
                }
            }
            A2[(size_t)((f - f0) * nchunk + c) * kTcRows + tid] = OP::pack(o);
        }
    }
}

// trace columns of D -> trace buffer row of element t (operand type)
template <typename OP>
__device__ void epi_traces(const TCArgs& A, uint32_t lane_tmem, typename OP::T* tr, int64_t t) {
    constexpr int V = OP::VPC;
    const int NT = A.d.NT;
    uint4* row = reinterpret_cast<uint4*>(tr + (size_t)t * NT);
    for (int j0 = 0; j0 < NT; j0 += 16) {
        float v[16];
        tc::tmem_ld16(lane_tmem + (uint32_t)j0, v);
#pragma unroll
        for (int q = 0; q < 16 / V; ++q) row[j0 / V + q] = OP::pack(v + V * q);
    }
}

// The update epilogue: per batch of up to 16 coefficients (48 values) the old
// fp32 field values are loaded first (12 float4, one per 4 values), then the
// accumulator columns; `op` applies the per-coefficient update (and energy
// partial); the new values are stored back to the tiled fp32 field in HBM and,
// with fp16 operands, to the fp16 operand copy of row length Kop (8 values per
// 16-byte chunk; values past the batch in its last chunk are padding, stored
// as 0; a batch of whole 4-coefficient groups may reach past Kop, those values
// are padding too and are not stored).
template <typename OP, typename Op>
__device__ void epi_update(uint32_t lane_tmem, float* field_tile, typename OP::T* op_tile, int N, int Kop, Op op) {
    const int tid = threadIdx.x;
    float4* F4 = reinterpret_cast<float4*>(field_tile);
    const int ngroups = (N + 3) / 4;
#pragma unroll 1
    for (int g0 = 0; g0 < ngroups; g0 += 4) {
        const int nq = 3 * min(4, ngroups - g0);
        // 16-column loads covering the batch's 4 nq columns only: the last one
        // ends at the padded output width (a multiple of 16), never past the
        // CTA's TMEM allocation
        const int nld = (4 * nq + 15) / 16;
        float4 hv[12];
#pragma unroll
        for (int q = 0; q < 12; ++q)
            if (q < nq) hv[q] = F4[(size_t)(3 * g0 + q) * kTcRows + tid];
        float dd[48];
#pragma unroll
        for (int s = 0; s < 3; ++s)
            if (s < nld) tc::tmem_ld16(lane_tmem + (uint32_t)(12 * g0 + 16 * s), dd + 16 * s);
        float* h = reinterpret_cast<float*>(hv);
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            if (c >= 4 * (nq / 3)) break;
            if (4 * g0 + c >= N) break;
            op(h + 3 * c, dd + 3 * c);
        }
#pragma unroll
        for (int q = 0; q < 12; ++q)
            if (q < nq) F4[(size_t)(3 * g0 + q) * kTcRows + tid] = hv[q];
        if constexpr (OP::VPC == 8) {
            // values [12 g0, 12 g0 + 4 nq) -> fp16 chunks from 12 g0 / 8 on
            uint4* O = reinterpret_cast<uint4*>(op_tile);
            const int nval = min(4 * nq, Kop - 12 * g0), nch = (nval + 7) / 8, ch0 = 3 * g0 / 2;
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                if (i >= nch) break;
                float w[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) w[q] = 8 * i + q < nval ? h[8 * i + q] : 0.f;
                O[(size_t)(ch0 + i) * kTcRows + tid] = OP::pack(w);
            }
        }
    }
}

// split an output range of up to 2 x 256 columns into MMAs (N <= 256)
__device__ void add_mmas(GemmDesc& G, int row0, int n, uint32_t dcol) {
    while (n > 0) {
        const int m = n > 256 ? 256 : n;
        G.row0[G.nmma] = row0;
        G.n[G.nmma] = m;
        G.dcol[G.nmma] = dcol;
        ++G.nmma;
        row0 += m;
        dcol += (uint32_t)m;
        n -= m;
    }
}

// make this thread's generic-proxy global stores visible to later bulk copies
__device__ __forceinline__ void fence_global_async() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

// One phase on every tile: IS_H = H-phase (update H from E), else E-phase.
//   GEMM1  D = in * Curl^T                 (in = E for the H-phase, H for the E-phase)
//   2 x    flux of two faces -> A2,  D += A2 * Lift^T
//   update out (= H or E) in HBM, FP32 energy partial
//   GEMM3  D = out_new * Tr^T  (A streamed back from L2) -> trace buffer of `out`
template <bool IS_H, typename OP>
__global__ void __launch_bounds__(128, 2) k_tc_phase(TCArgs A, double dt, double a_lo, double c_out, int energy) {
    using T = typename OP::T;
    extern __shared__ __align__(1024) uint8_t smem[];
    Ctl* ctl = reinterpret_cast<Ctl*>(smem);
    uint8_t* ring = smem + kHead;
    T* r2 = reinterpret_cast<T*>(smem + A.r2_offset);
    const int tid = threadIdx.x, warp = tid >> 5;
    const TCDims d = A.d;
    const int Kin = IS_H ? d.KEo : d.KHo;    // operand row length of the input field
    const int Kout = IS_H ? d.KH : d.KE;     // fp32 row length of the output field
    const int Kop = IS_H ? d.KHo : d.KEo;    // operand row length of the output field
    const int Nout = IS_H ? d.NC : d.NCE, Nfield = IS_H ? d.NH : d.NE;
    const uint8_t* in = static_cast<const uint8_t*>(IS_H ? A.Eop : A.Hop);
    float* out = IS_H ? A.H : A.E;
    T* out_op = static_cast<T*>(IS_H ? A.Hop : A.Eop);   // TF32: the fp32 field itself
    const T* tr_in = static_cast<const T*>(IS_H ? A.trE : A.trH);
    T* tr_out = static_cast<T*>(IS_H ? A.trH : A.trE);
    const uint8_t* Bc = static_cast<const uint8_t*>(IS_H ? A.B1H : A.B1E);
    const uint8_t* Bl = static_cast<const uint8_t*>(IS_H ? A.BliftH : A.BliftE);
    const uint8_t* Bt = static_cast<const uint8_t*>(IS_H ? A.BtrH : A.BtrE);
    double* part = IS_H ? A.partH : A.partE;
    setup(ctl, warp, A.tmem_cols);
    const uint32_t tmem = ctl->tmem;
    const uint32_t lane_tmem = tmem + ((uint32_t)(warp * 32) << 16);
    uint32_t g = 0, done_cnt = 0;
    double eacc = 0.0;
    const int half_steps = d.FB / OP::VPC;   // MMA K-steps of two faces (2 FB values)
    if (A.stall_test) {
        // failure injection: wait on the `load` barrier, which nothing arrives
        // at, until the limit runs out -- before any copy or MMA is issued, so
        // nothing is in flight when the kernel gives up
        if (tid == 0 && !tc::mbar_wait(&ctl->load, 0u, kStallTestLimit)) ctl->abort = 1;
        __syncthreads();
    }
    for (int tile = blockIdx.x; tile < A.ntiles && !ctl->abort; tile += gridDim.x) {
        const int64_t t = (int64_t)tile * kTcRows + tid;
        // GEMM1: curl (H-phase) or curl^T (E-phase) of the input field
        if (tid == 0) {
            GemmDesc G{};
            G.gA = in + (size_t)tile * Kin * kTcRows * sizeof(T);
            G.gB = Bc;
            G.lo_off = A.tab_lo;
            G.brows = Nout;
            G.nk = Kin / (2 * OP::VPC);
            add_mmas(G, 0, Nout, 0);
            if (!ring_gemm<OP>(ctl, ring, A.stage_bytes, g, G, tmem)) ctl->abort = 1;
        }
        if (!wait_done(ctl, done_cnt)) ctl->abort = 1;
        __syncthreads();
        if (ctl->abort) break;
        // flux and lift, two faces at a time
        for (int h = 0; h < 2; ++h) {
            epi_flux<OP>(A, 2 * h, tr_in, t, !IS_H, r2);
            epilogue_barrier();
            if (tid == 0) {
                GemmDesc G{};
                G.sA = tc::smem_u32(r2);
                G.gB = Bl + (size_t)h * half_steps * Nout * 32;
                G.lo_off = A.tab_lo;
                G.brows = Nout;
                G.nk = half_steps;
                G.acc_first = 1;
                add_mmas(G, 0, Nout, 0);
                if (!ring_gemm<OP>(ctl, ring, A.stage_bytes, g, G, tmem)) ctl->abort = 1;
            }
            if (!wait_done(ctl, done_cnt)) ctl->abort = 1;
            __syncthreads();
            if (ctl->abort) break;
        }
        if (ctl->abort) break;
        // update of the output field
        {
            const double* gg = A.geo + t * kGeoStride;
            const float gi0 = (float)gg[0], gi1 = (float)gg[1], gi2 = (float)gg[2], gi3 = (float)gg[3],
                        gi4 = (float)gg[4], gi5 = (float)gg[5];
            const float G0 = (float)gg[6], G1 = (float)gg[7], G2 = (float)gg[8], G3 = (float)gg[9],
                        G4 = (float)gg[10], G5 = (float)gg[11];
            const double mat = IS_H ? gg[kGeoMu] : gg[kGeoEps];
            const float sT = IS_H ? -(float)gg[kGeoSign] : (float)gg[kGeoSign];   // r = -s_T D (H), s_T D (E)
            const float s = (float)(dt * (IS_H ? gg[kGeoInvMu] : gg[kGeoInvEps]));
            const float co = (float)c_out, alo = (float)a_lo;
            float eloc = 0.f;
            epi_update<OP>(lane_tmem, out + (size_t)tile * Kout * kTcRows, out_op + (size_t)tile * Kop * kTcRows, Nfield, Kop,
                       [&](float* h, const float* dd) {
                           const float r0 = sT * dd[0], r1 = sT * dd[1], r2v = sT * dd[2];
                           const float d0 = s * (gi0 * r0 + gi1 * r1 + gi2 * r2v);
                           const float d1 = s * (gi1 * r0 + gi3 * r1 + gi4 * r2v);
                           const float d2 = s * (gi2 * r0 + gi4 * r1 + gi5 * r2v);
                           if (IS_H) {
                               // staggered pair (H_lo, H_hi) of the modified energy
                               if (energy) {
                                   const float l0 = h[0] - alo * d0, l1 = h[1] - alo * d1, l2 = h[2] - alo * d2;
                                   const float u0 = l0 + d0, u1 = l1 + d1, u2 = l2 + d2;
                                   eloc += l0 * (G0 * u0 + G1 * u1 + G2 * u2) + l1 * (G1 * u0 + G3 * u1 + G4 * u2) +
                                           l2 * (G2 * u0 + G4 * u1 + G5 * u2);
                               }
                               h[0] += co * d0;
                               h[1] += co * d1;
                               h[2] += co * d2;
                           } else {
                               h[0] += d0;
                               h[1] += d1;
                               h[2] += d2;
                               if (energy) {
                                   const float x0 = h[0], x1 = h[1], x2 = h[2];
                                   eloc += x0 * (G0 * x0 + G1 * x1 + G2 * x2) + x1 * (G1 * x0 + G3 * x1 + G4 * x2) +
                                           x2 * (G2 * x0 + G4 * x1 + G5 * x2);
                               }
                           }
                       });
            eacc += 0.5 * mat * (double)eloc;
        }
        fence_global_async();
        epilogue_barrier();
        // GEMM3: traces of the updated field for the other phase (A read back from L2)
        if (tid == 0) {
            GemmDesc G{};
            G.gA = reinterpret_cast<const uint8_t*>(out_op + (size_t)tile * Kop * kTcRows);
            G.gB = Bt;
            G.lo_off = A.tab_lo;
            G.brows = d.NT;
            G.nk = Kop / (2 * OP::VPC);
            add_mmas(G, 0, d.NT, 0);
            if (!ring_gemm<OP>(ctl, ring, A.stage_bytes, g, G, tmem)) ctl->abort = 1;
        }
        if (!wait_done(ctl, done_cnt)) ctl->abort = 1;
        __syncthreads();
        if (ctl->abort) break;
        epi_traces<OP>(A, lane_tmem, tr_out, t);
        epilogue_barrier();
    }
    if (ctl->abort && tid == 0) record_error(A.err);
    if (energy) block_sum_store(eacc, part);
    teardown(ctl, warp, A.tmem_cols);
}

// traces of E (which = 0; with `energy` also the energy partials of E) or H
// (which = 1) on tiles [tile0, tile1).
// With fp16 operands each thread first rewrites its element's fp16 copy of
// the field from the fp32 state (the state may have been changed from
// outside: import, sources, checkpoints); the copy then feeds the GEMM.
template <typename OP>
__global__ void __launch_bounds__(128, 2) k_tc_traces(TCArgs A, int which, int tile0, int tile1, int energy) {
    using T = typename OP::T;
    extern __shared__ __align__(1024) uint8_t smem[];
    Ctl* ctl = reinterpret_cast<Ctl*>(smem);
    uint8_t* ring = smem + kHead;
    const int tid = threadIdx.x, warp = tid >> 5;
    const TCDims d = A.d;
    setup(ctl, warp, A.tmem_cols);
    const uint32_t tmem = ctl->tmem;
    const uint32_t lane_tmem = tmem + ((uint32_t)(warp * 32) << 16);
    uint32_t g = 0, done_cnt = 0;
    const int K = which == 0 ? d.KE : d.KH, Ko = which == 0 ? d.KEo : d.KHo;
    const float* field = which == 0 ? A.E : A.H;
    T* field_op = static_cast<T*>(which == 0 ? A.Eop : A.Hop);
    double eacc = 0.0;
    for (int tile = tile0 + (int)blockIdx.x; tile < tile1; tile += gridDim.x) {
        const int64_t t = (int64_t)tile * kTcRows + tid;
        const float* ft = field + (size_t)tile * K * kTcRows;
        T* fo = field_op + (size_t)tile * Ko * kTcRows;
        if constexpr (OP::VPC == 8) {
            uint4* O = reinterpret_cast<uint4*>(fo);
            for (int q = 0; q < Ko / 8; ++q) {
                float w[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int k = 8 * q + i;
                    w[i] = k < K ? ft[((size_t)(k >> 2) * kTcRows + tid) * 4 + (k & 3)] : 0.f;
                }
                O[(size_t)q * kTcRows + tid] = OP::pack(w);
            }
            fence_global_async();
            __syncthreads();
        }
        if (tid == 0) {
            GemmDesc G{};
            G.gA = reinterpret_cast<const uint8_t*>(fo);
            G.gB = static_cast<const uint8_t*>(which == 0 ? A.BtrE : A.BtrH);
            G.lo_off = A.tab_lo;
            G.brows = d.NT;
            G.nk = Ko / (2 * OP::VPC);
            add_mmas(G, 0, d.NT, 0);
            if (!ring_gemm<OP>(ctl, ring, A.stage_bytes, g, G, tmem)) ctl->abort = 1;
        }
        if (which == 0 && energy) {
            const double* gg = A.geo + t * kGeoStride;
            const double G0 = gg[6], G1 = gg[7], G2 = gg[8], G3 = gg[9], G4 = gg[10], G5 = gg[11];
            for (int a = 0; a < d.NE; ++a) {
                double x[3];
                for (int m = 0; m < 3; ++m) {
                    const int k = 3 * a + m;
                    x[m] = ft[((size_t)(k >> 2) * kTcRows + tid) * 4 + (k & 3)];
                }
                eacc += 0.5 * gg[kGeoEps] *
                        (x[0] * (G0 * x[0] + G1 * x[1] + G2 * x[2]) + x[1] * (G1 * x[0] + G3 * x[1] + G4 * x[2]) +
                         x[2] * (G2 * x[0] + G4 * x[1] + G5 * x[2]));
            }
        }
        if (!wait_done(ctl, done_cnt)) ctl->abort = 1;
        __syncthreads();
        if (ctl->abort) break;
        epi_traces<OP>(A, lane_tmem, static_cast<T*>(which == 0 ? A.trE : A.trH), t);
        epilogue_barrier();
    }
    if (ctl->abort && tid == 0) record_error(A.err);
    if (which == 0 && energy) block_sum_store(eacc, A.partE);
    teardown(ctl, warp, A.tmem_cols);
}

// 1/2 (eps E, E) and 1/2 (mu H, H) partials of the tiled state
__global__ void k_tc_state_energy(TCArgs A) {
    const TCDims d = A.d;
    double eE = 0.0, eH = 0.0;
    const int64_t n = (int64_t)A.ntiles * kTcRows;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const double* gg = A.geo + t * kGeoStride;
        const double G0 = gg[6], G1 = gg[7], G2 = gg[8], G3 = gg[9], G4 = gg[10], G5 = gg[11];
        const int64_t tile = t / kTcRows, e = t % kTcRows;
        for (int which = 0; which < 2; ++which) {
            const int N = which == 0 ? d.NE : d.NH, K = which == 0 ? d.KE : d.KH;
            const float* base = (which == 0 ? A.E : A.H) + (size_t)tile * (K / 4) * kTcRows * 4;
            const double c = which == 0 ? gg[kGeoEps] : gg[kGeoMu];
            double acc = 0.0;
            for (int a = 0; a < N; ++a) {
                double x[3];
                for (int m = 0; m < 3; ++m) {
                    const int k = 3 * a + m;
                    x[m] = base[((size_t)(k >> 2) * kTcRows + e) * 4 + (k & 3)];
                }
                acc += x[0] * (G0 * x[0] + G1 * x[1] + G2 * x[2]) + x[1] * (G1 * x[0] + G3 * x[1] + G4 * x[2]) +
                       x[2] * (G2 * x[0] + G4 * x[1] + G5 * x[2]);
            }
            (which == 0 ? eE : eH) += 0.5 * c * acc;
        }
    }
    __shared__ double red[2][8];
    for (int o = 16; o > 0; o >>= 1) {
        eE += __shfl_down_sync(0xffffffffu, eE, o);
        eH += __shfl_down_sync(0xffffffffu, eH, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = eE;
        red[1][threadIdx.x >> 5] = eH;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a += red[0][w];
            b += red[1][w];
        }
        A.partE[blockIdx.x] = a;
        A.partH[blockIdx.x] = b;
    }
}

__global__ void k_tc_pack(const double* __restrict__ src, float* __restrict__ dst, const double* __restrict__ nrm,
                          int64_t nt, int N, int K) {
    const int64_t n = nt * 3 * N;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = i / (3 * N);
        const int rem = (int)(i - t * 3 * N);
        const int m = rem / N, a = rem - m * N;
        const int k = 3 * a + m;
        const double sc = nrm ? nrm[a] : 1.0;
        dst[(((t / kTcRows) * (K / 4) + (k >> 2)) * kTcRows + (t % kTcRows)) * 4 + (k & 3)] = (float)(src[i] * sc);
    }
}

__global__ void k_tc_unpack(const float* __restrict__ src, double* __restrict__ dst, const double* __restrict__ nrm,
                            int64_t nt, int N, int K) {
    const int64_t n = nt * 3 * N;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = i / (3 * N);
        const int rem = (int)(i - t * 3 * N);
        const int m = rem / N, a = rem - m * N;
        const int k = 3 * a + m;
        const double sc = nrm ? nrm[a] : 1.0;
        dst[i] = (double)src[(((t / kTcRows) * (K / 4) + (k >> 2)) * kTcRows + (t % kTcRows)) * 4 + (k & 3)] / sc;
    }
}

__global__ void k_split_half(const float* __restrict__ src, __half* __restrict__ hi, __half* __restrict__ lo, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const __half h = __float2half_rn(src[i]);
        hi[i] = h;
        lo[i] = __float2half_rn(src[i] - __half2float(h));
    }
}

__global__ void k_to_half(const float* __restrict__ src, __half* __restrict__ dst, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = __float2half_rn(src[i]);
}

int set_smem(const void* fn, size_t bytes) {
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) == cudaSuccess ? 0 : -1;
}

size_t smem_of(const TCArgs& a) {
    uint32_t sb, r2;
    return tc_smem_bytes(a.d, &sb, &r2);
}

}  // namespace

TCDims tc_dims(int NE, int NH, int N2H, bool f16, bool split) {
    TCDims d;
    d.NE = NE;
    d.NH = NH;
    d.N2H = N2H;
    d.layout = 1;
    d.f16 = f16 ? 1 : 0;
    d.bf16 = 0;
    d.NEp = d.NHp = d.G8 = d.G = 0;
    d.split = split && f16 ? 1 : 0;
    d.VPC = f16 ? 8 : 4;
    d.KE = padto(3 * NE, 24);
    d.KH = padto(3 * NH, 24);
    d.KEo = f16 ? padto(3 * NE, 16) : d.KE;
    d.KHo = f16 ? padto(3 * NH, 16) : d.KH;
    d.FB = padto(2 * N2H, d.VPC);   // whole 16-byte chunks, two faces = whole K-steps
    d.NT = 4 * d.FB;
    d.NC = padto(12 * ((NH + 3) / 4), 16);
    d.NCE = padto(12 * ((NE + 3) / 4), 16);
    return d;
}

uint32_t tc_tmem_cols(const TCDims& d) {
    const int need = std::max(std::max(d.NC, d.NCE), d.NT);
    uint32_t c = 32;
    while ((int)c < need) c <<= 1;
    return c;
}

uint32_t tc_tmem_reach(const TCDims& d) {
    int reach = std::max(std::max(d.NC, d.NCE), d.NT);   // GEMM outputs and trace reads
    for (int N : {d.NE, d.NH}) {                          // update epilogue batches
        const int ngroups = (N + 3) / 4;
        for (int g0 = 0; g0 < ngroups; g0 += 4) {
            const int nq = 3 * std::min(4, ngroups - g0);
            reach = std::max(reach, 12 * g0 + 16 * ((4 * nq + 15) / 16));
        }
    }
    return (uint32_t)reach;
}

size_t tc_smem_bytes(const TCDims& d, uint32_t* stage_bytes, uint32_t* r2_offset) {
    const int maxB = std::max(std::max(d.NC, d.NCE), d.NT);
    // A slice (128 rows) + B slice (rows), + the B lo slice with two-term tables
    const uint32_t stage = (uint32_t)(kTcRows + maxB * (d.split ? 2 : 1)) * 32u;
    const uint32_t r2 = (uint32_t)kTcRows * (uint32_t)(2 * d.FB) * (d.f16 ? 2u : 4u);   // flux of two faces
    *stage_bytes = stage;
    *r2_offset = kHead + kStages * stage;
    const size_t bytes = (size_t)kHead + kStages * stage + r2;
    // with more than 256 TMEM columns a CTA must have its SM to itself: ask for
    // enough shared memory that a second CTA cannot be resident
    return tc_tmem_cols(d) > 256 ? std::max<size_t>(bytes, 116 * 1024) : bytes;
}

namespace {

template <bool IS_H, typename OP>
int launch_phase(const TCArgs& a, int grid, double dt, double a_lo, double c_out, int energy, cudaStream_t s) {
    const size_t sm = smem_of(a);
    if (set_smem((const void*)k_tc_phase<IS_H, OP>, sm)) return -1;
    k_tc_phase<IS_H, OP><<<grid, 128, sm, s>>>(a, dt, a_lo, c_out, energy);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

template <typename OP>
int launch_traces(const TCArgs& a, int grid, int which, int tile0, int tile1, int energy, cudaStream_t s) {
    const size_t sm = smem_of(a);
    if (set_smem((const void*)k_tc_traces<OP>, sm)) return -1;
    k_tc_traces<OP><<<grid, 128, sm, s>>>(a, which, tile0, tile1, energy);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace

int tc_launch_phase_H(const TCArgs& a, int grid, double dt, double a_lo, double c_out, int energy, cudaStream_t s) {
    if (a.d.layout == 2) return tc2_launch_phase(a, true, grid, dt, a_lo, c_out, energy, s);
    return a.d.f16 ? launch_phase<true, OpF16>(a, grid, dt, a_lo, c_out, energy, s)
                   : launch_phase<true, OpTf32>(a, grid, dt, a_lo, c_out, energy, s);
}

int tc_launch_phase_E(const TCArgs& a, int grid, double dt, int energy, cudaStream_t s) {
    if (a.d.layout == 2) return tc2_launch_phase(a, false, grid, dt, 0.0, 1.0, energy, s);
    return a.d.f16 ? launch_phase<false, OpF16>(a, grid, dt, 0.0, 1.0, energy, s)
                   : launch_phase<false, OpTf32>(a, grid, dt, 0.0, 1.0, energy, s);
}

int tc_launch_traces(const TCArgs& a, int grid, int which, cudaStream_t s) {
    if (a.d.layout == 2) return tc2_launch_traces(a, which, grid, 0, a.ntiles, which == 0, s);
    return a.d.f16 ? launch_traces<OpF16>(a, grid, which, 0, a.ntiles, which == 0, s)
                   : launch_traces<OpTf32>(a, grid, which, 0, a.ntiles, which == 0, s);
}

int tc_launch_traces_tile(const TCArgs& a, int which, int tile, cudaStream_t s) {
    if (a.d.layout == 2) return tc2_launch_traces(a, which, 1, tile, tile + 1, 0, s);
    return a.d.f16 ? launch_traces<OpF16>(a, 1, which, tile, tile + 1, 0, s)
                   : launch_traces<OpTf32>(a, 1, which, tile, tile + 1, 0, s);
}

int tc_launch_to_half(const float* src, void* dst, size_t n, cudaStream_t s) {
    if (n == 0) return 0;
    const size_t blocks = std::min<size_t>((n + 255) / 256, 4096);
    k_to_half<<<(unsigned)blocks, 256, 0, s>>>(src, static_cast<__half*>(dst), n);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

int tc_launch_split_half(const float* src, void* hi, void* lo, size_t n, cudaStream_t s) {
    if (n == 0) return 0;
    const size_t blocks = std::min<size_t>((n + 255) / 256, 4096);
    k_split_half<<<(unsigned)blocks, 256, 0, s>>>(src, static_cast<__half*>(hi), static_cast<__half*>(lo), n);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

int tc_launch_state_energy(const TCArgs& a, int grid, cudaStream_t s) {
    if (a.d.layout == 2) return tc2_launch_state_energy(a, grid, s);
    k_tc_state_energy<<<grid, 128, 0, s>>>(a);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

int tc_launch_pack(const double* src, float* dst, const double* nrm, int64_t nt, int N, int K, cudaStream_t s) {
    const int64_t n = nt * 3 * N;
    if (n == 0) return 0;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 8192);
    k_tc_pack<<<(int)blocks, 256, 0, s>>>(src, dst, nrm, nt, N, K);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

int tc_launch_unpack(const float* src, double* dst, const double* nrm, int64_t nt, int N, int K, cudaStream_t s) {
    const int64_t n = nt * 3 * N;
    if (n == 0) return 0;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 8192);
    k_tc_unpack<<<(int)blocks, 256, 0, s>>>(src, dst, nrm, nt, N, K);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace dgm
