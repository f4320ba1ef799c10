// Tensor-core phase kernels with resident reference tables (sm_103a, tcgen05),
// 2-byte operands (fp16 or bf16), FP32 accumulation, fp32 state.
//
// The operator is the one of kernels.cu and tc_kernels.cu (Sec. 2.1 central
// flux, Sec. 3.2 reference curl and traces, Sec. 3.3.1 block inverse mass,
// Sec. 3 symplectic Euler), applied to tiles of 128 elements.  What differs
// is how the reference operators are stored and how the work is scheduled:
//
// * Component-separated tables.  The curl couples components only through
//   the three reference derivatives D_x, D_y, D_z (Sec. 3.2.2):
//     (curl E)_x = D_y E_z - D_z E_y, and cyclically,
//   and a face trace or lift (Sec. 3.2.3) acts on each component with the
//   same reference matrix Tr_f, the reference face tangents t_{f,i} (entries
//   -1, 0, 1) selecting and signing the components.  So every GEMM here is
//   (one field component) x (one small table), with the sign carried by the
//   MMA's negate-B bit; the whole table set of a phase (68 KB at p = 6 in
//   the H-phase, 84 KB in the E-phase) stays in shared memory for the life of
//   the CTA, and only the fields move.
// * Component-major state: element rows k = m Np + a (Np = N padded to 16),
//   [tile][k/4][128][4] floats and [tile][k/8][128][8] 2-byte operand copy,
//   so one field component of a tile is one contiguous K range.
// * Warp roles, one CTA per SM (persistent over tiles):
//     warp 0     MMA issuer (one thread)
//     warp 1     producer: tables once, then each tile's input operand copy
//                with one bulk copy, issued as soon as the region is free
//     WG1        update and trace epilogues (upe threads per element,
//                TMEM lanes = elements)
//     WG2        flux epilogue, one tile ahead of WG1: the jump (H-phase) or
//                average (E-phase) of the element's and its neighbours'
//                tangential traces, written as the A operand of the lift
//   Per tile:  M1 = curl + lift into the accumulator  ->  U = inverse mass,
//   update, energy partial; the updated field's operand copy goes to HBM and
//   into the operand region  ->  M2 = traces of the updated field  ->
//   T = trace buffer for the other phase.
//
// Every wait is bounded; on a timeout the kernel sets an abort flag that all
// roles see, skips the remaining work (every thread still passes every named
// barrier, so nothing waits forever), lets issued copies and MMAs complete,
// records the error word, frees its tensor memory and returns.

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>

#include "kernels.h"
#include "tc_kernels.h"
#include "tc_ptx.h"

namespace dgm {

__host__ __device__ TC2Smem tc2_smem(const TCDims& d, bool is_h) {
    const uint32_t npin = (uint32_t)(is_h ? d.NEp : d.NHp), npout = (uint32_t)(is_h ? d.NHp : d.NEp);
    TC2Smem L;
    L.curl = 3u * npin * npout * 2u;
    L.lift = 4u * npout * (uint32_t)d.G * 2u;
    L.trace = 4u * (uint32_t)d.G * npout * 2u;
    L.tab = L.curl + L.lift + L.trace;
    // the input field's operand tile, then (after the curl and lift) the updated field's
    L.sa = 3u * (npin > npout ? npin : npout) * 128u * 2u;
    L.sf = 8u * (uint32_t)d.G * 128u * 2u;
    L.o_tab = 1024u + 4096u;   // control block, then the MMA programs (128 entries of 32 bytes)
    L.o_sa = (L.o_tab + L.tab + 1023u) / 1024u * 1024u;
    L.o_sf = (L.o_sa + L.sa + 1023u) / 1024u * 1024u;
    // at least 116 KB: a second CTA on the same SM would find no tensor memory left
    const uint32_t need = L.o_sf + L.sf;
    L.total = need > 116u * 1024u ? need : 116u * 1024u;
    return L;
}

namespace {

constexpr long long kLimit2 = 4000000000LL;   // cycles before a wait gives up (~2 s)
constexpr long long kDrain2 = 200000000LL;
constexpr long long kStall2 = 2000000LL;      // ~1 ms: the injected wait's limit
constexpr int kErr2 = 1;
constexpr uint32_t kChunk = 128 * 16;         // one 8-value column chunk of a 128-row operand tile

// 2-byte operand types: packing and the MMA's source format code
template <bool BF>
struct Op2;
template <>
struct Op2<false> {
    static constexpr uint32_t fmt = 0;   // F16
    static __device__ __forceinline__ uint32_t pack(float a, float b) {
        const __half2 h = __floats2half2_rn(a, b);
        uint32_t u;
        memcpy(&u, &h, 4);
        return u;
    }
    static __device__ __forceinline__ float2 unpack(uint32_t u) {
        __half2 h;
        memcpy(&h, &u, 4);
        return __half22float2(h);
    }
};
template <>
struct Op2<true> {
    static constexpr uint32_t fmt = 1;   // BF16
    static __device__ __forceinline__ uint32_t pack(float a, float b) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        uint32_t u;
        memcpy(&u, &h, 4);
        return u;
    }
    static __device__ __forceinline__ float2 unpack(uint32_t u) {
        __nv_bfloat162 h;
        memcpy(&h, &u, 4);
        return __bfloat1622float2(h);
    }
};

struct Ctl2 {
    uint64_t tab_full;   // tables landed
    uint64_t sa_full;    // input operand tile landed (once per tile)
    uint64_t m1_done;    // curl + lift MMAs complete: accumulator ready, operand and flux regions free
    uint64_t sf_full;    // flux blocks written
    uint64_t u_done;     // update done: accumulator free, updated operand tile in shared memory
    uint64_t tr_full;    // trace MMAs complete: operand region free again
    uint64_t tr_empty;   // trace columns read
    uint64_t fin;        // issuer's last commit
    uint64_t never;      // failure injection: nothing arrives here
    uint32_t tmem;
    volatile int abort;
    double red[16];
};

// Bounded wait; false (and the abort flag set) on a timeout, false at once after an abort.
__device__ bool wait2(Ctl2* c, uint64_t* bar, uint32_t parity) {
    const long long t0 = clock64();
    while (!tc::mbar_try_wait(bar, parity)) {
        if (c->abort) return false;
        if (clock64() - t0 > kLimit2) {
            c->abort = 1;
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(bar)) : "memory");
}

// this thread's 16 bytes (and the line holding them) into L2, no register or wait
__device__ __forceinline__ void prefetch_l2_line(const void* p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ __forceinline__ void named_bar(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }

// kind::f16 instruction descriptor: D fp32, A = B = fp16 or bf16, K-major, M = 128, B optionally negated
__device__ __forceinline__ uint32_t idesc2(uint32_t fmt, int n, bool neg_b) {
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((neg_b ? 1u : 0u) << 14) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(128 >> 4) << 24);
}

// one MMA of a precomputed program: TMEM column, instruction descriptor,
// accumulate flag, shared-memory descriptors of A and B
struct MmaOp {
    uint32_t d, idesc, acc, pad;
    uint64_t a, b;
};
constexpr int kProgMax = 4096 / (int)sizeof(MmaOp);

// The whole issuing warp runs the program loop together and lane 0 issues each
// MMA (and the commits): with the warp converged the operands stay warp-uniform,
// and an MMA program ran about twice as fast as the same loop in one thread.
__device__ __forceinline__ void issue_op(const MmaOp& o, uint32_t tmem) {
    asm volatile(
        "{\n\t.reg .pred p, e;\n\t.reg .u32 l;\n\t"
        "mov.u32 l, %%laneid;\n\t"
        "setp.eq.u32 e, l, 0;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem + o.d),
        "l"(o.a), "l"(o.b), "r"(o.idesc), "r"(o.acc));
}

__device__ __forceinline__ void commit_lane0(uint64_t* bar) {
    asm volatile(
        "{\n\t.reg .pred e;\n\t.reg .u32 l;\n\t"
        "mov.u32 l, %%laneid;\n\t"
        "setp.eq.u32 e, l, 0;\n\t"
        "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n}\n" ::"r"(
            tc::smem_u32(bar))
        : "memory");
}

// wait2 for a whole warp: every lane gets the same answer
__device__ __forceinline__ bool wait2w(Ctl2* c, uint64_t* bar, uint32_t parity) {
    return __all_sync(0xffffffffu, wait2(c, bar, parity));
}

// three 8-column TMEM loads of this thread's lane, one wait
__device__ __forceinline__ void tmem_ld3x8(uint32_t a0, uint32_t a1, uint32_t a2, float* v) {
    uint32_t r[24];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%24];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8, %9, %10, %11, %12, %13, %14, %15}, [%25];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%16, %17, %18, %19, %20, %21, %22, %23}, [%26];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23])
        : "r"(a0), "r"(a1), "r"(a2));
#pragma unroll
    for (int i = 0; i < 24; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld8(uint32_t a, float* v) {
    uint32_t r[8];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
        : "r"(a));
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// curl chains (output component m): input component, table d, sign; H-phase
// (curl E)_x = D_y E_z - D_z E_y ...; E-phase (curl^T H)_x = D_z^T H_y - D_y^T H_z ...
__device__ __forceinline__ void curl_chain(bool is_h, int m, int j, int& in, int& d, bool& neg) {
    const int mp1 = (m + 1) % 3, mp2 = (m + 2) % 3;
    if (is_h) {   // +D_{m+1} E_{m+2} - D_{m+2} E_{m+1}
        in = j == 0 ? mp2 : mp1;
        d = j == 0 ? mp1 : mp2;
    } else {      // +D_{m+2}^T H_{m+1} - D_{m+1}^T H_{m+2}
        in = j == 0 ? mp1 : mp2;
        d = j == 0 ? mp2 : mp1;
    }
    neg = j == 1;
}

struct Dims2 {
    int Nin, Npin, Nout, Npout, G8, G, NT;
    uint32_t acc0, tr0;
    bool overlap;
};

template <bool IS_H>
__device__ Dims2 dims2(const TCArgs& A, uint32_t tr0) {
    const TCDims& d = A.d;
    Dims2 q;
    q.Nin = IS_H ? d.NE : d.NH;
    q.Npin = IS_H ? d.NEp : d.NHp;
    q.Nout = IS_H ? d.NH : d.NE;
    q.Npout = IS_H ? d.NHp : d.NEp;
    q.G8 = d.G8;
    q.G = d.G;
    q.NT = d.NT;
    q.acc0 = 0;
    q.tr0 = tr0;
    q.overlap = (uint32_t)(3 * q.Npout) > tr0;
    return q;
}

// MODE 0: phase (IS_H: H-phase, else E-phase); MODE 1: traces of the field
// (IS_H: H, else E) from its fp32 state, refreshing its operand copy.
template <bool IS_H, int MODE, bool BF>
__global__ void __launch_bounds__(384, 1)
    k_tc2(TCArgs A, double dt, double a_lo, double c_out, int energy, uint32_t tr0, int tile0, int tile1) {
    using OP = Op2<BF>;
    extern __shared__ __align__(1024) uint8_t smem[];
    Ctl2* ctl = reinterpret_cast<Ctl2*>(smem);
    const TC2Smem L = tc2_smem(A.d, IS_H);
    const Dims2 q = dims2<IS_H>(A, tr0);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint8_t* s_tab = smem + L.o_tab;
    uint8_t* s_sa = smem + L.o_sa;
    uint8_t* s_sf = smem + L.o_sf;
    const uint32_t a_tab = tc::smem_u32(s_tab), a_sa = tc::smem_u32(s_sa), a_sf = tc::smem_u32(s_sf);
    // tables of the phase: curl (3), lift (4), trace (4)
    const uint32_t a_curl = a_tab, a_lift = a_tab + L.curl, a_trace = a_tab + L.curl + L.lift;

    if (tid == 0) {
        uint64_t* bars = &ctl->tab_full;
        for (int b = 0; b < 9; ++b) tc::mbar_init(bars + b, 1);
        ctl->abort = 0;
        tc::fence_mbar_init();
        tc::fence_proxy_async();
    }
    if (warp == 0) {
        tc::tmem_alloc(&ctl->tmem, 512);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    if (A.stall_test) {
        // failure injection: nothing arrives at `never`; the wait runs out before
        // any copy or MMA is issued
        if (tid == 0 && !tc::mbar_wait(&ctl->never, 0u, kStall2)) ctl->abort = 1;
        __syncthreads();
    }
    const uint32_t tmem = ctl->tmem;
    const int first = tile0 + (int)blockIdx.x;
    const int stride = (int)gridDim.x;
    int ntile = 0;
    for (int tile = first; tile < tile1; tile += stride) ++ntile;

    float* st_out = IS_H ? A.H : A.E;
    uint8_t* op_out = static_cast<uint8_t*>(IS_H ? A.Hop : A.Eop);
    const uint8_t* op_in = static_cast<const uint8_t*>(IS_H ? A.Eop : A.Hop);
    const uint8_t* tr_in = static_cast<const uint8_t*>(IS_H ? A.trE : A.trH);
    uint8_t* tr_out = static_cast<uint8_t*>(IS_H ? A.trH : A.trE);
    const uint8_t* gtab = static_cast<const uint8_t*>(IS_H ? A.T2H : A.T2E);
    const uint32_t in_tile_bytes = (uint32_t)(3 * q.Npin) * 128u * 2u;
    const uint32_t out_tile_bytes = (uint32_t)(3 * q.Npout) * 128u * 2u;
    const int nbat = q.Npout / 8;                 // 8-coefficient batches of the output field

    if (warp == 1) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            bool tab_issued = false;
            int issued = 0;   // input tiles issued
            if (!ctl->abort) {
                const uint32_t off = MODE == 0 ? 0u : L.curl + L.lift;
                const uint32_t bytes = MODE == 0 ? L.tab : L.trace;
                tc::mbar_expect_tx(&ctl->tab_full, bytes);
                tc::bulk_g2s(s_tab + off, gtab + off, bytes, &ctl->tab_full);
                tab_issued = true;
                if (MODE == 0 && ntile > 0) {
                    tc::mbar_expect_tx(&ctl->sa_full, in_tile_bytes);
                    tc::bulk_g2s(s_sa, op_in + (size_t)first * in_tile_bytes, in_tile_bytes, &ctl->sa_full);
                    issued = 1;
                }
            }
            for (int it = 0; MODE == 0 && it + 1 < ntile; ++it) {
                // the operand region is free once the trace MMAs of tile it completed
                if (!wait2(ctl, &ctl->tr_full, (uint32_t)it & 1u)) break;
                tc::mbar_expect_tx(&ctl->sa_full, in_tile_bytes);
                tc::bulk_g2s(s_sa, op_in + (size_t)(first + (it + 1) * stride) * in_tile_bytes, in_tile_bytes,
                             &ctl->sa_full);
                issued = it + 2;
            }
            // nothing of ours may still be landing when shared memory is given up
            if (tab_issued) tc::mbar_wait(&ctl->tab_full, 0u, kDrain2);
            if (issued > 0) tc::mbar_wait(&ctl->sa_full, (uint32_t)(issued - 1) & 1u, kDrain2);
        }
    } else if (warp == 0) {
        // ------------------------------------------------------------ MMA issuer
        // The MMA programs are the same for every tile (fixed shared-memory
        // operands, fixed TMEM columns): lane 0 builds them once, then the warp
        // issues each entry with a handful of instructions.
        MmaOp* prog = reinterpret_cast<MmaOp*>(smem + 1024);
        int n1 = 0, n2 = 0;
        if (lane == 0) {
            const uint32_t fmt = OP::fmt;
            auto mk = [&](uint32_t dcol, uint32_t a, uint32_t b, uint32_t rows, int n, bool neg, bool acc) {
                MmaOp o;
                o.d = dcol;
                o.idesc = idesc2(fmt, n, neg);
                o.acc = acc ? 1u : 0u;
                o.pad = 0u;
                o.a = tc::sdesc(a, kChunk, 128u);
                o.b = tc::sdesc(b, rows * 16u, 128u);
                return o;
            };
            // Each accumulator's chain is issued in one run (the tensor cores were
            // measured faster on consecutive MMAs into one accumulator than on
            // MMAs interleaved across accumulators).
            if (MODE == 0) {
                const int ksin = q.Npin / 16, ksg = q.G / 16;
                for (int m = 0; m < 3; ++m) {
                    const uint32_t dcol = q.acc0 + (uint32_t)(m * q.Npout);
                    for (int j = 0; j < 2; ++j) {
                        int in, dd;
                        bool neg;
                        curl_chain(IS_H, m, j, in, dd, neg);
                        const uint32_t abase = a_sa + (uint32_t)(in * q.Npin / 8) * kChunk;
                        const uint32_t bbase = a_curl + (uint32_t)(dd * q.Npin * q.Npout * 2);
                        for (int s = 0; s < ksin; ++s)
                            prog[n1++] = mk(dcol, abase + (uint32_t)(2 * s) * kChunk,
                                            bbase + (uint32_t)(2 * s * q.Npout * 16), (uint32_t)q.Npout, q.Npout, neg,
                                            j > 0 || s > 0);
                    }
                    // lift: block (f, 0) with t2_{f,m}, block (f, 1) with -t1_{f,m}
                    for (int f = 0; f < 4; ++f)
                        for (int i = 0; i < 2; ++i) {
                            const int c = i == 0 ? A.tsgn[f][1][m] : -A.tsgn[f][0][m];
                            if (c == 0) continue;
                            const uint32_t abase = a_sf + (uint32_t)((2 * f + i) * (q.G / 8)) * kChunk;
                            const uint32_t bbase = a_lift + (uint32_t)(f * q.Npout * q.G * 2);
                            for (int s = 0; s < ksg; ++s)
                                prog[n1++] = mk(dcol, abase + (uint32_t)(2 * s) * kChunk,
                                                bbase + (uint32_t)(2 * s * q.Npout * 16), (uint32_t)q.Npout, q.Npout,
                                                c < 0, true);
                        }
                }
            }
            // traces of the updated field: block (f, i) = sum_m t_{f,i,m} Tr_f X_m
            {
                const int ksout = q.Npout / 16;
                for (int f = 0; f < 4; ++f)
                    for (int i = 0; i < 2; ++i) {
                        bool first = true;
                        for (int m = 0; m < 3; ++m) {
                            const int c = A.tsgn[f][i][m];
                            if (c == 0) continue;
                            const uint32_t abase = a_sa + (uint32_t)(m * q.Npout / 8) * kChunk;
                            const uint32_t dcol = q.tr0 + (uint32_t)((2 * f + i) * q.G);
                            const uint32_t bbase = a_trace + (uint32_t)(f * q.G * q.Npout * 2);
                            for (int s = 0; s < ksout; ++s) {
                                prog[n1 + n2++] = mk(dcol, abase + (uint32_t)(2 * s) * kChunk,
                                                     bbase + (uint32_t)(2 * s * q.G * 16), (uint32_t)q.G, q.G, c < 0,
                                                     !first);
                                first = false;
                            }
                        }
                    }
            }
            if (n1 + n2 > kProgMax) ctl->abort = 1;   // cannot happen for p <= 6 (at most 104 entries)
        }
        n1 = __shfl_sync(0xffffffffu, n1, 0);
        n2 = __shfl_sync(0xffffffffu, n2, 0);
        __syncwarp();
        bool ok = wait2w(ctl, &ctl->tab_full, 0u);
        for (int it = 0; it < ntile && ok; ++it) {
            if (MODE == 0) {
                ok = wait2w(ctl, &ctl->sa_full, (uint32_t)it & 1u) && wait2w(ctl, &ctl->sf_full, (uint32_t)it & 1u);
                if (ok && q.overlap && it > 0) ok = wait2w(ctl, &ctl->tr_empty, (uint32_t)(it - 1) & 1u);
                if (!ok) break;
                tc::tc_fence_after();
                for (int k = 0; k < n1; ++k) issue_op(prog[k], tmem);
                commit_lane0(&ctl->m1_done);
            }
            ok = wait2w(ctl, &ctl->u_done, (uint32_t)it & 1u);
            if (ok && (MODE == 1 || !q.overlap) && it > 0) ok = wait2w(ctl, &ctl->tr_empty, (uint32_t)(it - 1) & 1u);
            if (!ok) break;
            tc::tc_fence_after();
            for (int k = n1; k < n1 + n2; ++k) issue_op(prog[k], tmem);
            commit_lane0(&ctl->tr_full);
        }
        commit_lane0(&ctl->fin);
        tc::mbar_wait(&ctl->fin, 0u, kDrain2);
        __syncwarp();
    } else if (tid >= 128 && tid < 256) {
        // ------------------------------------------------------------ WG1: update
        // One thread per element (TMEM lane).  The fp32 state comes in 8-coefficient
        // batches (three components, six 16-byte loads) through a four-deep register
        // ring.  As soon as this tile's update is done the ring takes the next tile's
        // first four batches and the rest of that tile's state is prefetched into L2,
        // so both land while the traces and the next curl are computed.
        const int e = tid - 128;
        const uint32_t lane_t = tmem + ((uint32_t)((warp & 3) * 32) << 16);
        const int nvb = (q.Nout + 7) / 8;   // batches holding coefficients
        double eacc = 0.0;
        float4 r0[6], r1[6], r2[6], r3[6];
        auto tile_state = [&](int it) { return st_out + (size_t)(first + it * stride) * (3 * q.Npout) * 128; };
        auto load_b = [&](const float* st, int b, float4* v) {
            const float4* s4 = reinterpret_cast<const float4*>(st) + ((size_t)(2 * b) * 128 + e);
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                v[2 * m] = s4[(size_t)(m * q.Npout / 4) * 128];
                v[2 * m + 1] = s4[(size_t)(m * q.Npout / 4 + 1) * 128];
            }
        };
        auto load_ring = [&](const float* st) {
            if (0 < nvb) load_b(st, 0, r0);
            if (1 < nvb) load_b(st, 1, r1);
            if (2 < nvb) load_b(st, 2, r2);
            if (3 < nvb) load_b(st, 3, r3);
        };
        if (MODE == 0 && ntile > 0) load_ring(tile_state(0));
        for (int it = 0; it < ntile; ++it) {
            const int tile = first + it * stride;
            const int64_t t = (int64_t)tile * 128 + e;
            float* st = st_out + (size_t)tile * (3 * q.Npout) * 128;
            uint8_t* opg = op_out + (size_t)tile * out_tile_bytes;
            const float4* gp = reinterpret_cast<const float4*>(A.geoF + t * 16);
            const float4 g0 = gp[0], g1 = gp[1], g2 = gp[2], g3 = gp[3];
            const float Gi[6] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y};
            const float Gm[6] = {g1.z, g1.w, g2.x, g2.y, g2.z, g2.w};
            const double mat = IS_H ? (double)g3.y : (double)g3.x;
            float eloc = 0.f;
            if (MODE == 0) {
                const bool ok = wait2(ctl, &ctl->m1_done, (uint32_t)it & 1u);
                tc::tc_fence_after();
                const float sT = IS_H ? -g3.z : g3.z;   // r = -s_T D (H-phase), s_T D (E-phase)
                const float sc = (float)(dt / mat);
                const float co = (float)c_out, alo = (float)a_lo;
                auto process = [&](int b, float4* v) {
                    // the batch's values, updated in place: x[8 m + c] = coefficient 8 b + c of component m
                    float* x = reinterpret_cast<float*>(v);
                    float dd[24];
                    tmem_ld3x8(lane_t + q.acc0 + (uint32_t)(8 * b), lane_t + q.acc0 + (uint32_t)(q.Npout + 8 * b),
                               lane_t + q.acc0 + (uint32_t)(2 * q.Npout + 8 * b), dd);
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        if (8 * b + c >= q.Nout) break;
                        const float rr0 = sT * dd[c], rr1 = sT * dd[8 + c], rr2 = sT * dd[16 + c];
                        const float d0 = sc * (Gi[0] * rr0 + Gi[1] * rr1 + Gi[2] * rr2);
                        const float d1 = sc * (Gi[1] * rr0 + Gi[3] * rr1 + Gi[4] * rr2);
                        const float d2 = sc * (Gi[2] * rr0 + Gi[4] * rr1 + Gi[5] * rr2);
                        float& h0 = x[c];
                        float& h1 = x[8 + c];
                        float& h2 = x[16 + c];
                        if (IS_H) {
                            if (energy) {   // staggered pair (H_lo, H_hi) of the modified energy
                                const float l0 = h0 - alo * d0, l1 = h1 - alo * d1, l2 = h2 - alo * d2;
                                const float u0 = l0 + d0, u1 = l1 + d1, u2 = l2 + d2;
                                eloc += l0 * (Gm[0] * u0 + Gm[1] * u1 + Gm[2] * u2) +
                                        l1 * (Gm[1] * u0 + Gm[3] * u1 + Gm[4] * u2) +
                                        l2 * (Gm[2] * u0 + Gm[4] * u1 + Gm[5] * u2);
                            }
                            h0 += co * d0;
                            h1 += co * d1;
                            h2 += co * d2;
                        } else {
                            h0 += d0;
                            h1 += d1;
                            h2 += d2;
                            if (energy)
                                eloc += h0 * (Gm[0] * h0 + Gm[1] * h1 + Gm[2] * h2) +
                                        h1 * (Gm[1] * h0 + Gm[3] * h1 + Gm[4] * h2) +
                                        h2 * (Gm[2] * h0 + Gm[4] * h1 + Gm[5] * h2);
                        }
                    }
                    float4* s4 = reinterpret_cast<float4*>(st) + ((size_t)(2 * b) * 128 + e);
#pragma unroll
                    for (int m = 0; m < 3; ++m) {
                        s4[(size_t)(m * q.Npout / 4) * 128] = v[2 * m];
                        s4[(size_t)(m * q.Npout / 4 + 1) * 128] = v[2 * m + 1];
                    }
#pragma unroll
                    for (int m = 0; m < 3; ++m) {
                        float w[8];
#pragma unroll
                        for (int c = 0; c < 8; ++c) w[c] = 8 * b + c < q.Nout ? x[8 * m + c] : 0.f;
                        const uint4 o = make_uint4(OP::pack(w[0], w[1]), OP::pack(w[2], w[3]), OP::pack(w[4], w[5]),
                                                   OP::pack(w[6], w[7]));
                        const size_t off = ((size_t)(m * q.Npout / 8 + b) * 128 + e) * 16;
                        *reinterpret_cast<uint4*>(opg + off) = o;
                        *reinterpret_cast<uint4*>(s_sa + off) = o;
                    }
                };
                auto step = [&](int k, float4* v) {
                    if (k < nvb) {
                        process(k, v);
                        if (k + 4 < nvb) load_b(st, k + 4, v);
                    }
                };
                for (int k0 = 0; k0 < nvb && ok; k0 += 4) {
                    step(k0, r0);
                    step(k0 + 1, r1);
                    step(k0 + 2, r2);
                    step(k0 + 3, r3);
                }
                // batches of padding only: zero operand chunks for the trace GEMM
                for (int b = nvb; b < nbat && ok; ++b)
#pragma unroll
                    for (int m = 0; m < 3; ++m)
                        *reinterpret_cast<uint4*>(s_sa + ((size_t)(m * q.Npout / 8 + b) * 128 + e) * 16) =
                            make_uint4(0u, 0u, 0u, 0u);
                // the next tile: its first batches into the ring, the rest into L2
                if (it + 1 < ntile) {
                    const float* stn = tile_state(it + 1);
                    load_ring(stn);
                    for (int b = 4; b < nvb; ++b) {
                        const float* p4 = stn + ((size_t)(2 * b) * 128 + e) * 4;
#pragma unroll
                        for (int m = 0; m < 3; ++m) {
                            prefetch_l2_line(p4 + (size_t)(m * q.Npout / 4) * 128 * 4);
                            prefetch_l2_line(p4 + (size_t)(m * q.Npout / 4 + 1) * 128 * 4);
                        }
                    }
                }
            } else {
                // traces only: the operand copy of the field from its fp32 state
                // (changed from outside: import, sources, checkpoints), into the
                // operand region once the previous tile's trace MMAs have read it
                const bool ok = it == 0 || wait2(ctl, &ctl->tr_full, (uint32_t)(it - 1) & 1u);
                for (int b = 0; b < nbat && ok; ++b) {
                    const bool valid = 8 * b < q.Nout;
                    float x[24];
#pragma unroll
                    for (int m = 0; m < 3; ++m) {
                        if (valid) {
                            const float4* s4 = reinterpret_cast<const float4*>(st) +
                                               ((size_t)(m * q.Npout / 4 + 2 * b) * 128 + e);
                            const float4 v0 = s4[0], v1 = s4[128];
                            x[8 * m + 0] = v0.x; x[8 * m + 1] = v0.y; x[8 * m + 2] = v0.z; x[8 * m + 3] = v0.w;
                            x[8 * m + 4] = v1.x; x[8 * m + 5] = v1.y; x[8 * m + 6] = v1.z; x[8 * m + 7] = v1.w;
                        }
#pragma unroll
                        for (int c = 0; c < 8; ++c)
                            if (!valid || 8 * b + c >= q.Nout) x[8 * m + c] = 0.f;
                    }
                    if (energy && !IS_H && valid) {
#pragma unroll
                        for (int c = 0; c < 8; ++c) {
                            const float h0 = x[c], h1 = x[8 + c], h2 = x[16 + c];
                            eloc += h0 * (Gm[0] * h0 + Gm[1] * h1 + Gm[2] * h2) + h1 * (Gm[1] * h0 + Gm[3] * h1 + Gm[4] * h2) +
                                    h2 * (Gm[2] * h0 + Gm[4] * h1 + Gm[5] * h2);
                        }
                    }
#pragma unroll
                    for (int m = 0; m < 3; ++m) {
                        const uint4 o = make_uint4(OP::pack(x[8 * m], x[8 * m + 1]), OP::pack(x[8 * m + 2], x[8 * m + 3]),
                                                   OP::pack(x[8 * m + 4], x[8 * m + 5]),
                                                   OP::pack(x[8 * m + 6], x[8 * m + 7]));
                        const size_t off = ((size_t)(m * q.Npout / 8 + b) * 128 + e) * 16;
                        *reinterpret_cast<uint4*>(opg + off) = o;
                        *reinterpret_cast<uint4*>(s_sa + off) = o;
                    }
                }
            }
            eacc += 0.5 * mat * (double)eloc;
            // the updated operand tile in shared memory goes to the tensor cores
            tc::fence_proxy_async();
            tc::tc_fence_before();
            named_bar(1, 128);
            if (e == 0) mbar_arrive(&ctl->u_done);
        }
        if (energy) {
            for (int o = 16; o > 0; o >>= 1) eacc += __shfl_down_sync(0xffffffffu, eacc, o);
            if (lane == 0) ctl->red[warp & 3] = eacc;
            named_bar(1, 128);
            if (e == 0) {
                const double sum = ((ctl->red[0] + ctl->red[1]) + ctl->red[2]) + ctl->red[3];
                const bool h = MODE == 0 ? IS_H : false;
                (h ? A.partH : A.partE)[blockIdx.x] = sum;
            }
        }
    } else if (tid >= 256 && tid < 384) {
        // ------------------------------------------------------------ WG2: flux and traces
        // For tile it + 1: the jump (H-phase) or average (E-phase) of the
        // element's and its neighbours' tangential traces, written as the A
        // operand of the lift (the first two faces' loads are issued before the
        // wait for the flux blocks to be free, the last two after it).  Then,
        // for tile it: the traces of the updated field into the trace buffer.
        const int e = tid - 256;
        const uint32_t lane_t = tmem + ((uint32_t)((warp & 3) * 32) << 16);
        const int nG8 = q.G8 / 8, nG = q.G / 8;
        uint4 ov[2][6], nv[2][6];
        int4 nb4 = make_int4(-1, -1, -1, -1);
        auto load_pair = [&](int64_t t, int fp) {
#pragma unroll
            for (int ff = 0; ff < 2; ++ff) {
                const int f = 2 * fp + ff;
                const int32_t nb = fp == 0 ? (ff == 0 ? nb4.x : nb4.y) : (ff == 0 ? nb4.z : nb4.w);
                const uint4* own = reinterpret_cast<const uint4*>(tr_in + ((size_t)t * q.NT + f * 2 * q.G8) * 2);
                const uint4* src =
                    nb >= 0 ? reinterpret_cast<const uint4*>(tr_in + ((size_t)(nb >> 2) * q.NT + (nb & 3) * 2 * q.G8) * 2)
                            : own;
#pragma unroll
                for (int c = 0; c < 6; ++c)
                    if (c < 2 * nG8) {
                        ov[ff][c] = own[c];
                        nv[ff][c] = src[c];
                    }
            }
        };
        auto write_pair = [&](int fp) {
#pragma unroll
            for (int ff = 0; ff < 2; ++ff) {
                const int f = 2 * fp + ff;
                const bool pec = (fp == 0 ? (ff == 0 ? nb4.x : nb4.y) : (ff == 0 ? nb4.z : nb4.w)) < 0;
                const float sh = (float)A.sigma_hat[f];
#pragma unroll
                for (int c = 0; c < 6; ++c) {
                    if (c >= 2 * nG8) break;
                    const uint32_t ow[4] = {ov[ff][c].x, ov[ff][c].y, ov[ff][c].z, ov[ff][c].w};
                    const uint32_t nw[4] = {nv[ff][c].x, nv[ff][c].y, nv[ff][c].z, nv[ff][c].w};
                    uint32_t o[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const float2 v = OP::unpack(ow[k]), n = OP::unpack(nw[k]);
                        float a, b2;
                        if (IS_H) {   // jump: -sigma (v - n)/2, PEC ghost -sigma v
                            a = pec ? -sh * v.x : -sh * 0.5f * (v.x - n.x);
                            b2 = pec ? -sh * v.y : -sh * 0.5f * (v.y - n.y);
                        } else {      // average: sigma (v + n)/2, PEC sigma v
                            a = pec ? sh * v.x : sh * 0.5f * (v.x + n.x);
                            b2 = pec ? sh * v.y : sh * 0.5f * (v.y + n.y);
                        }
                        o[k] = OP::pack(a, b2);
                    }
                    // chunk c of the face block = tangent i = c / nG8, chunk c % nG8
                    const int i = c / nG8, cc = c - i * nG8;
                    *reinterpret_cast<uint4*>(s_sf + ((size_t)((2 * f + i) * nG + cc) * 128 + e) * 16) =
                        make_uint4(o[0], o[1], o[2], o[3]);
                }
            }
        };
        auto flux = [&](int it) {
            const int64_t t = (int64_t)(first + it * stride) * 128 + e;
            nb4 = *reinterpret_cast<const int4*>(A.nbr + t * 4);
            load_pair(t, 0);
            // the flux blocks are free once the lift of the previous tile completed
            const bool ok = it == 0 || wait2(ctl, &ctl->m1_done, (uint32_t)(it - 1) & 1u);
            if (ok) {
                write_pair(0);
                load_pair(t, 1);
                write_pair(1);
            }
            tc::fence_proxy_async();
            named_bar(2, 128);
            if (e == 0) mbar_arrive(&ctl->sf_full);
        };
        if (MODE == 0) {
            // the padding chunks of each flux block stay zero
            for (int blk = 0; blk < 8; ++blk)
                for (int c = nG8; c < nG; ++c)
                    *reinterpret_cast<uint4*>(s_sf + ((size_t)(blk * nG + c) * 128 + e) * 16) = make_uint4(0u, 0u, 0u, 0u);
            if (ntile > 0) flux(0);
        }
        for (int it = 0; it < ntile; ++it) {
            if (MODE == 0 && it + 1 < ntile) flux(it + 1);
            // trace epilogue of tile it: blocks (f, i) of the trace columns -> trace buffer row
            const int64_t t = (int64_t)(first + it * stride) * 128 + e;
            const bool ok = wait2(ctl, &ctl->tr_full, (uint32_t)it & 1u);
            tc::tc_fence_after();
            if (ok) {
                uint8_t* row = tr_out + (size_t)t * q.NT * 2;
                for (int blk = 0; blk < 8; ++blk)
                    for (int c = 0; c < nG8; ++c) {
                        float v[8];
                        tmem_ld8(lane_t + q.tr0 + (uint32_t)(blk * q.G + 8 * c), v);
                        *reinterpret_cast<uint4*>(row + (size_t)(blk * q.G8 + 8 * c) * 2) =
                            make_uint4(OP::pack(v[0], v[1]), OP::pack(v[2], v[3]), OP::pack(v[4], v[5]),
                                       OP::pack(v[6], v[7]));
                    }
            }
            tc::tc_fence_before();
            named_bar(2, 128);
            if (e == 0) mbar_arrive(&ctl->tr_empty);
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    if (tid == 0 && ctl->abort) atomicCAS(A.err, 0, kErr2);
    if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

__global__ void k_tc2_state_energy(TCArgs A) {
    const TCDims d = A.d;
    double eE = 0.0, eH = 0.0;
    const int64_t n = (int64_t)A.ntiles * 128;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const double* gg = A.geo + t * kGeoStride;
        const double G0 = gg[6], G1 = gg[7], G2 = gg[8], G3 = gg[9], G4 = gg[10], G5 = gg[11];
        const int64_t tile = t >> 7, e = t & 127;
        for (int which = 0; which < 2; ++which) {
            const int N = which == 0 ? d.NE : d.NH, Np = which == 0 ? d.NEp : d.NHp;
            const float* base = (which == 0 ? A.E : A.H) + (size_t)tile * 3 * Np * 128;
            double acc = 0.0;
            for (int a = 0; a < N; ++a) {
                double x[3];
                for (int m = 0; m < 3; ++m) {
                    const int k = m * Np + a;
                    x[m] = base[((size_t)(k >> 2) * 128 + e) * 4 + (k & 3)];
                }
                acc += x[0] * (G0 * x[0] + G1 * x[1] + G2 * x[2]) + x[1] * (G1 * x[0] + G3 * x[1] + G4 * x[2]) +
                       x[2] * (G2 * x[0] + G4 * x[1] + G5 * x[2]);
            }
            (which == 0 ? eE : eH) += 0.5 * (which == 0 ? gg[kGeoEps] : gg[kGeoMu]) * acc;
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

// canonical [t][3][N] doubles <-> component-major tiles, scaled by nrm[a] (import) / 1/nrm[a] (export)
__global__ void k_tc2_pack(const double* __restrict__ src, float* __restrict__ dst, const double* __restrict__ nrm,
                           int64_t nt, int N, int Np) {
    const int64_t n = nt * 3 * N;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = i / (3 * N);
        const int rem = (int)(i - t * 3 * N);
        const int m = rem / N, a = rem - m * N;
        const int k = m * Np + a;
        const double sc = nrm ? nrm[a] : 1.0;
        dst[(((t >> 7) * (3 * Np / 4) + (k >> 2)) * 128 + (t & 127)) * 4 + (k & 3)] = (float)(src[i] * sc);
    }
}

__global__ void k_tc2_unpack(const float* __restrict__ src, double* __restrict__ dst, const double* __restrict__ nrm,
                             int64_t nt, int N, int Np) {
    const int64_t n = nt * 3 * N;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = i / (3 * N);
        const int rem = (int)(i - t * 3 * N);
        const int m = rem / N, a = rem - m * N;
        const int k = m * Np + a;
        const double sc = nrm ? nrm[a] : 1.0;
        dst[i] = (double)src[(((t >> 7) * (3 * Np / 4) + (k >> 2)) * 128 + (t & 127)) * 4 + (k & 3)] / sc;
    }
}

__global__ void k_to_bf16(const float* __restrict__ src, __nv_bfloat16* __restrict__ dst, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = __float2bfloat16_rn(src[i]);
}

template <bool IS_H, int MODE, bool BF>
int launch2(const TCArgs& a, int grid, double dt, double a_lo, double c_out, int energy, int tile0, int tile1,
            cudaStream_t s) {
    const TC2Smem L = tc2_smem(a.d, IS_H);
    const void* fn = (const void*)k_tc2<IS_H, MODE, BF>;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total) != cudaSuccess) return -1;
    const int threads = 384;
    k_tc2<IS_H, MODE, BF><<<grid, threads, L.total, s>>>(a, dt, a_lo, c_out, energy, tc2_tr0(a.d, IS_H), tile0, tile1);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace


uint32_t tc2_tr0(const TCDims& d, bool is_h) {
    const uint32_t acc = 3u * (uint32_t)(is_h ? d.NHp : d.NEp);
    const uint32_t tr = 8u * (uint32_t)d.G;
    // after the accumulator when both fit; else at the end, overlapping it
    // (the next tile's curl then waits for the traces to be read)
    return acc + tr <= 512u ? acc : 512u - tr;
}

int tc2_launch_phase(const TCArgs& a, bool is_h, int grid, double dt, double a_lo, double c_out, int energy,
                     cudaStream_t s) {
    if (a.d.bf16)
        return is_h ? launch2<true, 0, true>(a, grid, dt, a_lo, c_out, energy, 0, a.ntiles, s)
                    : launch2<false, 0, true>(a, grid, dt, a_lo, c_out, energy, 0, a.ntiles, s);
    return is_h ? launch2<true, 0, false>(a, grid, dt, a_lo, c_out, energy, 0, a.ntiles, s)
                : launch2<false, 0, false>(a, grid, dt, a_lo, c_out, energy, 0, a.ntiles, s);
}

int tc2_launch_traces(const TCArgs& a, int which, int grid, int tile0, int tile1, int energy, cudaStream_t s) {
    // which = 0: E (the field the E-phase updates), 1: H
    if (a.d.bf16)
        return which == 0 ? launch2<false, 1, true>(a, grid, 0.0, 0.0, 0.0, energy, tile0, tile1, s)
                          : launch2<true, 1, true>(a, grid, 0.0, 0.0, 0.0, 0, tile0, tile1, s);
    return which == 0 ? launch2<false, 1, false>(a, grid, 0.0, 0.0, 0.0, energy, tile0, tile1, s)
                      : launch2<true, 1, false>(a, grid, 0.0, 0.0, 0.0, 0, tile0, tile1, s);
}

int tc2_launch_state_energy(const TCArgs& a, int grid, cudaStream_t s) {
    k_tc2_state_energy<<<grid, 128, 0, s>>>(a);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

int tc2_launch_pack(const double* src, float* dst, const double* nrm, int64_t nt, int N, int Np, cudaStream_t s) {
    const int64_t n = nt * 3 * N;
    if (n == 0) return 0;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 8192);
    k_tc2_pack<<<(int)blocks, 256, 0, s>>>(src, dst, nrm, nt, N, Np);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

int tc2_launch_unpack(const float* src, double* dst, const double* nrm, int64_t nt, int N, int Np, cudaStream_t s) {
    const int64_t n = nt * 3 * N;
    if (n == 0) return 0;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 8192);
    k_tc2_unpack<<<(int)blocks, 256, 0, s>>>(src, dst, nrm, nt, N, Np);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

int tc_launch_to_bf16(const float* src, void* dst, size_t n, cudaStream_t s) {
    if (n == 0) return 0;
    const size_t blocks = std::min<size_t>((n + 255) / 256, 4096);
    k_to_bf16<<<(unsigned)blocks, 256, 0, s>>>(src, static_cast<__nv_bfloat16*>(dst), n);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace dgm
