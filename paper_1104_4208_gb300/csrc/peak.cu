// dgm_measure_fp64_peak: the FP64 fused multiply-add rate of the device,
// measured with CUDA events.  It is the roofline denominator of the FP64
// path, whose phase kernels are bound by FP64 arithmetic rather than by
// memory.  Not part of the method of the paper.
//
// Every thread runs kChains independent multiply-add chains (enough
// independent instructions to keep the FP64 pipe issuing every cycle) for
// `iters` rounds; the grid fills every SM several times over.  The result of
// each chain is stored, so no chain can be removed as dead code.

#include <cuda_runtime.h>

#include <string>

#include "dgm_internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_fma_f64(double* __restrict__ out, int iters, double a, double b) {
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (double)(threadIdx.x + c) * 1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

int fail(const char* what, cudaError_t e) {
    dgm::set_error(std::string("dgm_measure_fp64_peak: ") + what + ": " + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? DGM_ERR_OOM : DGM_ERR_CUDA;
}

}  // namespace

extern "C" int dgm_measure_fp64_peak(int device, int repeats, double* tflops) {
    if (!tflops || repeats < 1) {
        dgm::set_error("dgm_measure_fp64_peak: bad argument");
        return DGM_ERR_INVALID_ARG;
    }
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return fail("cudaSetDevice", e);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const int blocks = sms * 8;
    const int iters = 4096;
    double* out = nullptr;
    if ((e = cudaMalloc(&out, (size_t)blocks * kThreads * sizeof(double))) != cudaSuccess) return fail("alloc", e);
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    // 0.999999 x + 1e-7 stays bounded; the values do not matter for the rate
    k_fma_f64<<<blocks, kThreads>>>(out, iters, 0.999999, 1e-7);   // warm-up
    double best_ms = 1e30;
    for (int r = 0; r < repeats && e == cudaSuccess; ++r) {
        cudaEventRecord(a);
        k_fma_f64<<<blocks, kThreads>>>(out, iters, 0.999999, 1e-7);
        cudaEventRecord(b);
        e = cudaEventSynchronize(b);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        if (e == cudaSuccess && ms < best_ms) best_ms = ms;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(out);
    if (e != cudaSuccess) return fail("kernel", e);
    const double flops = 2.0 * (double)blocks * kThreads * (double)iters * kChains;
    *tflops = flops / (best_ms * 1e-3) / 1e12;
    return DGM_OK;
}
