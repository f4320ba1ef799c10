// dgm_energy_noalloc: the discrete energy of a problem's current state,
// computed without allocating any device memory.
//
// Who needs it: applications that reserve all device memory up front for
// their own pool allocator and forbid further cudaMalloc/cudaFree calls (both
// calls synchronise the whole device and can fail once the pool owns the
// memory), and hosts that load this library as a plug-in inside such an
// application.  dgm_energy may allocate (its output slot is created on first
// use); this entry point never does.
//
// How: the energy kernels write one FP64 partial sum per thread block -- the
// H-phase kernel with dt = 0 on the CUDA-core precisions (FP64, FP32), the
// state-energy kernel on the tensor-core precisions (TC32, TC16; two sums, E
// and H, per block).  Here those partials go to a file-scope device array of
// fixed size instead of a buffer owned by the problem, and the fixed-order
// reduction writes the result to the caller's device pointer.  The array
// exists once per device for the lifetime of the process.  Its device address
// is looked up with cudaGetSymbolAddress on the first call made on each
// device (so make that first call before any stream capture); later calls
// reuse the address.
//
// Every call on a device shares the one array: two calls whose kernels overlap
// on the GPU (different streams, different problems) race on it and may return
// wrong energies.  Each block overwrites its own slot before the reduction
// reads it, so nothing left over from the previous call is ever read and the
// array needs no clearing.

#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "dgm_internal.h"
#include "kernels.h"
#include "problem.h"

namespace {

constexpr int kNoallocMaxBlocks = 4096;   // 32 KiB of FP64 partial sums per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_energy_scratch[kNoallocMaxBlocks];

std::mutex g_scratch_mu;
double* g_scratch_ptr[kMaxDevices] = {};

int scratch_for_current_device(double** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        dgm::set_error(std::string("dgm_energy_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
        return DGM_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        dgm::set_error("dgm_energy_noalloc: device index beyond the supported 64");
        return DGM_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_energy_scratch);
        if (e != cudaSuccess || !p) {
            dgm::set_error(std::string("dgm_energy_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            return DGM_ERR_CUDA;
        }
        g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_ptr[dev];
    return DGM_OK;
}

}  // namespace

extern "C" int dgm_energy_noalloc(dgm_problem* P, double* W_device, void* stream) {
    if (!P || !W_device) {
        dgm::set_error("dgm_energy_noalloc: null argument");
        return DGM_ERR_INVALID_ARG;
    }
    // partial sums this problem's energy kernels write: one per block of the
    // CUDA-core phase kernel, or an E and an H sum per tensor-core CTA
    const int nsums = P->tc ? 2 * P->tc_grid : P->grid;
    if (nsums > kNoallocMaxBlocks) {
        dgm::set_error("dgm_energy_noalloc: the problem uses " + std::to_string(nsums) +
                       " partial sums but the static scratch holds at most " +
                       std::to_string(kNoallocMaxBlocks));
        return DGM_ERR_INVALID_ARG;
    }
    // the scratch address belongs to the problem's device; make it current for
    // the look-up and the launches, then restore the caller's device
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) {
        dgm::set_error("dgm_energy_noalloc: cudaGetDevice failed");
        return DGM_ERR_CUDA;
    }
    if (prev != P->ctx->device && cudaSetDevice(P->ctx->device) != cudaSuccess) {
        dgm::set_error("dgm_energy_noalloc: cudaSetDevice failed");
        return DGM_ERR_CUDA;
    }
    double* scratch = nullptr;
    int rc = scratch_for_current_device(&scratch);
    if (rc == DGM_OK) {
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        int r;
        if (P->tc) {
            // the tiled state's 1/2 (eps E, E) and 1/2 (mu H, H) partials, E sums
            // first, then H sums -- the launch dgm_energy makes, redirected
            dgm::TCArgs a = P->tca;
            a.partE = scratch;
            a.partH = scratch + P->tc_grid;
            r = dgm::tc_launch_state_energy(a, P->tc_grid, s);
        } else {
            // dt = 0: the H-phase leaves H unchanged and its energy partial is
            // 1/2 (eps E, E) + 1/2 (mu H, H) -- the same launch dgm_energy makes
            r = P->fp32 ? dgm::launch_phase_H<float>(P->kf, P->grid, 0.0, 0.0, 0.0, scratch, s)
                        : dgm::launch_phase_H<double>(P->kd, P->grid, 0.0, 0.0, 0.0, scratch, s);
        }
        if (r == 0) r = dgm::launch_energy_reduce(scratch, nsums, W_device, s);
        if (r != 0) {
            dgm::set_error(std::string("dgm_energy_noalloc: launch failed: ") +
                           cudaGetErrorString(cudaGetLastError()));
            rc = DGM_ERR_CUDA;
        }
    }
    if (prev != P->ctx->device) cudaSetDevice(prev);
    return rc;
}
