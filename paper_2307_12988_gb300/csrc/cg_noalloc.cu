// cg_noalloc.cu -- reference-spectrum accumulation that allocates nothing.
//
// Some callers cannot allocate device memory when they need the reference
// spectrum: code running inside a real-time acquisition loop that must not
// stall on the allocator, processes whose device memory is already fully
// reserved by a memory pool they do not control, or hosts that only lend this
// library a stream and buffers.  For them this entry point keeps the
// per-block partial sums in a fixed array compiled into the library instead
// of the plan's own scratch.  The paper has no counterpart to this; it is an
// interface convenience of this library.
//
// The array lives in device memory of every GPU that loads the library, for
// as long as the process lives.  Host code may not use its name as a device
// address, so its address is looked up once per device with
// cudaGetSymbolAddress and cached; the first call on each device does that.
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "cg_internal.h"

namespace {

// 32768 doubles = 256 KiB of partial sums: rows of n_teeth values, one row
// per thread block of the accumulation kernel.
constexpr int kNoAllocScratchDoubles = 32768;
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_ref_scratch[kNoAllocScratchDoubles];

std::mutex g_scratch_mu;
double* g_scratch_addr[kMaxDevices] = {};

// Device address of g_ref_scratch on `dev` (looked up with `dev` current).
cudaError_t scratch_on(int dev, double** out)
{
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (g_scratch_addr[dev] == nullptr) {
        void* ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_ref_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = static_cast<double*>(ptr);
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

cg_status noalloc_fail(cg_status st, const char* msg)
{
    cg::set_last_error(msg);
    return st;
}

}  // namespace

extern "C" {

cg_status cg_reference_accumulate_noalloc(cg_plan_t plan, const int16_t* frames_dev, int64_t n,
                                          double* ref_dev, void* cuda_stream)
{
    cg::set_last_error("");
    if (!plan) return noalloc_fail(CG_ERR_ARG, "plan is NULL");
    if (n < 1) return noalloc_fail(CG_ERR_ARG, "need at least one reference frame");
    if (!frames_dev || (reinterpret_cast<uintptr_t>(frames_dev) & 1))
        return noalloc_fail(CG_ERR_ARG, "frames_dev must be a 2-byte aligned device pointer");
    if (!ref_dev || (reinterpret_cast<uintptr_t>(ref_dev) & 7))
        return noalloc_fail(CG_ERR_ARG, "ref_dev must be an 8-byte aligned device pointer");
    if (n > (int64_t(1) << 40) / plan->N) return noalloc_fail(CG_ERR_ARG, "n too large");
    const int T = plan->T;
    const int rows = kNoAllocScratchDoubles / T;
    if (rows < 1)
        return noalloc_fail(CG_ERR_ARG, "n_teeth exceeds the 32768-double static scratch");
    if (plan->device < 0 || plan->device >= kMaxDevices)
        return noalloc_fail(CG_ERR_UNSUPPORTED, "device ordinal beyond 63");

    int prev = -1;
    cudaError_t e = cudaGetDevice(&prev);
    if (e == cudaSuccess && prev != plan->device) e = cudaSetDevice(plan->device);
    double* scratch = nullptr;
    if (e == cudaSuccess) e = scratch_on(plan->device, &scratch);
    if (e == cudaSuccess)
        e = cg::launch_reference_into(plan, frames_dev, n, scratch, rows, ref_dev,
                                      static_cast<cudaStream_t>(cuda_stream));
    if (prev >= 0 && prev != plan->device) cudaSetDevice(prev);
    if (e != cudaSuccess) {
        return noalloc_fail(e == cudaErrorMemoryAllocation ? CG_ERR_NOMEM : CG_ERR_CUDA,
                            cudaGetErrorString(e));
    }
    return CG_OK;
}

}  // extern "C"
