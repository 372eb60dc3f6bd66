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
// address: cg_plan looks the address up (cudaGetSymbolAddress, the plan's
// device current), which also loads the array onto that device, and keeps it
// in the plan.  A plan made after a device reset therefore holds the address
// of that reset's reload; the entry point itself looks nothing up.
#include <cstdint>

#include <cuda_runtime.h>

#include "cg_internal.h"

namespace {

// 32768 doubles = 256 KiB of partial sums: rows of n_teeth values, one row
// per thread block of the accumulation kernel.
constexpr int kNoAllocScratchDoubles = 32768;

__device__ __align__(256) double g_ref_scratch[kNoAllocScratchDoubles];

cg_status noalloc_fail(cg_status st, const char* msg)
{
    cg::set_last_error(msg);
    return st;
}

// true when ptr is device (or managed) memory that the plan's device can use
bool on_plan_device(const void* ptr, int device)
{
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
        cudaGetLastError();   // clear the (non-sticky) error an unknown pointer leaves
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeDevice && at.device == device;
}

}  // namespace

namespace cg {

cudaError_t bind_noalloc_scratch(cg_plan_s* p)
{
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_ref_scratch);
    if (e != cudaSuccess) return e;
    p->noalloc_scratch = static_cast<double*>(ptr);
    return cudaSuccess;
}

}  // namespace cg

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
    if (!plan->noalloc_scratch) return noalloc_fail(CG_ERR_CUDA, "the plan holds no scratch address");
    if (!on_plan_device(frames_dev, plan->device))
        return noalloc_fail(CG_ERR_ARG, "frames_dev is not device memory of the plan's device");
    if (!on_plan_device(ref_dev, plan->device))
        return noalloc_fail(CG_ERR_ARG, "ref_dev is not device memory of the plan's device");

    int prev = -1;
    cudaError_t e = cudaGetDevice(&prev);
    if (e == cudaSuccess && prev != plan->device) e = cudaSetDevice(plan->device);
    if (e == cudaSuccess)
        e = cg::launch_reference_into(plan, frames_dev, n, plan->noalloc_scratch, rows, ref_dev,
                                      static_cast<cudaStream_t>(cuda_stream));
    if (prev >= 0 && prev != plan->device) cudaSetDevice(prev);
    if (e != cudaSuccess) {
        return noalloc_fail(e == cudaErrorMemoryAllocation ? CG_ERR_NOMEM : CG_ERR_CUDA,
                            cudaGetErrorString(e));
    }
    return CG_OK;
}

}  // extern "C"
