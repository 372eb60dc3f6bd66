// cg_stage.cuh -- asynchronous staging of a batch of frames (int16 or int8
// samples, contiguous in global memory) into shared memory with 16-byte
// cp.async copies; the ragged head and tail chunks go element by element.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace cg {

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem)
{
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem)
{
    const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Asynchronous staging of elements [e0, e0 + ne) of type S (int16 or int8
// samples) into raw: 16-byte chunks aligned in global memory go by cp.async,
// the ragged head/tail chunk by plain loads.  Returns the element offset of
// e0 inside raw.
template <class S>
__device__ __forceinline__ void copy_partial_chunk(uintptr_t pa, int c, uintptr_t p, uintptr_t pend, S* raw)
{
    constexpr int kPer = 16 / static_cast<int>(sizeof(S));
#pragma unroll
    for (int e = 0; e < kPer; ++e) {
        const uintptr_t ep = pa + 16 * static_cast<uintptr_t>(c) + sizeof(S) * e;
        if (ep >= p && ep < pend) raw[kPer * c + e] = *reinterpret_cast<const S*>(ep);
    }
}

template <class S>
__device__ __forceinline__ int stage_async(const S* frames, int64_t e0, int64_t ne, S* raw)
{
    const uintptr_t p = reinterpret_cast<uintptr_t>(frames + e0);
    const uintptr_t pa = p & ~static_cast<uintptr_t>(15);
    const uintptr_t pend = p + static_cast<uintptr_t>(ne) * sizeof(S);
    const int off = static_cast<int>((p - pa) / sizeof(S));
    const int nchunks = static_cast<int>((pend - pa + 15) >> 4);   // a batch is < 2 GiB
    const int first_whole = (p == pa) ? 0 : 1;
    const int end_whole = ((pend & 15) == 0) ? nchunks : nchunks - 1;   // whole chunks [first, end)
    const char* src = reinterpret_cast<const char*>(pa);
    char* dst = reinterpret_cast<char*>(raw);
    for (int c = first_whole + static_cast<int>(threadIdx.x); c < end_whole; c += blockDim.x)
        cp_async16(dst + 16 * c, src + 16 * c);
    // ragged first and last chunk, element by element
    if (threadIdx.x == 0 && first_whole == 1) copy_partial_chunk(pa, 0, p, pend, raw);
    if (threadIdx.x == blockDim.x - 1 && end_whole < nchunks && !(nchunks == 1 && first_whole == 1))
        copy_partial_chunk(pa, nchunks - 1, p, pend, raw);
    cp_async_commit();
    return off;
}

}  // namespace cg
