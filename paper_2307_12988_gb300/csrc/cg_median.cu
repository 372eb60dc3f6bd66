// cg_median.cu -- the paper's initial centre: a 7x7 median filter over the
// time x tooth image of a batch of spectra, then the lowest filtered value of
// each row ("Data Capture and Processing", initial-value paragraph; Fig. 3c).
//
// Image y[i][k]: frame i of the call (time order), tooth k; edges mirrored
// without repeating the edge sample's neighbour (index -1 -> 0, n -> n - 1,
// repeated for images smaller than the footprint); median = 25th smallest of
// the 49 values; ties in the row minimum go to the lowest tooth.  The centre
// written is x_k + shift (shift = q gamma for the Fano profile, whose minimum
// lies that far below its centre; 0 for the Lorentzian).
//
// Only the argmin of each filtered row is needed, so the kernel filters
// exactly only where the minimum can be.  Per block, R consecutive rows:
//   1. the (R + 6) x (T + 6) tile of y (mirrored rows and teeth) goes to
//      shared memory, so that no window needs an index mapping;
//   2. the median of each 7-row column segment (a pruned sorting network);
//   3. per row, bounds of each window's median: L(k) = min, U(k) = max of the
//      window's 7 column medians (at most 21 of the 49 values lie below the
//      smallest column median, at most 21 above the largest); windows with
//      L(k) <= min_k U(k) are candidates (about 12 of 99 at the paper rate);
//   4. the exact median t of the window of least U (sort its 7 columns, then
//      its 7 rows -- the matrix stays sorted both ways --, drop the 10
//      elements with more than 25 elements above or below them by position,
//      select the 15th smallest of the 29 left by forgetful selection);
//   5. every candidate is compared with t by counting its values below and
//      at or below t: a median below t (rare) is computed exactly and
//      competes by a 64-bit (value, tooth) atomicMin, a median equal to t
//      keeps its tooth by atomicMin; with no median below t, the first tooth
//      whose median equals t is the row's minimum;
//   6. c0 of each row into params[i][0].
// Every selection moves values without arithmetic, so the result is an
// element of the window, equal to the definition's.
#include <cstdint>
#include <cuda_runtime.h>

#include "cg_internal.h"

namespace cg {

namespace {

constexpr int kMedThreads = 256;
constexpr int kMaxKPerLane = 16;   // windows per lane in the bounds pass: T <= 512

__device__ __forceinline__ void cmpx(float& a, float& b)
{
    const float lo = fminf(a, b);
    b = fmaxf(a, b);
    a = lo;
}

// ascending sort of 7 values: 16 comparators in 6 layers (checked exhaustively
// on the 128 binary inputs, which suffices for a comparator network)
__device__ __forceinline__ void sort7(float (&v)[7])
{
    cmpx(v[0], v[6]); cmpx(v[2], v[3]); cmpx(v[4], v[5]);
    cmpx(v[0], v[2]); cmpx(v[1], v[4]); cmpx(v[3], v[6]);
    cmpx(v[0], v[1]); cmpx(v[2], v[5]); cmpx(v[3], v[4]);
    cmpx(v[1], v[2]); cmpx(v[4], v[6]);
    cmpx(v[2], v[3]); cmpx(v[4], v[5]);
    cmpx(v[1], v[2]); cmpx(v[3], v[4]); cmpx(v[5], v[6]);
}

// median of 7 values: the sorting network above pruned to the comparators
// that reach the middle output, each keeping only the outputs used later
// (22 min/max operations instead of 32; checked on the 128 binary inputs)
__device__ __forceinline__ float median7(float (&v)[7])
{
    cmpx(v[0], v[6]); cmpx(v[2], v[3]); cmpx(v[4], v[5]);
    cmpx(v[0], v[2]); cmpx(v[1], v[4]); cmpx(v[3], v[6]);
    v[1] = fmaxf(v[0], v[1]); cmpx(v[2], v[5]); cmpx(v[3], v[4]);
    v[2] = fmaxf(v[1], v[2]); v[4] = fminf(v[4], v[6]);
    v[3] = fmaxf(v[2], v[3]); v[4] = fminf(v[4], v[5]);
    return fminf(v[3], v[4]);
}

// median of N = 2M + 1 values by forgetful selection: the buffer v[t .. M+2)
// loses its minimum (to v[t]) and maximum (to v[M+1]) each step and takes the
// next input into v[M+1]; fully unrolled, so v stays in registers
template <int N>
__device__ __forceinline__ float forgetful_median(float (&v)[N])
{
    constexpr int M = N / 2;
#pragma unroll
    for (int t = 0; t < M - 1; ++t) {
        const int b = M + 2 - t;
#pragma unroll
        for (int i = 1; i < b; ++i) cmpx(v[t], v[t + i]);
#pragma unroll
        for (int i = 1; i < b - 1; ++i) cmpx(v[t + i], v[M + 1]);
        v[M + 1] = v[M + 2 + t];
    }
    cmpx(v[M - 1], v[M]);
    cmpx(v[M], v[M + 1]);
    cmpx(v[M - 1], v[M]);
    return v[M];
}

// mirrored index for i in [-3, n + 3): reflections until it lies in [0, n)
// (one for n >= 3; images smaller than the footprint take a few more)
__device__ __forceinline__ int mirror(int i, int n)
{
#pragma unroll 1
    for (int it = 0; it < 8 && (i < 0 || i >= n); ++it) i = i < 0 ? -1 - i : 2 * n - 1 - i;
    return i;
}

__device__ __forceinline__ int64_t mirror64(int64_t i, int64_t n)
{
#pragma unroll 1
    for (int it = 0; it < 8 && (i < 0 || i >= n); ++it) i = i < 0 ? -1 - i : 2 * n - 1 - i;
    return i;
}

// order-preserving map of a float onto unsigned integers
__device__ __forceinline__ uint32_t ord(float f)
{
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// exact median of the window whose top-left tile element is (r, k): the tile
// holds 3 mirrored columns on either side, so window k spans columns k..k+6
__device__ __forceinline__ float window_median(const float* tile, int S, int r, int k)
{
    float m[7][7];   // m[c][j]: column c, row j
#pragma unroll
    for (int c = 0; c < 7; ++c) {
#pragma unroll
        for (int j = 0; j < 7; ++j) m[c][j] = tile[(r + j) * S + k + c];
        sort7(m[c]);
    }
#pragma unroll
    for (int j = 0; j < 7; ++j) {
        float row[7];
#pragma unroll
        for (int c = 0; c < 7; ++c) row[c] = m[c][j];
        sort7(row);
#pragma unroll
        for (int c = 0; c < 7; ++c) m[c][j] = row[c];
    }
    // positions (j, c) with at most 24 elements certainly below and above
    float v[29];
    int q = 0;
#pragma unroll
    for (int j = 0; j < 7; ++j)
#pragma unroll
        for (int c = 0; c < 7; ++c)
            if ((j + 1) * (c + 1) <= 25 && (7 - j) * (7 - c) <= 25) v[q++] = m[c][j];
    return forgetful_median<29>(v);
}

__global__ void __launch_bounds__(kMedThreads) median_init_kernel(MedianArgs a)
{
    extern __shared__ __align__(16) unsigned char msm[];
    const int R = a.R, T = a.T, S = a.S;
    const int64_t n = a.n;
    const int W = T + 6;                                               // padded columns
    float* tile = reinterpret_cast<float*>(msm);                       // [R + 6][S], column j = tooth j - 3
    float* cm = tile + (R + 6) * S;                                    // [R][S]
    int* list = reinterpret_cast<int*>(cm + R * S);                    // [R T]
    unsigned long long* key = reinterpret_cast<unsigned long long*>(msm + a.sm_key);   // [R]
    int* count = reinterpret_cast<int*>(key + R);
    int* ka = count + 4;                                               // [R] first window of least U
    float* tq = reinterpret_cast<float*>(ka + R);                      // [R] its exact median
    int* tie = reinterpret_cast<int*>(tq + R);                         // [R] first window with median = tq
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    constexpr int kWarps = kMedThreads / 32;
    for (int64_t b = blockIdx.x; b * R < n; b += gridDim.x) {
        const int64_t i0 = b * R;
        const int rows = static_cast<int>((n - i0) < R ? (n - i0) : R);
        // 1. the tile: rows i0 - 3 .. i0 + rows + 2 and teeth -3 .. T + 2, mirrored
        for (int t = warp; t < rows + 6; t += kWarps) {
            const int64_t row = mirror64(i0 - 3 + t, n);
            const float* src = a.y ? a.y + row * T : a.amps + row * T;
            for (int j = lane; j < W; j += 32) {
                const int k = mirror(j - 3, T);
                tile[t * S + j] = a.y ? src[k] : __fmul_rn(src[k], a.inv_ref[k]);
            }
        }
        if (tid < R) {
            key[tid] = ~0ull;
            tie[tid] = 0x7fffffff;
        }
        if (tid == 0) *count = 0;
        __syncthreads();
        // 2. medians of the 7-row column segments
        for (int r = warp; r < rows; r += kWarps)
            for (int j = lane; j < W; j += 32) {
                float v[7];
#pragma unroll
                for (int q = 0; q < 7; ++q) v[q] = tile[(r + q) * S + j];
                cm[r * S + j] = median7(v);
            }
        __syncthreads();
        // 3. per row (one warp): bounds and the candidate windows
        for (int r = warp; r < rows; r += kWarps) {
            const float* cr = cm + r * S;
            float ustar = INFINITY;
            int kbest = 0x7fffffff;
            float lo[kMaxKPerLane];                // L(k) of this lane's windows
#pragma unroll
            for (int q = 0; q < kMaxKPerLane; ++q) {
                const int k = lane + 32 * q;
                lo[q] = INFINITY;
                if (k < T) {
                    float l = cr[k], hi = cr[k];
#pragma unroll
                    for (int d = 1; d < 7; ++d) {
                        l = fminf(l, cr[k + d]);
                        hi = fmaxf(hi, cr[k + d]);
                    }
                    lo[q] = l;
                    if (hi < ustar) {
                        ustar = hi;
                        kbest = k;
                    }
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float uo = __shfl_xor_sync(0xffffffffu, ustar, o);
                const int ko = __shfl_xor_sync(0xffffffffu, kbest, o);
                if (uo < ustar || (uo == ustar && ko < kbest)) {
                    ustar = uo;
                    kbest = ko;
                }
            }
            if (lane == 0) ka[r] = kbest < T ? kbest : 0;
#pragma unroll
            for (int q = 0; q < kMaxKPerLane; ++q) {
                const int k = lane + 32 * q;
                if (32 * q >= T) break;
                const bool cand = k < T && !(lo[q] > ustar);   // (non-finite rows keep every window)
                const unsigned bal = __ballot_sync(0xffffffffu, cand);
                int base = 0;
                if (lane == 0 && bal) base = atomicAdd(count, __popc(bal));
                base = __shfl_sync(0xffffffffu, base, 0);
                if (cand) list[base + __popc(bal & ((1u << lane) - 1u))] = (r << 16) | k;
            }
        }
        __syncthreads();
        // 4. the exact median t of each row's window of least U (an upper
        //    bound of the row minimum)
        if (tid < rows) tq[tid] = window_median(tile, S, tid, ka[tid]);
        __syncthreads();
        // 5. each candidate against t by counting: 25 or more values below t
        //    means a median below t (its exact median then competes by the
        //    (value, tooth) key); otherwise 25 or more values at or below t
        //    means a median equal to t (the first such tooth is kept).  With
        //    no median below t the minimum is t itself.
        const int nc = *count;
        for (int e = tid; e < nc; e += kMedThreads) {
            const int it = list[e];
            const int r = it >> 16, k = it & 0xffff;
            const float t = tq[r];
            int lt = 0, le = 0;
#pragma unroll
            for (int c = 0; c < 7; ++c)
#pragma unroll
                for (int j = 0; j < 7; ++j) {
                    const float v = tile[(r + j) * S + k + c];
                    lt += v < t ? 1 : 0;
                    le += v <= t ? 1 : 0;
                }
            if (lt >= 25) {
                const float med = window_median(tile, S, r, k);
                atomicMin(&key[r], (static_cast<unsigned long long>(ord(med)) << 32) | static_cast<unsigned>(k));
            } else if (le >= 25) {
                atomicMin(&tie[r], k);
            }
        }
        __syncthreads();
        // 6. the initial centres
        if (tid < rows) {
            const unsigned long long kv = key[tid];
            const unsigned kk = kv != ~0ull ? static_cast<unsigned>(kv & 0xffffffffull) : static_cast<unsigned>(tie[tid]);
            const int k = kk < static_cast<unsigned>(T) ? static_cast<int>(kk) : 0;
            a.params[(i0 + tid) * 4] = a.cx[k];
        }
        __syncthreads();
    }
}

}  // namespace

// Rows per block (32, 16, 8 or 4: the most whose tables fit in 100 KB of
// shared memory), the layout and the grid.
cudaError_t setup_median(cg_plan_s* p)
{
    p->median_ok = false;
    const int T = p->T;
    if (T > 32 * kMaxKPerLane) return cudaSuccess;
    const int S = (T + 6) | 1;
    MedianArgs& m = p->med;
    m = MedianArgs{};
    m.T = T;
    m.S = S;
    int R = 32;
    auto bytes = [&](int r) {
        const size_t tables = sizeof(float) * (static_cast<size_t>(r + 6) * S + static_cast<size_t>(r) * S) +
                              sizeof(int) * static_cast<size_t>(r) * T;
        return ((tables + 15) & ~static_cast<size_t>(15)) + 8 * r + 16 + 12 * r;
    };
    while (R > 4 && bytes(R) > 100 * 1024) R /= 2;
    m.R = R;
    const size_t tables = sizeof(float) * (static_cast<size_t>(R + 6) * S + static_cast<size_t>(R) * S) +
                          sizeof(int) * static_cast<size_t>(R) * T;
    m.sm_key = static_cast<int>((tables + 15) & ~static_cast<size_t>(15));
    m.sm_total = static_cast<int>(bytes(R));
    cudaError_t e;
    void* fn = reinterpret_cast<void*>(&median_init_kernel);
    if ((e = raise_smem_limit(fn, m.sm_total)) != cudaSuccess) return e;
    int occ = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kMedThreads, m.sm_total)) != cudaSuccess)
        return e;
    if (occ < 1) return cudaSuccess;
    p->grid_median = p->num_sms * occ;
    p->median_ok = true;
    return cudaSuccess;
}

cudaError_t launch_median(const cg_plan_s* p, const float* y, const float* amps, int64_t n, float* params,
                          cudaStream_t s)
{
    MedianArgs m = p->med;
    m.n = n;
    m.y = y;
    m.amps = amps;
    m.inv_ref = p->d.inv_ref;
    m.cx = p->d.median_cx;
    m.params = params;
    const int64_t nb = (n + m.R - 1) / m.R;
    const int grid = static_cast<int>(nb < p->grid_median ? nb : p->grid_median);
    void* args[] = {&m};
    return cudaLaunchKernel(reinterpret_cast<void*>(&median_init_kernel), dim3(grid), dim3(kMedThreads), args,
                            m.sm_total, s);
}

}  // namespace cg
