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
//      its 7 rows -- the matrix stays sorted both ways --, drop the 20
//      elements with 25 or more elements certainly above or below them by
//      position, select the 15th smallest of the 29 left with a merge
//      network pruned to that output);
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
#include "cg_net.cuh"
#include "cg_stage.cuh"

namespace cg {

namespace {

constexpr int kMedThreads = 256;
constexpr int kMaxTeeth = 512;     // 16 windows on each of 32 lanes in the bounds pass

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
    // positions (j, c) with at most 24 elements certainly below and above;
    // the 15th smallest of these 29 by the rank-pruned merge network (depth
    // <= 15, where a forgetful selection is a chain of ~440 dependent steps)
    float v[32];
    int q = 0;
#pragma unroll
    for (int j = 0; j < 7; ++j)
#pragma unroll
        for (int c = 0; c < 7; ++c)
            if ((j + 1) * (c + 1) <= 25 && (7 - j) * (7 - c) <= 25) v[q++] = m[c][j];
    v[29] = v[30] = v[31] = INFINITY;
    return rank_select<32, 29, 14>(v);
}

// LPR: lanes per row in the bounds pass, 16 windows each (T <= 16 LPR)
template <int LPR>
__global__ void __launch_bounds__(kMedThreads, 4) median_init_kernel(MedianArgs a)
{
    extern __shared__ __align__(16) unsigned char msm[];
    const int R = a.R, T = a.T, S = a.S;
    const int64_t n = a.n;
    const int W = T + 6;                                               // padded columns
    float* tile = reinterpret_cast<float*>(msm);                       // [R + 6][S], column j = tooth j - 3
    float* cm = tile + (R + 6) * S;                                    // [R][S]
    uint16_t* list = reinterpret_cast<uint16_t*>(cm + R * S);          // [R T]: (row << 9) | tooth
    unsigned long long* key = reinterpret_cast<unsigned long long*>(msm + a.sm_key);   // [R]
    int* count = reinterpret_cast<int*>(key + R);
    int* ka = count + 4;                                               // [R] first window of least U
    float* tq = reinterpret_cast<float*>(ka + R);                      // [R] its exact median
    int* tie = reinterpret_cast<int*>(tq + R);                         // [R] first window with median = tq
    int* mir = tie + R;                                                // [W] tooth of padded column j
    float* iref = reinterpret_cast<float*>(mir + W);                   // [T] 1 / reference
    float* raw = reinterpret_cast<float*>(msm + a.sm_raw);             // [(R + 6) T + 4] staged rows
    const float* src = a.y ? a.y : a.amps;
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    constexpr int kWarps = kMedThreads / 32;
    constexpr int kRPW = 32 / LPR;                                     // rows per warp in the bounds pass
    for (int j = tid; j < W; j += kMedThreads) mir[j] = mirror(j - 3, T);
    for (int k = tid; k < T; k += kMedThreads) iref[k] = a.y ? 1.0f : a.inv_ref[k];
    // the rows a block needs, [rlo, rhi): its own and 3 on either side, within
    // the image (mirrored rows are among them); staged by asynchronous 16-byte
    // copies, the next block's while the current one is filtered
    auto row_range = [&](int64_t bb, int64_t& rlo, int64_t& rhi) {
        const int64_t j0 = bb * R;
        const int64_t j1 = j0 + R < n ? j0 + R : n;
        rlo = j0 - 3 > 0 ? j0 - 3 : 0;
        rhi = j1 + 3 < n ? j1 + 3 : n;
    };
    int off = 0;
    if (static_cast<int64_t>(blockIdx.x) * R < n) {
        int64_t rlo, rhi;
        row_range(blockIdx.x, rlo, rhi);
        off = stage_async(src, rlo * T, (rhi - rlo) * T, raw);
    }
    __syncthreads();
    for (int64_t b = blockIdx.x; b * R < n; b += gridDim.x) {
        const int64_t i0 = b * R;
        const int rows = static_cast<int>((n - i0) < R ? (n - i0) : R);
        int64_t rlo, rhi;
        row_range(b, rlo, rhi);
        cp_async_wait_all();
        __syncthreads();
        // 1. the tile: rows i0 - 3 .. i0 + rows + 2 and teeth -3 .. T + 2,
        //    mirrored, normalised (x 1 when y is given: exact)
        for (int t = warp; t < rows + 6; t += kWarps) {
            const float* rr = raw + off + (mirror64(i0 - 3 + t, n) - rlo) * T;
            for (int j = lane; j < W; j += 32) {
                const int k = mir[j];
                tile[t * S + j] = __fmul_rn(rr[k], iref[k]);
            }
        }
        __syncthreads();
        // the staged rows are in the tile: the next block's rows go to raw
        {
            const int64_t bn = b + gridDim.x;
            if (bn * R < n) {
                int64_t nlo, nhi;
                row_range(bn, nlo, nhi);
                off = stage_async(src, nlo * T, (nhi - nlo) * T, raw);
            }
        }
        if (tid < R) {
            key[tid] = ~0ull;
            tie[tid] = 0x7fffffff;
        }
        if (tid == 0) *count = 0;
        __syncthreads();
        // 2. medians of the 7-row column segments: one thread per column and
        //    16 consecutive rows loads the column's 22 values once.  Two
        //    adjacent segments share 6 values: with s2 <= s3 their 3rd and 4th
        //    smallest, the median of the 6 and one more value x is
        //    min(max(x, s2), s3), so a pair costs one pruned 6-input selection
        //    and 4 operations
        for (int idx = tid; idx < W * ((rows + 15) / 16); idx += kMedThreads) {
            const int h = idx / W;
            const int j = idx - h * W;
            const int r0 = 16 * h;
            const int nr = rows - r0 < 16 ? rows - r0 : 16;
            float col[22];
#pragma unroll
            for (int q = 0; q < 22; ++q) col[q] = q < nr + 6 ? tile[(r0 + q) * S + j] : 0.f;
#pragma unroll
            for (int rr = 0; rr < 16; rr += 2) {
                if (rr + 1 < nr) {
                    float v[8];
#pragma unroll
                    for (int q = 0; q < 6; ++q) v[q] = col[rr + 1 + q];
                    rank_network<8, 6, 2, 3>(v);
                    cm[(r0 + rr) * S + j] = fminf(fmaxf(col[rr], v[2]), v[3]);
                    cm[(r0 + rr + 1) * S + j] = fminf(fmaxf(col[rr + 7], v[2]), v[3]);
                } else if (rr < nr) {
                    float v[7];
#pragma unroll
                    for (int q = 0; q < 7; ++q) v[q] = col[rr + q];
                    cm[(r0 + rr) * S + j] = median7(v);
                }
            }
        }
        __syncthreads();
        // 3. bounds and the candidate windows: LPR lanes per row, lane part p
        //    takes the 16 consecutive windows k0 = 16 p .. k0 + 15, which span
        //    the column medians c[k0 .. k0 + 21]; windows in fours share
        //    their middle four values (and pairs of the others), 3.25 min or
        //    max operations a window.  Pass 1: U and the row's least U (first
        //    window on ties, reduced over the row's lanes); pass 2: L and the
        //    windows with L <= U*
        for (int rg = warp * kRPW; rg < rows; rg += kWarps * kRPW) {   // (uniform over the warp)
            const int r = rg + lane / LPR;
            const int k0 = 16 * (lane % LPR);
            const bool rv = r < rows;
            const float* cr = cm + (rv ? r : 0) * S;
            float c[22];
#pragma unroll
            for (int q = 0; q < 22; ++q) c[q] = (rv && k0 + q < W) ? cr[k0 + q] : 0.f;
            float ustar = INFINITY;
            int kbest = 0x7fffffff;
#pragma unroll
            for (int g = 0; g < 16; g += 4) {
                const float m4 = fmaxf(fmaxf(c[g + 3], c[g + 4]), fmaxf(c[g + 5], c[g + 6]));
                const float p12 = fmaxf(c[g + 1], c[g + 2]), p78 = fmaxf(c[g + 7], c[g + 8]);
                const float u4[4] = {fmaxf(m4, fmaxf(c[g], p12)), fmaxf(m4, fmaxf(p12, c[g + 7])),
                                     fmaxf(m4, fmaxf(c[g + 2], p78)), fmaxf(m4, fmaxf(p78, c[g + 9]))};
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (rv && k0 + g + j < T && u4[j] < ustar) {
                        ustar = u4[j];
                        kbest = k0 + g + j;
                    }
            }
#pragma unroll
            for (int o = LPR / 2; o > 0; o >>= 1) {
                const float uo = __shfl_xor_sync(0xffffffffu, ustar, o);
                const int ko = __shfl_xor_sync(0xffffffffu, kbest, o);
                if (uo < ustar || (uo == ustar && ko < kbest)) {
                    ustar = uo;
                    kbest = ko;
                }
            }
            if (rv && k0 == 0) ka[r] = kbest < T ? kbest : 0;
            unsigned cand = 0;                     // bit q: window k0 + q
#pragma unroll
            for (int g = 0; g < 16; g += 4) {
                const float m4 = fminf(fminf(c[g + 3], c[g + 4]), fminf(c[g + 5], c[g + 6]));
                const float p12 = fminf(c[g + 1], c[g + 2]), p78 = fminf(c[g + 7], c[g + 8]);
                const float l4[4] = {fminf(m4, fminf(c[g], p12)), fminf(m4, fminf(p12, c[g + 7])),
                                     fminf(m4, fminf(c[g + 2], p78)), fminf(m4, fminf(p78, c[g + 9]))};
#pragma unroll
                for (int j = 0; j < 4; ++j)   // (non-finite rows keep every window)
                    if (rv && k0 + g + j < T && !(l4[j] > ustar)) cand |= 1u << (g + j);
            }
            const int mine = __popc(cand);
            int incl = mine;                       // inclusive prefix sum over the warp
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            const int total = __shfl_sync(0xffffffffu, incl, 31);
            int base = 0;
            if (lane == 0 && total > 0) base = atomicAdd(count, total);
            base = __shfl_sync(0xffffffffu, base, 0) + incl - mine;
            while (cand) {
                const int q = __ffs(cand) - 1;
                cand &= cand - 1;
                list[base++] = static_cast<uint16_t>((r << 9) | (k0 + q));
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
            const int r = it >> 9, k = it & 0x1ff;
            const float t = tq[r];
            // L(k) > t: the window's median exceeds t (no count needed)
            const float* cr = cm + r * S + k;
            float l = cr[0];
#pragma unroll
            for (int d = 1; d < 7; ++d) l = fminf(l, cr[d]);
            if (l > t) continue;
            // at or below t first: fewer than 25 means a median above t,
            // the usual case; only the others count the values below t
            int le = 0;
#pragma unroll
            for (int c = 0; c < 7; ++c)
#pragma unroll
                for (int j = 0; j < 7; ++j) le += tile[(r + j) * S + k + c] <= t ? 1 : 0;
            if (le < 25) continue;
            int lt = 0;
#pragma unroll
            for (int c = 0; c < 7; ++c)
#pragma unroll
                for (int j = 0; j < 7; ++j) lt += tile[(r + j) * S + k + c] < t ? 1 : 0;
            if (lt >= 25) {
                const float med = window_median(tile, S, r, k);
                atomicMin(&key[r], (static_cast<unsigned long long>(ord(med)) << 32) | static_cast<unsigned>(k));
            } else {
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

static void* median_fn(int T)
{
    if (T <= 128) return reinterpret_cast<void*>(&median_init_kernel<8>);
    if (T <= 256) return reinterpret_cast<void*>(&median_init_kernel<16>);
    return reinterpret_cast<void*>(&median_init_kernel<32>);
}

// Rows per block (32, 16, 8 or 4: the most whose tables fit in 100 KB of
// shared memory), the layout and the grid.
cudaError_t setup_median(cg_plan_s* p)
{
    p->median_ok = false;
    const int T = p->T;
    if (T > kMaxTeeth) return cudaSuccess;
    const int S = (T + 6) | 1;
    MedianArgs& m = p->med;
    m = MedianArgs{};
    m.T = T;
    m.S = S;
    int R = 32;
    auto bytes = [&](int r) {
        const size_t tables = sizeof(float) * (static_cast<size_t>(r + 6) * S + static_cast<size_t>(r) * S) +
                              sizeof(uint16_t) * static_cast<size_t>(r) * T;
        const size_t rest = ((tables + 15) & ~static_cast<size_t>(15)) + 8 * r + 16 + 12 * r + 4 * (T + 6) + 4 * T;
        const size_t raw = sizeof(float) * ((static_cast<size_t>(r + 6) * T + 4 + 3) & ~static_cast<size_t>(3));
        return ((rest + 15) & ~static_cast<size_t>(15)) + raw;
    };
    while (R > 4 && bytes(R) > 100 * 1024) R /= 2;
    m.R = R;
    const size_t tables = sizeof(float) * (static_cast<size_t>(R + 6) * S + static_cast<size_t>(R) * S) +
                          sizeof(uint16_t) * static_cast<size_t>(R) * T;
    m.sm_key = static_cast<int>((tables + 15) & ~static_cast<size_t>(15));
    {
        const size_t rest = static_cast<size_t>(m.sm_key) + 8 * R + 16 + 12 * R + 4 * (T + 6) + 4 * T;
        m.sm_raw = static_cast<int>((rest + 15) & ~static_cast<size_t>(15));
    }
    m.sm_total = static_cast<int>(bytes(R));
    cudaError_t e;
    void* fn = median_fn(T);
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
    return cudaLaunchKernel(median_fn(m.T), dim3(grid), dim3(kMedThreads), args, m.sm_total, s);
}

}  // namespace cg
