// cg_mlp_tc.cu -- inference of the learned initial guess on the tensor cores.
//
// For 128 normalised spectra at a time (one MMA M tile):
//     x = (y - in_mean) * in_scale                         (FP32, then BF16)
//     a1 = gelu(W1 x + b1),  a2 = gelu(W2 a1 + b2)          (BF16 x BF16 -> FP32 in TMEM)
//     p0 = (W3 a2 + b3) * out_scale + out_mean              (FP32 on the CUDA cores)
// with W1 (K zero-padded to 64 * nkb) and W2 stored as one BF16 matrix
// [512][256], streamed from L2 by TMA in 128-row x 64-column chunks through an
// S-stage mbarrier ring.  Persistent blocks, one per SM, with warp roles:
//   warps 0-7    epilogues: warp w reads TMEM lanes 32 (w % 4).. (rows) and
//                column half w / 4; layer 1: bias, GELU, BF16 into the a1
//                tile; layer 2: bias, GELU and the FP32 output layer;
//   warps 8-15   stage the next tile's spectra as BF16 into the input tile
//                (free again once the layer-1 products of the current tile
//                have read it);
//   warp 16      owns TMEM (layer-1 accumulator in columns 0-255, layer-2 in
//                256-511) and issues tcgen05.mma from one lane;
//   warp 17      issues the weight-chunk TMA loads from one lane.
// So the staging of tile t+1, the products of one layer and the epilogue of
// the other overlap.  The input and a1 tiles are K-major 128-byte-swizzled as
// the MMA reads them.  Every wait is bounded; on time-out the block records
// an error, stops issuing, drains its loads and frees its TMEM.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include "cg_internal.h"
#include "cg_tc.cuh"

namespace cg {

namespace {

constexpr int kMM = 128;                        // spectra per tile
constexpr int kHid = 256;                       // hidden width
constexpr int kChunkRows = 128;                 // weight rows per chunk (MMA N)
constexpr int kChunkBytes = kChunkRows * 64 * 2;
constexpr int kABytes = 4 * kMM * 64 * 2;       // one operand tile: 4 K blocks of 64
constexpr int kStagesMax = 6;
constexpr int kEpiWarps = 8;                    // epilogue warps (2 per TMEM lane quarter)
constexpr int kStageWarps = 8;                  // input staging warps
constexpr int kIssueWarp = kEpiWarps + kStageWarps;
constexpr int kLoadWarp = kIssueWarp + 1;
constexpr int kMlpThreads = (kLoadWarp + 1) * 32;
constexpr uint32_t kPolls = 1u << 22;
constexpr int kSlice = 16;                      // input rows per bulk copy
constexpr int kRawBytes = 2 * kSlice * 256 * 4; // two slices of up to 256 teeth

__device__ __forceinline__ bool wait_or_abort(uint64_t* bar, uint32_t parity, volatile int* abort_flag)
{
    const uint64_t t0 = tc::globaltimer_ns();
    for (uint32_t i = 0; i < kPolls; ++i) {
        if (tc::mbar_try_wait(bar, parity)) return true;
        if ((i & 255u) == 255u && (*abort_flag || tc::globaltimer_ns() - t0 > tc::kWaitLimitNs)) return false;
    }
    return false;
}

// GELU in its tanh form, evaluated as z / (1 + exp(-2 k (z + c z^3))), since
// 0.5 (1 + tanh(v)) = 1 / (1 + exp(-2 v)).  Unlike 1 + tanh, which cancels
// for negative z (an absolute tanh error of 2^-11 there shifted the trained
// network's outputs by 7 % of their scale), the quotient keeps its relative
// accuracy over the whole range; exp(+large) = inf gives the limit 0.
__device__ __forceinline__ float gelu_fast(float z)
{
    const float v = fmaf(0.044715f * z * z, z, z);
    float e;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(-2.0f * 0.7978845608028654f * 1.4426950408889634f * v));
    return __fdividef(z, 1.0f + e);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&h);
}

// GELU of two pre-activations as the BF16 pair the next layer's MMA reads.
__device__ __forceinline__ uint32_t gelu_bf16x2(float z0, float z1)
{
    return pack_bf16(gelu_fast(z0), gelu_fast(z1));
}

// byte offset of BF16 element (row, k) in a swizzled operand tile
__device__ __forceinline__ uint32_t a_off(int row, int k)
{
    const int kl = k & 63;
    return static_cast<uint32_t>((k >> 6) * (kMM * 128) + row * 128 + ((((kl >> 3) ^ (row & 7))) << 4) +
                                 ((kl & 7) << 1));
}

__global__ void __launch_bounds__(kMlpThreads, 1) mlp_infer_kernel(const __grid_constant__ CUtensorMap tmW, MlpArgs a)
{
    extern __shared__ __align__(1024) unsigned char msm_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(msm_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    unsigned char* Ain = sm;                       // staged input tile
    unsigned char* Ah = sm + kABytes;              // a1 tile
    float* raw = reinterpret_cast<float*>(sm + 2 * kABytes);        // [2][16][T] input rows as read
    unsigned char* Wst = sm + 2 * kABytes + kRawBytes;             // weight ring
    const int S = a.stages;
    const int T = a.T, nkb = a.nkb;
    // FP32 tables derived from the plan's: biases, the output layer
    // transposed (one 16-byte load per hidden unit) and per tooth
    // {1/ref (or 1 for y input), in_mean, in_scale, 0}
    float* b1s = reinterpret_cast<float*>(Wst + S * kChunkBytes);   // [256]
    float* b2s = b1s + kHid;                                         // [256]
    float4* w3t = reinterpret_cast<float4*>(b2s + kHid);            // [256]
    float* outs = reinterpret_cast<float*>(w3t + kHid);              // b3[4], out_mean[4], out_scale[4], pad
    float4* tooth = reinterpret_cast<float4*>(outs + 16);            // [T]
    float* red = reinterpret_cast<float*>(tooth + T);                // [2][128][4] output partials
    uint64_t* full = reinterpret_cast<uint64_t*>(red + 2 * kMM * 4);
    uint64_t* empty = full + kStagesMax;
    uint64_t* bars = empty + kStagesMax;
    uint64_t* a_full = bars + 0;      // input tile staged (staging threads)
    uint64_t* a_empty = bars + 1;     // layer-1 products done reading it (commit)
    uint64_t* acc1_full = bars + 2;   // layer-1 accumulator complete (commit)
    uint64_t* a1_full = bars + 3;     // a1 written, layer-1 accumulator read (epilogue threads)
    uint64_t* acc2_full = bars + 4;   // layer-2 accumulator complete (commit)
    uint64_t* acc2_empty = bars + 5;  // layer-2 accumulator read (epilogue threads)
    uint64_t* done = bars + 6;        // every product issued has completed
    uint64_t* red_full = bars + 7;    // [2] half 1's output partials written (128 threads)
    uint64_t* red_empty = bars + 9;   // [2] half 0 has read them (128 threads)
    uint64_t* raw_full = bars + 11;   // [2] a 16-row slice landed (bulk copy)
    uint64_t* raw_empty = bars + 13;  // [2] the slice was converted (staging threads)
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 15);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t ntiles = (a.n + kMM - 1) / kMM;
    const int my_tiles =
        static_cast<int64_t>(blockIdx.x) < ntiles ? static_cast<int>((ntiles - 1 - blockIdx.x) / gridDim.x) + 1 : 0;
    auto tile_f0 = [&](int it) { return (static_cast<int64_t>(blockIdx.x) + static_cast<int64_t>(it) * gridDim.x) * kMM; };
    const int n1 = 2 * nkb;      // layer-1 chunks: column half-major, K blocks within
    const int nch = n1 + 8;      // + layer-2 chunks, per tile
    for (int i = tid; i < kHid; i += blockDim.x) {
        b1s[i] = a.tab[kMlpTabB1 + i];
        b2s[i] = a.tab[kMlpTabB2 + i];
        w3t[i] = make_float4(a.tab[kMlpTabW3 + i], a.tab[kMlpTabW3 + kHid + i], a.tab[kMlpTabW3 + 2 * kHid + i],
                             a.tab[kMlpTabW3 + 3 * kHid + i]);
    }
    if (tid < 4) {
        outs[tid] = a.tab[kMlpTabB3 + tid];
        outs[4 + tid] = a.tab[kMlpTabOutMean + tid];
        outs[8 + tid] = a.tab[kMlpTabOutScale + tid];
    }
    for (int k = tid; k < T; k += blockDim.x)
        tooth[k] = make_float4(a.y ? 1.0f : a.inv_ref[k], a.tab[kMlpTabIn + k], a.tab[kMlpTabIn + T + k], 0.f);

    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        tc::mbar_init(a_full, kStageWarps * 32);
        tc::mbar_init(a_empty, 1);
        tc::mbar_init(acc1_full, 1);
        tc::mbar_init(a1_full, kEpiWarps * 32);
        tc::mbar_init(acc2_full, 1);
        tc::mbar_init(acc2_empty, kEpiWarps * 32);
        tc::mbar_init(done, 1);
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(&red_full[b], kMM);
            tc::mbar_init(&red_empty[b], kMM);
            tc::mbar_init(&raw_full[b], 1);
            tc::mbar_init(&raw_empty[b], kStageWarps * 32);
        }
        *abort_flag = 0;
        tc::fence_mbar_init();
    }
    if (warp == kIssueWarp) tc::tmem_alloc(tmem_slot, 2 * kHid);
    if (warp == kLoadWarp && lane == 0) tc::prefetch_tmap(&tmW);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    // chunk c of a tile -> layer, column half and K block
    auto chunk_geom = [&](int c, int& layer, int& nh, int& kb) {
        const int per = c < n1 ? nkb : 4;
        const int h = c < n1 ? c : c - n1;
        layer = c < n1 ? 0 : 1;
        nh = h / per;
        kb = h - nh * per;
    };

    if (warp == kLoadWarp) {
        // ---------------- weight chunks by TMA ----------------
        if (lane == 0) {
            int g = 0;
            bool ok = true;
            for (int it = 0; ok && it < my_tiles; ++it) {
                for (int c = 0; c < nch; ++c, ++g) {
                    const int s = g % S;
                    if (g >= S && !wait_or_abort(&empty[s], ((g / S) & 1u) ^ 1u, abort_flag)) {
                        *abort_flag = 1;
                        ok = false;
                        break;
                    }
                    int layer, nh, kb;
                    chunk_geom(c, layer, nh, kb);
                    tc::mbar_arrive_expect_tx(&full[s], kChunkBytes);
                    tc::tma_load_2d(Wst + s * kChunkBytes, &tmW, kb * 64, layer * kHid + nh * kChunkRows, &full[s]);
                }
            }
            // the last loads of every stage have landed before the block exits
            for (int q = g - S > 0 ? g - S : 0; q < g; ++q) (void)tc::mbar_wait(&full[q % S], (q / S) & 1u, kPolls);
        }
    } else if (warp == kIssueWarp) {
        // ---------------- MMA issue ----------------
        if (lane == 0) {
            const uint32_t idesc = tc::idesc_f16(kMM, kChunkRows, 1);
            int g = 0;
            bool ok = true;
            auto run = [&](int c0, int c1, unsigned char* A, uint32_t dcol) -> bool {
                for (int c = c0; c < c1; ++c, ++g) {
                    const int s = g % S;
                    if (!wait_or_abort(&full[s], (g / S) & 1u, abort_flag)) return false;
                    tc::tc_fence_after();
                    int layer, nh, kb;
                    chunk_geom(c, layer, nh, kb);
                    const uint32_t sa = tc::smem_u32(A) + kb * (kMM * 128);
                    const uint32_t sb = tc::smem_u32(Wst + s * kChunkBytes);
                    const uint32_t d = tmem + dcol + static_cast<uint32_t>(nh * kChunkRows);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        tc::mma_f16(d, tc::sdesc_sw128(sa + kk * 32), tc::sdesc_sw128(sb + kk * 32), idesc,
                                    (kb != 0 || kk != 0) ? 1u : 0u);
                    tc::mma_commit(&empty[s]);
                }
                return true;
            };
            for (int it = 0; ok && it < my_tiles; ++it) {
                const uint32_t ph = it & 1u;
                if (!wait_or_abort(a_full, ph, abort_flag)) { ok = false; break; }
                tc::tc_fence_after();
                if (!run(0, n1, Ain, 0)) { ok = false; break; }
                tc::mma_commit(a_empty);
                tc::mma_commit(acc1_full);
                if (!wait_or_abort(a1_full, ph, abort_flag)) { ok = false; break; }
                if (it >= 1 && !wait_or_abort(acc2_empty, ph ^ 1u, abort_flag)) { ok = false; break; }
                tc::tc_fence_after();
                if (!run(n1, nch, Ah, kHid)) { ok = false; break; }
                tc::mma_commit(acc2_full);
            }
            if (!ok) *abort_flag = 1;
            tc::mma_commit(done);   // arrives when every product issued above has completed
        }
    } else if (warp >= kEpiWarps) {
        // ---------------- input staging: (y - in_mean) * in_scale -> BF16 ----------------
        // The tile's rows arrive as 16-row slices by bulk copy into two raw
        // buffers (one slice ahead); each thread converts two (row, 8-tooth)
        // items of a slice into one 16-byte store of the swizzled tile.
        const int ls = tid - kEpiWarps * 32;          // 0 .. 255
        const bool scale_in = a.y == nullptr;
        const float* srcbase = scale_in ? a.amps : a.y;
        const int nslices = kMM / kSlice;
        const int nchunk8 = (T + 7) / 8;
        const uint32_t slice_bytes = static_cast<uint32_t>(kSlice * T * 4);
        // slice q of tile it: rows [f0 + 16 q, +16) clipped to n; a whole,
        // 16-byte-aligned slice goes by bulk copy, anything else by plain loads
        auto slice_rows = [&](int it, int q) {
            const int64_t r0 = tile_f0(it) + kSlice * q;
            const int64_t left = a.n - r0;
            return left <= 0 ? 0 : (left < kSlice ? static_cast<int>(left) : kSlice);
        };
        auto bulk_ok = [&](int it, int q) {
            const float* src = srcbase + (tile_f0(it) + kSlice * q) * T;
            return slice_rows(it, q) == kSlice && (slice_bytes & 15u) == 0 &&
                   (reinterpret_cast<uintptr_t>(src) & 15) == 0;
        };
        const int total_slices = my_tiles * nslices;
        int last_issued = -1;
        auto issue = [&](int gq) {   // by thread ls == 0
            const int it = gq / nslices, q = gq - it * nslices;
            const int b = gq & 1;
            if (gq >= 2 && !wait_or_abort(&raw_empty[b], ((gq >> 1) & 1u) ^ 1u, abort_flag)) return false;
            if (bulk_ok(it, q)) {
                tc::fence_proxy_async_smem();
                tc::mbar_arrive_expect_tx(&raw_full[b], slice_bytes);
                tc::bulk_g2s(raw + b * kSlice * 256, srcbase + (tile_f0(it) + kSlice * q) * T, slice_bytes,
                             &raw_full[b]);
            } else {
                // a slice read straight from global memory still completes its
                // phase, so no thread can run two slices ahead of the others
                tc::mbar_arrive(&raw_full[b]);
            }
            last_issued = gq;
            return true;
        };
        bool ok = true;
        if (ls == 0 && total_slices > 0) ok = issue(0);
        for (int gq = 0; ok && gq < total_slices; ++gq) {
            const int it = gq / nslices, q = gq - it * nslices;
            const int b = gq & 1;
            if (q == 0 && it >= 1 && !wait_or_abort(a_empty, (it - 1) & 1u, abort_flag)) { ok = false; break; }
            if (ls == 0 && gq + 1 < total_slices && !issue(gq + 1)) { ok = false; break; }
            const int nr = slice_rows(it, q);
            // a bulk-copied slice is read from shared memory; a ragged or
            // unaligned one straight from global memory by each thread
            const bool bulk = bulk_ok(it, q);
            if (!wait_or_abort(&raw_full[b], (gq >> 1) & 1u, abort_flag)) { ok = false; break; }
            auto convert = [&](const float* rb) {
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const int item = ls + 256 * j;            // 16 rows x 32 chunks of 8 teeth
                    const int r = item & (kSlice - 1), c = item >> 4;
                    const int row = kSlice * q + r;
                    uint32_t w[4] = {0u, 0u, 0u, 0u};
                    if (r < nr && c < nchunk8) {
                        const float* src = rb + r * T + 8 * c;
#pragma unroll
                        for (int e = 0; e < 8; e += 2) {
                            float x2[2];
#pragma unroll
                            for (int h = 0; h < 2; ++h) {
                                const int k = 8 * c + e + h;
                                float x = 0.f;
                                if (k < T) {
                                    const float4 tk = tooth[k];
                                    x = scale_in ? __fmul_rn(src[e + h], tk.x) : src[e + h];
                                    x = (x - tk.y) * tk.z;
                                }
                                x2[h] = x;
                            }
                            w[e >> 1] = pack_bf16(x2[0], x2[1]);
                        }
                    }
                    *reinterpret_cast<uint4*>(Ain + a_off(row, 8 * c)) = make_uint4(w[0], w[1], w[2], w[3]);
                }
            };
            if (bulk) {
                convert(raw + b * kSlice * 256);
            } else {
                convert(srcbase + (tile_f0(it) + kSlice * q) * T);
            }
            tc::mbar_arrive(&raw_empty[b]);
            if (q == nslices - 1) {
                tc::fence_proxy_async_smem();
                tc::mbar_arrive(a_full);
            }
        }
        if (!ok) *abort_flag = 1;
        // no copy may land after the block exits
        if (ls == 0) {
            for (int gq = last_issued - 1 > 0 ? last_issued - 1 : 0; gq <= last_issued; ++gq) {
                const int it = gq / nslices, q = gq - it * nslices;
                if (bulk_ok(it, q)) (void)tc::mbar_wait(&raw_full[gq & 1], (gq >> 1) & 1u, kPolls);
            }
        }
    } else {
        // ---------------- epilogues ----------------
        const int quarter = warp & 3, half = warp >> 2;
        const int row = quarter * 32 + lane;
        const uint32_t lane_base = tmem + (static_cast<uint32_t>(quarter * 32) << 16);
        bool ok = true;
        for (int it = 0; it < my_tiles; ++it) {
            const uint32_t ph = it & 1u;
            // layer 1: bias, GELU, BF16 into the a1 tile
            if (!wait_or_abort(acc1_full, ph, abort_flag)) { ok = false; break; }
            __syncwarp();
            tc::tc_fence_after();
            {
                unsigned char* rbase = Ah + row * 128;
                for (int cp = half * 4; cp < half * 4 + 4; ++cp) {
                    uint32_t raw[2][16];
                    tc::tmem_ld16_async(lane_base + 32 * cp, raw[0]);
                    tc::tmem_ld16_async(lane_base + 32 * cp + 16, raw[1]);
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int hh = 0; hh < 2; ++hh) {
                        const int cb = 2 * cp + hh;
                        uint32_t w[8];
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const int c = cb * 16 + 2 * i;
                            const float2 bb = *reinterpret_cast<const float2*>(b1s + c);
                            w[i] = gelu_bf16x2(__uint_as_float(raw[hh][2 * i]) + bb.x,
                                               __uint_as_float(raw[hh][2 * i + 1]) + bb.y);
                        }
                        unsigned char* base = rbase + (cb >> 2) * (kMM * 128);
                        const int c16 = (cb & 3) * 2;
                        *reinterpret_cast<uint4*>(base + ((c16 ^ (row & 7)) << 4)) = make_uint4(w[0], w[1], w[2], w[3]);
                        *reinterpret_cast<uint4*>(base + (((c16 + 1) ^ (row & 7)) << 4)) =
                            make_uint4(w[4], w[5], w[6], w[7]);
                    }
                }
            }
            tc::tc_fence_before();
            tc::fence_proxy_async_smem();
            tc::mbar_arrive(a1_full);
            // layer 2 and the FP32 output layer
            if (!wait_or_abort(acc2_full, ph, abort_flag)) { ok = false; break; }
            __syncwarp();
            tc::tc_fence_after();
            float o[4] = {0.f, 0.f, 0.f, 0.f};
            for (int cp = half * 4; cp < half * 4 + 4; ++cp) {
                uint32_t raw[2][16];
                tc::tmem_ld16_async(lane_base + kHid + 32 * cp, raw[0]);
                tc::tmem_ld16_async(lane_base + kHid + 32 * cp + 16, raw[1]);
                tc::tmem_wait_ld();
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const int c = cp * 32 + i;
                    const float h = gelu_fast(__uint_as_float(raw[i >> 4][i & 15]) + b2s[c]);
                    const float4 w3 = w3t[c];
                    o[0] = fmaf(w3.x, h, o[0]);
                    o[1] = fmaf(w3.y, h, o[1]);
                    o[2] = fmaf(w3.z, h, o[2]);
                    o[3] = fmaf(w3.w, h, o[3]);
                }
            }
            tc::tc_fence_before();
            tc::mbar_arrive(acc2_empty);
            // half 1 hands its partial sums to half 0 through a double buffer
            const int rb = it & 1;
            const uint32_t rph = (it >> 1) & 1u;
            float* rd = red + rb * (kMM * 4);
            if (half == 1) {
                if (it >= 2 && !wait_or_abort(&red_empty[rb], rph ^ 1u, abort_flag)) { ok = false; break; }
#pragma unroll
                for (int j = 0; j < 4; ++j) rd[row * 4 + j] = o[j];
                tc::mbar_arrive(&red_full[rb]);
                continue;
            }
            if (!wait_or_abort(&red_full[rb], rph, abort_flag)) { ok = false; break; }
            float po[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) po[j] = rd[row * 4 + j];
            tc::mbar_arrive(&red_empty[rb]);
            const int64_t f = tile_f0(it) + row;
            if (f < a.n) {
                float p[4];
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    p[j] = fmaf(o[j] + po[j] + outs[j], outs[8 + j], outs[4 + j]);
                p[1] = fminf(fmaxf(fabsf(p[1]), a.g_lo), a.g_hi);
                if (!(fabsf(p[0]) < INFINITY && fabsf(p[1]) < INFINITY && fabsf(p[2]) < INFINITY &&
                      fabsf(p[3]) < INFINITY)) {
                    // no usable guess: a flat start the polish cannot converge
                    // from, so the frame goes to the moment-guess fallback
                    p[0] = a.x_mid;
                    p[1] = a.g_lo;
                    p[2] = 0.f;
                    p[3] = 0.f;
                }
                float* q = a.p0 + f * 4;
                q[0] = p[0];
                q[1] = p[1];
                q[2] = p[2];
                q[3] = p[3];
                if (a.flags) a.flags[f] = 0;
            }
        }
        if (!ok) {
            *abort_flag = 1;
            if (tid == 0) atomicExch(a.err, 2);
        }
    }

    // ---- teardown: every product has completed before TMEM is freed ----
    tc::tc_fence_before();
    __syncthreads();
    if (warp == kIssueWarp) {
        (void)tc::mbar_wait(done, 0, kPolls);
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, 2 * kHid);
    }
}

PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

}  // namespace

int mlp_smem_bytes(int stages, int T)
{
    return 1024 + 2 * kABytes + kRawBytes + stages * kChunkBytes + 4 * (2 * kHid + 4 * kHid + 16 + 4 * T) +
           2 * 4 * 4 * kMM + 8 * (2 * kStagesMax + 15) + 16;
}

// Parses a cg_mlp_save blob, packs the BF16 weight matrix, the FP32 tables and
// the tensor map into the plan.
cudaError_t setup_mlp(cg_plan_s* p, const unsigned char* blob, size_t bytes, const char** why)
{
    *why = nullptr;
    if (bytes < static_cast<size_t>(kMlpHeaderBytes) || std::memcmp(blob, kMlpMagic, 8) != 0) {
        *why = "not a cg_mlp_save blob (bad magic)";
        return cudaErrorInvalidValue;
    }
    int32_t hdr[4];
    std::memcpy(hdr, blob + 8, sizeof(hdr));
    const int n_in = hdr[0], H = hdr[1], n_out = hdr[2];
    if (n_in != p->T || H != kHid || n_out != 4) {
        *why = "network shape must be n_teeth -> 256 -> 256 -> 4";
        return cudaErrorInvalidValue;
    }
    const int64_t np = static_cast<int64_t>(H) * n_in + H + static_cast<int64_t>(H) * H + H + 4 * H + 4;
    const size_t want = kMlpHeaderBytes + 4 * (2 * static_cast<size_t>(n_in) + 8 + static_cast<size_t>(np));
    if (bytes != want) {
        *why = "blob size does not match its header";
        return cudaErrorInvalidValue;
    }
    std::vector<float> f((bytes - kMlpHeaderBytes) / 4);
    std::memcpy(f.data(), blob + kMlpHeaderBytes, bytes - kMlpHeaderBytes);
    for (float v : f)
        if (!std::isfinite(v)) {
            *why = "blob holds a non-finite value";
            return cudaErrorInvalidValue;
        }
    const float* in_mean = f.data();
    const float* in_scale = in_mean + n_in;
    const float* out_mean = in_scale + n_in;
    const float* out_scale = out_mean + 4;
    const float* th = out_scale + 4;
    const float* W1 = th;
    const float* b1 = W1 + static_cast<size_t>(H) * n_in;
    const float* W2 = b1 + H;
    const float* b2 = W2 + static_cast<size_t>(H) * H;
    const float* W3 = b2 + H;
    const float* b3 = W3 + 4 * H;
    const int nkb = (n_in + 63) / 64;
    if (nkb > 4) {
        *why = "n_teeth > 256 is not supported by the inference kernel";
        return cudaErrorInvalidValue;
    }
    // [512][256] BF16: W1 rows (K zero-padded), then W2 rows
    std::vector<__nv_bfloat16> W(static_cast<size_t>(2 * kHid) * kHid, __float2bfloat16_rn(0.f));
    for (int h = 0; h < kHid; ++h) {
        for (int k = 0; k < n_in; ++k) W[static_cast<size_t>(h) * kHid + k] = __float2bfloat16_rn(W1[h * n_in + k]);
        for (int k = 0; k < kHid; ++k)
            W[static_cast<size_t>(kHid + h) * kHid + k] = __float2bfloat16_rn(W2[h * kHid + k]);
    }
    std::vector<float> tab(kMlpTabIn + 2 * n_in, 0.f);
    auto put = [&](int off, const float* src, int count) {
        for (int i = 0; i < count; ++i) tab[static_cast<size_t>(off + i)] = src[i];
    };
    put(kMlpTabB1, b1, kHid);
    put(kMlpTabB2, b2, kHid);
    put(kMlpTabW3, W3, 4 * kHid);
    put(kMlpTabB3, b3, 4);
    put(kMlpTabOutMean, out_mean, 4);
    put(kMlpTabOutScale, out_scale, 4);
    put(kMlpTabIn, in_mean, n_in);
    put(kMlpTabIn + n_in, in_scale, n_in);

    cudaError_t e;
    if (!p->d.mlp_W && (e = cudaMalloc(&p->d.mlp_W, W.size() * sizeof(__nv_bfloat16))) != cudaSuccess) return e;
    if (!p->d.mlp_tab && (e = cudaMalloc(&p->d.mlp_tab, tab.size() * sizeof(float))) != cudaSuccess) return e;
    if ((e = cudaMemcpy(p->d.mlp_W, W.data(), W.size() * sizeof(__nv_bfloat16), cudaMemcpyHostToDevice)) !=
        cudaSuccess)
        return e;
    if ((e = cudaMemcpy(p->d.mlp_tab, tab.data(), tab.size() * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess)
        return e;
    if (!p->d.err) {
        if ((e = cudaMalloc(&p->d.err, sizeof(int))) != cudaSuccess) return e;
        if ((e = cudaMemset(p->d.err, 0, sizeof(int))) != cudaSuccess) return e;
    }
    PFN_cuTensorMapEncodeTiled_v12000 enc = tmap_encoder();
    if (!enc) {
        *why = "cuTensorMapEncodeTiled is unavailable";
        return cudaErrorNotSupported;
    }
    cuuint64_t gdim[2] = {static_cast<cuuint64_t>(kHid), static_cast<cuuint64_t>(2 * kHid)};
    cuuint64_t gstride[1] = {static_cast<cuuint64_t>(kHid) * 2};
    cuuint32_t box[2] = {64, static_cast<cuuint32_t>(kChunkRows)};
    cuuint32_t estride[2] = {1, 1};
    CUresult r = enc(&p->mlp_map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, p->d.mlp_W, gdim, gstride, box, estride,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        *why = "tensor map encoding failed";
        return cudaErrorInvalidValue;
    }
    MlpArgs& m = p->ma;
    m.T = p->T;
    m.nkb = nkb;
    m.tab = p->d.mlp_tab;
    m.inv_ref = p->d.inv_ref;
    m.x_mid = static_cast<float>(p->x_mid);
    m.g_lo = static_cast<float>(0.5 * p->x_scale);
    m.g_hi = static_cast<float>(0.5 * (p->T - 1) * p->x_scale);
    // as many weight stages as fit beside the two operand tiles (at most 6)
    m.stages = kStagesMax;
    while (m.stages > 2 && mlp_smem_bytes(m.stages, p->T) > 227 * 1024) --m.stages;
    m.err = p->d.err;
    p->mlp_smem = mlp_smem_bytes(m.stages, p->T);
    if ((e = raise_smem_limit(reinterpret_cast<void*>(&mlp_infer_kernel), p->mlp_smem)) != cudaSuccess)
        return e;
    p->mlp_ok = true;
    return cudaSuccess;
}

cudaError_t launch_mlp(const cg_plan_s* p, const float* y, const float* amps, int64_t n, float* p0, int16_t* flags,
                       cudaStream_t s)
{
    MlpArgs m = p->ma;
    m.y = y;
    m.amps = amps;
    m.n = n;
    m.p0 = p0;
    m.flags = flags;
    const int64_t ntiles = (n + kMM - 1) / kMM;
    const unsigned grid = static_cast<unsigned>(ntiles < p->num_sms ? ntiles : p->num_sms);
    void* args[] = {const_cast<CUtensorMap*>(&p->mlp_map), &m};
    return cudaLaunchKernel(reinterpret_cast<void*>(&mlp_infer_kernel), dim3(grid), dim3(kMlpThreads), args, p->mlp_smem, s);
}

}  // namespace cg
