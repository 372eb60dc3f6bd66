// cg_mlp_tc.cu -- inference of the learned initial guess on the tensor cores.
//
// Per thread block: 128 normalised spectra (one MMA M tile) through
//     x = (y - in_mean) * in_scale                         (FP32, then BF16)
//     a1 = gelu(W1 x + b1),  a2 = gelu(W2 a1 + b2)          (BF16 x BF16 -> FP32 in TMEM)
//     p0 = (W3 a2 + b3) * out_scale + out_mean              (FP32 on the CUDA cores)
// with W1 (K zero-padded to 64 * nkb) and W2 stored as one BF16 matrix
// [512][256], streamed from L2 by TMA in 128-row x 64-column chunks through an
// S-stage mbarrier ring.  The spectra and then a1 are written by the threads
// into the K-major 128-byte-swizzled layout the MMA reads; the 256 hidden
// activations of a row live in 256 TMEM columns.
//   warps 0-7: stage the input tile and run both epilogues; warp w reads
//              TMEM lanes 32 (w % 4).. (rows) and column half w / 4, so the
//              second epilogue of half 0 overlaps the layer-2 MMAs of half 1;
//   warp 8:    owns TMEM; one lane issues the TMA loads and tcgen05.mma.
// Every wait is bounded; on time-out the block records an error, stops
// issuing, drains its loads and frees its TMEM.
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
constexpr int kABytes = 4 * kMM * 64 * 2;       // A operand: 4 K blocks of 64
constexpr int kStagesMax = 4;
constexpr int kEpiWarps = 8;                    // staging + epilogue warps (2 per TMEM lane quarter)
constexpr int kMlpThreads = (kEpiWarps + 1) * 32;  // + the TMA / MMA issuing warp
constexpr uint32_t kPolls = 1u << 22;

__device__ __forceinline__ bool wait_or_abort(uint64_t* bar, uint32_t parity, volatile int* abort_flag)
{
    for (uint32_t i = 0; i < kPolls; ++i) {
        if (tc::mbar_try_wait(bar, parity)) return true;
        if ((i & 1023u) == 1023u && *abort_flag) return false;
    }
    return false;
}

__device__ __forceinline__ float gelu_fast(float z)
{
    const float u = 0.7978845608028654f * fmaf(0.044715f * z * z, z, z);
    float t;
    asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(u));
    return 0.5f * z * (1.0f + t);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&h);
}

// byte offset of BF16 element (row, k) in the swizzled A operand
__device__ __forceinline__ uint32_t a_off(int row, int k)
{
    const int kl = k & 63;
    return static_cast<uint32_t>((k >> 6) * (kMM * 128) + row * 128 + ((((kl >> 3) ^ (row & 7))) << 4) +
                                 ((kl & 7) << 1));
}

__global__ void __launch_bounds__(kMlpThreads, 2) mlp_infer_kernel(const __grid_constant__ CUtensorMap tmW, MlpArgs a)
{
    extern __shared__ __align__(1024) unsigned char msm_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(msm_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    unsigned char* Abuf = sm;
    unsigned char* Wst = sm + kABytes;
    const int S = a.stages;
    const int T = a.T, nkb = a.nkb;
    float* tab = reinterpret_cast<float*>(Wst + S * kChunkBytes);   // FP32 tables, staged
    float* red = tab + kMlpTabIn + 2 * T;                            // [128][4] output partials
    uint64_t* full = reinterpret_cast<uint64_t*>(red + kMM * 4);
    uint64_t* empty = full + kStagesMax;
    uint64_t* done = empty + kStagesMax;                             // [2]: one per column half
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 2);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t f0 = static_cast<int64_t>(blockIdx.x) * kMM;
    const int n1 = 2 * nkb;      // layer-1 chunks: column half-major, K blocks within
    const int nch = n1 + 8;      // + layer-2 chunks
    const bool issuer = (warp == kEpiWarps && lane == 0);
    for (int i = tid; i < kMlpTabIn + 2 * T; i += blockDim.x) tab[i] = a.tab[i];

    if (issuer) {
        for (int s = 0; s < S; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        tc::mbar_init(&done[0], 1);
        tc::mbar_init(&done[1], 1);
        *abort_flag = 0;
        tc::fence_mbar_init();
        tc::prefetch_tmap(&tmW);
    }
    if (warp == kEpiWarps) tc::tmem_alloc(tmem_slot, kHid);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    // chunk g -> layer, column half and K block
    auto chunk_geom = [&](int g, int& layer, int& nh, int& kb) {
        const int per = g < n1 ? nkb : 4;
        const int h = g < n1 ? g : g - n1;
        layer = g < n1 ? 0 : 1;
        nh = h / per;
        kb = h - nh * per;
    };
    // issuer state
    int issued = 0, consumed = 0;
    auto load_chunk = [&](int g) {
        int layer, nh, kb;
        chunk_geom(g, layer, nh, kb);
        const int s = g % S;
        tc::mbar_arrive_expect_tx(&full[s], kChunkBytes);
        tc::tma_load_2d(Wst + s * kChunkBytes, &tmW, kb * 64, layer * kHid + nh * kChunkRows, &full[s]);
    };
    // chunk q's stage takes chunk q + S once q's MMAs have read it
    auto refill = [&](int q) -> bool {
        if (issued >= nch || issued != q + S) return true;
        if (!wait_or_abort(&empty[q % S], (q / S) & 1u, abort_flag)) return false;
        load_chunk(issued++);
        return true;
    };
    // MMAs of chunks [g0, g1)
    auto run_chunks = [&](int g0, int g1) -> bool {
        const uint32_t idesc = tc::idesc_f16(kMM, kChunkRows, 1);
        for (int g = g0; g < g1; ++g) {
            const int s = g % S;
            if (!wait_or_abort(&full[s], (g / S) & 1u, abort_flag)) return false;
            consumed = g + 1;
            tc::tc_fence_after();
            int layer, nh, kb;
            chunk_geom(g, layer, nh, kb);
            const uint32_t sa = tc::smem_u32(Abuf) + kb * (kMM * 128);
            const uint32_t sb = tc::smem_u32(Wst + s * kChunkBytes);
            const uint32_t d = tmem + static_cast<uint32_t>(nh * kChunkRows);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
                tc::mma_f16(d, tc::sdesc_sw128(sa + kk * 32), tc::sdesc_sw128(sb + kk * 32), idesc,
                            (kb != 0 || kk != 0) ? 1u : 0u);
            tc::mma_commit(&empty[s]);
            // refill the stage of the previous chunk (queued ahead of this
            // one), and at the end of the range this chunk's own stage
            if (g >= 1 && !refill(g - 1)) return false;
            if (g == g1 - 1 && !refill(g)) return false;
        }
        return true;
    };
    // one layer: column half 0, commit, column half 1, commit (the epilogue
    // of half 0 overlaps the MMAs of half 1); always commits, so that the
    // waiting warps are released also after an abort
    auto run_layer = [&](int g0, int per) {
        if (!*abort_flag && !run_chunks(g0, g0 + per)) *abort_flag = 1;
        tc::mma_commit(&done[0]);
        if (!*abort_flag && !run_chunks(g0 + per, g0 + 2 * per)) *abort_flag = 1;
        tc::mma_commit(&done[1]);
    };

    if (issuer) {
        for (; issued < S && issued < nch; ++issued) load_chunk(issued);
    }

    // epilogue warps: TMEM lane quarter (rows) and column half
    const int quarter = warp & 3, half = warp >> 2;
    const int row = quarter * 32 + lane;
    const uint32_t lane_base = tmem + (static_cast<uint32_t>(quarter * 32) << 16);

    // ---- stage the input tile: (y - in_mean) * in_scale -> BF16 ----
    if (warp < kEpiWarps) {
        const int64_t left = a.n - f0;
        const int rows = left < kMM ? static_cast<int>(left) : kMM;
        const float* src = (a.y ? a.y : a.amps) + f0 * T;
        const float* in_mean = tab + kMlpTabIn;
        const float* in_scale = in_mean + T;
        // the tile's rows are contiguous (and 16-byte aligned when the array
        // is, since a tile starts at a multiple of 128 rows): one flat
        // coalesced sweep, eight loads in flight per thread, (row, tooth)
        // tracked incrementally
        constexpr int kE = kEpiWarps * 32;
        const int total = rows * T;
        auto put = [&](float v, int r, int k) {
            float x = a.y ? v : __fmul_rn(v, __ldg(a.inv_ref + k));
            x = (x - in_mean[k]) * in_scale[k];
            *reinterpret_cast<__nv_bfloat16*>(Abuf + a_off(r, k)) = __float2bfloat16_rn(x);
        };
        if ((reinterpret_cast<uintptr_t>(src) & 15) == 0) {
            const float4* src4 = reinterpret_cast<const float4*>(src);
            const int total4 = total >> 2;
            const int qT = (4 * kE) / T, rT = (4 * kE) - qT * T;   // one step of 4 kE elements
            int r = (4 * tid) / T, k = 4 * tid - r * T;
            for (int j0 = 0; j0 < total4; j0 += 8 * kE) {
                float4 v[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int j = j0 + q * kE + tid;
                    v[q] = j < total4 ? __ldcs(src4 + j) : make_float4(0.f, 0.f, 0.f, 0.f);
                }
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    if (j0 + q * kE + tid < total4) {
                        const float e4[4] = {v[q].x, v[q].y, v[q].z, v[q].w};
                        int rr = r, kk = k;
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            put(e4[i], rr, kk);
                            if (++kk == T) {
                                kk = 0;
                                ++rr;
                            }
                        }
                    }
                    r += qT;
                    k += rT;
                    if (k >= T) {
                        k -= T;
                        ++r;
                    }
                }
            }
            for (int e = 4 * total4 + tid; e < total; e += kE) put(src[e], e / T, e - (e / T) * T);
        } else {
            int r = tid / T, k = tid - (tid / T) * T;
            for (int e0 = 0; e0 < total; e0 += 8 * kE) {
                float v[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int e = e0 + q * kE + tid;
                    v[q] = e < total ? __ldcs(src + e) : 0.f;
                }
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    if (e0 + q * kE + tid < total) put(v[q], r, k);
                    k += kE;
                    while (k >= T) {
                        k -= T;
                        ++r;
                    }
                }
            }
        }
        // K padding of every row and the rows past the end: zeros
        const int kpad = nkb * 64;
        if (half == 0) {
            if (row >= rows) {
                for (int k2 = 0; k2 < kpad; k2 += 8)
                    *reinterpret_cast<uint4*>(Abuf + a_off(row, k2)) = make_uint4(0u, 0u, 0u, 0u);
            } else {
                for (int k2 = T; k2 < kpad; ++k2)
                    *reinterpret_cast<__nv_bfloat16*>(Abuf + a_off(row, k2)) = __float2bfloat16_rn(0.f);
            }
        }
        tc::fence_proxy_async_smem();
    }
    __syncthreads();

    // ---- layer 1 ----
    if (issuer) run_layer(0, nkb);
    bool ok = true;
    if (warp < kEpiWarps) {
        // a1 overwrites the input tile, which every layer-1 MMA reads: both
        // halves wait for the whole layer (done[1] follows all of it)
        ok = wait_or_abort(&done[1], 0, abort_flag) && !*abort_flag;
        __syncwarp();
        tc::tc_fence_after();
        if (ok) {
            unsigned char* rbase = Abuf + row * 128;
            for (int cp = half * 4; cp < half * 4 + 4; ++cp) {
                // 32 columns per TMEM wait
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
                        w[i] = pack_bf16(gelu_fast(__uint_as_float(raw[hh][2 * i]) + tab[kMlpTabB1 + c]),
                                         gelu_fast(__uint_as_float(raw[hh][2 * i + 1]) + tab[kMlpTabB1 + c + 1]));
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
    }
    __syncthreads();

    // ---- layer 2, then the FP32 output layer ----
    if (issuer) {
        tc::tc_fence_after();
        run_layer(n1, 4);
    }
    if (warp < kEpiWarps) {
        ok = ok && wait_or_abort(&done[half], 1, abort_flag) && !*abort_flag;
        __syncwarp();
        tc::tc_fence_after();
        float o[4] = {0.f, 0.f, 0.f, 0.f};
        if (ok) {
            for (int cp = half * 4; cp < half * 4 + 4; ++cp) {
                uint32_t raw[2][16];
                tc::tmem_ld16_async(lane_base + 32 * cp, raw[0]);
                tc::tmem_ld16_async(lane_base + 32 * cp + 16, raw[1]);
                tc::tmem_wait_ld();
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const int c = cp * 32 + i;
                    const float h = gelu_fast(__uint_as_float(raw[i >> 4][i & 15]) + tab[kMlpTabB2 + c]);
#pragma unroll
                    for (int j = 0; j < 4; ++j) o[j] = fmaf(tab[kMlpTabW3 + j * kHid + c], h, o[j]);
                }
            }
        }
        if (half == 1) {
#pragma unroll
            for (int j = 0; j < 4; ++j) red[row * 4 + j] = o[j];
        }
        asm volatile("bar.sync 1, %0;\n" ::"n"(kEpiWarps * 32) : "memory");   // the epilogue warps only
        const int64_t f = f0 + row;
        if (half == 0 && ok && f < a.n) {
            float p[4];
#pragma unroll
            for (int j = 0; j < 4; ++j)
                p[j] = fmaf(o[j] + red[row * 4 + j] + tab[kMlpTabB3 + j], tab[kMlpTabOutScale + j],
                            tab[kMlpTabOutMean + j]);
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
        if (!ok && tid == 0) atomicExch(a.err, 2);
    }

    // ---- teardown: drain loads still in flight after an abort, free TMEM ----
    if (issuer && *abort_flag) {
        for (int g = consumed; g < issued; ++g) (void)tc::mbar_wait(&full[g % S], (g / S) & 1u, kPolls);
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == kEpiWarps) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, kHid);
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
    return 1024 + kABytes + stages * kChunkBytes + 4 * (kMlpTabIn + 2 * T) + 4 * 4 * kMM + 8 * (2 * kStagesMax + 2) +
           16;
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
    m.stages = 2;
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
    const unsigned grid = static_cast<unsigned>((n + kMM - 1) / kMM);
    void* args[] = {const_cast<CUtensorMap*>(&p->mlp_map), &m};
    return cudaLaunchKernel(reinterpret_cast<void*>(&mlp_infer_kernel), dim3(grid), dim3(kMlpThreads), args, p->mlp_smem, s);
}

}  // namespace cg
