// cg_gemm.cu -- split-precision DFT-at-teeth readout on the tensor cores.
//
// The tooth readout of the paper ("Data Capture and Processing": FFT of each
// row, then the tooth bins "selected and mapped") is recast as a dense product
//     C[frame][2t + {0,1}] = sum_n x[frame][n] * W[n][2t + {0,1}],
//     W[n][2t] = cos(2 pi b_t n / N),  W[n][2t+1] = -sin(2 pi b_t n / N),
// i.e. Re and Im of X at each tooth bin b_t, followed by |X| and the reference
// normalisation.  Precision split: W = W_hi + W_lo with both parts in FP16;
// 12-bit samples are exact in FP16 (two products per K step), full 16-bit
// samples are split x = 256 hi + lo with both parts exact in FP16 (four
// products).  Products accumulate in FP32 in tensor memory (TMEM).
//
// One thread block computes a 128-frame x NT-column tile (NT <= 256):
//   warps 0-3  stage the int16 samples of the tile's frames, convert them to
//              FP16 and store them in the K-major 128-byte-swizzled layout the
//              tensor core reads (frame rows are not 16-byte multiples, so no
//              TMA tensor map can address them), then run the epilogue;
//   warp 4     TMA-loads the W_hi / W_lo tiles (my own aligned layout);
//   warp 5     owns TMEM and issues tcgen05.mma from one lane;
// with an S-stage mbarrier pipeline.  Every wait is bounded: on time-out the
// block records an error code, stops issuing, drains what it issued and frees
// its TMEM.
#include <cstdint>
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include "cg_internal.h"
#include "cg_tc.cuh"

namespace cg {

namespace {

constexpr int kBM = 128;          // frames per tile (MMA M)
constexpr int kBK = 64;           // samples per K block (one 128-byte swizzle row)
constexpr int kPipeMax = 4;
constexpr uint32_t kMaxPolls = 1u << 22;

struct GemmSmem {
    int a_bytes, b_bytes, stage_bytes, stages;
};

__device__ __forceinline__ bool wait_or_abort(uint64_t* bar, uint32_t parity, volatile int* abort_flag)
{
    const uint64_t t0 = tc::globaltimer_ns();
    for (uint32_t i = 0; i < kMaxPolls; ++i) {
        if (tc::mbar_try_wait(bar, parity)) return true;
        if ((i & 255u) == 255u && (*abort_flag || tc::globaltimer_ns() - t0 > tc::kWaitLimitNs)) return false;
    }
    return false;
}

template <bool SPLITX>
__global__ void __launch_bounds__(192, 1) dft_gemm_kernel(const __grid_constant__ CUtensorMap tmB, GemmArgs a)
{
    extern __shared__ __align__(1024) unsigned char gsm_raw[];
    // 1024-byte alignment of the tiles (swizzle atoms)
    unsigned char* gsm = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(gsm_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    const int NT = a.ntile;
    const int S = a.stages;
    const int a_bytes = kBM * kBK * 2;           // one A tile (16 KiB)
    const int b_bytes = NT * kBK * 2;            // one B tile
    const int stage_bytes = (SPLITX ? 2 : 1) * a_bytes + 2 * b_bytes;
    uint64_t* full = reinterpret_cast<uint64_t*>(gsm + S * stage_bytes);   // samples staged
    uint64_t* bfull = full + kPipeMax;                                     // W tiles landed
    uint64_t* empty = bfull + kPipeMax;                                    // MMAs done
    uint64_t* done = empty + kPipeMax;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    // consecutive blocks are the column tiles of one frame tile: they run
    // together, so the frame tile's samples come from DRAM once
    const int64_t m0 = static_cast<int64_t>(blockIdx.x / a.n_ctiles) * kBM;
    const int nt = static_cast<int>(blockIdx.x % a.n_ctiles);
    const int nkb = a.nkb;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            tc::mbar_init(&full[s], 128);       // the 128 loader threads
            tc::mbar_init(&bfull[s], 1);        // the TMA issuer's expect_tx arrival
            tc::mbar_init(&empty[s], 1);        // one MMA commit
        }
        tc::mbar_init(done, 1);
        *abort_flag = 0;
        tc::fence_mbar_init();
    }
    if (warp == 5) tc::tmem_alloc(tmem_slot, a.tmem_cols);
    if (warp == 4 && lane == 0) tc::prefetch_tmap(&tmB);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp < 4) {
        // ---------------- sample loaders ----------------
        const int t = threadIdx.x;          // 0..127
        const int rsub = t >> 4;            // row within a pass of 8 rows
        const int c4 = t & 15;              // group of 4 samples
        const bool vec = a.vec8;
        // each thread owns 16 eight-byte pieces (4 samples) of every stage,
        // at the positions of the swizzled FP16 layout
        auto piece_off = [&](int pass) {
            const int r = pass * 8 + rsub;
            return r * 128 + (((c4 >> 1) ^ (r & 7)) << 4) + ((c4 & 1) << 3);
        };
        // convert the int16 samples held at As + off in place to FP16 (and the
        // split low parts to As + a_bytes + off)
        auto convert = [&](unsigned char* As, int off, const short (&v)[4]) {
            if (SPLITX) {
                __half hi[4], lo[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int hv = static_cast<int>(v[e]) >> 8;       // -128..127
                    const int lv = static_cast<int>(v[e]) & 0xff;     // 0..255
                    hi[e] = __int2half_rn(hv * 256);
                    lo[e] = __int2half_rn(lv);
                }
                *reinterpret_cast<uint2*>(As + off) = *reinterpret_cast<const uint2*>(hi);
                *reinterpret_cast<uint2*>(As + a_bytes + off) = *reinterpret_cast<const uint2*>(lo);
            } else {
                __half h[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) h[e] = __short2half_rn(v[e]);
                *reinterpret_cast<uint2*>(As + off) = *reinterpret_cast<const uint2*>(h);
            }
        };
        if (vec) {
            // raw samples stream in by cp.async D = S-1 K blocks ahead, straight
            // into their stage positions (zero-filled past the frame or the
            // matrix); each is converted in place right before its stage is
            // released to the tensor core
            const int D = S - 1;
            auto issue = [&](int kb) {
                if (kb < nkb && !*abort_flag) {
                    const int s = kb % S;
                    if (wait_or_abort(&empty[s], ((kb / S) & 1u) ^ 1u, abort_flag)) {
                        unsigned char* As = gsm + s * stage_bytes;
                        const int k = kb * kBK + 4 * c4;
#pragma unroll
                        for (int pass = 0; pass < kBM / 8; ++pass) {
                            const int64_t f = m0 + pass * 8 + rsub;
                            const bool in = (f < a.n) && (k < a.N);
                            const int16_t* src = in ? a.frames + f * a.N + k : a.frames;
                            tc::cp_async8_zfill(As + piece_off(pass), src, in ? 8u : 0u);
                        }
                    } else {
                        *abort_flag = 1;
                    }
                }
                tc::cp_async_commit();   // one group per K block, possibly empty
            };
            for (int j = 0; j < D; ++j) issue(j);
            for (int kb = 0; kb < nkb; ++kb) {
                issue(kb + D);
                tc::cp_async_wait_pending(D);   // the group of K block kb has landed
                if (*abort_flag) break;
                const int s = kb % S;
                unsigned char* As = gsm + s * stage_bytes;
#pragma unroll
                for (int pass = 0; pass < kBM / 8; ++pass) {
                    const int off = piece_off(pass);
                    const uint2 w = *reinterpret_cast<const uint2*>(As + off);
                    const short v[4] = {static_cast<short>(w.x & 0xffffu), static_cast<short>(w.x >> 16),
                                        static_cast<short>(w.y & 0xffffu), static_cast<short>(w.y >> 16)};
                    convert(As, off, v);
                }
                tc::fence_proxy_async_smem();
                tc::mbar_arrive(&full[s]);
            }
            tc::cp_async_wait_pending(0);
        } else {
            // frames not 8-byte aligned: element loads, synchronous
            for (int kb = 0; kb < nkb; ++kb) {
                const int s = kb % S;
                const uint32_t round = kb / S;
                if (!wait_or_abort(&empty[s], (round & 1u) ^ 1u, abort_flag)) {
                    *abort_flag = 1;
                    break;
                }
                unsigned char* As = gsm + s * stage_bytes;
                const int k = kb * kBK + 4 * c4;
#pragma unroll 4
                for (int pass = 0; pass < kBM / 8; ++pass) {
                    const int64_t f = m0 + pass * 8 + rsub;
                    short v[4] = {0, 0, 0, 0};
                    if (f < a.n) {
                        const int16_t* src = a.frames + f * a.N + k;
#pragma unroll
                        for (int e = 0; e < 4; ++e) v[e] = (k + e < a.N) ? src[e] : static_cast<short>(0);
                    }
                    convert(As, piece_off(pass), v);
                }
                tc::fence_proxy_async_smem();
                tc::mbar_arrive(&full[s]);
            }
        }
    } else if (warp == 4) {
        // ---------------- W tiles by TMA ----------------
        if (lane == 0) {
            const int a_part = (SPLITX ? 2 : 1) * a_bytes;
            int issued = 0;
            for (int kb = 0; kb < nkb; ++kb) {
                const int s = kb % S;
                const uint32_t round = kb / S;
                if (!wait_or_abort(&empty[s], (round & 1u) ^ 1u, abort_flag)) {
                    *abort_flag = 1;
                    break;
                }
                unsigned char* Bs = gsm + s * stage_bytes + a_part;
                tc::mbar_arrive_expect_tx(&bfull[s], 2u * static_cast<uint32_t>(b_bytes));
                tc::tma_load_2d(Bs, &tmB, kb * kBK, nt * NT, &bfull[s]);
                tc::tma_load_2d(Bs + b_bytes, &tmB, kb * kBK, a.nrows_total + nt * NT, &bfull[s]);
                issued = kb + 1;
            }
            // drain: the last load issued into each stage has landed
            for (int kb = issued - S > 0 ? issued - S : 0; kb < issued; ++kb)
                (void)tc::mbar_wait(&bfull[kb % S], (kb / S) & 1u, kMaxPolls);
        }
    } else {
        // ---------------- MMA issue ----------------
        if (lane == 0) {
            const uint32_t idesc = tc::idesc_f16(kBM, NT, 0);
            const int a_part = (SPLITX ? 2 : 1) * a_bytes;
            bool ok = true;
            for (int kb = 0; kb < nkb; ++kb) {
                const int s = kb % S;
                const uint32_t round = kb / S;
                if (!wait_or_abort(&full[s], round & 1u, abort_flag) ||
                    !wait_or_abort(&bfull[s], round & 1u, abort_flag)) {
                    *abort_flag = 1;
                    ok = false;
                    break;
                }
                tc::tc_fence_after();
                const uint32_t sa = tc::smem_u32(gsm + s * stage_bytes);
                const uint32_t sbh = sa + a_part;
                const uint32_t sbl = sbh + b_bytes;
                // K blocks alternate over n_acc accumulators (columns acc * acc_cols)
                const int acc = kb % a.n_acc;
                const uint32_t d = tmem + static_cast<uint32_t>(acc * a.acc_cols);
#pragma unroll
                for (int kk = 0; kk < kBK / 16; ++kk) {
                    const uint32_t koff = kk * 32;   // 16 elements of 2 bytes
                    const uint64_t ad = tc::sdesc_sw128(sa + koff);
                    const uint64_t bh = tc::sdesc_sw128(sbh + koff);
                    const uint64_t bl = tc::sdesc_sw128(sbl + koff);
                    tc::mma_f16(d, ad, bh, idesc, (kb >= a.n_acc || kk != 0) ? 1u : 0u);
                    tc::mma_f16(d, ad, bl, idesc, 1);
                    if (SPLITX) {
                        const uint64_t al = tc::sdesc_sw128(sa + a_bytes + koff);
                        tc::mma_f16(d, al, bh, idesc, 1);
                        tc::mma_f16(d, al, bl, idesc, 1);
                    }
                }
                tc::mma_commit(&empty[s]);
            }
            (void)ok;
            // arrives once every MMA issued above has completed (also on abort,
            // so TMEM is quiescent before it is freed)
            tc::mma_commit(done);
        }
    }

    if (warp < 4) {
        // ---------------- epilogue: TMEM -> |X| -> amps (and y) ----------------
        const bool ok = wait_or_abort(done, 0, abort_flag) && !*abort_flag;
        tc::tc_fence_after();
        if (ok) {
            const int r = warp * 32 + lane;
            const int64_t f = m0 + r;
            const uint32_t lane_base = tmem + (static_cast<uint32_t>(warp * 32) << 16);
            const int teeth_tile = NT / 2;
            const int nacc = nkb < a.n_acc ? nkb : a.n_acc;   // accumulators written
            for (int j = 0; j < NT / 16; ++j) {
                float v[16];
                tc::tmem_ld16(lane_base + 16 * j, v);
                for (int q = 1; q < nacc; ++q) {
                    float w[16];
                    tc::tmem_ld16(lane_base + static_cast<uint32_t>(q * a.acc_cols) + 16 * j, w);
#pragma unroll
                    for (int i = 0; i < 16; ++i) v[i] += w[i];
                }
                if (f < a.n) {
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const int tooth = nt * teeth_tile + 8 * j + i;
                        if (tooth < a.T) {
                            const float amp = sqrtf(fmaf(v[2 * i], v[2 * i], v[2 * i + 1] * v[2 * i + 1]));
                            if (a.amps) a.amps[f * a.T + tooth] = amp;
                            if (a.y) a.y[f * a.T + tooth] = __fmul_rn(amp, a.inv_ref[tooth]);
                        }
                    }
                }
            }
        } else if (threadIdx.x == 0) {
            atomicExch(a.err, 1);
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 5) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, a.tmem_cols);
    }
}

// ---------------------------------------------------------------------------
// Decoupled rings (12-bit samples, at most 256 output columns per tile):
// samples and twiddles go through separate mbarrier rings, so the sample ring
// can be deep (a.stages K blocks) while the twiddle ring holds kSB stages.
// HALVES = 1: 128-frame tiles, K blocks alternating over two accumulators
// (TMEM columns 0 and 256) that are summed at the end; HALVES = 2: 256-frame
// tiles whose two 128-frame halves share every twiddle stage, one
// accumulator per half.
//   warps 0 .. 4H-1  stage the samples (cp.async, in-place FP16) and run the
//                    epilogue (TMEM lane quarter w % 4, half w / 4);
//   warp 4H          TMA-loads the W_hi / W_lo tiles;
//   warp 4H+1        owns TMEM and issues tcgen05.mma from one lane.
// ---------------------------------------------------------------------------
constexpr int kSB = 2;       // twiddle stages (2 x NT x 128 B each)
constexpr int kSAMax = 8;    // sample stages at most

template <int HALVES>
__global__ void __launch_bounds__((4 * HALVES + 2) * 32, 1) dft_gemm_ring_kernel(const __grid_constant__ CUtensorMap tmB,
                                                                                 GemmArgs a)
{
    extern __shared__ __align__(1024) unsigned char gsm_raw[];
    unsigned char* gsm = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(gsm_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    constexpr int kLoaders = 128 * HALVES;
    const int NT = a.ntile;
    const int SA = a.stages;
    const int a_half = kBM * kBK * 2;            // 16 KiB: one 128-frame half of a K block
    const int a_stage = HALVES * a_half;
    const int b_bytes = NT * kBK * 2;            // one (hi or lo) twiddle tile
    const int b_stage = 2 * b_bytes;
    unsigned char* Aring = gsm;
    unsigned char* Bring = gsm + SA * a_stage;   // a_stage is a multiple of 1024
    uint64_t* fullA = reinterpret_cast<uint64_t*>(Bring + kSB * b_stage);
    uint64_t* emptyA = fullA + kSAMax;
    uint64_t* fullB = emptyA + kSAMax;
    uint64_t* emptyB = fullB + kSB;
    uint64_t* done = emptyB + kSB;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    // consecutive blocks are the column tiles of one frame tile: they run
    // together, so the frame tile's samples come from DRAM once
    const int64_t m0 = static_cast<int64_t>(blockIdx.x / a.n_ctiles) * (HALVES * kBM);
    const int nt = static_cast<int>(blockIdx.x % a.n_ctiles);
    const int nkb = a.nkb;
    constexpr int kTmaWarp = 4 * HALVES, kMmaWarp = 4 * HALVES + 1;

    if (threadIdx.x == 0) {
        for (int s = 0; s < SA; ++s) {
            tc::mbar_init(&fullA[s], kLoaders);   // every sample loader
            tc::mbar_init(&emptyA[s], 1);         // one MMA commit
        }
        for (int s = 0; s < kSB; ++s) {
            tc::mbar_init(&fullB[s], 1);          // the TMA issuer's expect_tx arrival
            tc::mbar_init(&emptyB[s], 1);
        }
        tc::mbar_init(done, 1);
        *abort_flag = 0;
        tc::fence_mbar_init();
    }
    if (warp == kMmaWarp) tc::tmem_alloc(tmem_slot, 512);
    if (warp == kTmaWarp && lane == 0) tc::prefetch_tmap(&tmB);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp < kTmaWarp) {
        // ---------------- sample loaders (cp.async D = SA - 2 blocks ahead) ----
        const int t = threadIdx.x & 127;
        const int half = threadIdx.x >> 7;
        const int rsub = t >> 4;            // row within a pass of 8 rows
        const int c4 = t & 15;              // group of 4 samples
        auto piece_off = [&](int pass) {
            const int r = pass * 8 + rsub;
            return half * a_half + r * 128 + (((c4 >> 1) ^ (r & 7)) << 4) + ((c4 & 1) << 3);
        };
        // two stages of slack: the block being converted and the block the
        // tensor core reads, so issuing never waits on the latest MMA
        const int D = SA - 2 > 0 ? SA - 2 : 1;
        auto issue = [&](int kb) {
            if (kb < nkb && !*abort_flag) {
                const int s = kb % SA;
                if (wait_or_abort(&emptyA[s], ((kb / SA) & 1u) ^ 1u, abort_flag)) {
                    unsigned char* As = Aring + s * a_stage;
                    const int k = kb * kBK + 4 * c4;
#pragma unroll
                    for (int pass = 0; pass < kBM / 8; ++pass) {
                        const int64_t f = m0 + half * kBM + pass * 8 + rsub;
                        const bool in = (f < a.n) && (k < a.N);
                        const int16_t* src = in ? a.frames + f * a.N + k : a.frames;
                        tc::cp_async8_zfill(As + piece_off(pass), src, in ? 8u : 0u);
                    }
                } else {
                    *abort_flag = 1;
                }
            }
            tc::cp_async_commit();   // one group per K block, possibly empty
        };
        for (int j = 0; j < D; ++j) issue(j);
        for (int kb = 0; kb < nkb; ++kb) {
            issue(kb + D);
            tc::cp_async_wait_pending(D > 3 ? 3 : D);
            if (D > 3) asm volatile("cp.async.wait_group 4;\n" ::: "memory");
            if (*abort_flag) break;
            unsigned char* As = Aring + (kb % SA) * a_stage;
#pragma unroll
            for (int pass = 0; pass < kBM / 8; ++pass) {
                const int off = piece_off(pass);
                const uint2 w = *reinterpret_cast<const uint2*>(As + off);
                __half h[4];
                h[0] = __short2half_rn(static_cast<short>(w.x & 0xffffu));
                h[1] = __short2half_rn(static_cast<short>(w.x >> 16));
                h[2] = __short2half_rn(static_cast<short>(w.y & 0xffffu));
                h[3] = __short2half_rn(static_cast<short>(w.y >> 16));
                *reinterpret_cast<uint2*>(As + off) = *reinterpret_cast<const uint2*>(h);
            }
            tc::fence_proxy_async_smem();
            tc::mbar_arrive(&fullA[kb % SA]);
        }
        tc::cp_async_wait_pending(0);
    } else if (warp == kTmaWarp) {
        // ---------------- twiddle tiles by TMA ----------------
        if (lane == 0) {
            int issued = 0;
            for (int kb = 0; kb < nkb; ++kb) {
                const int s = kb % kSB;
                if (!wait_or_abort(&emptyB[s], ((kb / kSB) & 1u) ^ 1u, abort_flag)) {
                    *abort_flag = 1;
                    break;
                }
                unsigned char* Bs = Bring + s * b_stage;
                tc::mbar_arrive_expect_tx(&fullB[s], static_cast<uint32_t>(b_stage));
                tc::tma_load_2d(Bs, &tmB, kb * kBK, nt * NT, &fullB[s]);
                tc::tma_load_2d(Bs + b_bytes, &tmB, kb * kBK, a.nrows_total + nt * NT, &fullB[s]);
                issued = kb + 1;
            }
            for (int kb = issued - kSB > 0 ? issued - kSB : 0; kb < issued; ++kb)
                (void)tc::mbar_wait(&fullB[kb % kSB], (kb / kSB) & 1u, kMaxPolls);
        }
    } else {
        // ---------------- MMA issue ----------------
        if (lane == 0) {
            const uint32_t idesc = tc::idesc_f16(kBM, NT, 0);
            for (int kb = 0; kb < nkb; ++kb) {
                const int sa = kb % SA, sb = kb % kSB;
                if (!wait_or_abort(&fullA[sa], (kb / SA) & 1u, abort_flag) ||
                    !wait_or_abort(&fullB[sb], (kb / kSB) & 1u, abort_flag)) {
                    *abort_flag = 1;
                    break;
                }
                tc::tc_fence_after();
                const uint32_t abase = tc::smem_u32(Aring + sa * a_stage);
                const uint32_t bh = tc::smem_u32(Bring + sb * b_stage);
                const uint32_t bl = bh + b_bytes;
#pragma unroll
                for (int h = 0; h < HALVES; ++h) {
                    // HALVES = 2: accumulator of half h; HALVES = 1: K blocks alternate
                    const int acc = HALVES == 2 ? h : (kb & 1);
                    const uint32_t d = tmem + static_cast<uint32_t>(acc * 256);
                    const bool first = HALVES == 2 ? (kb == 0) : (kb < 2);
#pragma unroll
                    for (int kk = 0; kk < kBK / 16; ++kk) {
                        const uint32_t koff = kk * 32;
                        const uint64_t ad = tc::sdesc_sw128(abase + h * a_half + koff);
                        tc::mma_f16(d, ad, tc::sdesc_sw128(bh + koff), idesc, (!first || kk != 0) ? 1u : 0u);
                        tc::mma_f16(d, ad, tc::sdesc_sw128(bl + koff), idesc, 1);
                    }
                }
                tc::mma_commit(&emptyA[sa]);
                tc::mma_commit(&emptyB[sb]);
            }
            tc::mma_commit(done);   // also on abort, so TMEM is quiescent before it is freed
        }
    }

    if (warp < kTmaWarp) {
        // ---------------- epilogue: TMEM -> |X| -> amps (and y) ----------------
        const bool ok = wait_or_abort(done, 0, abort_flag) && !*abort_flag;
        __syncwarp();
        tc::tc_fence_after();
        if (ok) {
            const int quarter = warp & 3, half = warp >> 2;
            const int64_t f = m0 + half * kBM + quarter * 32 + lane;
            const uint32_t lane_base = tmem + (static_cast<uint32_t>(quarter * 32) << 16);
            const int teeth_tile = NT / 2;
            for (int j = 0; j < NT / 16; ++j) {
                float v[16];
                tc::tmem_ld16(lane_base + static_cast<uint32_t>(half * 256) + 16 * j, v);
                if (HALVES == 1 && nkb > 1) {
                    float w[16];
                    tc::tmem_ld16(lane_base + 256 + 16 * j, w);
#pragma unroll
                    for (int i = 0; i < 16; ++i) v[i] += w[i];
                }
                if (f < a.n) {
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const int tooth = nt * teeth_tile + 8 * j + i;
                        if (tooth < a.T) {
                            const float amp = sqrtf(fmaf(v[2 * i], v[2 * i], v[2 * i + 1] * v[2 * i + 1]));
                            if (a.amps) a.amps[f * a.T + tooth] = amp;
                            if (a.y) a.y[f * a.T + tooth] = __fmul_rn(amp, a.inv_ref[tooth]);
                        }
                    }
                }
            }
        } else if (threadIdx.x == 0) {
            atomicExch(a.err, 1);
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == kMmaWarp) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, 512);
    }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encoder()
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

// Builds the split twiddle matrix [2 x rows_total][Kpad] (FP16, K contiguous),
// its tensor map and the launch geometry.  Called from cg_plan.
cudaError_t setup_gemm(cg_plan_s* p)
{
    const int N = p->N, T = p->T;
    const int split = p->gemm_split_x;
    // output columns: 2 per tooth, tiles of NT <= 224 columns (multiple of 16)
    const int cols = 2 * T;
    int ntiles = (cols + 223) / 224;
    int NT = ((cols + ntiles - 1) / ntiles + 15) / 16 * 16;
    const int rows_total = NT * ntiles;
    const int nkb = (N + kBK - 1) / kBK;
    const int Kpad = nkb * kBK;
    std::vector<__half> W(static_cast<size_t>(2) * rows_total * Kpad, __float2half_rn(0.f));
    const double two_pi = 6.28318530717958647692528676655900577;
    for (int t = 0; t < T; ++t) {
        const long long b = p->bins[t];
        for (int n = 0; n < N; ++n) {
            const double ang = two_pi * static_cast<double>((b * n) % N) / N;
            const double w[2] = {std::cos(ang), -std::sin(ang)};
            for (int c = 0; c < 2; ++c) {
                const __half hi = __float2half_rn(static_cast<float>(w[c]));
                const __half lo = __float2half_rn(static_cast<float>(w[c] - static_cast<double>(__half2float(hi))));
                const size_t row = static_cast<size_t>(2 * t + c);
                W[row * Kpad + n] = hi;
                W[(rows_total + row) * Kpad + n] = lo;
            }
        }
    }
    cudaError_t e = cudaMalloc(&p->d.gemm_W, W.size() * sizeof(__half));
    if (e != cudaSuccess) return e;
    e = cudaMemcpy(p->d.gemm_W, W.data(), W.size() * sizeof(__half), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
    if ((e = cudaMalloc(&p->d.err, sizeof(int))) != cudaSuccess) return e;
    if ((e = cudaMemset(p->d.err, 0, sizeof(int))) != cudaSuccess) return e;

    PFN_cuTensorMapEncodeTiled_v12000 enc = get_encoder();
    if (!enc) return cudaErrorNotSupported;
    cuuint64_t gdim[2] = {static_cast<cuuint64_t>(Kpad), static_cast<cuuint64_t>(2 * rows_total)};
    cuuint64_t gstride[1] = {static_cast<cuuint64_t>(Kpad) * 2};
    cuuint32_t box[2] = {static_cast<cuuint32_t>(kBK), static_cast<cuuint32_t>(NT)};
    cuuint32_t estride[2] = {1, 1};
    CUresult r = enc(&p->gemm_map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, p->d.gemm_W, gdim, gstride, box, estride,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;

    GemmArgs& g = p->ga;
    g.N = N;
    g.T = T;
    g.nkb = nkb;
    g.ntile = NT;
    g.n_ctiles = ntiles;
    g.nrows_total = rows_total;
    // FP32 accumulation error grows with the coherent partial sum; alternate
    // the K blocks over as many accumulators as fit in the 512 TMEM columns
    // (up to 4) and add them in FP32 at the end
    g.acc_cols = NT <= 32 ? 32 : NT <= 64 ? 64 : NT <= 128 ? 128 : 256;
    g.n_acc = 512 / g.acc_cols;
    if (g.n_acc > 4) g.n_acc = 4;
    g.tmem_cols = g.acc_cols * g.n_acc;
    g.inv_ref = p->d.inv_ref;
    g.err = p->d.err;
    const int a_bytes = kBM * kBK * 2, b_bytes = NT * kBK * 2;
    const int stage_bytes = (split ? 2 : 1) * a_bytes + 2 * b_bytes;
    int stages = (227 * 1024 - 2048) / stage_bytes;
    if (stages > kPipeMax) stages = kPipeMax;
    if (stages < 2) return cudaErrorInvalidValue;
    g.stages = stages;
    p->gemm_smem = 1024 + stages * stage_bytes + 8 * (3 * kPipeMax + 1) + 16;
    p->gemm_ntiles = ntiles;
    // decoupled-ring kernel: 12-bit samples, NT <= 256; 256-frame tiles (one
    // accumulator per half) only while FP32 accumulation over N samples stays
    // well within the error bound, else 128-frame tiles alternating two
    // accumulators; as many sample stages as shared memory holds
    p->gemm_ring = !split && NT <= 256 && N <= 4096;
    if (p->gemm_ring) {
        p->gemm_halves = (N <= 1536) ? 2 : 1;
        const int a_stage = p->gemm_halves * a_bytes;
        const int fixed = 1024 + kSB * 2 * b_bytes + 8 * (2 * kSAMax + 2 * kSB + 1) + 16;
        int sa = (227 * 1024 - fixed) / a_stage;
        if (sa > kSAMax) sa = kSAMax;
        if (sa < 3) {
            p->gemm_ring = false;
        } else {
            p->gemm_ring_stages = sa;
            p->gemm_ring_smem = fixed + sa * a_stage;
            void* rk = p->gemm_halves == 2 ? reinterpret_cast<void*>(&dft_gemm_ring_kernel<2>)
                                           : reinterpret_cast<void*>(&dft_gemm_ring_kernel<1>);
            cudaError_t e2 = raise_smem_limit(rk, p->gemm_ring_smem);
            if (e2 != cudaSuccess) return e2;
        }
    }
    void* fn = split ? reinterpret_cast<void*>(&dft_gemm_kernel<true>) : reinterpret_cast<void*>(&dft_gemm_kernel<false>);
    return raise_smem_limit(fn, p->gemm_smem);
}

cudaError_t launch_gemm_readout(const cg_plan_s* p, const int16_t* frames, int64_t n, float* amps, float* y,
                                cudaStream_t s)
{
    GemmArgs g = p->ga;
    g.frames = frames;
    g.n = n;
    g.amps = amps;
    g.y = y;
    g.vec8 = (reinterpret_cast<uintptr_t>(frames) & 7) == 0 && (p->N % 4) == 0;
    if (p->gemm_ring && g.vec8) {
        const int H = p->gemm_halves;
        g.stages = p->gemm_ring_stages;
        dim3 grid2(static_cast<unsigned>((n + H * kBM - 1) / (H * kBM) * p->gemm_ntiles));
        void* args2[] = {const_cast<CUtensorMap*>(&p->gemm_map), &g};
        void* rk = H == 2 ? reinterpret_cast<void*>(&dft_gemm_ring_kernel<2>)
                          : reinterpret_cast<void*>(&dft_gemm_ring_kernel<1>);
        return cudaLaunchKernel(rk, grid2, dim3((4 * H + 2) * 32), args2, p->gemm_ring_smem, s);
    }
    dim3 grid(static_cast<unsigned>((n + kBM - 1) / kBM * p->gemm_ntiles));
    void* fn = p->gemm_split_x ? reinterpret_cast<void*>(&dft_gemm_kernel<true>)
                               : reinterpret_cast<void*>(&dft_gemm_kernel<false>);
    void* args[] = {const_cast<CUtensorMap*>(&p->gemm_map), &g};
    return cudaLaunchKernel(fn, grid, dim3(192), args, p->gemm_smem, s);
}

}  // namespace cg
