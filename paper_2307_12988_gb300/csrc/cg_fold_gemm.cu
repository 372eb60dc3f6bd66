// cg_fold_gemm.cu -- folded DFT-at-teeth readout on the tensor cores, for
// comb geometries whose tooth bins lie in one residue pair +-r mod 10
// (N = 10 L, L even).
//
// The tooth readout of the paper ("Data Capture and Processing": FFT of each
// row, the tooth bins selected and mapped, normalised by the reference) needs
// X at bins b = 10 q + r only.  With n = m + L j (m < L, j < 10):
//     X_{10q+r} = sum_m W_L^{q m} z_m,
//     z_m = W_N^{r m} sum_j x_{m + L j} W_10^{r j},
// so each frame is first folded to L complex values z_m (CUDA cores, integer
// sums and the W_10 symmetry w_{j+5} = (-1)^r w_j), then the L-point DFT at
// the teeth' q is a dense product on the tensor cores:
//     Re X_k = sum_m [zr_m, zi_m] . [cos, sin](2 pi q_k m / L)
//     Im X_k = sum_m [zi_m, -zr_m] . [cos, sin](2 pi q_k m / L)
// One twiddle row per tooth serves both parts: the A operand carries every
// frame twice (variant 0 = [zr, zi], variant 1 = [zi, -zr]) and the two
// variants accumulate into two TMEM accumulators.  Precision: z and the
// twiddles are split into FP16 hi + lo; three products (hi.hi, hi.lo, lo.hi)
// accumulate in FP32.  z is scaled by 1/8 first (an exact power of two) so
// full-range int16 samples stay inside FP16; |X| is scaled back.
//
// Persistent blocks of 13 warps, one 128-frame tile at a time:
//   warps 0-3   epilogue: TMEM -> |X| -> amps / y through a small staging
//               buffer for coalesced stores (TMEM lane quarter = warp);
//   warps 4-11  fold: 32-bit sample-pair loads (double-buffered in registers
//               one K block ahead; the next tile is prefetched into L2),
//               fold, twiddle, FP16 split, swizzled stores into the A ring;
//   warp 12     TMA-loads the twiddles once (resident for the whole kernel),
//               owns TMEM and issues tcgen05.mma from one lane.
// Two accumulator pairs alternate between tiles, so the epilogue of one tile
// overlaps the products of the next.  Every wait is bounded: on time-out the
// block records an error word, stops issuing, drains and frees its TMEM.
#include <cmath>
#include <cstdint>
#include <vector>
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include "cg_internal.h"
#include "cg_tc.cuh"

namespace cg {

namespace {

constexpr int kFM = 128;              // frames per tile (MMA M)
constexpr int kFK = 32;               // FP16 elements per K block (one 64-byte swizzled row)
constexpr int kEpiWarps = 4;
constexpr int kFoldWarps = 8;
constexpr int kIssueWarp = kEpiWarps + kFoldWarps;
constexpr int kFoldThreads = (kIssueWarp + 1) * 32;
constexpr int kItems = kFM * (kFK / 4) / (kFoldWarps * 32);   // (frame, output pair) items per thread
constexpr int kRowStep = kFoldWarps * 4;                          // frame rows covered by one item round
constexpr int kAtile = kFM * kFK * 2;  // 8 KiB: one variant, one (hi or lo) part of a K block
constexpr int kAstage = 4 * kAtile;    // two variants x (hi, lo)
constexpr int kStagesMax = 6;
constexpr int kStageLd = 17;           // epilogue staging row stride (floats)
constexpr uint32_t kPolls = 1u << 22;
constexpr float kZScale = 0.125f;

static_assert(kItems * kFoldWarps * 32 == kFM * (kFK / 4), "fold items must cover a K block");

// bounded wait (kPolls polls)
__device__ __forceinline__ bool wait_or_abort(uint64_t* bar, uint32_t parity, volatile int* abort_flag)
{
    const uint64_t t0 = tc::globaltimer_ns();
    for (uint32_t i = 0; i < kPolls; ++i) {
        if (tc::mbar_try_wait(bar, parity)) return true;
        if ((i & 255u) == 255u && (*abort_flag || tc::globaltimer_ns() - t0 > tc::kWaitLimitNs)) return false;
    }
    return false;
}

// fold of one output: x[j] = x_{m + L j}; returns sum_j x_j W_10^(r j) with
// D_j = x_j + s x_{j+5}, E = D_1 + s D_4 ..., s = (-1)^r (see the fast readout)
template <int SG>
__device__ __forceinline__ float2 fold10(const int (&x)[10], float c1, float s1, float c2, float s2)
{
    const int D0 = x[0] + SG * x[5], D1 = x[1] + SG * x[6], D2 = x[2] + SG * x[7];
    const int D3 = x[3] + SG * x[8], D4 = x[4] + SG * x[9];
    const int E1 = D1 + SG * D4, F1 = D1 - SG * D4;
    const int E2 = D2 + SG * D3, F2 = D2 - SG * D3;
    float2 fz;
    fz.x = fmaf(static_cast<float>(E2), c2, fmaf(static_cast<float>(E1), c1, static_cast<float>(D0)));
    fz.y = fmaf(static_cast<float>(F2), s2, static_cast<float>(F1) * s1);
    return fz;
}

__device__ __forceinline__ uint32_t h2_bits(__half2 h) { return *reinterpret_cast<uint32_t*>(&h); }
// [re, im] (low, high halves) -> [im, -re]
__device__ __forceinline__ uint32_t rot_variant(uint32_t w) { return __byte_perm(w, 0u, 0x1032) ^ 0x80000000u; }

template <int SG>
__global__ void __launch_bounds__(kFoldThreads, 1) fold_gemm_kernel(const __grid_constant__ CUtensorMap tmW, FoldArgs a)
{
    extern __shared__ __align__(1024) unsigned char fsm_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(fsm_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    const int NT = a.ntile, nkb = a.nkb, S = a.stages, T = a.T, L = a.L;
    const int wtile = NT * kFK * 2;                       // one (hi or lo) K block of W
    unsigned char* Ws = sm + a.sm_W;                      // [nkb][hi, lo][NT][64 B]
    unsigned char* As = sm + a.sm_A;                      // [S][variant][hi, lo][128][64 B]
    float* stg = reinterpret_cast<float*>(sm + a.sm_stage);
    float2* tw = reinterpret_cast<float2*>(sm + a.sm_tw);  // [nkb * 16] W_N^(r m) / 8, zero past L
    float* iref = reinterpret_cast<float*>(sm + a.sm_iref);
    uint64_t* wfull = reinterpret_cast<uint64_t*>(sm + a.sm_bar);
    uint64_t* afull = wfull + 1;
    uint64_t* aempty = afull + kStagesMax;
    uint64_t* accfull = aempty + kStagesMax;
    uint64_t* accempty = accfull + 2;
    uint64_t* done = accempty + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t ntiles = (a.n + kFM - 1) / kFM;
    const int my_tiles =
        static_cast<int64_t>(blockIdx.x) < ntiles ? static_cast<int>((ntiles - 1 - blockIdx.x) / gridDim.x) + 1 : 0;

    for (int i = threadIdx.x; i < nkb * (kFK / 2); i += blockDim.x) {
        const float2 t = i < L ? a.twN[i] : make_float2(0.f, 0.f);
        tw[i] = make_float2(t.x * a.z_scale, t.y * a.z_scale);
    }
    for (int i = threadIdx.x; i < T; i += blockDim.x) iref[i] = a.inv_ref[i];
    if (threadIdx.x == 0) {
        tc::mbar_init(wfull, 1);
        for (int s = 0; s < S; ++s) {
            tc::mbar_init(&afull[s], kFoldWarps * 32);
            tc::mbar_init(&aempty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(&accfull[b], 1);
            tc::mbar_init(&accempty[b], kEpiWarps);
        }
        tc::mbar_init(done, 1);
        *abort_flag = 0;
        tc::fence_mbar_init();
    }
    if (warp == kIssueWarp) tc::tmem_alloc(tmem_slot, a.tmem_cols);
    if (warp == kIssueWarp && lane == 0) tc::prefetch_tmap(&tmW);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == kIssueWarp) {
        // ---------------- twiddles by TMA, then MMA issue ----------------
        if (lane == 0) {
            tc::mbar_arrive_expect_tx(wfull, static_cast<uint32_t>(2 * nkb * wtile));
            for (int kb = 0; kb < nkb; ++kb) {
                tc::tma_load_2d(Ws + (2 * kb) * wtile, &tmW, kb * kFK, 0, wfull);
                tc::tma_load_2d(Ws + (2 * kb + 1) * wtile, &tmW, kb * kFK, NT, wfull);
            }
            bool ok = wait_or_abort(wfull, 0, abort_flag);
            if (!ok) *abort_flag = 1;
            const uint32_t idesc = tc::idesc_f16(kFM, NT, 0);
            int g = 0;
            for (int it = 0; ok && it < my_tiles; ++it) {
                const int b = it & 1;
                if (!wait_or_abort(&accempty[b], ((it >> 1) & 1u) ^ 1u, abort_flag)) {
                    *abort_flag = 1;
                    ok = false;
                    break;
                }
                tc::tc_fence_after();
                const uint32_t d0 = tmem + static_cast<uint32_t>(2 * b * a.acc_stride);
                for (int kb = 0; kb < nkb; ++kb, ++g) {
                    const int s = g % S;
                    if (!wait_or_abort(&afull[s], (g / S) & 1u, abort_flag)) {
                        *abort_flag = 1;
                        ok = false;
                        break;
                    }
                    tc::tc_fence_after();
                    const uint32_t abase = tc::smem_u32(As + s * kAstage);
                    const uint32_t wh = tc::smem_u32(Ws + (2 * kb) * wtile), wl = wh + wtile;
#pragma unroll
                    for (int kk = 0; kk < kFK / 16; ++kk) {
                        const uint32_t koff = kk * 32;
#pragma unroll
                        for (int v = 0; v < 2; ++v) {
                            const uint32_t d = d0 + static_cast<uint32_t>(v * a.acc_stride);
                            const uint64_t ah = tc::sdesc_sw64(abase + (2 * v) * kAtile + koff);
                            const uint64_t al = tc::sdesc_sw64(abase + (2 * v + 1) * kAtile + koff);
                            tc::mma_f16(d, ah, tc::sdesc_sw64(wh + koff), idesc, (kb | kk) ? 1u : 0u);
                            tc::mma_f16(d, ah, tc::sdesc_sw64(wl + koff), idesc, 1u);
                            tc::mma_f16(d, al, tc::sdesc_sw64(wh + koff), idesc, 1u);
                        }
                    }
                    tc::mma_commit(&aempty[s]);
                }
                if (!ok) break;
                tc::mma_commit(&accfull[b]);
            }
            // arrives when every MMA issued above has completed (also on abort)
            tc::mma_commit(done);
            if (!ok) (void)tc::mbar_wait(wfull, 0, kPolls);   // no TMA write in flight at exit
        }
    } else if (warp >= kEpiWarps) {
        // ---------------- fold ----------------
        const int t = threadIdx.x - kEpiWarps * 32;    // 0 .. 32 kFoldWarps - 1
        const int fr = t >> 3;                          // frame row (+ kRowStep i)
        const int pm = t & 7;                           // output pair: m = 16 kb + 2 pm
        const int halfL = L >> 1;
        const int nsteps = my_tiles * nkb;
        const uint32_t* fw = reinterpret_cast<const uint32_t*>(a.frames);   // 4-byte aligned
        auto tile_f0 = [&](int it) { return (static_cast<int64_t>(blockIdx.x) + static_cast<int64_t>(it) * gridDim.x) * kFM; };
        auto prefetch_tile = [&](int it) {
            if (it >= my_tiles) return;
            const int64_t f0 = tile_f0(it);
            const int64_t f1 = (f0 + kFM < a.n) ? f0 + kFM : a.n;
            uintptr_t lo = reinterpret_cast<uintptr_t>(a.frames + f0 * a.N);
            uintptr_t hi = reinterpret_cast<uintptr_t>(a.frames + f1 * a.N);
            lo = (lo + 15) & ~static_cast<uintptr_t>(15);
            hi &= ~static_cast<uintptr_t>(15);
            for (uintptr_t p = lo; p < hi; p += 65536) {
                const uintptr_t e = (hi - p) < 65536 ? hi : p + 65536;
                tc::prefetch_l2_bulk(reinterpret_cast<const void*>(p), static_cast<uint32_t>(e - p));
            }
        };
        auto load = [&](int g, uint32_t (&w)[kItems][10]) {
            const int it = g / nkb, kb = g - it * nkb;
            const int64_t f0 = tile_f0(it);
            const int m = kb * (kFK / 2) + 2 * pm;
#pragma unroll
            for (int i = 0; i < kItems; ++i) {
                const int64_t f = f0 + fr + kRowStep * i;
                const bool in = f < a.n && m < L;
                const uint32_t* src = fw + (in ? (f * a.N + m) >> 1 : 0);
#pragma unroll
                for (int j = 0; j < 10; ++j) w[i][j] = in ? __ldg(src + j * halfL) : 0u;
            }
        };
        auto step = [&](int g, const uint32_t (&w)[kItems][10]) -> bool {
            const int s = g % S;
            const int it = g / nkb, kb = g - it * nkb;
            if (kb == 0 && t == 0) prefetch_tile(it + 1);
            if (g >= S && !wait_or_abort(&aempty[s], ((g / S) & 1u) ^ 1u, abort_flag)) {
                *abort_flag = 1;
                return false;
            }
            unsigned char* A0 = As + s * kAstage;
            const float4 tw2 = *reinterpret_cast<const float4*>(tw + kb * (kFK / 2) + 2 * pm);
#pragma unroll
            for (int i = 0; i < kItems; ++i) {
                const int r = fr + kRowStep * i;
                uint32_t hw[2], lw[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    int x[10];
#pragma unroll
                    for (int j = 0; j < 10; ++j)
                        x[j] = h ? (static_cast<int>(w[i][j]) >> 16) : static_cast<int>(static_cast<short>(w[i][j] & 0xffffu));
                    const float2 fz = fold10<SG>(x, a.c1, a.s1, a.c2, a.s2);
                    const float2 tn = h ? make_float2(tw2.z, tw2.w) : make_float2(tw2.x, tw2.y);
                    const float zr = fmaf(fz.x, tn.x, -fz.y * tn.y);
                    const float zi = fmaf(fz.x, tn.y, fz.y * tn.x);
                    const __half2 hh = __floats2half2_rn(zr, zi);
                    const float2 hf = __half22float2(hh);
                    hw[h] = h2_bits(hh);
                    lw[h] = h2_bits(__floats2half2_rn(zr - hf.x, zi - hf.y));
                }
                const int off = r * 64 + (((pm >> 1) ^ ((r >> 1) & 3)) << 4) + ((pm & 1) << 3);
                *reinterpret_cast<uint2*>(A0 + off) = make_uint2(hw[0], hw[1]);
                *reinterpret_cast<uint2*>(A0 + kAtile + off) = make_uint2(lw[0], lw[1]);
                *reinterpret_cast<uint2*>(A0 + 2 * kAtile + off) = make_uint2(rot_variant(hw[0]), rot_variant(hw[1]));
                *reinterpret_cast<uint2*>(A0 + 3 * kAtile + off) = make_uint2(rot_variant(lw[0]), rot_variant(lw[1]));
            }
            tc::fence_proxy_async_smem();
            tc::mbar_arrive(&afull[s]);
            return true;
        };
        if (t == 0) prefetch_tile(0);
        uint32_t wa[kItems][10], wb[kItems][10];
        if (nsteps > 0) load(0, wa);
        for (int g = 0; g < nsteps; g += 2) {
            if (g + 1 < nsteps) load(g + 1, wb);
            if (!step(g, wa)) break;
            if (g + 1 >= nsteps) break;
            if (g + 2 < nsteps) load(g + 2, wa);
            if (!step(g + 1, wb)) break;
        }
    } else {
        // ---------------- epilogue ----------------
        float* st = stg + warp * 32 * kStageLd;
        const uint32_t lane_base = tmem + (static_cast<uint32_t>(warp * 32) << 16);
        const int nch = (T + 15) / 16;
        bool ok = true;
        for (int it = 0; it < my_tiles; ++it) {
            const int b = it & 1;
            if (!wait_or_abort(&accfull[b], (it >> 1) & 1u, abort_flag)) {
                *abort_flag = 1;
                ok = false;
                break;
            }
            __syncwarp();
            tc::tc_fence_after();
            const int64_t fb = (static_cast<int64_t>(blockIdx.x) + static_cast<int64_t>(it) * gridDim.x) * kFM + warp * 32;
            const int nvalid = (a.n - fb) >= 32 ? 32 : static_cast<int>(a.n - fb > 0 ? a.n - fb : 0);
            const uint32_t cre = lane_base + static_cast<uint32_t>(2 * b * a.acc_stride);
            const uint32_t cim = cre + static_cast<uint32_t>(a.acc_stride);
            for (int c = 0; c < nch; ++c) {
                uint32_t re[16], im[16];
                tc::tmem_ld16_async(cre + 16 * c, re);
                tc::tmem_ld16_async(cim + 16 * c, im);
                tc::tmem_wait_ld();
                const int k0 = 16 * c;
                const int kc = (T - k0) < 16 ? T - k0 : 16;
                float amp[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const float xr = __uint_as_float(re[i]), xi = __uint_as_float(im[i]);
                    amp[i] = sqrtf(fmaf(xr, xr, xi * xi)) * a.out_scale;
                }
#pragma unroll
                for (int o = 0; o < 2; ++o) {
                    float* out = o ? a.y : a.amps;
                    if (!out) continue;
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        st[lane * kStageLd + i] = o ? __fmul_rn(amp[i], iref[(k0 + i) < T ? k0 + i : 0]) : amp[i];
                    __syncwarp();
                    const int kk = lane & 15;
#pragma unroll 4
                    for (int q = 0; q < 16; ++q) {
                        const int rr = 2 * q + (lane >> 4);
                        if (rr < nvalid && kk < kc) out[(fb + rr) * T + k0 + kk] = st[rr * kStageLd + kk];
                    }
                    __syncwarp();
                }
            }
            tc::tc_fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&accempty[b]);
        }
        if (!ok && lane == 0) atomicExch(a.err, 1);
    }

    tc::tc_fence_before();
    __syncthreads();
    if (warp == kIssueWarp) {
        (void)tc::mbar_wait(done, 0, kPolls);
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, a.tmem_cols);
    }
}

PFN_cuTensorMapEncodeTiled_v12000 fold_encoder()
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

void* fold_fn(int sign)
{
    return sign < 0 ? reinterpret_cast<void*>(&fold_gemm_kernel<-1>) : reinterpret_cast<void*>(&fold_gemm_kernel<1>);
}

}  // namespace

// Builds the split twiddle matrix [hi, lo][NT][Kpad] (FP16, K contiguous:
// element 2m = cos, 2m+1 = sin of 2 pi q_k m / L for tooth row k), its tensor
// map, the shared-memory layout and the grid.  Leaves fold_ok false when the
// geometry does not admit the folded readout (not a radix-10 coset, odd L,
// more than 128 teeth, or twiddles beyond shared memory).
cudaError_t setup_fold(cg_plan_s* p, const std::vector<int>& zidx)
{
    p->fold_ok = false;
    const int N = p->N, T = p->T, L = p->L;
    if (p->kind != CG_FFT_COSET || p->M != 10 || N != 10 * L || (L & 1)) return cudaSuccess;
    const int NT = (T + 15) / 16 * 16;
    if (NT > 128) return cudaSuccess;
    const int nkb = (2 * L + kFK - 1) / kFK;
    const int Kpad = nkb * kFK;
    const int acc_stride = NT <= 32 ? 32 : NT <= 64 ? 64 : 128;

    FoldArgs& f = p->fo;
    int off = 0;
    f.sm_W = off; off += nkb * 2 * NT * kFK * 2;                 // multiple of 1024 (NT % 16 == 0)
    f.sm_A = off;
    int fixed = 0;
    const int stage_b = kEpiWarps * 32 * kStageLd * 4;
    const int tw_b = nkb * (kFK / 2) * 8;
    const int iref_b = (4 * T + 15) / 16 * 16;
    const int bar_b = 8 * (1 + 2 * kStagesMax + 4 + 1) + 16;
    fixed = stage_b + tw_b + iref_b + bar_b;
    const int limit = 227 * 1024 - 1024;
    int S = (limit - off - fixed) / kAstage;
    if (S > kStagesMax) S = kStagesMax;
    if (S < 2) return cudaSuccess;
    off += S * kAstage;
    f.sm_stage = off; off += stage_b;
    f.sm_tw = off; off += tw_b;
    f.sm_iref = off; off += iref_b;
    f.sm_bar = off; off += bar_b;
    f.sm_total = off + 1024;

    std::vector<__half> W(static_cast<size_t>(2) * NT * Kpad, __float2half_rn(0.f));
    const double two_pi = 6.28318530717958647692528676655900577;
    for (int k = 0; k < T; ++k) {
        const long long q = zidx[k];
        for (int m = 0; m < L; ++m) {
            const double ang = two_pi * static_cast<double>((q * m) % L) / L;
            const double w[2] = {std::cos(ang), std::sin(ang)};
            for (int c = 0; c < 2; ++c) {
                const __half hi = __float2half_rn(static_cast<float>(w[c]));
                const __half lo = __float2half_rn(static_cast<float>(w[c] - static_cast<double>(__half2float(hi))));
                W[static_cast<size_t>(k) * Kpad + 2 * m + c] = hi;
                W[static_cast<size_t>(NT + k) * Kpad + 2 * m + c] = lo;
            }
        }
    }
    cudaError_t e = cudaMalloc(&p->d.fold_W, W.size() * sizeof(__half));
    if (e != cudaSuccess) return e;
    if ((e = cudaMemcpy(p->d.fold_W, W.data(), W.size() * sizeof(__half), cudaMemcpyHostToDevice)) != cudaSuccess)
        return e;
    if (!p->d.err) {
        if ((e = cudaMalloc(&p->d.err, sizeof(int))) != cudaSuccess) return e;
        if ((e = cudaMemset(p->d.err, 0, sizeof(int))) != cudaSuccess) return e;
    }
    PFN_cuTensorMapEncodeTiled_v12000 enc = fold_encoder();
    if (!enc) return cudaErrorNotSupported;
    cuuint64_t gdim[2] = {static_cast<cuuint64_t>(Kpad), static_cast<cuuint64_t>(2 * NT)};
    cuuint64_t gstride[1] = {static_cast<cuuint64_t>(Kpad) * 2};
    cuuint32_t box[2] = {static_cast<cuuint32_t>(kFK), static_cast<cuuint32_t>(NT)};
    cuuint32_t estride[2] = {1, 1};
    CUresult r = enc(&p->fold_map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, p->d.fold_W, gdim, gstride, box, estride,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;

    f.N = N;
    f.T = T;
    f.L = L;
    f.nkb = nkb;
    f.ntile = NT;
    f.acc_stride = acc_stride;
    f.tmem_cols = 4 * acc_stride;
    f.stages = S;
    f.z_scale = kZScale;
    f.out_scale = 1.0f / kZScale;
    for (int j = 1; j <= 2; ++j) {
        const double ang = -two_pi * static_cast<double>((p->r0 * j) % 10) / 10.0;
        (j == 1 ? f.c1 : f.c2) = static_cast<float>(std::cos(ang));
        (j == 1 ? f.s1 : f.s2) = static_cast<float>(std::sin(ang));
    }
    f.twN = p->d.tw_n1;
    f.inv_ref = p->d.inv_ref;
    f.err = p->d.err;
    p->fold_sign = (p->r0 & 1) ? -1 : 1;
    if ((e = raise_smem_limit(fold_fn(p->fold_sign), f.sm_total)) != cudaSuccess) return e;
    int occ = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fold_fn(p->fold_sign), kFoldThreads, f.sm_total)) !=
        cudaSuccess)
        return e;
    if (occ < 1) return cudaSuccess;
    p->grid_fold = p->num_sms;   // one persistent block per SM (TMEM: 4 x acc_stride columns)
    p->fold_ok = true;
    return cudaSuccess;
}

cudaError_t launch_fold_readout(const cg_plan_s* p, const int16_t* frames, int64_t n, float* amps, float* y,
                                cudaStream_t s)
{
    FoldArgs f = p->fo;
    f.frames = frames;
    f.n = n;
    f.amps = amps;
    f.y = y;
    const int64_t ntiles = (n + kFM - 1) / kFM;
    const unsigned grid = static_cast<unsigned>(ntiles < p->grid_fold ? ntiles : p->grid_fold);
    void* args[] = {const_cast<CUtensorMap*>(&p->fold_map), &f};
    return cudaLaunchKernel(fold_fn(p->fold_sign), dim3(grid), dim3(kFoldThreads), args, f.sm_total, s);
}

}  // namespace cg
