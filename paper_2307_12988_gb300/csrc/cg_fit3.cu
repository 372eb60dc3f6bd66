// cg_fit3.cu -- Levenberg-Marquardt fit of the Lorentzian cavity model with
// each frame's spectrum in shared memory and the point arithmetic on packed
// FP32 pairs.
//
// Paper: "Data Capture and Processing", fit paragraphs: each normalised
// spectrum is fit by Levenberg-Marquardt, at most 20 iterations, tolerance
// 1e-6.  The damped step, the acceptance and convergence rules and the
// outputs are those of fit2_kernel (cg_fast.cu); what differs is the layout
// of the work:
//  * G lanes per frame (a group) and 32 / G frames in flight per warp; the
//    groups pull frames from the warp's task one by one as their previous
//    frame ends, so no group waits for another frame's iterations;
//  * each group owns two row slots in shared memory.  While it fits the
//    frame in one, a single bulk copy (cp.async.bulk, completing on that
//    slot's mbarrier) brings its next frame's row into the other: the
//    16-byte-aligned window around the row, so tooth 0 lands at offset
//    o in [0, 3] of the slot.  Starting a frame costs a barrier wait and a
//    few scalars; no row is copied into registers;
//  * the teeth are taken in pairs (2i, 2i + 1) -- lane gl of a group owns the
//    pairs gl, gl + G, ... -- and a pair is evaluated with packed FP32x2
//    arithmetic (one instruction for both points).  Each of the 14 sums of
//    J^T J, J^T r and chi^2 is a pair whose halves are added at the end, so
//    the summation order depends on the tooth index only, not on where the
//    frame lies in memory: a frame's result is the same in any batch.
//  * per pair, one 16-byte table entry gives both abscissae and both
//    1 / reference values (1 when the normalised spectra are given);
//  * the point is evaluated in e = (u - c) / g: L = 1 / (1 + e^2) takes two
//    packed operations and a reciprocal; the centre column L q d (q the
//    reciprocal of (u - c)^2 + g^2) equals L^2 e / g and the width column
//    L q d^2 equals L (1 - L), so per point the sums are of L^2, L^3, L^4,
//    L, L jc', L^2 jc', jc'^2, jc', L r, jc' r, L^2 r, r, r^2 with
//    jc' = L^2 e (13 instead of 14, and no separate L q product); the 14
//    sums of the textbook normal equations follow from them per frame.
//
// MODEL 1 is the paper's Fano profile (centre free, scale A and offset B
// boxed, asymmetry q and width g fixed; an active set holds a bound
// parameter whose gradient points out of its box, and the trial point is
// clamped onto the box), as fit2_kernel<G, PPL, EXACT, 1>: per point
// F = (q + e)^2 / (1 + e^2) and jc' = (q + e)(1 - q e) / (1 + e^2)^2, the
// centre column being -2 A jc' / g; 9 sums (jc' jc', jc' F, jc', F F, F,
// jc' r, F r, r, r r).  Its starting centre is the given one (the median
// filter's) or the lowest tooth of the frame (first on ties) moved by q g.
#include <cstdint>
#include <cuda_runtime.h>

#include "cg_fit.cuh"
#include "cg_internal.h"
#include "cg_tc.cuh"

namespace cg {
namespace {

__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 dup2(float v) { return make_float2(v, v); }
// a product rounded on its own: the normalised spectrum amps / ref must
// round exactly as the readout rounds it.  Two scalar __fmul_rn, which are
// never fused into the following subtraction (a packed product measured
// fused there, giving fma(amps, 1/ref, -B) without y but y - B with it)
__device__ __forceinline__ float2 mul2_rounded(float2 a, float2 b)
{
    return make_float2(__fmul_rn(a.x, b.x), __fmul_rn(a.y, b.y));
}

// The 14 sums of fit2_kernel (L L, L jc, L jg, L, jc jc, jc jg, jc, jg jg,
// jg, L r, jc r, jg r, r, r r with jc = L q d and jg = jc d) from the 13
// sums over L, L^2 and jc' = L^2 e = g jc, using jg = L - L^2.
__device__ __forceinline__ void sums_from_powers(const float (&w)[13], float ig, LmSums& S)
{
    S.v[0] = w[0];                                  // L L
    S.v[1] = w[4] * ig;                             // L jc
    S.v[2] = w[0] - w[1];                           // L jg = L^2 - L^3
    S.v[3] = w[3];                                  // L
    S.v[4] = w[6] * (ig * ig);                      // jc jc
    S.v[5] = (w[4] - w[5]) * ig;                    // jc jg
    S.v[6] = w[7] * ig;                             // jc
    S.v[7] = fmaf(-2.0f, w[1], w[0]) + w[2];        // jg jg = L^2 - 2 L^3 + L^4
    S.v[8] = w[3] - w[0];                           // jg = L - L^2
    S.v[9] = w[8];                                  // L r
    S.v[10] = w[9] * ig;                            // jc r
    S.v[11] = w[8] - w[10];                         // jg r = L r - L^2 r
    S.v[12] = w[11];                                // r
    S.v[13] = w[12];                                // r r
}

template <int G, int T>
struct Fit3Shape {
    static constexpr int kGroups = 32 / G;                      // frames in flight per warp
    static constexpr int kPairs = (T + 1) / 2;                  // tooth pairs (the last is half empty for odd T)
    static constexpr int kPPL = (kPairs + G - 1) / G;           // pairs per lane
    static constexpr int kTab = G * kPPL;                       // table entries (padded pairs included)
    static constexpr int kWin = ((4 * T + 12 + 15) / 16) * 4;   // floats of the largest 16-byte window (o = 3)
    // slot stride: >= the window, a multiple of 4 floats (16-byte slot starts)
    // and an odd multiple of 4, so the slots of the 8 groups of a half warp
    // start on distinct 4-bank quads
    static constexpr int kRS = (kWin % 8 == 4) ? kWin : kWin + 4;
    static constexpr int kSlots = 2 * kGroups;                  // per warp
};

template <int G, int T, int MODEL>
__global__ void __launch_bounds__(256, 2) fit3_kernel(Fit2Args a)
{
    constexpr int kW = MODEL == 1 ? 9 : 13;   // sums per point
    using S = Fit3Shape<G, T>;
    extern __shared__ __align__(16) float4 f3sm[];
    float4* tab = f3sm;
    const int nwarps = static_cast<int>(blockDim.x) >> 5;
    uint64_t* bars_all = reinterpret_cast<uint64_t*>(f3sm + S::kTab);
    float* slots_all = reinterpret_cast<float*>(bars_all + nwarps * S::kSlots);
    const int warp = static_cast<int>(threadIdx.x) >> 5;
    const int lane = static_cast<int>(threadIdx.x) & 31;
    const int gl = lane & (G - 1);
    const int grp = lane / G;
    const int leader_lane = lane & ~(G - 1);
    uint64_t* bars = bars_all + warp * S::kSlots;
    float* slots = slots_all + static_cast<size_t>(warp) * S::kSlots * S::kRS;

    // pair table (u_2i, u_2i+1, w_2i, w_2i+1), w = 1 / ref (1 for given y);
    // padding teeth get a far abscissa and w = 0 (finite, masked below)
    for (int i = static_cast<int>(threadIdx.x); i < S::kTab; i += static_cast<int>(blockDim.x)) {
        float v[4];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int k = 2 * i + h;
            v[h] = k < T ? a.u[k] : 65536.0f;
            v[2 + h] = k < T ? (a.y ? 1.0f : a.inv_ref[k]) : 0.0f;
        }
        tab[i] = make_float4(v[0], v[1], v[2], v[3]);
    }
    if (threadIdx.x == 0) {
        for (int i = 0; i < nwarps * S::kSlots; ++i) tc::mbar_init(&bars_all[i], 1);
        tc::fence_mbar_init();
    }
    __syncthreads();

    // the last pair of a lane may hold teeth beyond T: their terms are zeroed
    const int ilast = gl + G * (S::kPPL - 1);
    const float2 wlast = make_float2(2 * ilast < T ? 1.0f : 0.0f, 2 * ilast + 1 < T ? 1.0f : 0.0f);
    const int klast0 = 2 * ilast < T ? 2 * ilast : 0;
    const int klast1 = 2 * ilast + 1 < T ? 2 * ilast + 1 : 0;

    const float* src_base = a.y ? a.y : a.amps;
    const uintptr_t buf_lo = reinterpret_cast<uintptr_t>(src_base);
    const uintptr_t buf_hi = buf_lo + static_cast<uintptr_t>(a.n_rows) * T * sizeof(float);
    const float inv_scale = 1.0f / a.x_scale;
    int64_t n = a.n;
    if (a.list_n) {
        const int64_t c = *a.list_n;
        n = c < n ? c : n;
    }
    int64_t next = 0, end = 0;   // the warp's current task [next, end)
    int64_t f = -1, fr = -1;     // task index and row of the frame being fit
    int64_t fn = -1, frn = -1;   // the group's next frame (its copy in flight)
    float pn[4] = {0.f, 1.f, 0.f, 0.f};   // its starting point, loaded when claimed
    int flagn = 0;
    int cs = 0;                  // slot parity of the current frame
    int oc = 0, on = 0;          // offset of tooth 0 in the current / next slot
    uint32_t ph = 0;             // phase parity of the group's two slot barriers
    float p[4] = {0.f, 1.f, 0.f, 0.f};
    float lambda = a.lambda0, chi2 = 0.f;
    Normal Nm;
#pragma unroll
    for (int i = 0; i < 10; ++i) Nm.H[i] = 0.f;
#pragma unroll
    for (int i = 0; i < 4; ++i) Nm.b[i] = 0.f;
    int it = 0, st = kMaxIter, flag = 0;
    bool fresh = false, failed = false;

    while (true) {
        // ---- a group without a frame starts its next one ----
        if (f < 0 && fn >= 0) {
            const int nx = cs ^ 1;
            const int sl = grp + S::kGroups * nx;
            if (!tc::mbar_wait(&bars[sl], (ph >> nx) & 1u, 1u << 22)) failed = true;
            ph ^= 1u << nx;
            cs = nx;
            f = fn;
            fr = frn;
            oc = on;
            fn = frn = -1;
            fresh = true;
            if constexpr (MODEL == 1) {
                float c0;
                if (a.p0) {
                    c0 = (pn[0] - a.x_mid) * inv_scale;
                } else {
                    // the lowest tooth of the normalised spectrum (first on
                    // ties), the group's lanes scanning their pairs
                    const float* row = slots + (grp + S::kGroups * cs) * S::kRS + oc;
                    float best = INFINITY;
                    int bk = 0x7fffffff;
#pragma unroll 4
                    for (int j = 0; j < S::kPPL; ++j) {
                        const int i = gl + G * j;
                        const float4 tb = tab[i];
                        if (2 * i < T) {
                            const float v = __fmul_rn(row[2 * i], tb.z);
                            if (v < best) { best = v; bk = 2 * i; }
                        }
                        if (2 * i + 1 < T) {
                            const float v = __fmul_rn(row[2 * i + 1], tb.w);
                            if (v < best) { best = v; bk = 2 * i + 1; }
                        }
                    }
                    // (only the starting groups are here: shuffle within the group)
                    const unsigned gmask = G == 32 ? kFull : (((1u << G) - 1u) << leader_lane);
#pragma unroll
                    for (int o = G / 2; o > 0; o >>= 1) {
                        const float ob = __shfl_xor_sync(gmask, best, o);
                        const int ok = __shfl_xor_sync(gmask, bk, o);
                        if (ob < best || (ob == best && ok < bk)) {
                            best = ob;
                            bk = ok;
                        }
                    }
                    c0 = (bk < T ? a.u[bk] : 0.f) + a.fano_shift;
                }
                p[0] = c0;
                p[1] = a.fano_g;
                p[2] = fminf(fmaxf(a.fano_A0, a.fano_Alo), a.fano_Ahi);
                p[3] = fminf(fmaxf(a.fano_B0, a.fano_Blo), a.fano_Bhi);
                flag = 0;
            } else {
                p[0] = (pn[0] - a.x_mid) * inv_scale;
                p[1] = pn[1] * inv_scale;
                p[2] = pn[2];
                p[3] = pn[3];
                flag = flagn;
            }
            lambda = a.lambda0;
            it = 0;
            st = kMaxIter;
        }
        if (__any_sync(kFull, failed)) break;
        // ---- groups without a next frame claim one; its row goes to the free slot ----
        unsigned need = __ballot_sync(kFull, gl == 0 && fn < 0);
        while (need != 0 && next < n) {
            if (next >= end) {
                unsigned long long t = 0;
                if (lane == 0) t = atomicAdd(a.counter, 1ULL);
                t = __shfl_sync(kFull, t, 0);
                next = static_cast<int64_t>(t) * a.task;
                if (next >= n) {
                    next = end = n;
                    break;
                }
                end = next + a.task < n ? next + a.task : n;
            }
            const int cnt = __popc(need);
            const int64_t avail = end - next;
            const int take = static_cast<int>(avail < cnt ? avail : cnt);
            const int rank = __popc(need & ((1u << leader_lane) - 1u));
            if (((need >> leader_lane) & 1u) && rank < take) {
                fn = next + rank;
                frn = a.list ? static_cast<int64_t>(a.list[fn]) : fn;
                // (params rows need only 4-byte alignment: scalar loads)
                if (a.p0) {
                    const float* q = a.p0 + frn * 4;
                    pn[0] = q[0];
                    pn[1] = q[1];
                    pn[2] = q[2];
                    pn[3] = q[3];
                }
                flagn = a.flags_in ? (a.flags_in[frn] & kInitFlat) : 0;
                const float* src = src_base + frn * T;
                const uintptr_t ad = reinterpret_cast<uintptr_t>(src);
                const uintptr_t a16 = ad & ~static_cast<uintptr_t>(15);
                const uintptr_t e16 = (ad + 4u * T + 15u) & ~static_cast<uintptr_t>(15);
                on = static_cast<int>((ad - a16) >> 2);
                const int sl = grp + S::kGroups * (cs ^ 1);
                float* dst = slots + sl * S::kRS;
                if (gl == 0) {
                    if (a16 >= buf_lo && e16 <= buf_hi) {
                        // the slot's last generic reads precede this async write
                        tc::fence_proxy_async_smem();
                        tc::mbar_arrive_expect_tx(&bars[sl], static_cast<uint32_t>(e16 - a16));
                        tc::bulk_g2s(dst, reinterpret_cast<const void*>(a16), static_cast<uint32_t>(e16 - a16),
                                     &bars[sl]);
                    } else {
                        // the first or last row of an unaligned buffer: the
                        // window would leave it, so the row goes by plain loads
                        for (int k = 0; k < T; ++k) dst[on + k] = src[k];
                        tc::mbar_arrive(&bars[sl]);
                    }
                }
            }
            next += take;
            need = __ballot_sync(kFull, gl == 0 && fn < 0);
        }
        if (!__any_sync(kFull, f >= 0 || fn >= 0)) break;

        // ---- trial point ----
        float pe[4] = {p[0], p[1], p[2], p[3]};
        bool done = false;
        const bool trial = f >= 0 && !fresh;
        if (a.solve_f64) {
            // the normal equations solved in FP64 (the tensor-core form): FP64
            // is scarce, so with several lanes per frame the group's leader
            // solves and the group takes its step (shuffles outside the branch)
            float d4[4] = {0.f, 0.f, 0.f, 0.f};
            int okl = 0;
            if (trial && gl == 0) {
                if constexpr (MODEL == 1) {
                    int held = 0;
                    if ((p[2] <= a.fano_Alo && Nm.b[1] < 0.f) || (p[2] >= a.fano_Ahi && Nm.b[1] > 0.f)) held |= 2;
                    if ((p[3] <= a.fano_Blo && Nm.b[2] < 0.f) || (p[3] >= a.fano_Bhi && Nm.b[2] > 0.f)) held |= 4;
                    float d3[3] = {0.f, 0.f, 0.f};
                    okl = lm_solve3<double>(Nm, lambda, held, d3) ? 1 : 0;
                    d4[0] = d3[0];
                    d4[1] = d3[1];
                    d4[2] = d3[2];
                } else {
                    okl = lm_solve4_f64(Nm, lambda, d4) ? 1 : 0;
                }
            }
            if constexpr (G > 1) {
                okl = __shfl_sync(kFull, okl, leader_lane);
#pragma unroll
                for (int i = 0; i < 4; ++i) d4[i] = __shfl_sync(kFull, d4[i], leader_lane);
            }
            if (trial) {
                if (okl) {
                    if constexpr (MODEL == 1) {
                        pe[0] = p[0] + d4[0];
                        pe[2] = fminf(fmaxf(p[2] + d4[1], a.fano_Alo), a.fano_Ahi);
                        pe[3] = fminf(fmaxf(p[3] + d4[2], a.fano_Blo), a.fano_Bhi);
                    } else {
#pragma unroll
                        for (int i = 0; i < 4; ++i) pe[i] = p[i] + d4[i];
                    }
                } else {
                    st = kSingular;
                    done = true;
                }
            }
        } else if (trial) {
            if constexpr (MODEL == 1) {
                // a scale or offset on its bound with the gradient pointing
                // outward is held for this step (active set); c steps freely,
                // A and B are clamped onto their boxes
                int held = 0;
                if ((p[2] <= a.fano_Alo && Nm.b[1] < 0.f) || (p[2] >= a.fano_Ahi && Nm.b[1] > 0.f)) held |= 2;
                if ((p[3] <= a.fano_Blo && Nm.b[2] < 0.f) || (p[3] >= a.fano_Bhi && Nm.b[2] > 0.f)) held |= 4;
                float d3[3] = {0.f, 0.f, 0.f};
                if (lm_solve3<float>(Nm, lambda, held, d3)) {
                    pe[0] = p[0] + d3[0];
                    pe[2] = fminf(fmaxf(p[2] + d3[1], a.fano_Alo), a.fano_Ahi);
                    pe[3] = fminf(fmaxf(p[3] + d3[2], a.fano_Blo), a.fano_Bhi);
                } else {
                    st = kSingular;
                    done = true;
                }
            } else {
                float delta[4] = {0.f, 0.f, 0.f, 0.f};
                if (lm_solve4_fast(Nm, lambda, delta)) {
#pragma unroll
                    for (int i = 0; i < 4; ++i) pe[i] = p[i] + delta[i];
                } else {
                    st = kSingular;
                    done = true;
                }
            }
        }
        // ---- sums at the trial point over the lane's tooth pairs ----
        const float* row = slots + (grp + S::kGroups * cs) * S::kRS + oc;
        // (any fixed 1/g is a consistent width for the model below)
        const float igs = MODEL == 1 ? a.fano_inv_g : rcp_fast(pe[1]);
        const float2 ig = dup2(igs);
        const float2 ncig = dup2(-pe[0] * igs);
        const float2 one = dup2(1.0f);
        const float2 nA = dup2(-pe[2]);
        const float2 nB = dup2(-pe[3]);
        float2 s[kW];
        if constexpr (MODEL == 1) {
            const float2 qq = dup2(a.fano_q);
            const float2 nq = dup2(-a.fano_q);
#pragma unroll
            for (int j = 0; j < S::kPPL; ++j) {
                const int i = gl + G * j;
                const float4 tb = tab[i];
                float2 yv;
                if (j < S::kPPL - 1) {
                    yv = make_float2(row[2 * i], row[2 * i + 1]);
                } else {
                    yv = make_float2(row[klast0], row[klast1]);
                    yv = make_float2(wlast.x != 0.f ? yv.x : 0.f, wlast.y != 0.f ? yv.y : 0.f);
                }
                yv = mul2_rounded(yv, make_float2(tb.z, tb.w));
                const float2 e = fma2(make_float2(tb.x, tb.y), ig, ncig);
                const float2 E = fma2(e, e, one);
                const float2 id = make_float2(rcp_fast(E.x), rcp_fast(E.y));
                const float2 qe = add2(e, qq);
                float2 F = mul2(mul2(qe, qe), id);
                const float2 yb = add2(yv, nB);
                float2 r = fma2(nA, F, yb);
                // (q + e)(1 - q e) / (1 + e^2)^2: -g / (2 A) x the centre column
                float2 jc = mul2(mul2(qe, fma2(nq, e, one)), mul2(id, id));
                if (j == S::kPPL - 1) {
                    F = mul2(F, wlast);
                    jc = mul2(jc, wlast);
                    r = mul2(r, wlast);
                }
                if (j == 0) {
                    s[0] = mul2(jc, jc);
                    s[1] = mul2(jc, F);
                    s[2] = jc;
                    s[3] = mul2(F, F);
                    s[4] = F;
                    s[5] = mul2(jc, r);
                    s[6] = mul2(F, r);
                    s[7] = r;
                    s[8] = mul2(r, r);
                } else {
                    s[0] = fma2(jc, jc, s[0]);
                    s[1] = fma2(jc, F, s[1]);
                    s[2] = add2(s[2], jc);
                    s[3] = fma2(F, F, s[3]);
                    s[4] = add2(s[4], F);
                    s[5] = fma2(jc, r, s[5]);
                    s[6] = fma2(F, r, s[6]);
                    s[7] = add2(s[7], r);
                    s[8] = fma2(r, r, s[8]);
                }
            }
        } else {
    #pragma unroll
            for (int j = 0; j < S::kPPL; ++j) {
                const int i = gl + G * j;
                const float4 tb = tab[i];
                float2 yv;
                if (j < S::kPPL - 1) {
                    yv = make_float2(row[2 * i], row[2 * i + 1]);
                } else {
                    yv = make_float2(row[klast0], row[klast1]);
                    yv = make_float2(wlast.x != 0.f ? yv.x : 0.f, wlast.y != 0.f ? yv.y : 0.f);
                }
                yv = mul2_rounded(yv, make_float2(tb.z, tb.w));
                const float2 e = fma2(make_float2(tb.x, tb.y), ig, ncig);
                const float2 E = fma2(e, e, one);
                float2 L = make_float2(rcp_fast(E.x), rcp_fast(E.y));
                // (y - B) is exact while y and B agree within a factor of two
                const float2 yb = add2(yv, nB);
                float2 r = fma2(nA, L, yb);
                float2 L2 = mul2(L, L);
                float2 jc = mul2(L2, e);   // g x the centre column's L q d
                if (j == S::kPPL - 1) {
                    L = mul2(L, wlast);
                    L2 = mul2(L2, wlast);
                    jc = mul2(jc, wlast);
                    r = mul2(r, wlast);
                }
                if (j == 0) {   // the first pair starts the sums (no zeroing)
                    s[0] = L2;
                    s[1] = mul2(L2, L);
                    s[2] = mul2(L2, L2);
                    s[3] = L;
                    s[4] = mul2(L, jc);
                    s[5] = mul2(L2, jc);
                    s[6] = mul2(jc, jc);
                    s[7] = jc;
                    s[8] = mul2(L, r);
                    s[9] = mul2(jc, r);
                    s[10] = mul2(L2, r);
                    s[11] = r;
                    s[12] = mul2(r, r);
                } else {
                    s[0] = add2(s[0], L2);
                    s[1] = fma2(L2, L, s[1]);
                    s[2] = fma2(L2, L2, s[2]);
                    s[3] = add2(s[3], L);
                    s[4] = fma2(L, jc, s[4]);
                    s[5] = fma2(L2, jc, s[5]);
                    s[6] = fma2(jc, jc, s[6]);
                    s[7] = add2(s[7], jc);
                    s[8] = fma2(L, r, s[8]);
                    s[9] = fma2(jc, r, s[9]);
                    s[10] = fma2(L2, r, s[10]);
                    s[11] = add2(s[11], r);
                    s[12] = fma2(r, r, s[12]);
                }
            }
        }
        float w[kW];
#pragma unroll
        for (int i = 0; i < kW; ++i) w[i] = s[i].x + s[i].y;
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
#pragma unroll
            for (int i = 0; i < kW; ++i) w[i] += __shfl_xor_sync(kFull, w[i], o);
        }
        // ---- LM bookkeeping (as fit2_kernel) ----
        // the sums of the normal equations (and chi^2 in v[13])
        LmSums Sm;
        if constexpr (MODEL == 1) {
            // the centre column is kappa jc' with kappa = -2 A / g
            const float ka = -2.0f * pe[2] * igs;
            Sm.v[0] = w[0] * (ka * ka);
            Sm.v[1] = w[1] * ka;
            Sm.v[2] = w[2] * ka;
            Sm.v[3] = w[3];
            Sm.v[4] = w[4];
            Sm.v[5] = w[5] * ka;
            Sm.v[6] = w[6];
            Sm.v[7] = w[7];
            Sm.v[13] = w[8];
        } else {
            sums_from_powers(w, igs, Sm);
        }
        auto normal = [&](Normal& N) {
            if constexpr (MODEL == 1)
                make_normal_fano(Sm, T, N);
            else
                make_normal_fast(Sm, pe[1], pe[2], T, N);
        };
        if (f >= 0 && !done) {
            const float chi2t = Sm.v[13];
            if (fresh) {
                chi2 = chi2t;
                if (!(chi2t < INFINITY)) {
                    st = kNonfinite;
                    done = true;
                } else {
                    normal(Nm);
                    if (a.max_iter <= 0) done = true;
                }
            } else {
                ++it;
                if (!(chi2t < INFINITY)) {
                    lambda *= 10.0f;
                } else if (chi2_settled(chi2t, chi2, a.tol, p[2], p[3])) {
                    if (chi2t <= chi2) {
#pragma unroll
                        for (int i = 0; i < 4; ++i) p[i] = pe[i];
                        chi2 = chi2t;
                    }
                    st = kConverged;
                    done = true;
                } else if (chi2t < chi2) {
#pragma unroll
                    for (int i = 0; i < 4; ++i) p[i] = pe[i];
                    chi2 = chi2t;
                    normal(Nm);
                    lambda *= 0.1f;
                } else {
                    lambda *= 10.0f;
                }
                if (!done && it >= a.max_iter) done = true;
            }
        }
        fresh = false;
        if (f >= 0 && done) {
            if (gl == 0) {
                float* po = a.params + fr * 4;
                po[0] = fmaf(a.x_scale, p[0], a.x_mid);
                po[1] = a.x_scale * fabsf(p[1]);
                po[2] = p[2];
                po[3] = p[3];
                if (a.rss) a.rss[fr] = chi2;
                if (a.iters) a.iters[fr] = static_cast<int16_t>(it + a.iters_base);
                if (a.status) a.status[fr] = static_cast<int16_t>(st | flag | a.status_or);
                if (a.fb_list && (st == kMaxIter || st == kSingular))
                    a.fb_list[atomicAdd(a.fb_count, 1)] = static_cast<int>(fr);
            }
            f = -1;
        }
    }
    // no copy may land after the block exits: wait (bounded) for the copies
    // still in flight (after a failed wait only)
    if (fn >= 0) {
        const int nx = cs ^ 1;
        tc::mbar_wait(&bars[grp + S::kGroups * nx], (ph >> nx) & 1u, 1u << 22);
    }
    if (failed && lane == 0 && a.err) atomicExch(a.err, 4);
}

template <int G, int T, int MODEL>
void* fit3_fn()
{
    return reinterpret_cast<void*>(&fit3_kernel<G, T, MODEL>);
}

template <int G, int T>
size_t fit3_bytes(int warps)
{
    using S = Fit3Shape<G, T>;
    return sizeof(float4) * S::kTab + static_cast<size_t>(warps) * S::kSlots * (sizeof(uint64_t) + sizeof(float) * S::kRS);
}

struct Fit3Inst {
    int G, T, model;
    int f64;   // 1: the instance for the FP64 solve (one lane per frame where it fits)
    void* (*fn)();
    size_t (*bytes)(int);
};
// the workload geometries: 21 teeth (one lane per frame), 99 (two lanes),
// 201 and 221 (four lanes)
// (the Fano profile at the paper's 99 teeth)
// (FP64 solve: one lane per frame at 21 and 99 teeth, so that all 32 lanes
// of a warp solve at once; at 201 and 221 teeth the slots of one lane per
// frame do not fit, and the group leaders solve)
const Fit3Inst kFit3[] = {
    {1, 21, 0, 0, fit3_fn<1, 21, 0>, fit3_bytes<1, 21>},
    {2, 99, 0, 0, fit3_fn<2, 99, 0>, fit3_bytes<2, 99>},
    {4, 201, 0, 0, fit3_fn<4, 201, 0>, fit3_bytes<4, 201>},
    {4, 221, 0, 0, fit3_fn<4, 221, 0>, fit3_bytes<4, 221>},
    {2, 99, 1, 0, fit3_fn<2, 99, 1>, fit3_bytes<2, 99>},
    {1, 21, 0, 1, fit3_fn<1, 21, 0>, fit3_bytes<1, 21>},
    {1, 99, 0, 1, fit3_fn<1, 99, 0>, fit3_bytes<1, 99>},
    {4, 201, 0, 1, fit3_fn<4, 201, 0>, fit3_bytes<4, 201>},
    {4, 221, 0, 1, fit3_fn<4, 221, 0>, fit3_bytes<4, 221>},
    {1, 99, 1, 1, fit3_fn<1, 99, 1>, fit3_bytes<1, 99>},
};

const Fit3Inst* fit3_find(int T, int model, int f64)
{
    for (const Fit3Inst& f : kFit3)
        if (f.T == T && f.model == model && f.f64 == f64) return &f;
    return nullptr;
}

}  // namespace

// Chooses the shared-memory kernel for the plan when one is instantiated for
// its tooth count: lanes per frame, warps per block (the most that let two
// blocks share an SM), its grid.  Leaves fit3_ok false otherwise.
cudaError_t setup_fit3(cg_plan_s* p)
{
    p->fit3_ok = false;
    const Fit3Inst* fi = fit3_find(p->T, p->opts.model, p->solve_f64 ? 1 : 0);
    if (!fi) return cudaSuccess;
    int smem_sm = 0, smem_block = 0;
    cudaError_t e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, p->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_block, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device);
    if (e != cudaSuccess) return e;
    int warps = 8;
    while (warps > 1 && (2 * (fi->bytes(warps) + 1024) > static_cast<size_t>(smem_sm) ||
                         fi->bytes(warps) > static_cast<size_t>(smem_block)))
        --warps;
    const size_t bytes = fi->bytes(warps);
    if (bytes > static_cast<size_t>(smem_block)) return cudaSuccess;
    void* fn = fi->fn();
    if ((e = raise_smem_limit(fn, static_cast<int>(bytes))) != cudaSuccess) return e;
    int occ = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, 32 * warps, bytes)) != cudaSuccess) return e;
    if (occ < 1) return cudaSuccess;
    p->fit3_G = fi->G;
    p->fit3_warps = warps;
    p->fit3_smem = static_cast<int>(bytes);
    p->grid_fit3 = p->num_sms * occ;
    p->fit3_ok = true;
    return cudaSuccess;
}

cudaError_t launch_fit3(const cg_plan_s* p, Fit2Args a, cudaStream_t s)
{
    const Fit3Inst* fi = fit3_find(p->T, p->opts.model, p->solve_f64 ? 1 : 0);
    if (!fi || !p->fit3_ok) return cudaErrorInvalidValue;
    const int gpw = 32 / fi->G;   // groups per warp
    a.task = 2 * gpw;
    const int64_t tasks = (a.n + a.task - 1) / a.task;
    const int64_t blocks = (tasks + p->fit3_warps - 1) / p->fit3_warps;
    const int grid = static_cast<int>(blocks < p->grid_fit3 ? blocks : p->grid_fit3);
    cudaError_t e = cudaMemsetAsync(a.counter, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    void* args[] = {&a};
    return cudaLaunchKernel(fi->fn(), dim3(grid), dim3(32 * p->fit3_warps), args, p->fit3_smem, s);
}

}  // namespace cg
