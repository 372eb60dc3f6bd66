// cg_fast.cu -- the throughput path for comb geometries whose tooth bins lie in
// one residue pair +-r mod 10 (every 1 us-frame workload: N = 10 P Q).
//
// fast_readout_kernel<P, Q, PAIR>: cast + coset transform + tooth readout +
//   moment initial guess for a batch of frames per thread block:
//   * the next batch's int16 samples stream into shared memory with cp.async
//     while the current batch is transformed;
//   * stage 1 (one thread per frame and residue a < P, or per pair a, a+1):
//     the radix-10 fold of the samples at n1 = a + P b, using the symmetry
//     W_10^(r (n2+5)) = -W_10^(r n2) for odd r, times W_N^(r n1), then a Q-point
//     DFT over b in registers and the twiddle W_L^(u a);
//   * stage 2 (one thread per frame and u < Q): a P-point DFT over a gives
//     Z[u + Q v] = X_{10 (u + Q v) + r}; teeth read their |Z|;
//   * amplitudes leave coalesced; the moment initial guess of each frame is
//     written as its starting parameters.
// fit2_kernel<G, PPL>: Levenberg-Marquardt with each lane's PPL points in
//   registers; the groups of a warp pull frames from the warp's task one by one
//   as their previous frame finishes, so no group waits for another frame's
//   iterations.
//
// Paper: "Data Capture and Processing" (cast on the GPU, FFT per 1 us row,
// tooth selection and mapping, reference normalisation, LM fit).
#include <algorithm>
#include <cstdint>
#include <cuda_runtime.h>

#include "cg_fft.cuh"
#include "cg_fit.cuh"
#include "cg_internal.h"
#include "cg_net.cuh"
#include "cg_stage.cuh"
#include "cg_tc.cuh"

namespace cg {

template <int P, int Q, class S>
__global__ void __launch_bounds__(128) fast_readout_kernel(FastArgs a)
{
    constexpr int L = P * Q;
    constexpr int MH = 5;                     // M / 2 with M = 10
    // long Q-point transforms: the fold runs as its own stage with one item
    // per output (balanced over the block) and the Q-point DFTs read it back
    constexpr bool kSplitFold = Q > 11;
    extern __shared__ __align__(16) unsigned char sm[];
    float2* twL = reinterpret_cast<float2*>(sm + a.sm_twL);
    float2* twN = reinterpret_cast<float2*>(sm + a.sm_twN);
    int* tom = reinterpret_cast<int*>(sm + a.sm_tom);
    float* iref = reinterpret_cast<float*>(sm + a.sm_iref);
    S* raw = reinterpret_cast<S*>(sm + a.sm_raw);
    const S* frames = static_cast<const S*>(a.frames);
    float2* Yb = reinterpret_cast<float2*>(sm + a.sm_Y);
    const int T = a.T, N = a.N, F = a.F;
    for (int i = threadIdx.x; i < L; i += blockDim.x) {
        twL[i] = a.twL[i];
        twN[i] = a.twN[i];
        tom[i] = a.tooth_of_m[i];
    }
    for (int i = threadIdx.x; i < T; i += blockDim.x) iref[i] = a.inv_ref[i];
    // fold twiddles w_j = W_10^(r j): with s = (-1)^r, w_{5-j} = s conj(w_j), so
    // sum_j D_j w_j = D_0 + (E_1 c_1 + E_2 c_2) + i (F_1 s_1 + F_2 s_2) where
    // D_j = x_j + s x_{j+5}, E_j = D_j + s D_{5-j}, F_j = D_j - s D_{5-j}
    const float c1 = a.twM[1].x, s1 = a.twM[1].y, c2 = a.twM[2].x, s2 = a.twM[2].y;
    const int sg = a.pair_isign;

    const int64_t nb = (a.n_frames + F - 1) / F;
    int64_t b = blockIdx.x;
    int off = 0;
    if (b < nb) {
        const int nf0 = static_cast<int>((a.n_frames - b * F) < F ? (a.n_frames - b * F) : F);
        off = stage_async(frames, b * F * static_cast<int64_t>(N), static_cast<int64_t>(nf0) * N, raw);
    }
    for (; b < nb; b += gridDim.x) {
        const int64_t f0 = b * F;
        const int nf = static_cast<int>((a.n_frames - f0) < F ? (a.n_frames - f0) : F);
        cp_async_wait_all();
        __syncthreads();
        int offn = 0;
        if constexpr (kSplitFold) {
            // ---------------- stage 0: the fold, one item per output m ------
            for (int item = threadIdx.x; item < nf * L; item += blockDim.x) {
                const int f = item / L;
                const int m = item - f * L;
                const S* xp = raw + off + f * N + m;
                int D[MH];
#pragma unroll
                for (int j = 0; j < MH; ++j) D[j] = static_cast<int>(xp[L * j]) + sg * static_cast<int>(xp[L * (j + MH)]);
                const int E1 = D[1] + sg * D[4], F1 = D[1] - sg * D[4];
                const int E2 = D[2] + sg * D[3], F2 = D[2] - sg * D[3];
                float2 fz;
                fz.x = fmaf(static_cast<float>(E2), c2, fmaf(static_cast<float>(E1), c1, static_cast<float>(D[0])));
                fz.y = fmaf(static_cast<float>(F2), s2, static_cast<float>(F1) * s1);
                Yb[f * L + m] = cmul(fz, twN[m]);
            }
            __syncthreads();
            // raw is free: start the next batch's samples
            const int64_t bn = b + gridDim.x;
            if (bn < nb) {
                const int nfn = static_cast<int>((a.n_frames - bn * F) < F ? (a.n_frames - bn * F) : F);
                offn = stage_async(frames, bn * F * static_cast<int64_t>(N), static_cast<int64_t>(nfn) * N, raw);
            }
            // ---------------- stage 1: Q-point DFT over b, twiddle (in place) --
            for (int item = threadIdx.x; item < nf * P; item += blockDim.x) {
                const int f = item / P;
                const int a0 = item - f * P;
                float2* Yf = Yb + f * L + a0;
                float2 z[Q];
#pragma unroll
                for (int bq = 0; bq < Q; ++bq) z[bq] = Yf[P * bq];
                Dft<Q>::run(z);
#pragma unroll
                for (int u = 0; u < Q; ++u) Yf[u * P] = u ? cmul(z[u], twL[u * a0]) : z[u];
            }
            __syncthreads();
        } else {
            // ---------------- stage 1: fold, Q-point DFT, twiddle ----------------
            for (int item = threadIdx.x; item < nf * P; item += blockDim.x) {
                const int f = item / P;
                const int a0 = item - f * P;
                const S* xs = raw + off + f * N + a0;
                float2 z[Q];
#pragma unroll
                for (int bq = 0; bq < Q; ++bq) {
                    const S* xp = xs + P * bq;
                    int D[MH];
#pragma unroll
                    for (int j = 0; j < MH; ++j) D[j] = static_cast<int>(xp[L * j]) + sg * static_cast<int>(xp[L * (j + MH)]);
                    const int E1 = D[1] + sg * D[4], F1 = D[1] - sg * D[4];
                    const int E2 = D[2] + sg * D[3], F2 = D[2] - sg * D[3];
                    float2 fz;
                    fz.x = fmaf(static_cast<float>(E2), c2, fmaf(static_cast<float>(E1), c1, static_cast<float>(D[0])));
                    fz.y = fmaf(static_cast<float>(F2), s2, static_cast<float>(F1) * s1);
                    z[bq] = cmul(fz, twN[a0 + P * bq]);
                }
                Dft<Q>::run(z);
                float2* Yf = Yb + f * L + a0;
#pragma unroll
                for (int u = 0; u < Q; ++u) Yf[u * P] = u ? cmul(z[u], twL[u * a0]) : z[u];
            }
            __syncthreads();
            // raw is free: start the next batch's samples
            const int64_t bn = b + gridDim.x;
            if (bn < nb) {
                const int nfn = static_cast<int>((a.n_frames - bn * F) < F ? (a.n_frames - bn * F) : F);
                offn = stage_async(frames, bn * F * static_cast<int64_t>(N), static_cast<int64_t>(nfn) * N, raw);
            }
        }
        // ---------------- stage 2: P-point DFT over a, tooth magnitudes -------
        for (int item = threadIdx.x; item < nf * Q; item += blockDim.x) {
            const int f = item / Q;
            const int u = item - f * Q;
            const float2* Yf = Yb + f * L + u * P;
            float2 z[P];
#pragma unroll
            for (int q = 0; q < P; q += 2) {
                const float4 v = *reinterpret_cast<const float4*>(Yf + q);
                z[q] = make_float2(v.x, v.y);
                z[q + 1] = make_float2(v.z, v.w);
            }
            Dft<P>::run(z);
            // straight to global memory: the items of a frame hold runs of
            // consecutive bins, i.e. runs of consecutive (or reversed) teeth
            const int64_t orow = (f0 + f) * T;
#pragma unroll
            for (int v = 0; v < P; ++v) {
                const int k = tom[u + Q * v];
                if (k >= 0) {
                    const float av = cabs_approx(z[v]);
                    if (a.amps) a.amps[orow + k] = av;
                    if (a.y) a.y[orow + k] = __fmul_rn(av, iref[k]);
                }
            }
        }
        // (the next batch's stages start after the barrier at the loop top)
        off = offn;
    }
    cp_async_wait_all();
}

// ---------------------------------------------------------------------------
// moment initial guess, one lane per frame
// ---------------------------------------------------------------------------
// Moment initial guess from the baseline B0 (the median of the outer teeth):
// d = y - B0, s = sign of the largest |d|, w = max(s d, 0); c0 = centroid of
// w over the abscissa, A0 = s max w, g0 = area / (pi |A0|) clamped to
// [du / 2, span / 2]; a flat spectrum gives c0 = u_mid and a flag.  y(k)
// returns tooth k's normalised value, u(k) its abscissa.
template <class Y, class U>
__device__ __forceinline__ void moment_finish(Y y, U u, int T, float B0, float u_mid, float du, float span,
                                              float x_mid, float x_scale, float* po, int16_t* flag_out)
{
    // one pass: the extreme deviation and the excess sums of both signs (the
    // sign picks one set at the end; each sum sees the same terms in the same
    // order as a second pass would)
    float best = -1.f;
    float dbest = y(0) - B0;
    float Wp = 0.f, Wup = 0.f, wmaxp = 0.f, Wn = 0.f, Wun = 0.f, wmaxn = 0.f;
    for (int k = 0; k < T; ++k) {
        const float d = y(k) - B0;
        const float dv = fabsf(d);
        if (dv > best) {
            best = dv;
            dbest = d;
        }
        const float wp = fmaxf(d, 0.f), wn = fmaxf(-d, 0.f);
        const float uk = u(k);
        Wp += wp;
        Wup = fmaf(wp, uk, Wup);
        wmaxp = fmaxf(wmaxp, wp);
        Wn += wn;
        Wun = fmaf(wn, uk, Wun);
        wmaxn = fmaxf(wmaxn, wn);
    }
    const float sgn = dbest >= 0.f ? 1.0f : -1.0f;
    const float W = sgn > 0.f ? Wp : Wn, Wu = sgn > 0.f ? Wup : Wun, wmax = sgn > 0.f ? wmaxp : wmaxn;
    float c0, g0, A0;
    int flag = 0;
    if (!(W > 0.f)) {
        c0 = u_mid;
        g0 = 0.5f * du;
        A0 = 0.f;
        flag = kInitFlat;
    } else {
        A0 = sgn * wmax;
        g0 = W * du / (3.14159265358979f * fabsf(A0));
        g0 = fminf(fmaxf(g0, 0.5f * du), 0.5f * span);
        c0 = Wu / W;
    }
    po[0] = fmaf(x_scale, c0, x_mid);
    po[1] = x_scale * g0;
    po[2] = A0;
    po[3] = B0;
    if (flag_out) *flag_out = static_cast<int16_t>(flag);
}

// A warp takes 32 consecutive frames at a time: their normalised spectra
// (row stride odd, so the lanes' reads of one tooth fall on distinct banks)
// arrive in shared memory by one bulk copy per 32 rows, double-buffered so the
// next rows land while these are read (else by coalesced loads); each lane
// then computes its frame's guess as the oracle defines it: baseline = median
// of the outer fifth (sorted with the network, +inf padding), sign of the
// largest deviation, centroid / extreme / area of the one-signed excess.
// NOUT > 0: the outer set has NOUT teeth (a compile-time count): its median
// comes from the merge network pruned to the two middle ranks; NOUT = 0 sorts
// the NPAD wires (a.n_outer real, the rest +infinity) fully
template <int NPAD, int NOUT>
__global__ void __launch_bounds__(128) init_kernel(InitArgs a)
{
    extern __shared__ __align__(16) float ism[];
    const int T = a.T, TS = a.row_stride;
    float* us = ism;
    float* iref = us + T;
    int* outer = reinterpret_cast<int*>(iref + T);
    // per warp two mbarriers and two 32-row buffers (task t lands in buffer
    // t % 2 while the other one is read)
    const int warp = threadIdx.x >> 5;
    uint64_t* bars = reinterpret_cast<uint64_t*>(ism + ((2 * T + a.n_outer + 3) & ~3)) + 2 * warp;
    float* rows0 = reinterpret_cast<float*>(reinterpret_cast<uint64_t*>(ism + ((2 * T + a.n_outer + 3) & ~3)) + 8) +
                   warp * 2 * 32 * TS;
    const int lane = threadIdx.x & 31;
    if (lane == 0) {
        tc::mbar_init(&bars[0], 1);
        tc::mbar_init(&bars[1], 1);
        tc::fence_mbar_init();
    }
    for (int i = threadIdx.x; i < T; i += blockDim.x) {
        us[i] = a.u[i];
        iref[i] = a.inv_ref[i];
    }
    for (int i = threadIdx.x; i < a.n_outer; i += blockDim.x) outer[i] = a.outer_idx[i];
    __syncthreads();
    constexpr OddEvenNet<NPAD> net{};
    const int64_t nwarps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
    int64_t n = a.n;
    if (a.list_n) {
        const int64_t c = *a.list_n;
        n = c < n ? c : n;
    }
    const float* srcbase = a.y ? a.y : a.amps;
    // a whole task of 32 contiguous rows goes by one bulk copy (16-byte
    // aligned: 32 rows of odd T floats are 128 T bytes)
    auto bulk_ok = [&](int64_t task) {
        return a.bulk && !a.list && (task + 1) * 32 <= n &&
               (reinterpret_cast<uintptr_t>(srcbase + task * 32 * T) & 15) == 0;
    };
    auto issue = [&](int64_t task, int b) {
        if (lane == 0) {
            tc::fence_proxy_async_smem();   // generic reads of the buffer are ordered before the copy
            tc::mbar_arrive_expect_tx(&bars[b], static_cast<uint32_t>(32 * T * 4));
            tc::bulk_g2s(rows0 + b * 32 * TS, srcbase + task * 32 * T, static_cast<uint32_t>(32 * T * 4), &bars[b]);
        }
    };
    uint32_t phase = 0u, pending = 0u;   // bit b: buffer b's parity / a copy in flight
    int64_t task = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + warp;
    if (task * 32 < n && bulk_ok(task)) {
        issue(task, 0);
        pending |= 1u;
    }
    bool failed = false;
    for (int b = 0; task * 32 < n; task += nwarps, b ^= 1) {
        float* rows = rows0 + b * 32 * TS;
        const int64_t f0 = task * 32;
        const int nf = (n - f0) < 32 ? static_cast<int>(n - f0) : 32;
        // the next task's copy goes out before this one is read
        const int64_t nt = task + nwarps;
        __syncwarp();
        if (nt * 32 < n && bulk_ok(nt)) {
            issue(nt, b ^ 1);
            pending |= 1u << (b ^ 1);
        }
        const bool in_smem_raw = (pending >> b) & 1u;   // rows hold y, or amps still to be scaled
        if (in_smem_raw) {
            if (!tc::mbar_wait(&bars[b], (phase >> b) & 1u, 1u << 24)) {
                failed = true;
                break;
            }
            phase ^= 1u << b;
            pending &= ~(1u << b);
        } else if (a.list) {
            // listed frames (the fallback pass): one coalesced row at a time
            for (int f = 0; f < nf; ++f) {
                const int64_t fr = a.list[f0 + f];
                const float* src = srcbase + fr * T;
                for (int k = lane; k < T; k += 32) rows[f * TS + k] = a.y ? src[k] : __fmul_rn(src[k], iref[k]);
            }
        } else {
            // the 32 rows are contiguous in global memory: one flat coalesced
            // sweep, eight loads in flight per lane, (frame, tooth) tracked
            // incrementally
            const float* src = srcbase + f0 * T;
            const int total = nf * T;
            auto put = [&](float v, int f, int k) { rows[f * TS + k] = a.y ? v : __fmul_rn(v, iref[k]); };
            if ((reinterpret_cast<uintptr_t>(src) & 15) == 0) {
                // 16-byte loads (a task starts at a multiple of 32 rows, so
                // the block is aligned whenever the array is)
                const float4* src4 = reinterpret_cast<const float4*>(src);
                const int total4 = total >> 2;
                const int qT = 128 / T, rT = 128 - qT * T;   // one step of 32 lanes x 4 values
                int f = (4 * lane) / T, k = 4 * lane - ((4 * lane) / T) * T;
                for (int j0 = 0; j0 < total4; j0 += 8 * 32) {
                    float4 v[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int jj = j0 + q * 32 + lane;
                        v[q] = jj < total4 ? src4[jj] : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        if (j0 + q * 32 + lane < total4) {
                            const float e4[4] = {v[q].x, v[q].y, v[q].z, v[q].w};
                            int ff = f, kk = k;
#pragma unroll
                            for (int i = 0; i < 4; ++i) {
                                put(e4[i], ff, kk);
                                if (++kk == T) {
                                    kk = 0;
                                    ++ff;
                                }
                            }
                        }
                        f += qT;
                        k += rT;
                        if (k >= T) {
                            k -= T;
                            ++f;
                        }
                    }
                }
                for (int e = 4 * total4 + lane; e < total; e += 32) put(src[e], e / T, e - (e / T) * T);
            } else {
                int f = lane / T, k = lane - (lane / T) * T;
                for (int e0 = 0; e0 < total; e0 += 8 * 32) {
                    float v[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int e = e0 + q * 32 + lane;
                        v[q] = e < total ? src[e] : 0.f;
                    }
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int e = e0 + q * 32 + lane;
                        if (e < total) put(v[q], f, k);
                        k += 32;
                        while (k >= T) {
                            k -= T;
                            ++f;
                        }
                    }
                }
            }
        }
        __syncwarp();
        if (lane < nf) {
            const int64_t fo = a.list ? static_cast<int64_t>(a.list[f0 + lane]) : f0 + lane;
            const float* r = rows + lane * TS;
            // bulk-copied magnitudes are normalised here, as the staging does
            const bool scale = in_smem_raw && !a.y;
            auto yk = [&](int k) { return scale ? __fmul_rn(r[k], iref[k]) : r[k]; };
            float v[NPAD];
            float B0;
            if constexpr (NOUT > 0) {
#pragma unroll
                for (int i = 0; i < NPAD; ++i) v[i] = i < NOUT ? yk(outer[i]) : INFINITY;
                constexpr int kLo = (NOUT - 1) / 2, kHi = NOUT / 2;
                rank_network<NPAD, NOUT, kLo, kHi>(v);
                B0 = 0.5f * (v[kLo] + v[kHi]);
            } else {
#pragma unroll
                for (int i = 0; i < NPAD; ++i) v[i] = (i < a.n_outer) ? yk(outer[i]) : INFINITY;
#pragma unroll
                for (int c = 0; c < OddEvenNet<NPAD>::kCount; ++c) {
                    const float lo = fminf(v[net.lo[c]], v[net.hi[c]]);
                    const float hi = fmaxf(v[net.lo[c]], v[net.hi[c]]);
                    v[net.lo[c]] = lo;
                    v[net.hi[c]] = hi;
                }
                const int rlo = (a.n_outer - 1) >> 1, rhi = a.n_outer >> 1;
                float vlo = 0.f, vhi = 0.f;
#pragma unroll
                for (int i = 0; i < NPAD; ++i) {
                    vlo = (i == rlo) ? v[i] : vlo;
                    vhi = (i == rhi) ? v[i] : vhi;
                }
                B0 = 0.5f * (vlo + vhi);
            }
            moment_finish(yk, [&](int k) { return us[k]; }, T, B0, a.u_mid, a.du, a.span, a.x_mid, a.x_scale,
                          a.p0_out + fo * 4, a.flag_out ? a.flag_out + fo : nullptr);
        }
    }
    // no copy may land after the block exits
    __syncwarp();
    for (int b = 0; b < 2; ++b)
        if (((pending >> b) & 1u) && !tc::mbar_wait(&bars[b], (phase >> b) & 1u, 1u << 24)) failed = true;
    if (failed && lane == 0 && a.err) atomicExch(a.err, 2);
}

// ---------------------------------------------------------------------------
// fit2: LM with each lane's spectrum points in registers and a per-warp frame
// queue.  EXACT: PPL == ceil(T / G), so only the last point of a lane can lie
// beyond T.
// ---------------------------------------------------------------------------
template <int G, int PPL, bool EXACT, int MODEL>
__global__ void __launch_bounds__(G == 1 ? 128 : 256, G == 1 ? 3 : 2) fit2_kernel(Fit2Args a)
{
    extern __shared__ __align__(16) float fsm[];
    const int T = a.T;
    float* us = fsm;
    float* iref = fsm + T;
    // per lane a slot of PPL points (odd stride: conflict-free) for the
    // group's next frame, copied asynchronously while the current one is fit
    // (G >= 2; one lane per frame runs the shared-memory kernel instead)
    constexpr bool kPrefetch = G >= 2;
    constexpr int kSlot = PPL | 1;
    float* const slot = kPrefetch ? fsm + 2 * T + static_cast<int>(threadIdx.x) * kSlot : nullptr;
    for (int i = threadIdx.x; i < T; i += blockDim.x) {
        us[i] = a.u[i];
        iref[i] = a.inv_ref[i];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int gl = lane & (G - 1);
    const int leader_lane = lane & ~(G - 1);
    const float inv_scale = 1.0f / a.x_scale;
    int64_t next = 0, end = 0;   // current task [next, end); tasks come from a.counter
    int64_t n = a.n;
    if (a.list_n) {
        const int64_t c = *a.list_n;
        n = c < n ? c : n;
    }

    int64_t f = -1, fr = -1;     // task index, frame index being fit
    int64_t fn = -1, frn = -1;   // the group's next frame (copy in flight)
    float yv[PPL];
#pragma unroll
    for (int j = 0; j < PPL; ++j) yv[j] = 0.f;
    float p[4] = {0.f, 1.f, 0.f, 0.f};
    float lambda = a.lambda0, chi2 = 0.f;
    Normal Nm;
#pragma unroll
    for (int i = 0; i < 10; ++i) Nm.H[i] = 0.f;
#pragma unroll
    for (int i = 0; i < 4; ++i) Nm.b[i] = 0.f;
    int it = 0, st = kMaxIter, flag = 0;
    bool fresh = false;

    while (true) {
        // ---- hand frames to groups (a group's lanes agree): with prefetch a
        //      group claims its next frame while fitting the current one ----
        unsigned need = __ballot_sync(kFull, gl == 0 && (kPrefetch ? fn < 0 : f < 0));
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
                if constexpr (kPrefetch) {
                    fn = next + rank;
                    frn = a.list ? static_cast<int64_t>(a.list[fn]) : fn;
                    const float* src = (a.y ? a.y : a.amps) + frn * T;
#pragma unroll
                    for (int j = 0; j < PPL; ++j) {
                        const int k = gl + G * j;
                        if (k < T) cp_async4(slot + j, src + k);
                    }
                } else {
                    f = next + rank;
                    fresh = true;
                }
            }
            next += take;
            need = __ballot_sync(kFull, gl == 0 && (kPrefetch ? fn < 0 : f < 0));
        }
        // p, flag, lambda and counters of a frame that starts now
        auto start_frame = [&]() {
            if constexpr (MODEL == 1) {
                // a given centre (the median-filter guess), else the lowest
                // tooth of the group's frame (first on ties); the profile's
                // minimum (e = -q) moved onto the centre
                float best = INFINITY;
                int bk = 0x7fffffff;
#pragma unroll
                for (int j = 0; j < PPL; ++j) {
                    const int k = gl + G * j;
                    if (((EXACT && j < PPL - 1) || k < T) && yv[j] < best) {
                        best = yv[j];
                        bk = k;
                    }
                }
                const unsigned gmask = G == 32 ? kFull : (((1u << G) - 1u) << leader_lane);
#pragma unroll
                for (int o = G / 2; o > 0; o >>= 1) {
                    const float ob = __shfl_xor_sync(gmask, best, o);
                    const int ok2 = __shfl_xor_sync(gmask, bk, o);
                    if (ob < best || (ob == best && ok2 < bk)) {
                        best = ob;
                        bk = ok2;
                    }
                }
                p[0] = a.p0 ? (a.p0[fr * 4] - a.x_mid) * inv_scale : (bk < T ? us[bk] : 0.f) + a.fano_shift;
                p[1] = a.fano_g;
                p[2] = fminf(fmaxf(a.fano_A0, a.fano_Alo), a.fano_Ahi);
                p[3] = fminf(fmaxf(a.fano_B0, a.fano_Blo), a.fano_Bhi);
                flag = 0;
            } else {
                const float* q = a.p0 + fr * 4;
                p[0] = (q[0] - a.x_mid) * inv_scale;
                p[1] = q[1] * inv_scale;
                p[2] = q[2];
                p[3] = q[3];
                flag = a.flags_in ? (a.flags_in[fr] & kInitFlat) : 0;
            }
            lambda = a.lambda0;
            it = 0;
            st = kMaxIter;
        };
        if constexpr (kPrefetch) {
            cp_async_commit();
            // a group with no current frame starts its next one
            if (f < 0 && fn >= 0) {
                f = fn;
                fr = frn;
                fn = frn = -1;
                fresh = true;
                cp_async_wait_all();
#pragma unroll
                for (int j = 0; j < PPL; ++j) {
                    const int k = gl + G * j;
                    yv[j] = (k < T) ? (a.y ? slot[j] : __fmul_rn(slot[j], iref[k])) : 0.f;
                }
                start_frame();
            }
            if (!__any_sync(kFull, f >= 0 || fn >= 0)) break;
        } else {
            if (!__any_sync(kFull, f >= 0)) break;
            if (fresh) {
                fr = a.list ? static_cast<int64_t>(a.list[f]) : f;
                if (a.y) {
                    const float* src = a.y + fr * T;
#pragma unroll
                    for (int j = 0; j < PPL; ++j) {
                        const int k = gl + G * j;
                        yv[j] = (k < T) ? src[k] : 0.f;
                    }
                } else {
                    const float* src = a.amps + fr * T;
#pragma unroll
                    for (int j = 0; j < PPL; ++j) {
                        const int k = gl + G * j;
                        yv[j] = (k < T) ? __fmul_rn(src[k], iref[k]) : 0.f;
                    }
                }
                start_frame();
            }
        }
        // ---- trial point ----
        float pe[4] = {p[0], p[1], p[2], p[3]};
        bool done = false;
        const bool trial = (f >= 0 && !fresh);
        float delta[4] = {0.f, 0.f, 0.f, 0.f};
        bool ok = true;
        // the solve of the model's free parameters (Fano: c, A, B into delta[0..2])
        auto solve = [&](bool f64) -> bool {
            if constexpr (MODEL == 1) {
                // a scale or offset on its bound with the gradient pointing
                // outward is held for this step (active set)
                int held = 0;
                if ((p[2] <= a.fano_Alo && Nm.b[1] < 0.f) || (p[2] >= a.fano_Ahi && Nm.b[1] > 0.f)) held |= 2;
                if ((p[3] <= a.fano_Blo && Nm.b[2] < 0.f) || (p[3] >= a.fano_Bhi && Nm.b[2] > 0.f)) held |= 4;
                float d3[3] = {0.f, 0.f, 0.f};
                const bool r = f64 ? lm_solve3<double>(Nm, lambda, held, d3) : lm_solve3<float>(Nm, lambda, held, d3);
                delta[0] = d3[0];
                delta[1] = d3[1];
                delta[2] = d3[2];
                return r;
            } else {
                return f64 ? lm_solve4_f64(Nm, lambda, delta) : lm_solve4_fast(Nm, lambda, delta);
            }
        };
        if (G > 1 && a.solve_f64) {
            // FP64 is scarce: the group's leader solves, the group takes its step
            int okl = 0;
            if (trial && gl == 0) okl = solve(true) ? 1 : 0;
            okl = __shfl_sync(kFull, okl, leader_lane);
#pragma unroll
            for (int i = 0; i < 4; ++i) delta[i] = __shfl_sync(kFull, delta[i], leader_lane);
            ok = okl != 0;
        } else if (trial) {
            ok = solve(a.solve_f64 != 0);
        }
        if (trial) {
            if (ok) {
                if constexpr (MODEL == 1) {
                    // c steps freely; A and B are clamped onto their boxes
                    pe[0] = p[0] + delta[0];
                    pe[2] = fminf(fmaxf(p[2] + delta[1], a.fano_Alo), a.fano_Ahi);
                    pe[3] = fminf(fmaxf(p[3] + delta[2], a.fano_Blo), a.fano_Bhi);
                } else {
#pragma unroll
                    for (int i = 0; i < 4; ++i) pe[i] = p[i] + delta[i];
                }
            } else {
                st = kSingular;
                done = true;
            }
        }
        // ---- sums at the trial point (every lane takes part) ----
        LmSums S;
#pragma unroll
        for (int i = 0; i < 14; ++i) S.v[i] = 0.f;
        const float g2 = pe[1] * pe[1];
#pragma unroll
        for (int j = 0; j < PPL; ++j) {
            const int k = gl + G * j;
            if ((EXACT && j < PPL - 1) || k < T) {
                if constexpr (MODEL == 1)
                    accum_point_fano(us[k], yv[j], pe[0], a.fano_inv_g, a.fano_q, pe[2], pe[3], S);
                else
                    accum_point(us[k], yv[j], pe[0], g2, pe[2], pe[3], S);
            }
        }
        if constexpr (G > 1) reduce_sums<G>(S);
        // ---- LM bookkeeping ----
        auto normal = [&](const LmSums& Sx, const float (&px)[4], Normal& N) {
            if constexpr (MODEL == 1)
                make_normal_fano(Sx, T, N);
            else
                make_normal_fast(Sx, px[1], px[2], T, N);
        };
        if (f >= 0 && !done) {
            const float chi2t = S.v[13];
            if (fresh) {
                chi2 = chi2t;
                if (!(chi2t < INFINITY)) {
                    st = kNonfinite;
                    done = true;
                } else {
                    normal(S, pe, Nm);
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
                    normal(S, pe, Nm);
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
                if (a.fb_list && (st == kMaxIter || st == kSingular)) a.fb_list[atomicAdd(a.fb_count, 1)] = static_cast<int>(fr);
            }
            f = -1;
        }
    }
    if constexpr (kPrefetch) cp_async_wait_all();
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
template <int P, int Q, class S>
static void* fast_fn() { return reinterpret_cast<void*>(&fast_readout_kernel<P, Q, S>); }

// the instantiated coset readouts: L = 10 Q with Q in {10, 11, 22, 25};
// int16 samples, and int8 samples for the 8-bit 2200-sample frame (Q = 22)
void* fast_readout_ptr(int Q, int sample_bytes)
{
    if (sample_bytes == 1) return Q == 22 ? fast_fn<10, 22, int8_t>() : nullptr;
    switch (Q) {
    case 10: return fast_fn<10, 10, int16_t>();
    case 11: return fast_fn<10, 11, int16_t>();
    case 22: return fast_fn<10, 22, int16_t>();
    case 25: return fast_fn<10, 25, int16_t>();
    default: return nullptr;
    }
}

// the outer-set sizes of the workload geometries (21, 99, 201 and 221 teeth:
// the outer fifth with ties kept) have their own pruned median
void* init_ptr(int npad, int n_outer)
{
    switch (n_outer) {
    case 6: return reinterpret_cast<void*>(&init_kernel<8, 6>);
    case 20: return reinterpret_cast<void*>(&init_kernel<32, 20>);
    case 42: return reinterpret_cast<void*>(&init_kernel<64, 42>);
    case 46: return reinterpret_cast<void*>(&init_kernel<64, 46>);
    default: break;
    }
    switch (npad) {
    case 8: return reinterpret_cast<void*>(&init_kernel<8, 0>);
    case 16: return reinterpret_cast<void*>(&init_kernel<16, 0>);
    case 32: return reinterpret_cast<void*>(&init_kernel<32, 0>);
    case 64: return reinterpret_cast<void*>(&init_kernel<64, 0>);
    default: return nullptr;
    }
}

template <int G, int PPL, bool EXACT, int MODEL = 0>
static void* fit2_fn() { return reinterpret_cast<void*>(&fit2_kernel<G, PPL, EXACT, MODEL>); }

// Instantiated (G, PPL): exact fits for the workload geometries
// (T = 21, 99 with G = 4; T = 201, 221 with G = 8; T = 21, 99, 201, 221 with
// G = 16, 32) and a general ladder with full tail checks; model 1 (the Fano
// lineshape) for the two- to eight-lane entries.
struct Fit2Inst {
    int G, PPL;
    bool exact;
    int model;
    void* (*fn)();
};
static const Fit2Inst kFit2[] = {
    {2, 50, true, 0, fit2_fn<2, 50, true>},   {2, 11, true, 0, fit2_fn<2, 11, true>},
    {4, 6, true, 0, fit2_fn<4, 6, true>},     {4, 25, true, 0, fit2_fn<4, 25, true>},
    {8, 26, true, 0, fit2_fn<8, 26, true>},   {8, 28, true, 0, fit2_fn<8, 28, true>},
    {8, 3, true, 0, fit2_fn<8, 3, true>},     {8, 13, true, 0, fit2_fn<8, 13, true>},
    {16, 2, true, 0, fit2_fn<16, 2, true>},   {16, 7, true, 0, fit2_fn<16, 7, true>},
    {16, 13, true, 0, fit2_fn<16, 13, true>}, {16, 14, true, 0, fit2_fn<16, 14, true>},
    {32, 1, true, 0, fit2_fn<32, 1, true>},   {32, 4, true, 0, fit2_fn<32, 4, true>},
    {32, 7, true, 0, fit2_fn<32, 7, true>},
    {4, 56, true, 0, fit2_fn<4, 56, true>},   {4, 51, true, 0, fit2_fn<4, 51, true>},
    {2, 24, false, 0, fit2_fn<2, 24, false>}, {2, 32, false, 0, fit2_fn<2, 32, false>},
    {2, 50, false, 0, fit2_fn<2, 50, false>},
    {4, 8, false, 0, fit2_fn<4, 8, false>},   {4, 16, false, 0, fit2_fn<4, 16, false>},
    {4, 32, false, 0, fit2_fn<4, 32, false>}, {8, 8, false, 0, fit2_fn<8, 8, false>},
    {8, 16, false, 0, fit2_fn<8, 16, false>}, {8, 32, false, 0, fit2_fn<8, 32, false>},
    {16, 8, false, 0, fit2_fn<16, 8, false>}, {16, 16, false, 0, fit2_fn<16, 16, false>},
    {32, 8, false, 0, fit2_fn<32, 8, false>},
    // the Fano lineshape
    {2, 50, true, 1, fit2_fn<2, 50, true, 1>},   {2, 11, true, 1, fit2_fn<2, 11, true, 1>},
    {4, 6, true, 1, fit2_fn<4, 6, true, 1>},     {4, 25, true, 1, fit2_fn<4, 25, true, 1>},
    {4, 56, true, 1, fit2_fn<4, 56, true, 1>},   {4, 51, true, 1, fit2_fn<4, 51, true, 1>},
    {8, 26, true, 1, fit2_fn<8, 26, true, 1>},   {8, 28, true, 1, fit2_fn<8, 28, true, 1>},
    {2, 24, false, 1, fit2_fn<2, 24, false, 1>}, {2, 32, false, 1, fit2_fn<2, 32, false, 1>},
    {2, 50, false, 1, fit2_fn<2, 50, false, 1>}, {4, 32, false, 1, fit2_fn<4, 32, false, 1>},
    {8, 32, false, 1, fit2_fn<8, 32, false, 1>},
};

void* fit2_ptr(int G, int PPL, bool exact, int model)
{
    if (G == 1) return model == 0 ? fit1_ptr() : nullptr;
    for (const Fit2Inst& f : kFit2)
        if (f.G == G && f.PPL == PPL && f.exact == exact && f.model == model) return f.fn();
    return nullptr;
}

// smallest instantiated PPL for (G, T); *exact tells whether it is ceil(T/G)
int fit2_ppl(int G, int T, bool* exact, int model)
{
    if (G == 1) {   // the lane-per-frame kernel keeps spectra in shared memory
        *exact = true;
        return model == 0 ? T : 0;
    }
    const int need = (T + G - 1) / G;
    for (const Fit2Inst& f : kFit2)
        if (f.G == G && f.exact && f.PPL == need && f.model == model) {
            *exact = true;
            return need;
        }
    int best = 0;
    for (const Fit2Inst& f : kFit2)
        if (f.G == G && !f.exact && f.model == model && f.PPL >= need && (best == 0 || f.PPL < best)) best = f.PPL;
    *exact = false;
    return best;
}

int fit2_threads(int G) { return G == 1 ? 128 : 256; }
size_t fit2_smem(int G, int T, int model);

int init_npad(int n_outer)
{
    for (int np : {8, 16, 32, 64})
        if (n_outer <= np) return np;
    return 0;
}

static cudaError_t launch_fast(const cg_plan_s* p, const void* frames, int sample_bytes, int64_t n, float* amps,
                               float* y, cudaStream_t s)
{
    FastArgs a = sample_bytes == 1 ? p->fa8 : p->fa;
    a.frames = frames;
    a.n_frames = n;
    a.amps = amps;
    a.y = y;
    const int64_t nb = (n + a.F - 1) / a.F;
    const int gmax = sample_bytes == 1 ? p->grid_fast8 : p->grid_fast;
    const int grid = static_cast<int>(nb < gmax ? nb : gmax);
    void* args[] = {&a};
    return cudaLaunchKernel(fast_readout_ptr(p->Q, sample_bytes), dim3(grid), dim3(128), args, a.sm_total, s);
}

cudaError_t launch_fast_readout(const cg_plan_s* p, const int16_t* frames, int64_t n, float* amps,
                                float* y, cudaStream_t s)
{
    return launch_fast(p, frames, 2, n, amps, y, s);
}

cudaError_t launch_fast_readout_i8(const cg_plan_s* p, const int8_t* frames, int64_t n, float* amps, float* y,
                                   cudaStream_t s)
{
    return launch_fast(p, frames, 1, n, amps, y, s);
}

cudaError_t launch_init(const cg_plan_s* p, const float* y, const float* amps, int64_t n,
                        float* p0_out, int16_t* flag_out, cudaStream_t s, const int* list,
                        const int* list_n)
{
    InitArgs a = p->ia;
    a.n = n;
    a.y = y;
    a.amps = amps;
    a.p0_out = p0_out;
    a.flag_out = flag_out;
    a.list = list;
    a.list_n = list_n;
    a.bulk = (p->T & 1) ? 1 : 0;
    a.err = p->d.err;
    const int64_t tasks = (n + 31) / 32;
    const int64_t blocks = (tasks + 3) / 4;
    const int grid = static_cast<int>(blocks < p->grid_init ? blocks : p->grid_init);
    void* args[] = {&a};
    return cudaLaunchKernel(init_ptr(p->init_npad, p->n_outer), dim3(grid), dim3(128), args, p->init_smem, s);
}

cudaError_t launch_fit2(const cg_plan_s* p, const float* y, const float* amps, int64_t n,
                        const float* p0, const int16_t* flags_in, float* params, float* rss,
                        int16_t* iters, int16_t* status, cudaStream_t s, const FitLaunch& fl)
{
    Fit2Args a{};
    a.n = n;
    a.T = p->T;
    a.y = y;
    a.amps = amps;
    a.inv_ref = p->d.inv_ref;
    a.u = p->d.u;
    a.p0 = p0;
    a.flags_in = flags_in;
    a.x_mid = static_cast<float>(p->x_mid);
    a.x_scale = static_cast<float>(p->x_scale);
    a.max_iter = fl.max_iter >= 0 ? fl.max_iter : p->opts.max_iter;
    a.tol = static_cast<float>(p->opts.tol);
    a.lambda0 = static_cast<float>(p->opts.lambda0);
    a.params = params;
    a.rss = rss;
    a.iters = iters;
    a.status = status;
    a.list = fl.list;
    a.list_n = fl.list_n;
    a.fb_list = fl.fb_list;
    a.fb_count = fl.fb_count;
    a.iters_base = fl.iters_base;
    a.status_or = fl.status_or;
    if (p->opts.model == CG_MODEL_FANO) {
        // the Fano parameters on the fit's normalised abscissa u = (x - x_mid) / x_scale
        const double g = p->opts.fano_gamma / p->x_scale;
        a.fano_q = static_cast<float>(p->opts.fano_q);
        a.fano_g = static_cast<float>(g);
        a.fano_inv_g = static_cast<float>(1.0 / g);
        a.fano_shift = static_cast<float>(p->opts.fano_q * g);
        const double A0 = p->opts.fano_A, B0 = p->opts.fano_B, bx = p->opts.fano_box;
        a.fano_A0 = static_cast<float>(A0);
        a.fano_B0 = static_cast<float>(B0);
        a.fano_Alo = static_cast<float>(std::min(A0 * (1.0 - bx), A0 * (1.0 + bx)));
        a.fano_Ahi = static_cast<float>(std::max(A0 * (1.0 - bx), A0 * (1.0 + bx)));
        a.fano_Blo = static_cast<float>(std::min(B0 * (1.0 - bx), B0 * (1.0 + bx)));
        a.fano_Bhi = static_cast<float>(std::max(B0 * (1.0 - bx), B0 * (1.0 + bx)));
    }
    a.row_stride = p->T | 1;
    a.counter = p->d.fit_counter;
    a.solve_f64 = p->solve_f64;
    a.n_rows = n;
    a.err = p->d.err;
    // the shared-memory kernel where one is instantiated for the tooth count,
    // lineshape and solve precision (the Lorentzian from a given guess; the
    // Fano profile from a given centre or its lowest tooth)
    if (p->fit3_ok && (p0 != nullptr || p->opts.model == CG_MODEL_FANO)) return launch_fit3(p, a, s);
    // tasks are claimed dynamically: a few frames per lane group per task
    const int gpw = 32 / p->G2;                   // groups per warp
    a.task = 2 * gpw;
    const int threads = fit2_threads(p->G2);
    const int wpb = threads / 32;                 // warps per block
    const int64_t tasks = (n + a.task - 1) / a.task;
    const int64_t blocks = (tasks + wpb - 1) / wpb;
    const int grid = static_cast<int>(blocks < p->grid_fit2 ? blocks : p->grid_fit2);
    cudaError_t e = cudaMemsetAsync(a.counter, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    void* args[] = {&a};
    return cudaLaunchKernel(fit2_ptr(p->G2, p->PPL, p->ppl_exact, p->opts.model), dim3(grid), dim3(threads), args,
                            fit2_smem(p->G2, p->T, p->opts.model), s);
}

size_t fit2_smem(int G, int T, int model)
{
    // G == 1: abscissa table, 4 warps x [2][32] row slots, 4 x 32 slot offsets;
    // G > 1: abscissa and 1 / reference tables, one PPL prefetch slot per thread
    if (G == 1) return sizeof(float) * (T + 4 * 64 * (T | 1)) + sizeof(int) * 4 * 32;
    bool exact = false;
    const int ppl = fit2_ppl(G, T, &exact, model);
    return sizeof(float) * (2 * T + (G >= 2 ? static_cast<size_t>(fit2_threads(G)) * (ppl | 1) : 0));
}

}  // namespace cg
