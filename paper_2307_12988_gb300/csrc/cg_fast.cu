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
#include <cstdint>
#include <cuda_runtime.h>

#include "cg_fft.cuh"
#include "cg_fit.cuh"
#include "cg_internal.h"

namespace cg {

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem)
{
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Asynchronous staging of int16 elements [e0, e0 + ne) into raw: 16-byte
// chunks aligned in global memory go by cp.async, the ragged head/tail chunk
// by plain loads.  Returns the element offset of e0 inside raw.
__device__ __forceinline__ int stage_async(const int16_t* frames, int64_t e0, int64_t ne, int16_t* raw)
{
    const char* p = reinterpret_cast<const char*>(frames + e0);
    const uintptr_t pa = reinterpret_cast<uintptr_t>(p) & ~static_cast<uintptr_t>(15);
    const int off = static_cast<int>((reinterpret_cast<uintptr_t>(p) - pa) >> 1);
    const char* pend = p + ne * 2;
    const int64_t nchunks = (static_cast<int64_t>(reinterpret_cast<uintptr_t>(pend) - pa) + 15) >> 4;
    for (int64_t c = threadIdx.x; c < nchunks; c += blockDim.x) {
        const char* cp = reinterpret_cast<const char*>(pa) + 16 * c;
        if (cp >= p && cp + 16 <= pend) {
            cp_async16(reinterpret_cast<char*>(raw) + 16 * c, cp);
        } else {
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const char* ep = cp + 2 * e;
                if (ep >= p && ep < pend) raw[8 * c + e] = *reinterpret_cast<const int16_t*>(ep);
            }
        }
    }
    cp_async_commit();
    return off;
}

template <int P, int Q>
__global__ void __launch_bounds__(128) fast_readout_kernel(FastArgs a, FitArgs fa)
{
    constexpr int L = P * Q;
    constexpr int MH = 5;                     // M / 2 with M = 10
    extern __shared__ __align__(16) unsigned char sm[];
    float2* twL = reinterpret_cast<float2*>(sm + a.sm_twL);
    float2* twN = reinterpret_cast<float2*>(sm + a.sm_twN);
    int* tom = reinterpret_cast<int*>(sm + a.sm_tom);
    float* iref = reinterpret_cast<float*>(sm + a.sm_iref);
    float* us = reinterpret_cast<float*>(sm + a.sm_u);
    int16_t* raw = reinterpret_cast<int16_t*>(sm + a.sm_raw);
    float2* Yb = reinterpret_cast<float2*>(sm + a.sm_Y);
    float* amp_s = reinterpret_cast<float*>(sm + a.sm_amps);
    float* y_s = reinterpret_cast<float*>(sm + a.sm_y);
    const int T = a.T, N = a.N, F = a.F;
    for (int i = threadIdx.x; i < L; i += blockDim.x) {
        twL[i] = a.twL[i];
        twN[i] = a.twN[i];
        tom[i] = a.tooth_of_m[i];
    }
    for (int i = threadIdx.x; i < T; i += blockDim.x) {
        iref[i] = a.inv_ref[i];
        us[i] = a.u[i];
    }
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
        off = stage_async(a.frames, b * F * static_cast<int64_t>(N), static_cast<int64_t>(nf0) * N, raw);
    }
    for (; b < nb; b += gridDim.x) {
        const int64_t f0 = b * F;
        const int nf = static_cast<int>((a.n_frames - f0) < F ? (a.n_frames - f0) : F);
        cp_async_wait_all();
        __syncthreads();
        // ---------------- stage 1: fold, Q-point DFT, twiddle ----------------
        for (int item = threadIdx.x; item < nf * P; item += blockDim.x) {
            const int f = item / P;
            const int a0 = item - f * P;
            const int16_t* xs = raw + off + f * N + a0;
            float2 z[Q];
#pragma unroll
            for (int bq = 0; bq < Q; ++bq) {
                const int16_t* xp = xs + P * bq;
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
        int offn = 0;
        if (bn < nb) {
            const int nfn = static_cast<int>((a.n_frames - bn * F) < F ? (a.n_frames - bn * F) : F);
            offn = stage_async(a.frames, bn * F * static_cast<int64_t>(N), static_cast<int64_t>(nfn) * N, raw);
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
#pragma unroll
            for (int v = 0; v < P; ++v) {
                const int k = tom[u + Q * v];
                if (k >= 0) amp_s[f * T + k] = sqrtf(fmaf(z[v].x, z[v].x, z[v].y * z[v].y));
            }
        }
        __syncthreads();
        // ---------------- outputs (coalesced) and normalised spectra ----------
        for (int i = threadIdx.x; i < nf * T; i += blockDim.x) {
            const int f = i / T;
            const int k = i - f * T;
            const float av = amp_s[i];
            const float yv = av * iref[k];
            y_s[i] = yv;
            if (a.amps) a.amps[f0 * T + i] = av;
            if (a.y) a.y[f0 * T + i] = yv;
        }
        __syncthreads();
        // ---------------- moment initial guess, 8 lanes per frame -------------
        {
            constexpr int GI = 8;
            const int ngroups = blockDim.x / GI;
            const int group = threadIdx.x / GI;
            const int warp_first_group = (threadIdx.x & ~31) / GI;
            for (int base = 0; base < nf; base += ngroups) {
                if (base + warp_first_group >= nf) break;   // warp-uniform
                const int fi = base + group;
                const bool valid = fi < nf;
                float p[4];
                int flag = 0;
                moment_init<GI>(y_s + (valid ? fi : 0) * T, us, fa, p, flag);
                if (valid && (threadIdx.x & (GI - 1)) == 0) {
                    float* po = a.p0_out + (f0 + fi) * 4;
                    po[0] = fmaf(fa.x_scale, p[0], fa.x_mid);
                    po[1] = fa.x_scale * fabsf(p[1]);
                    po[2] = p[2];
                    po[3] = p[3];
                    if (a.flag_out) a.flag_out[f0 + fi] = static_cast<int16_t>(flag);
                }
            }
        }
        off = offn;
    }
    cp_async_wait_all();
}

// ---------------------------------------------------------------------------
// fit2: register-resident LM with a per-warp frame queue
// ---------------------------------------------------------------------------
template <int G, int PPL>
__global__ void __launch_bounds__(256, 2) fit2_kernel(Fit2Args a)
{
    const int lane = threadIdx.x & 31;
    const int gl = lane & (G - 1);
    const int leader_lane = lane & ~(G - 1);
    const int T = a.T;
    float uv[PPL];
#pragma unroll
    for (int j = 0; j < PPL; ++j) {
        const int k = gl + G * j;
        uv[j] = (k < T) ? a.u[k] : 0.f;
    }
    const int64_t nwarps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
    int64_t task = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
    int64_t next = task * a.task;
    int64_t end = next + a.task < a.n ? next + a.task : a.n;
    if (next >= a.n) next = end = a.n;

    int64_t f = -1;
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
        // ---- hand frames to idle groups (all lanes of a group agree) ----
        unsigned need = __ballot_sync(kFull, gl == 0 && f < 0);
        while (need != 0 && next < a.n) {
            if (next >= end) {
                task += nwarps;
                next = task * a.task;
                if (next >= a.n) {
                    next = end = a.n;
                    break;
                }
                end = next + a.task < a.n ? next + a.task : a.n;
            }
            const int cnt = __popc(need);
            const int64_t avail = end - next;
            const int take = static_cast<int>(avail < cnt ? avail : cnt);
            const int rank = __popc(need & ((1u << leader_lane) - 1u));
            if (((need >> leader_lane) & 1u) && rank < take) {
                f = next + rank;
                fresh = true;
            }
            next += take;
            need = __ballot_sync(kFull, gl == 0 && f < 0);
        }
        if (!__any_sync(kFull, f >= 0)) break;

        if (fresh) {
            const float* src = a.y ? a.y + f * T : a.amps + f * T;
#pragma unroll
            for (int j = 0; j < PPL; ++j) {
                const int k = gl + G * j;
                yv[j] = (k < T) ? (a.y ? src[k] : src[k] * a.inv_ref[k]) : 0.f;
            }
            const float* q = a.p0 + f * 4;
            p[0] = (q[0] - a.x_mid) / a.x_scale;
            p[1] = q[1] / a.x_scale;
            p[2] = q[2];
            p[3] = q[3];
            flag = a.flags_in ? (a.flags_in[f] & kInitFlat) : 0;
            lambda = a.lambda0;
            it = 0;
            st = kMaxIter;
        }
        // ---- trial point ----
        float pe[4] = {p[0], p[1], p[2], p[3]};
        bool done = false;
        if (f >= 0 && !fresh) {
            float delta[4];
            if (lm_solve4(Nm, lambda, delta)) {
#pragma unroll
                for (int i = 0; i < 4; ++i) pe[i] = p[i] + delta[i];
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
            if (gl + G * j < T) accum_point(uv[j], yv[j], pe[0], g2, pe[2], pe[3], S);
        }
        reduce_sums<G>(S);
        // ---- LM bookkeeping ----
        if (f >= 0 && !done) {
            const float chi2t = S.v[13];
            if (fresh) {
                fresh = false;
                chi2 = chi2t;
                if (!(chi2t < INFINITY)) {
                    st = kNonfinite;
                    done = true;
                } else {
                    make_normal(S, pe[1], pe[2], T, Nm);
                    if (a.max_iter <= 0) done = true;
                }
            } else {
                ++it;
                if (!(chi2t < INFINITY)) {
                    lambda *= 10.0f;
                } else if (fabsf(chi2t - chi2) <= a.tol * chi2) {
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
                    make_normal(S, pe[1], pe[2], T, Nm);
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
                float* po = a.params + f * 4;
                po[0] = fmaf(a.x_scale, p[0], a.x_mid);
                po[1] = a.x_scale * fabsf(p[1]);
                po[2] = p[2];
                po[3] = p[3];
                if (a.rss) a.rss[f] = chi2;
                if (a.iters) a.iters[f] = static_cast<int16_t>(it);
                if (a.status) a.status[f] = static_cast<int16_t>(st | flag);
            }
            f = -1;
        }
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
template <int P, int Q>
static void* fast_fn() { return reinterpret_cast<void*>(&fast_readout_kernel<P, Q>); }

void* fast_readout_ptr(int Q)
{
    switch (Q) {
    case 10: return fast_fn<10, 10>();
    case 11: return fast_fn<10, 11>();
    case 22: return fast_fn<10, 22>();
    case 25: return fast_fn<10, 25>();
    default: return nullptr;
    }
}

template <int G, int PPL>
static void* fit2_fn() { return reinterpret_cast<void*>(&fit2_kernel<G, PPL>); }

void* fit2_ptr(int G, int PPL)
{
    switch (G * 1000 + PPL) {
    case 4008: return fit2_fn<4, 8>();
    case 4016: return fit2_fn<4, 16>();
    case 4025: return fit2_fn<4, 25>();
    case 4032: return fit2_fn<4, 32>();
    case 8004: return fit2_fn<8, 4>();
    case 8008: return fit2_fn<8, 8>();
    case 8016: return fit2_fn<8, 16>();
    case 8028: return fit2_fn<8, 28>();
    case 8032: return fit2_fn<8, 32>();
    case 16004: return fit2_fn<16, 4>();
    case 16008: return fit2_fn<16, 8>();
    case 16016: return fit2_fn<16, 16>();
    case 32004: return fit2_fn<32, 4>();
    case 32008: return fit2_fn<32, 8>();
    default: return nullptr;
    }
}

int fit2_ppl(int G, int T)
{
    static const int kG4[] = {8, 16, 25, 32};
    static const int kG8[] = {4, 8, 16, 28, 32};
    static const int kG16[] = {4, 8, 16};
    static const int kG32[] = {4, 8};
    const int need = (T + G - 1) / G;
    const int* list = nullptr;
    int cnt = 0;
    switch (G) {
    case 4: list = kG4; cnt = 4; break;
    case 8: list = kG8; cnt = 5; break;
    case 16: list = kG16; cnt = 3; break;
    case 32: list = kG32; cnt = 2; break;
    default: return 0;
    }
    for (int i = 0; i < cnt; ++i)
        if (list[i] >= need) return list[i];
    return 0;
}

cudaError_t launch_fast_readout(const cg_plan_s* p, const int16_t* frames, int64_t n, float* amps,
                                float* y, float* p0_out, int16_t* flag_out, cudaStream_t s)
{
    FastArgs a = p->fa;
    a.frames = frames;
    a.n_frames = n;
    a.amps = amps;
    a.y = y;
    a.p0_out = p0_out;
    a.flag_out = flag_out;
    FitArgs fa = make_fit_args(p);
    const int64_t nb = (n + a.F - 1) / a.F;
    const int grid = static_cast<int>(nb < p->grid_fast ? nb : p->grid_fast);
    void* args[] = {&a, &fa};
    return cudaLaunchKernel(fast_readout_ptr(p->Q), dim3(grid), dim3(128), args, a.sm_total, s);
}

cudaError_t launch_fit2(const cg_plan_s* p, const float* y, const float* amps, int64_t n,
                        const float* p0, const int16_t* flags_in, float* params, float* rss,
                        int16_t* iters, int16_t* status, cudaStream_t s)
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
    a.max_iter = p->opts.max_iter;
    a.tol = static_cast<float>(p->opts.tol);
    a.lambda0 = static_cast<float>(p->opts.lambda0);
    a.params = params;
    a.rss = rss;
    a.iters = iters;
    a.status = status;
    const int warps_total = p->grid_fit2 * 8;
    const int gpw = 32 / p->G2;  // groups per warp
    int64_t per = (n + warps_total - 1) / warps_total;
    if (per < 2 * gpw) per = 2 * gpw;
    per = ((per + gpw - 1) / gpw) * gpw;
    a.task = static_cast<int>(per);
    const int64_t tasks = (n + per - 1) / per;
    const int64_t blocks = (tasks + 7) / 8;
    const int grid = static_cast<int>(blocks < p->grid_fit2 ? blocks : p->grid_fit2);
    void* args[] = {&a};
    return cudaLaunchKernel(fit2_ptr(p->G2, p->PPL), dim3(grid), dim3(256), args, 0, s);
}

}  // namespace cg
