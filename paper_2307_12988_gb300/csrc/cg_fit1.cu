// cg_fit1.cu -- Levenberg-Marquardt with one lane per frame.
//
// Paper ("Data Capture and Processing"): each normalised spectrum is fit by
// Levenberg-Marquardt, at most 20 iterations, tolerance 1e-6.  Here every lane
// of a warp fits its own frame, so a pass needs no reduction and no solve
// replicated over lanes: per tooth the lane evaluates the model, its Jacobian
// and the 14 running sums of J^T J, J^T r and chi^2 (cg_fit.cuh).
//
// Frames are handed out dynamically and one frame ahead: every lane keeps one
// claimed frame in flight besides the one it is fitting.  The rows claimed in
// a pass belong to consecutive frames, contiguous in memory, so the whole
// warp copies them with coalesced 4-byte cp.async into the claimers' spare
// shared-memory slots; the copy lands behind the pass's arithmetic and is
// waited for at the end of the pass.  Slots are laid out [parity][lane][tooth]
// with an odd row stride, so the 32 lanes reading tooth k touch 32 banks; the
// abscissa table is a broadcast read.
#include <cstdint>
#include <cuda_runtime.h>

#include "cg_fit.cuh"
#include "cg_internal.h"

namespace cg {

namespace {

__device__ __forceinline__ void cp_async4(void* smem, const void* gmem)
{
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit1() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all1() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

}  // namespace

__global__ void __launch_bounds__(128) fit1_kernel(Fit2Args a)
{
    extern __shared__ __align__(16) float fsm[];
    const int T = a.T, TS = a.row_stride;
    const int nw = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    float* us = fsm;
    float* slots = fsm + T + warp * 64 * TS;                        // [2][32][TS]
    int* dst_of = reinterpret_cast<int*>(fsm + T + nw * 64 * TS) + warp * 32;
    for (int i = threadIdx.x; i < T; i += blockDim.x) us[i] = a.u[i];
    __syncthreads();
    const float inv_scale = 1.0f / a.x_scale;
    const float* src_rows = a.y ? a.y : a.amps;
    const bool scale_rows = (a.y == nullptr);

    int64_t n = a.n;
    if (a.list_n) {
        const int64_t c = *a.list_n;
        n = c < n ? c : n;
    }
    int64_t next = 0, end = 0;      // the warp's current task [next, end)
    int64_t cur = -1, nxt = -1;     // task being fit / claimed task in flight
    int64_t cur_f = -1, nxt_f = -1; // their frame indices (list[task] for a frame list)
    int par = 0;                    // cur's slot is par * 32 + lane
    bool fitting = false, fresh = false;
    float q0[4] = {0.f, 1.f, 0.f, 0.f};   // start parameters of nxt
    int qflag = 0;
    float p[4] = {0.f, 1.f, 0.f, 0.f};
    float lambda = a.lambda0, chi2 = 0.f;
    Normal Nm;
#pragma unroll
    for (int i = 0; i < 10; ++i) Nm.H[i] = 0.f;
#pragma unroll
    for (int i = 0; i < 4; ++i) Nm.b[i] = 0.f;
    int it = 0, st = kMaxIter, flag = 0;

    while (true) {
        // ---- claim (at most one contiguous run per pass) for lanes with no
        //      frame in flight; consecutive frames go to ascending lanes ----
        unsigned got = 0;
        int64_t first = 0;
        {
            const unsigned need = __ballot_sync(kFull, nxt < 0);
            if (need != 0 && next < n) {
                if (next >= end) {
                    unsigned long long t = 0;
                    if (lane == 0) t = atomicAdd(a.counter, 1ULL);
                    t = __shfl_sync(kFull, t, 0);
                    next = static_cast<int64_t>(t) * a.task;
                    if (next >= n) next = n;
                    end = next + a.task < n ? next + a.task : n;
                }
                if (next < end) {
                    const int cnt = __popc(need);
                    const int64_t avail = end - next;
                    const int take = static_cast<int>(avail < cnt ? avail : cnt);
                    const int rank = __popc(need & ((1u << lane) - 1u));
                    const bool gets = ((need >> lane) & 1u) && rank < take;
                    if (gets) {
                        nxt = next + rank;
                        nxt_f = a.list ? static_cast<int64_t>(a.list[nxt]) : nxt;
                        const float* q = a.p0 + nxt_f * 4;
                        q0[0] = q[0];
                        q0[1] = q[1];
                        q0[2] = q[2];
                        q0[3] = q[3];
                        qflag = a.flags_in ? (a.flags_in[nxt_f] & kInitFlat) : 0;
                    }
                    got = __ballot_sync(kFull, gets);
                    first = next;
                    next += take;
                }
            }
        }
        if (!__any_sync(kFull, cur >= 0 || nxt >= 0)) break;
        // ---- coalesced asynchronous copy of the claimed rows ----
        dst_of[lane] = ((par ^ 1) * 32 + lane) * TS;
        __syncwarp();
        if (got != 0 && a.list) {
            // listed frames are not contiguous: one coalesced row per claimer
            unsigned m = got;
            while (m != 0) {
                const int l = __ffs(m) - 1;
                m &= m - 1;
                const int64_t rf = __shfl_sync(kFull, nxt_f, l);
                const float* src = src_rows + rf * T;
                float* dst = slots + dst_of[l];
                for (int k = lane; k < T; k += 32) cp_async4(dst + k, src + k);
            }
        } else if (got != 0) {
            const float* src = src_rows + first * T;
            const int total = __popc(got) * T;
            int r = lane / T, k = lane - r * T;
            unsigned m = got;
            for (int q = 0; q < r; ++q) m &= m - 1;
            for (int e = lane; e < total; e += 32) {
                cp_async4(slots + dst_of[__ffs(m) - 1] + k, src + e);
                k += 32;
                while (k >= T) {
                    k -= T;
                    m &= m - 1;
                }
            }
        }
        cp_async_commit1();
        // ---- start the current frame ----
        if (cur >= 0 && !fitting) {
            p[0] = (p[0] - a.x_mid) * inv_scale;    // p holds the abscissa-unit start
            p[1] = p[1] * inv_scale;
            lambda = a.lambda0;
            it = 0;
            st = kMaxIter;
            fitting = true;
            fresh = true;
        }
        // ---- trial point ----
        float pe[4] = {p[0], p[1], p[2], p[3]};
        bool done = false;
        if (fitting && !fresh) {
            float delta[4];
            if (a.solve_f64 ? lm_solve4_f64(Nm, lambda, delta) : lm_solve4_fast(Nm, lambda, delta)) {
#pragma unroll
                for (int i = 0; i < 4; ++i) pe[i] = p[i] + delta[i];
            } else {
                st = kSingular;
                done = true;
            }
        }
        // ---- sums over the frame's teeth ----
        const float* my = slots + (par * 32 + lane) * TS;
        const float c = pe[0], g2 = pe[1] * pe[1], A = pe[2], B = pe[3];
        LmSums S;
#pragma unroll
        for (int i = 0; i < 14; ++i) S.v[i] = 0.f;
        if (scale_rows) {
            const float* ir = a.inv_ref;
#pragma unroll 4
            for (int k = 0; k < T; ++k) accum_point(us[k], __fmul_rn(my[k], __ldg(ir + k)), c, g2, A, B, S);
        } else {
#pragma unroll 4
            for (int k = 0; k < T; ++k) accum_point(us[k], my[k], c, g2, A, B, S);
        }
        // ---- LM bookkeeping ----
        if (fitting && !done) {
            const float chi2t = S.v[13];
            if (fresh) {
                chi2 = chi2t;
                if (!(chi2t < INFINITY)) {
                    st = kNonfinite;
                    done = true;
                } else {
                    make_normal_fast(S, pe[1], pe[2], T, Nm);
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
                    make_normal_fast(S, pe[1], pe[2], T, Nm);
                    lambda *= 0.1f;
                } else {
                    lambda *= 10.0f;
                }
                if (!done && it >= a.max_iter) done = true;
            }
        }
        fresh = false;
        if (fitting && done) {
            float* po = a.params + cur_f * 4;
            po[0] = fmaf(a.x_scale, p[0], a.x_mid);
            po[1] = a.x_scale * fabsf(p[1]);
            po[2] = p[2];
            po[3] = p[3];
            if (a.rss) a.rss[cur_f] = chi2;
            if (a.iters) a.iters[cur_f] = static_cast<int16_t>(it + a.iters_base);
            if (a.status) a.status[cur_f] = static_cast<int16_t>(st | flag | a.status_or);
            if (a.fb_list && (st == kMaxIter || st == kSingular))
                a.fb_list[atomicAdd(a.fb_count, 1)] = static_cast<int>(cur_f);
            fitting = false;
            cur = -1;
        }
        // ---- rows copied this pass are complete; promote the frame in flight ----
        cp_async_wait_all1();
        __syncwarp();
        if (cur < 0 && nxt >= 0) {
            cur = nxt;
            cur_f = nxt_f;
            nxt = -1;
            par ^= 1;
#pragma unroll
            for (int i = 0; i < 4; ++i) p[i] = q0[i];
            flag = qflag;
        }
    }
    cp_async_wait_all1();
}

}  // namespace cg

namespace cg {
void* fit1_ptr() { return reinterpret_cast<void*>(&fit1_kernel); }
}  // namespace cg
