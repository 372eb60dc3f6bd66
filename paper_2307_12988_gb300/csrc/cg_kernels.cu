// cg_kernels.cu -- the plain-path kernels: cast + shared-memory FFT + tooth
// readout (+ normalisation), the same fused with the per-frame LM fit, the
// standalone fit, and the reference-spectrum accumulation.
//
// Paper ("Data Capture and Processing"): integer samples are cast to floats on
// the GPU "to minimize the quantity of data transferred", rows of N samples
// are Fourier transformed, the tooth bins are selected and mapped to the
// optical spectrum, divided by the averaged reference and fit.
#include <cstdint>
#include <cuda_runtime.h>

#include "cg_fft.cuh"
#include "cg_fit.cuh"
#include "cg_internal.h"

namespace cg {

// ---------------------------------------------------------------------------
// staging of a batch's int16 samples into shared memory.  The byte range
// [p, pend) of the batch is covered by 16-byte chunks aligned in global
// memory; whole chunks inside the range move as one 16-byte load, the ragged
// head and tail element by element.  Returns the element offset of the first
// sample in `raw`.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int stage_raw(const int16_t* frames, int64_t e0, int64_t ne,
                                         int16_t* raw)
{
    const char* p = reinterpret_cast<const char*>(frames + e0);
    const uintptr_t pa = reinterpret_cast<uintptr_t>(p) & ~static_cast<uintptr_t>(15);
    const int off = static_cast<int>((reinterpret_cast<uintptr_t>(p) - pa) >> 1);
    const char* pend = p + ne * 2;
    const int64_t nchunks = (static_cast<int64_t>(reinterpret_cast<uintptr_t>(pend) - pa) + 15) >> 4;
    uint4* raw4 = reinterpret_cast<uint4*>(raw);
    for (int64_t c = threadIdx.x; c < nchunks; c += blockDim.x) {
        const char* cp = reinterpret_cast<const char*>(pa) + 16 * c;
        if (cp >= p && cp + 16 <= pend) {
            raw4[c] = __ldcs(reinterpret_cast<const uint4*>(cp));
        } else {
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const char* ep = cp + 2 * e;
                if (ep >= p && ep < pend) raw[8 * c + e] = *reinterpret_cast<const int16_t*>(ep);
            }
        }
    }
    return off;
}

// tables into shared memory (once per block)
__device__ __forceinline__ void load_tables(const ReadoutArgs& a, unsigned char* sm)
{
    float2* twL = reinterpret_cast<float2*>(sm + a.sm_twL);
    for (int i = threadIdx.x; i < a.L; i += blockDim.x) twL[i] = a.tw_L[i];
    if (a.kind == CG_FFT_COSET) {
        float2* twM = reinterpret_cast<float2*>(sm + a.sm_twM);
        float2* twn1 = reinterpret_cast<float2*>(sm + a.sm_twn1);
        for (int i = threadIdx.x; i < a.M; i += blockDim.x) twM[i] = a.tw_M[i];
        for (int i = threadIdx.x; i < a.L; i += blockDim.x) twn1[i] = a.tw_n1[i];
    } else {
        float2* twb = reinterpret_cast<float2*>(sm + a.sm_twb);
        for (int i = threadIdx.x; i < a.T; i += blockDim.x) twb[i] = a.tw_b[i];
    }
    int* zidx = reinterpret_cast<int*>(sm + a.sm_zidx);
    float* iref = reinterpret_cast<float*>(sm + a.sm_iref);
    float* us = reinterpret_cast<float*>(sm + a.sm_u);
    for (int i = threadIdx.x; i < a.T; i += blockDim.x) {
        zidx[i] = a.zidx[i];
        iref[i] = a.inv_ref[i];
        us[i] = a.u[i];
    }
}

// cast + transform of nf frames (staged at raw + off) into the L-point
// complex spectrum; returns the buffer holding the result.
__device__ __forceinline__ const float2* transform_batch(const ReadoutArgs& a, unsigned char* sm,
                                                         const int16_t* raw, int off, int nf)
{
    float2* bufA = reinterpret_cast<float2*>(sm + a.sm_a);
    float2* bufB = reinterpret_cast<float2*>(sm + a.sm_b);
    const float2* twL = reinterpret_cast<const float2*>(sm + a.sm_twL);
    const int L = a.L, N = a.N;
    if (a.kind == CG_FFT_COSET) {
        const float2* twM = reinterpret_cast<const float2*>(sm + a.sm_twM);
        const float2* twn1 = reinterpret_cast<const float2*>(sm + a.sm_twn1);
        const int M = a.M;
        for (int item = threadIdx.x; item < nf * L; item += blockDim.x) {
            const int f = item / L;
            const int n1 = item - f * L;
            const int16_t* xs = raw + off + f * N + n1;
            float2 acc = make_float2(0.f, 0.f);
            for (int n2 = 0; n2 < M; ++n2) {
                const float v = static_cast<float>(xs[n2 * L]);
                const float2 w = twM[n2];
                acc.x = fmaf(v, w.x, acc.x);
                acc.y = fmaf(v, w.y, acc.y);
            }
            bufA[f * a.fstride + n1] = cmul(acc, twn1[n1]);
        }
    } else {
        for (int item = threadIdx.x; item < nf * L; item += blockDim.x) {
            const int f = item / L;
            const int n = item - f * L;
            const int16_t* xs = raw + off + f * N + 2 * n;
            bufA[f * a.fstride + n] = make_float2(static_cast<float>(xs[0]), static_cast<float>(xs[1]));
        }
    }
    __syncthreads();
    const float2* cur = bufA;
    float2* nxt = bufB;
    int Ns = 1;
    for (int s = 0; s < a.nst; ++s) {
        const int R = a.radix[s];
        stockham_dispatch(R, cur, nxt, L, Ns, nf, a.fstride, twL);
        __syncthreads();
        Ns *= R;
        const float2* t = cur;
        cur = nxt;
        nxt = const_cast<float2*>(t);
    }
    return cur;
}

// tooth magnitude of frame f, tooth k from the transformed buffer
__device__ __forceinline__ float tooth_amp(const ReadoutArgs& a, const unsigned char* sm,
                                           const float2* Z, int k)
{
    const int* zidx = reinterpret_cast<const int*>(sm + a.sm_zidx);
    float2 X;
    if (a.kind == CG_FFT_COSET) {
        X = Z[zidx[k]];
    } else {
        const int b = zidx[k];
        const int L = a.L;
        const int i1 = (b == L) ? 0 : b;
        const int i2 = (b == 0) ? 0 : L - b;
        const float2 Zb = Z[i1];
        const float2 Zr = Z[i2];
        // even part E = (Zb + conj Zr)/2, odd part O = (Zb - conj Zr)/(2i)
        const float2 E = make_float2(0.5f * (Zb.x + Zr.x), 0.5f * (Zb.y - Zr.y));
        const float2 Dd = make_float2(0.5f * (Zb.x - Zr.x), 0.5f * (Zb.y + Zr.y));
        const float2 O = make_float2(Dd.y, -Dd.x);
        const float2 W = reinterpret_cast<const float2*>(sm + a.sm_twb)[k];
        X = cadd(E, cmul(W, O));
    }
    return sqrtf(fmaf(X.x, X.x, X.y * X.y));
}

// ---------------------------------------------------------------------------
// readout kernel: MODE 0 = amps/y to global, MODE 1 = fused LM fit,
// MODE 2 = reference accumulation (per-block FP64 partial sums)
// ---------------------------------------------------------------------------
template <int MODE, int G>
__global__ void __launch_bounds__(kThreads) readout_kernel(ReadoutArgs a, FitArgs fa)
{
    extern __shared__ __align__(16) unsigned char sm[];
    load_tables(a, sm);
    int16_t* raw = reinterpret_cast<int16_t*>(sm + a.sm_raw);
    float* ys = reinterpret_cast<float*>(sm + a.sm_y);
    const float* iref = reinterpret_cast<const float*>(sm + a.sm_iref);
    const float* us = reinterpret_cast<const float*>(sm + a.sm_u);
    double* acc = reinterpret_cast<double*>(sm + a.sm_acc);
    if (MODE == 2)
        for (int k = threadIdx.x; k < a.T; k += blockDim.x) acc[k] = 0.0;
    const int64_t nb = (a.n_frames + a.F - 1) / a.F;
    const int T = a.T;
    for (int64_t b = blockIdx.x; b < nb; b += gridDim.x) {
        const int64_t f0 = b * a.F;
        const int nf = static_cast<int>((a.n_frames - f0) < a.F ? (a.n_frames - f0) : a.F);
        __syncthreads();
        const int off = stage_raw(a.frames, f0 * a.N, static_cast<int64_t>(nf) * a.N, raw);
        __syncthreads();
        const float2* Z = transform_batch(a, sm, raw, off, nf);
        for (int item = threadIdx.x; item < nf * T; item += blockDim.x) {
            const int f = item / T;
            const int k = item - f * T;
            const float amp = tooth_amp(a, sm, Z + f * a.fstride, k);
            const int64_t o = (f0 + f) * T + k;
            if (MODE == 2) {
                atomicAdd(&acc[k], static_cast<double>(amp));
            } else {
                const float yv = __fmul_rn(amp, iref[k]);
                if (a.amps) a.amps[o] = amp;
                if (a.y) a.y[o] = yv;
                if (MODE == 1) ys[f * a.ystride + k] = yv;
            }
        }
        if (MODE == 1) {
            __syncthreads();
            const int ngroups = blockDim.x / G;
            const int group = threadIdx.x / G;
            const int warp_first_group = (threadIdx.x & ~31) / G;
            for (int base = 0; base < nf; base += ngroups) {
                if (base + warp_first_group >= nf) break;   // warp-uniform
                const int fi = base + group;
                const bool valid = fi < nf;
                const int fs = valid ? fi : 0;
                fit_group<G>(ys + fs * a.ystride, us, fa, f0 + fs, valid);
            }
        }
    }
    if (MODE == 2) {
        __syncthreads();
        for (int k = threadIdx.x; k < T; k += blockDim.x) a.ref_part[blockIdx.x * T + k] = acc[k];
    }
}

// standalone fit: groups of G lanes, one frame each, spectra staged in smem
template <int G>
__global__ void __launch_bounds__(kThreads) fit_kernel(FitArgs fa, int ystride)
{
    extern __shared__ __align__(16) unsigned char sm[];
    float* us = reinterpret_cast<float*>(sm);
    const int T = fa.T;
    float* ys = us + ((T + 3) & ~3);
    for (int k = threadIdx.x; k < T; k += blockDim.x) us[k] = fa.u[k];
    const int fpb = blockDim.x / G;
    const int group = threadIdx.x / G;
    const int64_t nrounds = (fa.n + fpb - 1) / fpb;
    for (int64_t r = blockIdx.x; r < nrounds; r += gridDim.x) {
        const int64_t f0 = r * fpb;
        const int nf = static_cast<int>((fa.n - f0) < fpb ? (fa.n - f0) : fpb);
        __syncthreads();
        for (int i = threadIdx.x; i < nf * T; i += blockDim.x) {
            const int f = i / T;
            const int k = i - f * T;
            ys[f * ystride + k] = fa.y ? fa.y[f0 * T + i] : __fmul_rn(fa.amps_in[f0 * T + i], fa.inv_ref[k]);
        }
        __syncthreads();
        const bool valid = group < nf;
        fit_group<G>(ys + (valid ? group : 0) * ystride, us, fa, f0 + (valid ? group : 0), valid);
    }
}

// sum of per-block partials -> mean reference spectrum
__global__ void ref_reduce_kernel(const double* part, int rows, int T, double inv_n, double* out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= T) return;
    double s = 0.0;
    for (int r = 0; r < rows; ++r) s += part[static_cast<int64_t>(r) * T + k];
    out[k] = s * inv_n;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
FitArgs make_fit_args(const cg_plan_s* p)
{
    FitArgs f{};
    f.T = p->T;
    f.u = p->d.u;
    f.inv_ref = p->d.inv_ref;
    f.outer_idx = p->d.outer_idx;
    f.n_outer = p->n_outer;
    f.u_mid = p->u_mid;
    f.du = p->du;
    f.span = p->span;
    f.x_mid = static_cast<float>(p->x_mid);
    f.x_scale = static_cast<float>(p->x_scale);
    f.max_iter = p->opts.max_iter;
    f.tol = static_cast<float>(p->opts.tol);
    f.lambda0 = static_cast<float>(p->opts.lambda0);
    return f;
}

template <int MODE, int G>
static void* readout_fn() { return reinterpret_cast<void*>(&readout_kernel<MODE, G>); }

static void* readout_ptr(int mode, int G)
{
    switch (mode * 100 + G) {
    case 4: return readout_fn<0, 4>();
    case 8: return readout_fn<0, 8>();
    case 16: return readout_fn<0, 16>();
    case 32: return readout_fn<0, 32>();
    case 104: return readout_fn<1, 4>();
    case 108: return readout_fn<1, 8>();
    case 116: return readout_fn<1, 16>();
    case 132: return readout_fn<1, 32>();
    case 204: return readout_fn<2, 4>();
    case 208: return readout_fn<2, 8>();
    case 216: return readout_fn<2, 16>();
    case 232: return readout_fn<2, 32>();
    default: return nullptr;
    }
}

static void* fit_ptr(int G)
{
    switch (G) {
    case 4: return reinterpret_cast<void*>(&fit_kernel<4>);
    case 8: return reinterpret_cast<void*>(&fit_kernel<8>);
    case 16: return reinterpret_cast<void*>(&fit_kernel<16>);
    case 32: return reinterpret_cast<void*>(&fit_kernel<32>);
    default: return nullptr;
    }
}

static int fit_ystride(int T, int G)
{
    // stride == G (mod 32) keeps the groups of one warp on distinct banks
    int s = T;
    const int want = G % 32;
    while (s % 32 != want) ++s;
    return s;
}

cudaError_t configure_kernels(cg_plan_s* p)
{
    cudaError_t e;
    const int G = p->G;
    for (int mode = 0; mode < 3; ++mode) {
        void* fn = readout_ptr(mode, G);
        if (!fn) return cudaErrorInvalidValue;
        e = raise_smem_limit(fn, p->ra.sm_total);
        if (e != cudaSuccess) return e;
    }
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, readout_ptr(0, G), kThreads, p->ra.sm_total);
    if (e != cudaSuccess) return e;
    p->grid_readout = p->num_sms * (occ > 0 ? occ : 1);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, readout_ptr(1, G), kThreads, p->ra.sm_total);
    if (e != cudaSuccess) return e;
    p->grid_fused = p->num_sms * (occ > 0 ? occ : 1);
    const int ys = fit_ystride(p->T, G);
    const int fit_smem = static_cast<int>(sizeof(float)) * (((p->T + 3) & ~3) + (kThreads / G) * ys);
    e = raise_smem_limit(fit_ptr(G), fit_smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fit_ptr(G), kThreads, fit_smem);
    if (e != cudaSuccess) return e;
    p->grid_fit = p->num_sms * (occ > 0 ? occ : 1);
    return cudaSuccess;
}

static int grid_for(int64_t n_frames, int F, int cap)
{
    const int64_t nb = (n_frames + F - 1) / F;
    return static_cast<int>(nb < cap ? nb : cap);
}

cudaError_t launch_readout(const cg_plan_s* p, const int16_t* frames, int64_t n, float* amps,
                           float* y, cudaStream_t s)
{
    ReadoutArgs a = p->ra;
    a.frames = frames;
    a.n_frames = n;
    a.amps = amps;
    a.y = y;
    FitArgs fa = make_fit_args(p);
    const int grid = grid_for(n, a.F, p->grid_readout);
    void* args[] = {&a, &fa};
    return cudaLaunchKernel(readout_ptr(0, p->G), dim3(grid), dim3(kThreads), args, a.sm_total, s);
}

cudaError_t launch_fused(const cg_plan_s* p, const int16_t* frames, int64_t n, float* amps,
                         float* y, float* params, float* rss, int16_t* iters, int16_t* status,
                         cudaStream_t s)
{
    ReadoutArgs a = p->ra;
    a.frames = frames;
    a.n_frames = n;
    a.amps = amps;
    a.y = y;
    FitArgs fa = make_fit_args(p);
    fa.n = n;
    fa.params = params;
    fa.rss = rss;
    fa.iters = iters;
    fa.status = status;
    const int grid = grid_for(n, a.F, p->grid_fused);
    void* args[] = {&a, &fa};
    return cudaLaunchKernel(readout_ptr(1, p->G), dim3(grid), dim3(kThreads), args, a.sm_total, s);
}

cudaError_t launch_fit(const cg_plan_s* p, const float* y, const float* amps, int64_t n,
                       const float* p0, float* params, float* rss, int16_t* iters,
                       int16_t* status, cudaStream_t s)
{
    FitArgs fa = make_fit_args(p);
    fa.n = n;
    fa.y = y;
    fa.amps_in = amps;
    fa.p0 = p0;
    fa.params = params;
    fa.rss = rss;
    fa.iters = iters;
    fa.status = status;
    const int G = p->G;
    int ys = fit_ystride(p->T, G);
    const int fpb = kThreads / G;
    const int fit_smem = static_cast<int>(sizeof(float)) * (((p->T + 3) & ~3) + fpb * ys);
    const int64_t rounds = (n + fpb - 1) / fpb;
    const int grid = static_cast<int>(rounds < p->grid_fit ? rounds : p->grid_fit);
    void* args[] = {&fa, &ys};
    return cudaLaunchKernel(fit_ptr(G), dim3(grid), dim3(kThreads), args, fit_smem, s);
}

cudaError_t launch_reference(const cg_plan_s* p, const int16_t* frames, int64_t n, cudaStream_t s)
{
    ReadoutArgs a = p->ra;
    a.frames = frames;
    a.n_frames = n;
    a.amps = nullptr;
    a.y = nullptr;
    a.ref_part = p->d.ref_part;
    FitArgs fa = make_fit_args(p);
    int grid = grid_for(n, a.F, p->grid_readout);
    if (grid > p->d.ref_part_rows) grid = p->d.ref_part_rows;
    void* args[] = {&a, &fa};
    cudaError_t e = cudaLaunchKernel(readout_ptr(2, p->G), dim3(grid), dim3(kThreads), args,
                                     a.sm_total, s);
    if (e != cudaSuccess) return e;
    const int tb = 128;
    ref_reduce_kernel<<<(p->T + tb - 1) / tb, tb, 0, s>>>(p->d.ref_part, grid, p->T,
                                                          1.0 / static_cast<double>(n), p->d.ref_out);
    return cudaGetLastError();
}

cudaError_t preload_reference_kernels(const cg_plan_s* p)
{
    // querying a kernel's attributes loads its module (lazy loading), so the
    // first launch later needs no module load
    cudaFuncAttributes fa{};
    cudaError_t e = cudaFuncGetAttributes(&fa, readout_ptr(2, p->G));
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, reinterpret_cast<const void*>(&ref_reduce_kernel));
    return e;
}

cudaError_t launch_reference_into(const cg_plan_s* p, const int16_t* frames, int64_t n,
                                  double* part, int max_rows, double* out, cudaStream_t s)
{
    ReadoutArgs a = p->ra;
    a.frames = frames;
    a.n_frames = n;
    a.amps = nullptr;
    a.y = nullptr;
    a.ref_part = part;
    FitArgs fa = make_fit_args(p);
    int grid = grid_for(n, a.F, p->grid_readout);
    if (grid > max_rows) grid = max_rows;
    void* args[] = {&a, &fa};
    cudaError_t e = cudaLaunchKernel(readout_ptr(2, p->G), dim3(grid), dim3(kThreads), args,
                                     a.sm_total, s);
    if (e != cudaSuccess) return e;
    const int tb = 128;
    ref_reduce_kernel<<<(p->T + tb - 1) / tb, tb, 0, s>>>(part, grid, p->T,
                                                          1.0 / static_cast<double>(n), out);
    return cudaGetLastError();
}

}  // namespace cg
