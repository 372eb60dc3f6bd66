// cg_pow2.cu -- tooth readout for frames whose teeth share no residue class
// (the full real transform) when N = 2 L with L = 1024, 2048 or 4096.
//
// Paper ("Data Capture and Processing"): each row of N samples is Fourier
// transformed and the tooth bins are read.  The real row is packed as L
// complex values z_n = x_{2n} + i x_{2n+1}; the L-point DFT is factored as
// L = 16 x 16 x R3 (R3 = L / 256) and run in three register passes with
// compile-time sizes, L / 16 threads per frame and 16 values per thread:
//   pass 1  n = n1 + (L/16) n2:  DFT16 over n2 -> k2, twiddle W_L^{n1 k2};
//   pass 2  n1 = m1 + R3 m2:     DFT16 over m2 -> j,  twiddle W_{L/16}^{m1 j};
//   pass 3                        DFT_R3 over m1 -> j',
// so that Z[k2 + 16 j + 256 j'] = sum_n z_n W_L^{n k}.  Between passes the
// values go through a padded shared buffer (row stride 17 R3 complex values,
// conflict-free for every access pattern above); the last pass writes Z at
// position k + k / 16.  The real-FFT split X_b = E + W_N^b O is evaluated only
// at the teeth.  Samples of the next batch stream in with cp.async while the
// current batch is transformed.
#include <cstdint>
#include <cuda_runtime.h>

#include "cg_fft.cuh"
#include "cg_internal.h"
#include "cg_stage.cuh"

namespace cg {

namespace {

constexpr int kPow2Threads = 256;

template <int L>
struct Pow2Plan {
    static constexpr int TPF = L / 16;             // threads per frame
    static constexpr int FPB = kPow2Threads / TPF;  // frames per block pass
    static constexpr int R3 = L / 256;
    static constexpr int RS = 17 * R3;             // exchange row stride (complex values)
    static constexpr int BUF = 16 * RS;            // = L + L / 16
    static constexpr int PP = 256 / TPF;           // pass-3 (k2, j) pairs per thread
    static constexpr int N = 2 * L;
};

__device__ __forceinline__ int zpos(int k) { return k + (k >> 4); }

template <int L>
__global__ void __launch_bounds__(kPow2Threads) pow2_readout_kernel(ReadoutArgs a)
{
    using P = Pow2Plan<L>;
    constexpr int TPF = P::TPF, FPB = P::FPB, R3 = P::R3, RS = P::RS, BUF = P::BUF, PP = P::PP, N = P::N;
    extern __shared__ __align__(16) unsigned char sm[];
    const int T = a.T;
    // pass twiddles laid out so a warp reads consecutive entries:
    // tw1[k2][n1] = W_L^{n1 k2}, tw2[j][m1] = W_{L/16}^{m1 j}
    float2* tw1 = reinterpret_cast<float2*>(sm);                       // [16][L/16]
    float2* tw2 = tw1 + L;                                             // [16][R3]
    float2* twb = tw2 + 16 * R3;                                       // [T] W_N^{b_k}
    int* bins = reinterpret_cast<int*>(twb + T);                       // [T]
    float* iref = reinterpret_cast<float*>(bins + T);                  // [T]
    float2* S = reinterpret_cast<float2*>(sm + a.sm_a);                // [FPB][BUF]
    int16_t* raw0 = reinterpret_cast<int16_t*>(sm + a.sm_raw);         // [2][FPB N + 16]
    constexpr int kRawStride = FPB * N + 16;
    for (int i = threadIdx.x; i < L; i += blockDim.x) {
        const int k2 = i / TPF, n1 = i - k2 * TPF;
        tw1[i] = a.tw_L[n1 * k2];
    }
    for (int i = threadIdx.x; i < 16 * R3; i += blockDim.x) {
        const int j = i / R3, m1 = i - j * R3;
        tw2[i] = a.tw_L[16 * m1 * j];
    }
    for (int i = threadIdx.x; i < T; i += blockDim.x) {
        twb[i] = a.tw_b[i];
        bins[i] = a.zidx[i];
        iref[i] = a.inv_ref[i];
    }
    const int fs = threadIdx.x / TPF;      // frame slot
    const int lt = threadIdx.x % TPF;      // thread within the frame
    float2* Sf = S + fs * BUF;
    const int64_t nb = (a.n_frames + FPB - 1) / FPB;
    int64_t b = blockIdx.x;
    int buf = 0;
    int off_cur = 0;   // element offset of the current batch inside its buffer
    if (b < nb) {
        const int nf0 = static_cast<int>((a.n_frames - b * FPB) < FPB ? (a.n_frames - b * FPB) : FPB);
        off_cur = stage_async(a.frames, b * FPB * static_cast<int64_t>(N), static_cast<int64_t>(nf0) * N, raw0);
    }
    for (; b < nb; b += gridDim.x, buf ^= 1) {
        const int64_t f0 = b * FPB;
        const int nf = static_cast<int>((a.n_frames - f0) < FPB ? (a.n_frames - f0) : FPB);
        // the next batch streams into the other buffer (a possibly empty group)
        const int64_t bn = b + gridDim.x;
        int off_next = 0;
        if (bn < nb) {
            const int nfn = static_cast<int>((a.n_frames - bn * FPB) < FPB ? (a.n_frames - bn * FPB) : FPB);
            off_next = stage_async(a.frames, bn * FPB * static_cast<int64_t>(N), static_cast<int64_t>(nfn) * N,
                                   raw0 + (buf ^ 1) * kRawStride);
        } else {
            cp_async_commit();
        }
        asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        __syncthreads();
        const bool live = fs < nf;
        // ---- pass 1: DFT16 over n2, twiddle W_L^{n1 k2} ----
        {
            float2 z[16];
            const uint32_t* rw = reinterpret_cast<const uint32_t*>(raw0 + buf * kRawStride + off_cur + fs * N);
#pragma unroll
            for (int n2 = 0; n2 < 16; ++n2) {
                const uint32_t w = live ? rw[lt + TPF * n2] : 0u;
                z[n2] = make_float2(static_cast<float>(static_cast<short>(w & 0xffffu)),
                                    static_cast<float>(static_cast<short>(w >> 16)));
            }
            Dft<16>::run(z);
#pragma unroll
            for (int k2 = 1; k2 < 16; ++k2) z[k2] = cmul(z[k2], tw1[k2 * TPF + lt]);
#pragma unroll
            for (int k2 = 0; k2 < 16; ++k2) Sf[k2 * RS + lt] = z[k2];
        }
        __syncthreads();
        // ---- pass 2: DFT16 over m2, twiddle W_{L/16}^{m1 j} ----
        {
            const int k2 = lt / R3, m1 = lt % R3;
            float2 z[16];
#pragma unroll
            for (int m2 = 0; m2 < 16; ++m2) z[m2] = Sf[k2 * RS + m1 + R3 * m2];
            Dft<16>::run(z);
#pragma unroll
            for (int j = 1; j < 16; ++j) z[j] = cmul(z[j], tw2[j * R3 + m1]);
            __syncthreads();
#pragma unroll
            for (int j = 0; j < 16; ++j) Sf[k2 * RS + 17 * m1 + j] = z[j];
        }
        __syncthreads();
        // ---- pass 3: DFT_R3 over m1; Z[k2 + 16 j + 256 j'] at zpos ----
        {
            const int j = lt & 15;
            float2 v[PP][R3];
#pragma unroll
            for (int p = 0; p < PP; ++p) {
                const int k2 = (lt >> 4) + (TPF / 16) * p;
#pragma unroll
                for (int m1 = 0; m1 < R3; ++m1) v[p][m1] = Sf[k2 * RS + 17 * m1 + j];
            }
            __syncthreads();
#pragma unroll
            for (int p = 0; p < PP; ++p) {
                const int k2 = (lt >> 4) + (TPF / 16) * p;
                Dft<R3>::run(v[p]);
#pragma unroll
                for (int jj = 0; jj < R3; ++jj) Sf[zpos(k2 + 16 * j + 256 * jj)] = v[p][jj];
            }
        }
        __syncthreads();
        // ---- teeth: real-FFT split at the tooth bins, coalesced outputs ----
        for (int item = threadIdx.x; item < nf * T; item += blockDim.x) {
            const int f = item / T;
            const int k = item - f * T;
            const float2* Z = S + f * BUF;
            const int bb = bins[k];
            const int i1 = (bb == L) ? 0 : bb;
            const int i2 = (bb == 0) ? 0 : L - bb;
            const float2 Zb = Z[zpos(i1)];
            const float2 Zr = Z[zpos(i2)];
            // E = (Zb + conj Zr) / 2, O = (Zb - conj Zr) / (2 i), X_b = E + W_N^b O
            const float2 E = make_float2(0.5f * (Zb.x + Zr.x), 0.5f * (Zb.y - Zr.y));
            const float2 Dd = make_float2(0.5f * (Zb.x - Zr.x), 0.5f * (Zb.y + Zr.y));
            const float2 O = make_float2(Dd.y, -Dd.x);
            const float2 X = cadd(E, cmul(twb[k], O));
            const float amp = cabs_approx(X);
            const int64_t o = (f0 + f) * T + k;
            if (a.amps) a.amps[o] = amp;
            if (a.y) a.y[o] = __fmul_rn(amp, iref[k]);
        }
        off_cur = off_next;
    }
    cp_async_wait_all();
}

template <int L>
void* pow2_fn()
{
    return reinterpret_cast<void*>(&pow2_readout_kernel<L>);
}

void* pow2_ptr(int L)
{
    switch (L) {
    case 1024: return pow2_fn<1024>();
    case 2048: return pow2_fn<2048>();
    case 4096: return pow2_fn<4096>();
    default: return nullptr;
    }
}

int pow2_fpb(int L) { return kPow2Threads / (L / 16); }

}  // namespace

// Chooses the power-of-two readout for full real transforms with L = N / 2 in
// {1024, 2048, 4096}: shared-memory layout (twiddles and tooth tables, two
// sample buffers, the exchange buffers) and the grid; leaves pow2_ok false
// otherwise.
cudaError_t setup_pow2(cg_plan_s* p)
{
    p->pow2_ok = false;
    if (p->kind != CG_FFT_FULL || p->M != 2) return cudaSuccess;
    const int L = p->L, T = p->T;
    void* fn = pow2_ptr(L);
    if (!fn) return cudaSuccess;
    const int fpb = pow2_fpb(L);
    const int N = 2 * L;
    ReadoutArgs& r = p->pa;
    r = p->ra;
    int off = 8 * L + 8 * 16 * (L / 256) + 8 * T + 4 * T + 4 * T;
    off = (off + 15) & ~15;
    r.sm_a = off;
    off += fpb * (L + L / 16) * 8;
    r.sm_raw = off;
    off += 2 * (fpb * N + 16) * 2;
    r.sm_total = (off + 15) & ~15;
    cudaError_t e;
    if ((e = raise_smem_limit(fn, r.sm_total)) != cudaSuccess) return e;
    int occ = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kPow2Threads, r.sm_total)) != cudaSuccess)
        return e;
    if (occ < 1) return cudaSuccess;
    p->grid_pow2 = p->num_sms * occ;
    p->pow2_ok = true;
    return cudaSuccess;
}

cudaError_t launch_pow2_readout(const cg_plan_s* p, const int16_t* frames, int64_t n, float* amps, float* y,
                                cudaStream_t s)
{
    ReadoutArgs r = p->pa;
    r.frames = frames;
    r.n_frames = n;
    r.amps = amps;
    r.y = y;
    const int fpb = pow2_fpb(p->L);
    const int64_t nb = (n + fpb - 1) / fpb;
    const int grid = static_cast<int>(nb < p->grid_pow2 ? nb : p->grid_pow2);
    void* args[] = {&r};
    return cudaLaunchKernel(pow2_ptr(p->L), dim3(grid), dim3(kPow2Threads), args, r.sm_total, s);
}

}  // namespace cg
