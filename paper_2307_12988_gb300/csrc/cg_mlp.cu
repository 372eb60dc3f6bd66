// cg_mlp.cu -- training side of the learned initial guess: a multilayer
// perceptron n_in -> H -> H -> n_out (tanh-form GELU, linear output, MSE loss)
// trained on the GPU by the library's own kernels: a tensor-core matrix
// product (FP32 operands split into TF32 pairs, FP32 accumulation) with fused
// bias / activation / activation-derivative epilogues,
// column sums for the bias gradients, the MSE gradient with a fixed-order
// loss reduction, a minibatch gather and Adam.  Every result is computed by
// one thread in a fixed order (no atomics), so training is deterministic.
//
// The paper seeds each LM fit from filtered data and notes that the iteration
// count depends on the quality of that seed; the network learns the seed.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include <cuda_runtime.h>

#include "cg_internal.h"
#include "cg_tc.cuh"

struct cg_mlp_s {
    int device = 0;
    int n_in = 0, H = 0, n_out = 0, max_batch = 0;
    int64_t np = 0;
    int64_t step = 0;                 // Adam steps taken
    float* theta = nullptr;           // [np] parameters
    float* grad = nullptr;            // [np]
    float* m = nullptr;               // [np] Adam first moment
    float* v = nullptr;               // [np] Adam second moment
    // activations and gradients of one batch
    float *xb = nullptr, *tb = nullptr;          // gathered batch [max_batch][n_in / n_out]
    float *z1 = nullptr, *a1 = nullptr, *z2 = nullptr, *a2 = nullptr, *out = nullptr;
    float *g_out = nullptr, *g_z2 = nullptr, *g_z1 = nullptr;
    float* part = nullptr;            // [kLossBlocks] loss partial sums
    float* loss = nullptr;            // [1]
    float* ws = nullptr;              // K-split partial sums of the weight gradients
    int* err = nullptr;               // [1] set by a matrix-product block whose bounded wait ran out
    std::vector<float> in_mean, in_scale, out_mean, out_scale;
};

namespace cg {
namespace {

constexpr int kLossBlocks = 256;
constexpr float kGeluK = 0.7978845608028654f;   // sqrt(2 / pi)
constexpr float kGeluC = 0.044715f;

enum { kEpiNone = 0, kEpiBias = 1, kEpiBiasGelu = 2, kEpiGeluGrad = 3 };

__device__ __forceinline__ float gelu_f(float z)
{
    const float t = tanhf(kGeluK * fmaf(kGeluC * z * z, z, z));
    return 0.5f * z * (1.0f + t);
}
__device__ __forceinline__ float gelu_grad_f(float z)
{
    const float t = tanhf(kGeluK * fmaf(kGeluC * z * z, z, z));
    return 0.5f * (1.0f + t) + 0.5f * z * (1.0f - t * t) * kGeluK * fmaf(3.0f * kGeluC, z * z, 1.0f);
}

// ---------------------------------------------------------------------------
// C[m][n] = epilogue(sum_k opA(m,k) opB(k,n)) on the tensor cores.
// opA(m,k) = TA ? A[k][m] : A[m][k];  opB(k,n) = TB ? B[n][k] : B[k][n].
// Each FP32 operand is split x = hi + lo with hi = tf32(x) and lo =
// tf32(x - hi) (x - hi is exact in FP32), and C takes hi*hi + hi*lo + lo*hi
// (tcgen05.mma kind::tf32, FP32 accumulation in tensor memory): the dropped
// lo*lo and the rounding of lo are each about 2^-22 of |x y|, near FP32's own
// rounding, where one TF32 product would lose 2^-11 (the three-product TF32
// split is a standard way to recover FP32 accuracy from TF32 units).
//
// One block per 128 x bn output tile (bn = 16 .. 128) and K range.  Eight
// worker warps copy 32-element K blocks of both operands straight into the
// K-major 128-byte-swizzled tile with 4-byte cp.async (any layout, any
// alignment; out-of-range elements zero-filled), two blocks ahead of the one
// they split in place (hi rounded where it lies, lo beside it) for the MMAs;
// three buffers, and the MMAs of one block run while the next is split.
// Warp 8 owns TMEM and issues the MMAs from one lane; the workers then read
// the accumulator out through shared memory and apply the epilogue row by
// row.  With gridDim.z > 1, block z takes the z-th K range and writes its
// raw sum to ws[z][M][N]; a second kernel adds the ranges in order of z.
// Every sum has a fixed order, so training stays deterministic.  Waits are
// bounded; on a time-out the block sets the object's error word and writes
// nothing.
// Epilogue: kEpiBias C = acc + bias[n]; kEpiBiasGelu C = z = acc + bias[n],
// C2 = gelu(z); kEpiGeluGrad C = acc * gelu'(aux[m][n]).
// ---------------------------------------------------------------------------
constexpr int kGM = 128;            // rows per tile (MMA M)
constexpr int kGK = 32;             // K elements per block (one 128-byte swizzle row of FP32)
constexpr int kGN = 128;            // columns per tile at most (MMA N)
constexpr int kGStages = 3;
constexpr int kGWorkerWarps = 8;    // copy / split / epilogue warps
constexpr int kGProducers = 32 * kGWorkerWarps;
constexpr int kGThreads = kGProducers + 32;   // + the MMA warp
constexpr int kGMaxSplit = 8;       // K ranges of one output tile at most
constexpr uint32_t kGPolls = 1u << 22;
constexpr int kGTile = kGM * kGK * 4;            // 16 KiB: one (hi or lo) tile of A or of B
constexpr int kGStage = 4 * kGTile;              // A hi, A lo, B hi, B lo
constexpr int kGSmem = 1024 + kGStages * kGStage + 128;
constexpr int kGPitch = kGN + 1;                 // epilogue rows in shared memory (floats)
static_assert(kGM * kGPitch * 4 <= kGStages * kGStage, "epilogue tile must fit in the operand buffers");

// bounded wait; with watch_abort it also gives up once another thread has
// set the block's abort flag
__device__ __forceinline__ bool tg_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag, bool watch_abort)
{
    const uint64_t t0 = tc::globaltimer_ns();
    for (uint32_t i = 0; i < kGPolls; ++i) {
        if (tc::mbar_try_wait(bar, parity)) return true;
        if ((i & 255u) == 255u &&
            ((watch_abort && *abort_flag) || tc::globaltimer_ns() - t0 > tc::kWaitLimitNs))
            return false;
    }
    return false;
}

// barrier of the worker threads (named barrier 1) that also returns whether
// any of them passed `flag` true: the same answer in every thread
__device__ __forceinline__ bool producers_any(bool flag)
{
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n"
        " bar.red.or.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(r)
        : "r"(flag ? 1u : 0u), "n"(kGProducers)
        : "memory");
    return r != 0;
}
__device__ __forceinline__ void producers_sync() { asm volatile("bar.sync 1, %0;\n" ::"n"(kGProducers) : "memory"); }

// FP32 -> TF32, round to nearest (ties away), as a 32-bit pattern with the
// low 13 mantissa bits zero
__device__ __forceinline__ float tf32_rn(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// cp.async of rows [row0, row0 + nrows) x K elements [k0, k0 + 32) of an
// operand into the K-major 128-byte-swizzled tile `dst` (element (r, k) at
// byte r * 128 + 16 * ((k / 4) ^ (r % 8)) + 4 * (k % 4)); elements outside
// rows_total x K are zero-filled.  KMAJOR: element (r, k) at src[r * ld + k];
// worker warp w copies rows w, w + 8, ..., lane = k (128 contiguous bytes a
// row).  Else element (r, k) at src[k * ld + r]; warp w copies 8-row groups
// w, w + 8, ..., lane = (r % 8) + 8 (k % 4) over the 8 groups of 4 k (32-byte
// segments, and no two lanes on one shared-memory bank).  nrows is a
// multiple of 8.
template <bool KMAJOR>
__device__ __forceinline__ void tg_copy(unsigned char* dst, const float* __restrict__ src, int ld, int rows_total,
                                        int row0, int nrows, int K, int k0, int t)
{
    const int w = t >> 5, lane = t & 31;
    if (KMAJOR) {
        const int gk = k0 + lane;
        const bool kin = gk < K;
        for (int r = w; r < nrows; r += kGWorkerWarps) {
            const int gr = row0 + r;
            const bool in = kin && gr < rows_total;
            const float* g = in ? src + static_cast<int64_t>(gr) * ld + gk : src;
            tc::cp_async4_zfill(dst + r * 128 + ((((lane >> 2) ^ (r & 7))) << 4) + ((lane & 3) << 2), g, in ? 4u : 0u);
        }
    } else {
        const int rl = lane & 7, kl = lane >> 3;
        for (int rb = w; rb < (nrows >> 3); rb += kGWorkerWarps) {
            const int r = rb * 8 + rl;
            const int gr = row0 + r;
            const bool rin = gr < rows_total;
            unsigned char* d = dst + r * 128 + (kl << 2);
#pragma unroll
            for (int kq = 0; kq < 8; ++kq) {
                const int gk = k0 + kq * 4 + kl;
                const bool in = rin && gk < K;
                const float* g = in ? src + static_cast<int64_t>(gk) * ld + gr : src;
                tc::cp_async4_zfill(d + ((kq ^ rl) << 4), g, in ? 4u : 0u);
            }
        }
    }
}

// split the FP32 values of a tile in place: hi <- tf32(x), lo <- tf32(x - hi)
__device__ __forceinline__ void tg_split(unsigned char* hi, unsigned char* lo, int bytes, int t)
{
    for (int o = t * 16; o < bytes; o += kGProducers * 16) {
        const float4 x = *reinterpret_cast<const float4*>(hi + o);
        float4 h, l;
        h.x = tf32_rn(x.x);
        h.y = tf32_rn(x.y);
        h.z = tf32_rn(x.z);
        h.w = tf32_rn(x.w);
        l.x = tf32_rn(x.x - h.x);
        l.y = tf32_rn(x.y - h.y);
        l.z = tf32_rn(x.z - h.z);
        l.w = tf32_rn(x.w - h.w);
        *reinterpret_cast<float4*>(hi + o) = h;
        *reinterpret_cast<float4*>(lo + o) = l;
    }
}

template <bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(kGThreads, 1) tgemm_kernel(int M, int N, int K, int bn, int kb_per,
                                                             const float* __restrict__ A,
                                                             int lda, const float* __restrict__ B, int ldb,
                                                             float* __restrict__ C, int ldc,
                                                             const float* __restrict__ bias,
                                                             const float* __restrict__ aux, float* __restrict__ C2,
                                                             float* __restrict__ ws, int* err)
{
    extern __shared__ __align__(1024) unsigned char tg_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(tg_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(sm + kGStages * kGStage);
    uint64_t* empty = full + kGStages;
    uint64_t* done = empty + kGStages;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * kGM, n0 = blockIdx.x * bn;
    const int ncols = N - n0 < bn ? N - n0 : bn;
    const int BN = (ncols + 15) & ~15;               // MMA N: a multiple of 16
    const int nkb_all = (K + kGK - 1) / kGK;
    const int kb0 = blockIdx.z * kb_per;
    const int nkb = nkb_all - kb0 < kb_per ? nkb_all - kb0 : kb_per;   // >= 1 (host)
    auto stage = [&](int s) { return sm + s * kGStage; };   // A hi | A lo | B hi | B lo

    if (threadIdx.x == 0) {
        for (int s = 0; s < kGStages; ++s) {
            tc::mbar_init(&full[s], kGProducers);
            tc::mbar_init(&empty[s], 1);
        }
        tc::mbar_init(done, 1);
        *abort_flag = 0;
        tc::fence_mbar_init();
    }
    if (warp == kGWorkerWarps) tc::tmem_alloc(tmem_slot, kGN);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp < kGWorkerWarps) {
        const int t = threadIdx.x;
        auto issue = [&](int b) {   // block b (local index) into stage b % kGStages
            unsigned char* st = stage(b % kGStages);
            const int k0 = (kb0 + b) * kGK;
            tg_copy<!TA>(st, A, lda, M, m0, kGM, K, k0, t);
            tg_copy<TB>(st + 2 * kGTile, B, ldb, N, n0, BN, K, k0, t);
        };
        issue(0);
        tc::cp_async_commit();
        if (nkb > 1) issue(1);
        tc::cp_async_commit();
        for (int kb = 0; kb < nkb; ++kb) {
            tc::cp_async_wait_pending(1);    // this thread's copies of block kb have landed
            producers_sync();                // ... and every other worker's
            unsigned char* st = stage(kb % kGStages);
            tg_split(st, st + kGTile, kGM * 128, t);
            tg_split(st + 2 * kGTile, st + 3 * kGTile, BN * 128, t);
            tc::fence_proxy_async_smem();
            tc::mbar_arrive(&full[kb % kGStages]);
            // refill the buffer of block kb - 1 with block kb + 2 once its
            // MMAs are done (they run while block kb was being split)
            const int nb = kb + 2;
            bool ok = true;
            if (nb < nkb && nb >= kGStages)
                ok = tg_wait(&empty[nb % kGStages], (nb / kGStages - 1) & 1u, abort_flag, true);
            if (!ok) *abort_flag = 1;
            if (producers_any(!ok)) break;   // every worker leaves together
            if (nb < nkb) issue(nb);
            tc::cp_async_commit();
        }
        tc::cp_async_wait_pending(0);        // nothing in flight past this point
    } else if (lane == 0) {
        const uint32_t idesc = tc::idesc_tf32(kGM, BN);
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb % kGStages;
            if (!tg_wait(&full[s], (kb / kGStages) & 1u, abort_flag, true)) {
                *abort_flag = 1;
                break;
            }
            tc::tc_fence_after();
            const uint32_t ah = tc::smem_u32(stage(s)), al = ah + kGTile;
            const uint32_t bh = ah + 2 * kGTile, bl = ah + 3 * kGTile;
#pragma unroll
            for (int kk = 0; kk < kGK / 8; ++kk) {
                const uint32_t ko = kk * 32;   // 8 TF32 elements of 4 bytes
                tc::mma_tf32(tmem, tc::sdesc_sw128(ah + ko), tc::sdesc_sw128(bh + ko), idesc,
                             (kb > 0 || kk > 0) ? 1u : 0u);
                tc::mma_tf32(tmem, tc::sdesc_sw128(ah + ko), tc::sdesc_sw128(bl + ko), idesc, 1u);
                tc::mma_tf32(tmem, tc::sdesc_sw128(al + ko), tc::sdesc_sw128(bh + ko), idesc, 1u);
            }
            tc::mma_commit(&empty[s]);
        }
        tc::mma_commit(done);   // also on abort: TMEM is quiescent before it is read or freed
    }

    if (warp < kGWorkerWarps) {
        // the MMA lane commits `done` on every path, so this wait does not
        // watch the abort flag: TMEM is quiescent once it returns true
        __syncwarp();
        const bool waited = tg_wait(done, 0, abort_flag, false);
        const bool failed = producers_any(!waited || *abort_flag);   // same answer in every worker
        tc::tc_fence_after();
        if (!failed) {
            // the accumulator -> shared memory (the operand buffers are free:
            // every MMA and every copy has completed): warp w reads TMEM lanes
            // 32 (w % 4) .. + 31, 16-column chunks w / 4, w / 4 + 2, ...;
            // then rows go out whole, so that loads of aux and stores of C
            // coalesce: warp w takes rows 16 w .. 16 w + 15
            float* T = reinterpret_cast<float*>(sm);
            const int quarter = warp & 3, half = warp >> 2;
            const uint32_t lane_base = tmem + (static_cast<uint32_t>(quarter * 32) << 16);
            for (int j = half; j < BN / 16; j += 2) {
                float v[16];
                tc::tmem_ld16(lane_base + 16 * j, v);
#pragma unroll
                for (int i = 0; i < 16; ++i) T[(quarter * 32 + lane) * kGPitch + 16 * j + i] = v[i];
            }
            producers_sync();
            float* part = gridDim.z > 1 ? ws + static_cast<int64_t>(blockIdx.z) * M * N : nullptr;
            const int rw = warp * 16;                       // first tile row of this warp
            const int rows = M - (m0 + rw) < 16 ? M - (m0 + rw) : 16;
            constexpr int kQ = kGN / 32;   // columns of a lane
            float bq[kQ];
#pragma unroll
            for (int q = 0; q < kQ; ++q) {
                const int c = lane + 32 * q;
                bq[q] = ((EPI == kEpiBias || EPI == kEpiBiasGelu) && c < ncols) ? bias[n0 + c] : 0.f;
            }
            // four rows at a time: every load of a group is issued before its
            // values are used
            for (int r0 = 0; r0 < rows; r0 += 4) {
                float av[4][kQ];
#pragma unroll
                for (int rr = 0; rr < 4; ++rr)
#pragma unroll
                    for (int q = 0; q < kQ; ++q) {
                        const int r = r0 + rr, c = lane + 32 * q;
                        av[rr][q] = (EPI == kEpiGeluGrad && r < rows && c < ncols)
                                        ? aux[static_cast<int64_t>(m0 + rw + r) * ldc + n0 + c]
                                        : 0.f;
                    }
#pragma unroll
                for (int rr = 0; rr < 4; ++rr) {
                    const int r = r0 + rr;
                    if (r >= rows) break;
                    const int64_t m = m0 + rw + r;
#pragma unroll
                    for (int q = 0; q < kQ; ++q) {
                        const int c = lane + 32 * q;
                        if (c >= ncols) continue;
                        float v = T[(rw + r) * kGPitch + c];
                        if (part) {
                            part[m * N + n0 + c] = v;
                            continue;
                        }
                        const int64_t o = m * ldc + n0 + c;
                        if (EPI == kEpiBias || EPI == kEpiBiasGelu) v += bq[q];
                        if (EPI == kEpiGeluGrad) v *= gelu_grad_f(av[rr][q]);
                        C[o] = v;
                        if (EPI == kEpiBiasGelu) C2[o] = gelu_f(v);
                    }
                }
            }
        } else if (threadIdx.x == 0 && err) {
            atomicExch(err, 1);
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == kGWorkerWarps) {
        __syncwarp();
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, kGN);
    }
}

// C[m][n] = sum over z < splits of ws[z][m][n], in order of z
__global__ void split_sum_kernel(const float* __restrict__ ws, int splits, int64_t mn, float* __restrict__ C)
{
    for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < mn;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        float s = ws[e];
        for (int z = 1; z < splits; ++z) s += ws[z * mn + e];
        C[e] = s;
    }
}

// out[n] = sum over rows m of A[m][n]: block (32 x 32) per 32 columns; thread
// (x, y) adds rows y, y + 32, ... of column x in order, then thread (x, 0)
// adds the 32 partial sums in order of y (fixed order: deterministic)
__global__ void __launch_bounds__(1024) colsum_kernel(const float* __restrict__ A, int M, int N,
                                                      float* __restrict__ out)
{
    __shared__ float part[32][33];
    const int n = blockIdx.x * 32 + threadIdx.x;
    float s = 0.f;
    if (n < N)
        for (int m = threadIdx.y; m < M; m += 32) s += A[static_cast<int64_t>(m) * N + n];
    part[threadIdx.y][threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.y == 0 && n < N) {
        float t = part[0][threadIdx.x];
        for (int y = 1; y < 32; ++y) t += part[y][threadIdx.x];
        out[n] = t;
    }
}

// g = 2 (o - t) / count; part[block] = the block's sum of (o - t)^2
__global__ void __launch_bounds__(256) mse_kernel(const float* __restrict__ o, const float* __restrict__ t,
                                                   int64_t count, float* __restrict__ g, float* __restrict__ part)
{
    __shared__ float red[256];
    const float scale = 2.0f / static_cast<float>(count);
    float s = 0.f;
    for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < count;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const float d = o[e] - t[e];
        g[e] = scale * d;
        s = fmaf(d, d, s);
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// loss = sum of the partials / count, written to loss[0] and (optionally) copy[0]
__global__ void __launch_bounds__(256) loss_final_kernel(const float* __restrict__ part, int nparts, int64_t count,
                                                         float* __restrict__ loss, float* __restrict__ copy)
{
    __shared__ float red[256];
    float s = 0.f;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) s += part[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const float l = red[0] / static_cast<float>(count);
        loss[0] = l;
        if (copy) copy[0] = l;
    }
}

__global__ void adam_kernel(float* __restrict__ theta, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int64_t np, float lr, float b1, float b2, float eps, float bc1,
                            float bc2)
{
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < np;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const float gi = g[i];
        const float mi = fmaf(b1, m[i], (1.0f - b1) * gi);
        const float vi = fmaf(b2, v[i], (1.0f - b2) * gi * gi);
        m[i] = mi;
        v[i] = vi;
        theta[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    }
}

// dst[r][:] = src[idx[r]][:] for r < rows (an index outside [0, n_src) gives a zero row)
__global__ void gather_rows_kernel(const float* __restrict__ src, int64_t n_src, const int32_t* __restrict__ idx,
                                   int rows, int width, float* __restrict__ dst)
{
    const int64_t total = static_cast<int64_t>(rows) * width;
    for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int r = static_cast<int>(e / width);
        const int c = static_cast<int>(e - static_cast<int64_t>(r) * width);
        const int64_t i = idx[r];
        dst[e] = (i >= 0 && i < n_src) ? src[i * width + c] : 0.f;
    }
}

// ws: scratch of kGMaxSplit * M * N floats, or null (no K split).  Only
// products without an epilogue are split.
template <bool TA, bool TB, int EPI>
cudaError_t sgemm(int M, int N, int K, const float* A, int lda, const float* B, int ldb, float* C, int ldc,
                  const float* bias, const float* aux, float* C2, float* ws, int* err, cudaStream_t s)
{
    if (M <= 0 || N <= 0) return cudaSuccess;
    if (K <= 0) return cudaErrorInvalidValue;
    void* fn = reinterpret_cast<void*>(&tgemm_kernel<TA, TB, EPI>);
    cudaError_t e = raise_smem_limit(fn, kGSmem);
    if (e != cudaSuccess) return e;
    // Tile width bn (128, 64, 32 or 16 columns) and K ranges: the pair with
    // the least modelled time, waves x (a fixed cost + per K block the A tile
    // and a bn-row B tile + the epilogue of bn columns), in units of one
    // 128-row operand tile; K ranges of 4 blocks at least and only for
    // products without an epilogue.  These products are small, so filling
    // the SMs matters more than re-reading A once per column tile from L2.
    static int n_sm = 0;
    if (n_sm == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n_sm < 1)
            n_sm = 1;
    }
    const int tiles_m = (M + kGM - 1) / kGM;
    const int nkb = (K + kGK - 1) / kGK;
    const int max_split = (EPI == kEpiNone && ws && ldc == N) ? std::min(kGMaxSplit, std::max(1, nkb / 4)) : 1;
    int bn = kGN, kb_per = nkb, splits = 1;
    double best = 0.0;
    for (int w = kGN; w >= 16; w >>= 1) {
        for (int sp = 1; sp <= max_split; ++sp) {
            const int per = (nkb + sp - 1) / sp;
            const int sp_eff = (nkb + per - 1) / per;
            const int64_t ctas = static_cast<int64_t>(tiles_m) * ((N + w - 1) / w) * sp_eff;
            const double waves = static_cast<double>((ctas + n_sm - 1) / n_sm);
            const double tm = waves * (3.0 + per * (1.0 + w / 128.0) + 2.0 * w / 128.0) + (sp_eff > 1 ? 1.0 : 0.0);
            if (best == 0.0 || tm < best) {
                best = tm;
                bn = w;
                kb_per = per;
                splits = sp_eff;
            }
        }
    }
    const int tiles_n = (N + bn - 1) / bn;
    dim3 grid(tiles_n, tiles_m, splits);
    tgemm_kernel<TA, TB, EPI><<<grid, kGThreads, kGSmem, s>>>(M, N, K, bn, kb_per, A, lda, B, ldb, C, ldc, bias,
                                                              aux, C2, ws, err);
    if (splits > 1) {
        const int64_t mn = static_cast<int64_t>(M) * N;
        const int blocks = static_cast<int>(std::min<int64_t>((mn + 255) / 256, 1024));
        split_sum_kernel<<<blocks, 256, 0, s>>>(ws, splits, mn, C);
    }
    return cudaGetLastError();
}

struct Offsets {
    int64_t W1, b1, W2, b2, W3, b3;
};
Offsets offsets(const cg_mlp_s* m)
{
    Offsets o;
    o.W1 = 0;
    o.b1 = o.W1 + static_cast<int64_t>(m->H) * m->n_in;
    o.W2 = o.b1 + m->H;
    o.b2 = o.W2 + static_cast<int64_t>(m->H) * m->H;
    o.W3 = o.b2 + m->H;
    o.b3 = o.W3 + static_cast<int64_t>(m->n_out) * m->H;
    return o;
}

// forward of rows x [n][n_in] (n <= max_batch) into the object's activations
cudaError_t forward_batch(cg_mlp_s* m, const float* x, int n, float* out, cudaStream_t s)
{
    const Offsets o = offsets(m);
    const float* th = m->theta;
    cudaError_t e = sgemm<false, true, kEpiBiasGelu>(n, m->H, m->n_in, x, m->n_in, th + o.W1, m->n_in, m->z1,
                                                     m->H, th + o.b1, nullptr, m->a1, nullptr, m->err, s);
    if (e == cudaSuccess)
        e = sgemm<false, true, kEpiBiasGelu>(n, m->H, m->H, m->a1, m->H, th + o.W2, m->H, m->z2, m->H,
                                             th + o.b2, nullptr, m->a2, nullptr, m->err, s);
    if (e == cudaSuccess)
        e = sgemm<false, true, kEpiBias>(n, m->n_out, m->H, m->a2, m->H, th + o.W3, m->H, out, m->n_out,
                                         th + o.b3, nullptr, nullptr, nullptr, m->err, s);
    return e;
}

cudaError_t backward_batch(cg_mlp_s* m, const float* x, const float* t, int n, float* loss_copy, cudaStream_t s)
{
    const Offsets o = offsets(m);
    const float* th = m->theta;
    float* g = m->grad;
    const int H = m->H, ni = m->n_in, no = m->n_out;
    cudaError_t e = forward_batch(m, x, n, m->out, s);
    if (e != cudaSuccess) return e;
    const int64_t count = static_cast<int64_t>(n) * no;
    mse_kernel<<<kLossBlocks, 256, 0, s>>>(m->out, t, count, m->g_out, m->part);
    loss_final_kernel<<<1, 256, 0, s>>>(m->part, kLossBlocks, count, m->loss, loss_copy);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // output layer: dW3 = g_out^T a2, db3 = colsum(g_out)
    e = sgemm<true, false, kEpiNone>(no, H, n, m->g_out, no, m->a2, H, g + o.W3, H, nullptr, nullptr, nullptr,
                                     m->ws, m->err, s);
    if (e != cudaSuccess) return e;
    colsum_kernel<<<(no + 31) / 32, dim3(32, 32), 0, s>>>(m->g_out, n, no, g + o.b3);
    // g_z2 = (g_out W3) * gelu'(z2)
    e = sgemm<false, false, kEpiGeluGrad>(n, H, no, m->g_out, no, th + o.W3, H, m->g_z2, H, nullptr, m->z2,
                                          nullptr, nullptr, m->err, s);
    if (e != cudaSuccess) return e;
    e = sgemm<true, false, kEpiNone>(H, H, n, m->g_z2, H, m->a1, H, g + o.W2, H, nullptr, nullptr, nullptr,
                                     m->ws, m->err, s);
    if (e != cudaSuccess) return e;
    colsum_kernel<<<(H + 31) / 32, dim3(32, 32), 0, s>>>(m->g_z2, n, H, g + o.b2);
    // g_z1 = (g_z2 W2) * gelu'(z1)
    e = sgemm<false, false, kEpiGeluGrad>(n, H, H, m->g_z2, H, th + o.W2, H, m->g_z1, H, nullptr, m->z1, nullptr,
                                          nullptr, m->err, s);
    if (e != cudaSuccess) return e;
    e = sgemm<true, false, kEpiNone>(H, ni, n, m->g_z1, H, x, ni, g + o.W1, ni, nullptr, nullptr, nullptr,
                                     m->ws, m->err, s);
    if (e != cudaSuccess) return e;
    colsum_kernel<<<(H + 31) / 32, dim3(32, 32), 0, s>>>(m->g_z1, n, H, g + o.b1);
    return cudaGetLastError();
}

cudaError_t adam(cg_mlp_s* m, float lr, float b1, float b2, float eps, cudaStream_t s)
{
    m->step += 1;
    const float bc1 = static_cast<float>(1.0 - std::pow(static_cast<double>(b1), static_cast<double>(m->step)));
    const float bc2 = static_cast<float>(1.0 - std::pow(static_cast<double>(b2), static_cast<double>(m->step)));
    const int blocks = static_cast<int>(std::min<int64_t>((m->np + 255) / 256, 1024));
    adam_kernel<<<blocks, 256, 0, s>>>(m->theta, m->grad, m->m, m->v, m->np, lr, b1, b2, eps, bc1, bc2);
    return cudaGetLastError();
}

uint64_t splitmix64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

cg_status fail_m(cg_status st, const char* msg)
{
    set_last_error(msg);
    return st;
}
cg_status cuda_fail_m(cudaError_t e, const char* what)
{
    static thread_local char buf[256];
    std::snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
    set_last_error(buf);
    return e == cudaErrorMemoryAllocation ? CG_ERR_NOMEM : CG_ERR_CUDA;
}

void free_mlp(cg_mlp_s* m)
{
    for (float* q : {m->theta, m->grad, m->m, m->v, m->xb, m->tb, m->z1, m->a1, m->z2, m->a2, m->out, m->g_out,
                     m->g_z2, m->g_z1, m->part, m->loss, m->ws})
        if (q) cudaFree(q);
    if (m->err) cudaFree(m->err);
    delete m;
}

// after a device synchronisation: CG_ERR_TIMEOUT (and the word cleared) when a
// matrix-product block gave up waiting since the last check
cg_status take_err(cg_mlp_s* m, const char* what)
{
    int h = 0;
    cudaError_t e = cudaMemcpy(&h, m->err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && h != 0) e = cudaMemset(m->err, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_fail_m(e, what);
    if (h != 0) {
        static thread_local char buf[256];
        std::snprintf(buf, sizeof(buf), "%s: a matrix-product wait ran out; results since the last check are invalid",
                      what);
        return fail_m(CG_ERR_TIMEOUT, buf);
    }
    return CG_OK;
}

}  // namespace
}  // namespace cg

using namespace cg;

extern "C" {

int64_t cg_mlp_param_count(int n_in, int n_hidden, int n_out)
{
    if (n_in < 1 || n_hidden < 1 || n_out < 1) return 0;
    const int64_t H = n_hidden;
    return H * n_in + H + H * H + H + static_cast<int64_t>(n_out) * H + n_out;
}

cg_status cg_mlp_create(cg_mlp_t* out, int n_in, int n_hidden, int n_out, int max_batch, uint64_t seed)
{
    if (!out) return fail_m(CG_ERR_ARG, "mlp is NULL");
    *out = nullptr;
    if (n_in < 1 || n_in > 1024) return fail_m(CG_ERR_ARG, "n_in must be in [1, 1024]");
    if (n_hidden < 1 || n_hidden > 1024) return fail_m(CG_ERR_ARG, "n_hidden must be in [1, 1024]");
    if (n_out < 1 || n_out > 16) return fail_m(CG_ERR_ARG, "n_out must be in [1, 16]");
    if (max_batch < 1 || max_batch > (1 << 20)) return fail_m(CG_ERR_ARG, "max_batch must be in [1, 2^20]");
    cg_mlp_s* m = new (std::nothrow) cg_mlp_s;
    if (!m) return fail_m(CG_ERR_NOMEM, "host allocation failed");
    cudaGetDevice(&m->device);
    m->n_in = n_in;
    m->H = n_hidden;
    m->n_out = n_out;
    m->max_batch = max_batch;
    m->np = cg_mlp_param_count(n_in, n_hidden, n_out);
    m->in_mean.assign(n_in, 0.f);
    m->in_scale.assign(n_in, 1.f);
    m->out_mean.assign(n_out, 0.f);
    m->out_scale.assign(n_out, 1.f);
    const int64_t B = max_batch, H = n_hidden;
    struct {
        float** p;
        int64_t count;
    } allocs[] = {{&m->theta, m->np}, {&m->grad, m->np}, {&m->m, m->np},       {&m->v, m->np},
                  {&m->xb, B * n_in}, {&m->tb, B * n_out}, {&m->z1, B * H},    {&m->a1, B * H},
                  {&m->z2, B * H},    {&m->a2, B * H},     {&m->out, B * n_out}, {&m->g_out, B * n_out},
                  {&m->g_z2, B * H},  {&m->g_z1, B * H},   {&m->part, kLossBlocks}, {&m->loss, 1},
                  {&m->ws, kGMaxSplit * std::max({H * H, H * n_in, H * n_out})}};
    for (auto& a : allocs) {
        cudaError_t e = cudaMalloc(a.p, sizeof(float) * a.count);
        if (e != cudaSuccess) {
            free_mlp(m);
            return cuda_fail_m(e, "cg_mlp_create");
        }
    }
    if (cudaError_t e = cudaMalloc(&m->err, sizeof(int)); e != cudaSuccess) {
        free_mlp(m);
        return cuda_fail_m(e, "cg_mlp_create");
    }
    // weights ~ U(-1/sqrt(fan_in), 1/sqrt(fan_in)) from SplitMix64(seed ^ index), biases 0
    std::vector<float> th(static_cast<size_t>(m->np), 0.f);
    const Offsets o = offsets(m);
    auto fill = [&](int64_t off, int64_t count, int fan_in) {
        const double bound = 1.0 / std::sqrt(static_cast<double>(fan_in));
        for (int64_t i = 0; i < count; ++i) {
            const uint64_t r = splitmix64(seed * 0x100000001B3ull + static_cast<uint64_t>(off + i));
            const double u = static_cast<double>(r >> 11) * (1.0 / 9007199254740992.0);   // [0, 1)
            th[static_cast<size_t>(off + i)] = static_cast<float>((2.0 * u - 1.0) * bound);
        }
    };
    fill(o.W1, H * n_in, n_in);
    fill(o.W2, H * H, n_hidden);
    fill(o.W3, static_cast<int64_t>(n_out) * H, n_hidden);
    cudaError_t e = cudaMemcpy(m->theta, th.data(), sizeof(float) * m->np, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(m->m, 0, sizeof(float) * m->np);
    if (e == cudaSuccess) e = cudaMemset(m->v, 0, sizeof(float) * m->np);
    if (e == cudaSuccess) e = cudaMemset(m->grad, 0, sizeof(float) * m->np);
    if (e == cudaSuccess) e = cudaMemset(m->err, 0, sizeof(int));
    if (e != cudaSuccess) {
        free_mlp(m);
        return cuda_fail_m(e, "cg_mlp_create");
    }
    *out = m;
    return CG_OK;
}

void cg_mlp_destroy(cg_mlp_t m)
{
    if (!m) return;
    cudaDeviceSynchronize();
    free_mlp(m);
}

cg_status cg_mlp_get_params(cg_mlp_t m, float* host, int64_t count)
{
    if (!m || !host) return fail_m(CG_ERR_ARG, "mlp or params_host is NULL");
    if (count != m->np) return fail_m(CG_ERR_ARG, "count != cg_mlp_param_count");
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(host, m->theta, sizeof(float) * count, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? take_err(m, "cg_mlp_get_params") : cuda_fail_m(e, "cg_mlp_get_params");
}

cg_status cg_mlp_set_params(cg_mlp_t m, const float* host, int64_t count)
{
    if (!m || !host) return fail_m(CG_ERR_ARG, "mlp or params_host is NULL");
    if (count != m->np) return fail_m(CG_ERR_ARG, "count != cg_mlp_param_count");
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(m->theta, host, sizeof(float) * count, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(m->m, 0, sizeof(float) * m->np);
    if (e == cudaSuccess) e = cudaMemset(m->v, 0, sizeof(float) * m->np);
    m->step = 0;
    return e == cudaSuccess ? CG_OK : cuda_fail_m(e, "cg_mlp_set_params");
}

cg_status cg_mlp_forward(cg_mlp_t m, const float* x, int64_t n, float* out, void* stream)
{
    if (!m) return fail_m(CG_ERR_ARG, "mlp is NULL");
    if (n < 0) return fail_m(CG_ERR_ARG, "n < 0");
    if (n == 0) return CG_OK;
    if (!x || !out) return fail_m(CG_ERR_ARG, "x_dev and out_dev are required");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    for (int64_t r0 = 0; r0 < n; r0 += m->max_batch) {
        const int rows = static_cast<int>(std::min<int64_t>(m->max_batch, n - r0));
        cudaError_t e = forward_batch(m, x + r0 * m->n_in, rows, out + r0 * m->n_out, s);
        if (e != cudaSuccess) return cuda_fail_m(e, "cg_mlp_forward");
    }
    return CG_OK;
}

cg_status cg_mlp_backward(cg_mlp_t m, const float* x, const float* t, int64_t n, float* loss_dev, float* grad_dev,
                          void* stream)
{
    if (!m) return fail_m(CG_ERR_ARG, "mlp is NULL");
    if (n < 1 || n > m->max_batch) return fail_m(CG_ERR_ARG, "n must be in [1, max_batch]");
    if (!x || !t) return fail_m(CG_ERR_ARG, "x_dev and t_dev are required");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = backward_batch(m, x, t, static_cast<int>(n), loss_dev, s);
    if (e == cudaSuccess && grad_dev)
        e = cudaMemcpyAsync(grad_dev, m->grad, sizeof(float) * m->np, cudaMemcpyDeviceToDevice, s);
    return e == cudaSuccess ? CG_OK : cuda_fail_m(e, "cg_mlp_backward");
}

cg_status cg_mlp_adam(cg_mlp_t m, float lr, float b1, float b2, float eps, void* stream)
{
    if (!m) return fail_m(CG_ERR_ARG, "mlp is NULL");
    if (!(lr >= 0.f) || !(b1 >= 0.f && b1 < 1.f) || !(b2 >= 0.f && b2 < 1.f) || !(eps > 0.f))
        return fail_m(CG_ERR_ARG, "Adam hyper-parameters out of range");
    cudaError_t e = adam(m, lr, b1, b2, eps, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? CG_OK : cuda_fail_m(e, "cg_mlp_adam");
}

cg_status cg_mlp_train_epoch(cg_mlp_t m, const float* x, const float* t, int64_t n, const int32_t* perm, int batch,
                             float lr, float* losses, void* stream)
{
    if (!m) return fail_m(CG_ERR_ARG, "mlp is NULL");
    if (n < 1) return fail_m(CG_ERR_ARG, "n < 1");
    if (!x || !t || !perm) return fail_m(CG_ERR_ARG, "x_dev, t_dev and perm_dev are required");
    if (batch < 1 || batch > m->max_batch) return fail_m(CG_ERR_ARG, "batch must be in [1, max_batch]");
    if (!(lr >= 0.f)) return fail_m(CG_ERR_ARG, "lr < 0");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int64_t b = 0;
    for (int64_t r0 = 0; r0 < n; r0 += batch, ++b) {
        const int rows = static_cast<int>(std::min<int64_t>(batch, n - r0));
        const int gx = static_cast<int>(std::min<int64_t>((static_cast<int64_t>(rows) * m->n_in + 255) / 256, 2048));
        const int gt = static_cast<int>(std::min<int64_t>((static_cast<int64_t>(rows) * m->n_out + 255) / 256, 2048));
        gather_rows_kernel<<<gx, 256, 0, s>>>(x, n, perm + r0, rows, m->n_in, m->xb);
        gather_rows_kernel<<<gt, 256, 0, s>>>(t, n, perm + r0, rows, m->n_out, m->tb);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = backward_batch(m, m->xb, m->tb, rows, losses ? losses + b : nullptr, s);
        if (e == cudaSuccess) e = adam(m, lr, 0.9f, 0.999f, 1e-8f, s);
        if (e != cudaSuccess) return cuda_fail_m(e, "cg_mlp_train_epoch");
    }
    return CG_OK;
}

cg_status cg_mlp_set_norm(cg_mlp_t m, const float* in_mean, const float* in_scale, const float* out_mean,
                          const float* out_scale)
{
    if (!m || !in_mean || !in_scale || !out_mean || !out_scale) return fail_m(CG_ERR_ARG, "NULL argument");
    for (int i = 0; i < m->n_in; ++i)
        if (!std::isfinite(in_mean[i]) || !std::isfinite(in_scale[i])) return fail_m(CG_ERR_ARG, "non-finite input norm");
    for (int i = 0; i < m->n_out; ++i)
        if (!std::isfinite(out_mean[i]) || !std::isfinite(out_scale[i]))
            return fail_m(CG_ERR_ARG, "non-finite output norm");
    m->in_mean.assign(in_mean, in_mean + m->n_in);
    m->in_scale.assign(in_scale, in_scale + m->n_in);
    m->out_mean.assign(out_mean, out_mean + m->n_out);
    m->out_scale.assign(out_scale, out_scale + m->n_out);
    return CG_OK;
}

cg_status cg_mlp_save(cg_mlp_t m, void* blob, size_t cap, size_t* bytes_out)
{
    if (!m || !bytes_out) return fail_m(CG_ERR_ARG, "mlp or bytes_out is NULL");
    const size_t floats = 2 * static_cast<size_t>(m->n_in) + 2 * static_cast<size_t>(m->n_out) + m->np;
    const size_t total = kMlpHeaderBytes + 4 * floats;
    *bytes_out = total;
    if (!blob) return CG_OK;
    if (cap < total) return fail_m(CG_ERR_ARG, "blob capacity too small");
    std::vector<float> th(static_cast<size_t>(m->np));
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(th.data(), m->theta, sizeof(float) * m->np, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail_m(e, "cg_mlp_save");
    if (cg_status st = take_err(m, "cg_mlp_save"); st != CG_OK) return st;
    unsigned char* b = static_cast<unsigned char*>(blob);
    std::memcpy(b, kMlpMagic, 8);
    const int32_t hdr[4] = {m->n_in, m->H, m->n_out, 0};
    std::memcpy(b + 8, hdr, sizeof(hdr));
    size_t off = kMlpHeaderBytes;
    auto put = [&](const float* src, size_t count) {
        std::memcpy(b + off, src, 4 * count);
        off += 4 * count;
    };
    put(m->in_mean.data(), m->n_in);
    put(m->in_scale.data(), m->n_in);
    put(m->out_mean.data(), m->n_out);
    put(m->out_scale.data(), m->n_out);
    put(th.data(), th.size());
    return CG_OK;
}

}  // extern "C"
