// cg_mlp.cu -- training side of the learned initial guess: a multilayer
// perceptron n_in -> H -> H -> n_out (tanh-form GELU, linear output, MSE loss)
// trained on the GPU by the library's own FP32 kernels: a tiled SIMT matrix
// product with fused bias / activation / activation-derivative epilogues,
// column sums for the bias gradients, the MSE gradient with a fixed-order
// loss reduction, a minibatch gather and Adam.  Every result is computed by
// one thread in a fixed order (no atomics), so training is deterministic.
//
// The paper seeds each LM fit from filtered data and notes that the iteration
// count depends on the quality of that seed; the network learns the seed.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include <cuda_runtime.h>

#include "cg_internal.h"

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
    std::vector<float> in_mean, in_scale, out_mean, out_scale;
};

namespace cg {
namespace {

constexpr int kTile = 64;
constexpr int kTK = 16;
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

// C[m][n] = sum_k opA(m,k) opB(k,n), 64 x 64 tile per block, 4 x 4 per thread.
// opA(m,k) = TA ? A[k][m] : A[m][k];  opB(k,n) = TB ? B[n][k] : B[k][n].
// Epilogue: kEpiBias C = acc + bias[n]; kEpiBiasGelu C = z = acc + bias[n],
// C2 = gelu(z); kEpiGeluGrad C = acc * gelu'(aux[m][n]).
template <bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(256) sgemm_kernel(int M, int N, int K, const float* __restrict__ A, int lda,
                                                    const float* __restrict__ B, int ldb, float* __restrict__ C,
                                                    int ldc, const float* __restrict__ bias,
                                                    const float* __restrict__ aux, float* __restrict__ C2)
{
    __shared__ float As[kTK][kTile + 4];
    __shared__ float Bs[kTK][kTile + 4];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int m0 = blockIdx.y * kTile, n0 = blockIdx.x * kTile;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int k0 = 0; k0 < K; k0 += kTK) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int i = threadIdx.x + 256 * r;
            int mm, kk;
            if (TA) { mm = i & 63; kk = i >> 6; }   // A[k][m]: contiguous in m
            else { kk = i & 15; mm = i >> 4; }      // A[m][k]: contiguous in k
            const int gm = m0 + mm, gk = k0 + kk;
            float v = 0.f;
            if (gm < M && gk < K)
                v = TA ? A[static_cast<int64_t>(gk) * lda + gm] : A[static_cast<int64_t>(gm) * lda + gk];
            As[kk][mm] = v;
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int i = threadIdx.x + 256 * r;
            int nn, kk;
            if (TB) { kk = i & 15; nn = i >> 4; }   // B[n][k]: contiguous in k
            else { nn = i & 63; kk = i >> 6; }      // B[k][n]: contiguous in n
            const int gn = n0 + nn, gk = k0 + kk;
            float v = 0.f;
            if (gn < N && gk < K)
                v = TB ? B[static_cast<int64_t>(gn) * ldb + gk] : B[static_cast<int64_t>(gk) * ldb + gn];
            Bs[kk][nn] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kTK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + ty * 4 + i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tx * 4 + j;
            if (n >= N) continue;
            const int64_t o = static_cast<int64_t>(m) * ldc + n;
            float r = acc[i][j];
            if (EPI == kEpiBias || EPI == kEpiBiasGelu) r += bias[n];
            if (EPI == kEpiGeluGrad) r *= gelu_grad_f(aux[o]);
            C[o] = r;
            if (EPI == kEpiBiasGelu) C2[o] = gelu_f(r);
        }
    }
}

// out[n] = sum over rows m of A[m][n] (one thread per column, rows in order)
__global__ void colsum_kernel(const float* __restrict__ A, int M, int N, float* __restrict__ out)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.f;
    for (int m = 0; m < M; ++m) s += A[static_cast<int64_t>(m) * N + n];
    out[n] = s;
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

template <bool TA, bool TB, int EPI>
cudaError_t sgemm(int M, int N, int K, const float* A, int lda, const float* B, int ldb, float* C, int ldc,
                  const float* bias, const float* aux, float* C2, cudaStream_t s)
{
    dim3 grid((N + kTile - 1) / kTile, (M + kTile - 1) / kTile);
    sgemm_kernel<TA, TB, EPI><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, aux, C2);
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
                                                     m->H, th + o.b1, nullptr, m->a1, s);
    if (e == cudaSuccess)
        e = sgemm<false, true, kEpiBiasGelu>(n, m->H, m->H, m->a1, m->H, th + o.W2, m->H, m->z2, m->H,
                                             th + o.b2, nullptr, m->a2, s);
    if (e == cudaSuccess)
        e = sgemm<false, true, kEpiBias>(n, m->n_out, m->H, m->a2, m->H, th + o.W3, m->H, out, m->n_out,
                                         th + o.b3, nullptr, nullptr, s);
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
    e = sgemm<true, false, kEpiNone>(no, H, n, m->g_out, no, m->a2, H, g + o.W3, H, nullptr, nullptr, nullptr, s);
    if (e != cudaSuccess) return e;
    colsum_kernel<<<(no + 127) / 128, 128, 0, s>>>(m->g_out, n, no, g + o.b3);
    // g_z2 = (g_out W3) * gelu'(z2)
    e = sgemm<false, false, kEpiGeluGrad>(n, H, no, m->g_out, no, th + o.W3, H, m->g_z2, H, nullptr, m->z2,
                                          nullptr, s);
    if (e != cudaSuccess) return e;
    e = sgemm<true, false, kEpiNone>(H, H, n, m->g_z2, H, m->a1, H, g + o.W2, H, nullptr, nullptr, nullptr, s);
    if (e != cudaSuccess) return e;
    colsum_kernel<<<(H + 127) / 128, 128, 0, s>>>(m->g_z2, n, H, g + o.b2);
    // g_z1 = (g_z2 W2) * gelu'(z1)
    e = sgemm<false, false, kEpiGeluGrad>(n, H, H, m->g_z2, H, th + o.W2, H, m->g_z1, H, nullptr, m->z1, nullptr,
                                          s);
    if (e != cudaSuccess) return e;
    e = sgemm<true, false, kEpiNone>(H, ni, n, m->g_z1, H, x, ni, g + o.W1, ni, nullptr, nullptr, nullptr, s);
    if (e != cudaSuccess) return e;
    colsum_kernel<<<(H + 127) / 128, 128, 0, s>>>(m->g_z1, n, H, g + o.b1);
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
                     m->g_z2, m->g_z1, m->part, m->loss})
        if (q) cudaFree(q);
    delete m;
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
                  {&m->g_z2, B * H},  {&m->g_z1, B * H},   {&m->part, kLossBlocks}, {&m->loss, 1}};
    for (auto& a : allocs) {
        cudaError_t e = cudaMalloc(a.p, sizeof(float) * a.count);
        if (e != cudaSuccess) {
            free_mlp(m);
            return cuda_fail_m(e, "cg_mlp_create");
        }
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
    return e == cudaSuccess ? CG_OK : cuda_fail_m(e, "cg_mlp_get_params");
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
