// cg_psd.cu -- displacement power spectral density of the fitted-centre
// series and the fit of the mechanical resonance (f0, Q) to it (paper,
// "Experimental Results", Fig. 6: PSDs for 1 s, 10 s and 10 min of data and
// the resonance frequency and quality factor fitted to them).
//
// PSD: Welch's method -- segments of M = 2L samples advanced by L, segment
// mean removed, periodic Hann window, |rfft|^2 averaged over the complete
// segments, one-sided density (factor 2 except at DC and M/2) / (fs sum w^2).
// psd_welch_kernel<L>: one segment per block pass, L/16 threads; the
// segment's L packed complex values z_n = x_2n + i x_2n+1 stay in shared
// memory (one pad per 16 values against bank conflicts) through in-place
// Stockham stages of radix 16 (and one smaller radix), each thread holding
// 16 values in registers between a stage's read and write, twiddles of all
// but a final small-radix stage from a shared table; the real-FFT split X_k = E_k + W_M^k O_k gives |X_k|^2 for
// k = 0..L, which each thread accumulates in FP64 registers over all the
// segments its block takes; per-block partials are summed and scaled by
// psd_reduce_kernel.
//
// Resonance: S(f) = A f0^4 / ((f0^2 - f^2)^2 + (f f0 / Q)^2) + B fitted to
// ln S over the bins of a band by Levenberg-Marquardt in FP64 (one block:
// per-point sums reduced in shared memory, the 4x4 solve on one thread);
// initial values from the band (largest bin, smallest bin, half-height
// width); standard errors from diag(H^-1) chi^2 / (n - 4).
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>
#include <cuda_runtime.h>

#include "cg_fft.cuh"
#include "cg_internal.h"

struct cg_psd_s {
    int device = 0;
    int L = 0;                 // complex transform length (M / 2)
    int grid = 0;              // blocks of the Welch kernel
    size_t smem = 0;
    double sum_w2 = 0.0;       // sum of the squared window
    float* win = nullptr;      // [M]
    float2* twL = nullptr;     // [L] W_L^m
    float2* twM = nullptr;     // [L + 1] W_M^k
    double* part = nullptr;    // [grid][L + 1] per-block sums of |X_k|^2
};

namespace cg {

namespace {

struct PsdArgs {
    const float* x;
    int64_t stride;            // elements between consecutive samples
    int64_t K;                 // segments
    const float* win;
    const float2* twL;
    const float2* twM;
    double* part;
};

// position of complex value i in the exchange buffer: one pad per 16 values,
// so the first stage's 16-value-stride writes fall on distinct banks
__device__ __forceinline__ int zp(int i) { return i + (i >> 4); }

// twiddles: W_L^(q s) for q < min(L, 4096), s = max(1, L / 4096), in shared
// memory (every stage but a last one of radix < 16 at L > 4096 indexes a
// multiple of s); that last stage reads the full table from global memory
template <int L>
struct TwShared {
    static constexpr int kStride = L > 4096 ? L / 4096 : 1;
    static constexpr int kSize = L > 4096 ? 4096 : L;
};

template <int R>
struct StageShape {
    static constexpr int kPerThread = 16 / R;   // butterflies per thread
};

// one in-place Stockham stage of radix R over the L values in z
// twiddle source of a stage: 0 the global table, 1 the shared W_L^(q s)
// table, 2 the shared W_256^q table (the Ns = 16 stage: consecutive frames
// read consecutive entries instead of entries 16 apart)
template <int L, int R, int kTw>
__device__ __forceinline__ void stage_inplace(float2* z, int Ns, const float2* __restrict__ ts,
                                              const float2* __restrict__ t256, const float2* __restrict__ twL)
{
    constexpr int NT = L / 16, per = L / R, NB = StageShape<R>::kPerThread;
    const int t = threadIdx.x;
    float2 a[NB][R];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int j = t + NT * b;
#pragma unroll
        for (int r = 0; r < R; ++r) a[b][r] = z[zp(j + r * per)];
    }
    __syncthreads();
    const int twstep = L / (Ns * R);
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int j = t + NT * b;
        const int k = j & (Ns - 1);
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                const int m = r * k * twstep;
                const float2 w = kTw == 2   ? t256[r * k]
                                 : kTw == 1 ? ts[m / TwShared<L>::kStride]
                                            : __ldg(&twL[m]);
                a[b][r] = cmul(a[b][r], w);
            }
        }
        Dft<R>::run(a[b]);
        const int idx = (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) z[zp(idx + r * Ns)] = a[b][r];
    }
    __syncthreads();
}

template <int L>
__global__ void __launch_bounds__(L / 16) psd_welch_kernel(PsdArgs a)
{
    constexpr int NT = L / 16, M = 2 * L;
    extern __shared__ __align__(16) float2 z[];   // [L + L/16] (padded), then the twiddle table
    float2* ts = z + L + L / 16;                  // [TwShared<L>::kSize]
    float2* t256 = ts + TwShared<L>::kSize;       // [256] W_256^q
    __shared__ double red[NT / 32];
    const int t = threadIdx.x;
    for (int i = t; i < TwShared<L>::kSize; i += NT) ts[i] = a.twL[i * TwShared<L>::kStride];
    for (int i = t; i < 256; i += NT) t256[i] = a.twL[i * (L / 256)];
    // FP64 sums of |X_k|^2 in registers; at L = 16384 (1024 threads, 64
    // registers each) in the block's own L2-resident row of part instead
    constexpr bool kRowAcc = L == 16384;
    double* row = a.part + static_cast<int64_t>(blockIdx.x) * (L + 1);
    double acc[kRowAcc ? 1 : 17];
#pragma unroll
    for (int j = 0; j < (kRowAcc ? 1 : 17); ++j) acc[j] = 0.0;
    if constexpr (kRowAcc) {
#pragma unroll
        for (int j = 0; j < 16; ++j) row[t + NT * j] = 0.0;
        if (t == 0) row[L] = 0.0;
    }
    for (int64_t s = blockIdx.x; s < a.K; s += gridDim.x) {
        const float* x = a.x + s * static_cast<int64_t>(L) * a.stride;
        float2 v[16];
        float sum = 0.0f;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int64_t n = t + NT * j;
            v[j] = make_float2(__ldg(x + 2 * n * a.stride), __ldg(x + (2 * n + 1) * a.stride));
            sum += v[j].x + v[j].y;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if ((t & 31) == 0) red[t >> 5] = sum;
        __syncthreads();
        double tot = 0.0;
#pragma unroll 1
        for (int w = 0; w < NT / 32; ++w) tot += red[w];
        const float mean = static_cast<float>(tot / M);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int n = t + NT * j;
            z[zp(n)] = make_float2((v[j].x - mean) * __ldg(a.win + 2 * n), (v[j].y - mean) * __ldg(a.win + 2 * n + 1));
        }
        __syncthreads();
        // L = 16^3 * Rl (Rl = 2, 4) or 16^2 * 8
        stage_inplace<L, 16, 1>(z, 1, ts, t256, a.twL);
        stage_inplace<L, 16, 2>(z, 16, ts, t256, a.twL);
        if constexpr (L == 2048) {
            stage_inplace<L, 8, 1>(z, 256, ts, t256, a.twL);
        } else {
            stage_inplace<L, 16, 1>(z, 256, ts, t256, a.twL);
            if constexpr (L == 8192) stage_inplace<L, 2, 0>(z, 4096, ts, t256, a.twL);
            if constexpr (L == 16384) stage_inplace<L, 4, 0>(z, 4096, ts, t256, a.twL);
        }
        // real-FFT split at every bin k = 0..L
#pragma unroll
        for (int j = 0; j < 17; ++j) {
            const int k = t + NT * j;
            if (j < 16 || t == 0) {
                const int kk = (j == 16) ? L : k;
                const float2 Zb = z[zp(kk & (L - 1))];
                const float2 Zr = z[zp((L - kk) & (L - 1))];
                const float2 E = make_float2(0.5f * (Zb.x + Zr.x), 0.5f * (Zb.y - Zr.y));
                const float2 Dd = make_float2(0.5f * (Zb.x - Zr.x), 0.5f * (Zb.y + Zr.y));
                const float2 O = make_float2(Dd.y, -Dd.x);
                const float2 X = cadd(E, cmul(__ldg(&a.twM[kk]), O));
                const double P = static_cast<double>(fmaf(X.x, X.x, X.y * X.y));
                if constexpr (kRowAcc)
                    row[kk] += P;
                else
                    acc[j] += P;
            }
        }
        __syncthreads();
    }
    if constexpr (!kRowAcc) {
#pragma unroll
        for (int j = 0; j < 16; ++j) row[t + NT * j] = acc[j];
        if (t == 0) row[L] = acc[16];
    }
}

__global__ void psd_reduce_kernel(const double* part, int nblk, int L, double scale, double* psd)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > L) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[static_cast<int64_t>(b) * (L + 1) + k];
    psd[k] = s * scale * ((k == 0 || k == L) ? 1.0 : 2.0);
}

template <int L>
void* welch_fn()
{
    return reinterpret_cast<void*>(&psd_welch_kernel<L>);
}

void* welch_ptr(int L)
{
    switch (L) {
    case 2048: return welch_fn<2048>();
    case 4096: return welch_fn<4096>();
    case 8192: return welch_fn<8192>();
    case 16384: return welch_fn<16384>();
    default: return nullptr;
    }
}

// ---------------------------------------------------------------------------
// resonance fit
// ---------------------------------------------------------------------------
constexpr int kResThreads = 256;

struct ResArgs {
    const double* psd;
    int k0, np;                // first bin and bins in the band
    double df;
    int max_iter;
    double tol, lambda0;
    double* out;               // [12]
};

// per-point sums: 10 of J^T J (upper), 4 of J^T r, chi^2, bad-point count
struct ResSums {
    double v[16];
};

__device__ __forceinline__ void res_point(double f, double S, const double (&p)[4], ResSums& s)
{
    const double f0 = p[0], Q = p[1], A = p[2], B = p[3];
    const double u = f0 * f0 - f * f;
    const double c = f * f0 / Q;
    const double D = u * u + c * c;
    const double f04 = f0 * f0 * f0 * f0;
    const double g = f04 / D;
    const double m = A * g + B;
    if (!(m > 0.0) || !(m < INFINITY)) {
        s.v[15] += 1.0;
        return;
    }
    const double dD0 = 4.0 * f0 * u + 2.0 * f * f * f0 / (Q * Q);
    const double dDQ = -2.0 * c * c / Q;
    const double im = 1.0 / m;
    double J[4];
    J[0] = A * (4.0 * f0 * f0 * f0 / D - f04 * dD0 / (D * D)) * im;
    J[1] = -A * f04 * dDQ / (D * D) * im;
    J[2] = g * im;
    J[3] = im;
    const double r = log(S) - log(m);
    int q = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = i; j < 4; ++j) s.v[q++] += J[i] * J[j];
#pragma unroll
    for (int i = 0; i < 4; ++i) s.v[10 + i] += J[i] * r;
    s.v[14] += r * r;
}

// (H + lambda diag H) d = g, Jacobi-scaled Cholesky; false if not positive definite
__device__ bool res_solve(const double* Hu, const double* g, double lambda, double* d)
{
    double H[4][4];
    int q = 0;
    for (int i = 0; i < 4; ++i)
        for (int j = i; j < 4; ++j) H[i][j] = H[j][i] = Hu[q++];
    double s[4];
    for (int i = 0; i < 4; ++i) {
        if (!(H[i][i] > 0.0) || !(H[i][i] < INFINITY)) return false;
        s[i] = 1.0 / sqrt(H[i][i]);
    }
    double Mx[4][4], Lc[4][4] = {};
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) Mx[i][j] = (i == j) ? 1.0 + lambda : H[i][j] * s[i] * s[j];
    for (int j = 0; j < 4; ++j) {
        double v = Mx[j][j];
        for (int k = 0; k < j; ++k) v -= Lc[j][k] * Lc[j][k];
        if (!(v > 0.0)) return false;
        Lc[j][j] = sqrt(v);
        for (int i = j + 1; i < 4; ++i) {
            double w = Mx[i][j];
            for (int k = 0; k < j; ++k) w -= Lc[i][k] * Lc[j][k];
            Lc[i][j] = w / Lc[j][j];
        }
    }
    double zz[4], u[4];
    for (int i = 0; i < 4; ++i) {
        double v = g[i] * s[i];
        for (int k = 0; k < i; ++k) v -= Lc[i][k] * zz[k];
        zz[i] = v / Lc[i][i];
    }
    for (int i = 3; i >= 0; --i) {
        double v = zz[i];
        for (int k = i + 1; k < 4; ++k) v -= Lc[k][i] * u[k];
        u[i] = v / Lc[i][i];
    }
    for (int i = 0; i < 4; ++i) d[i] = u[i] * s[i];
    return true;
}

// diag(H^-1) by Gauss-Jordan on the 4x4 matrix; false if singular
__device__ bool res_inv_diag(const double* Hu, double* dg)
{
    double A[4][8];
    int q = 0;
    for (int i = 0; i < 4; ++i)
        for (int j = i; j < 4; ++j) A[i][j] = A[j][i] = Hu[q++];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) A[i][4 + j] = (i == j) ? 1.0 : 0.0;
    for (int c = 0; c < 4; ++c) {
        int piv = c;
        for (int r = c + 1; r < 4; ++r)
            if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
        if (!(fabs(A[piv][c]) > 0.0)) return false;
        for (int j = 0; j < 8; ++j) {
            const double tmp = A[c][j];
            A[c][j] = A[piv][j];
            A[piv][j] = tmp;
        }
        const double ip = 1.0 / A[c][c];
        for (int j = 0; j < 8; ++j) A[c][j] *= ip;
        for (int r = 0; r < 4; ++r)
            if (r != c) {
                const double fct = A[r][c];
                for (int j = 0; j < 8; ++j) A[r][j] -= fct * A[c][j];
            }
    }
    for (int i = 0; i < 4; ++i) dg[i] = A[i][4 + i];
    return true;
}

__global__ void __launch_bounds__(kResThreads) resonance_fit_kernel(ResArgs a)
{
    __shared__ double red[kResThreads / 32][16];
    __shared__ ResSums tot;
    __shared__ double sp[4];        // parameters at which the sums are taken
    __shared__ int s_ctl;           // 0 continue, 1 stop
    const int t = threadIdx.x;
    const double* S = a.psd + a.k0;
    // sums over the band at sp -> tot (all threads take part)
    auto sums = [&]() {
        ResSums s;
#pragma unroll
        for (int i = 0; i < 16; ++i) s.v[i] = 0.0;
        const double p[4] = {sp[0], sp[1], sp[2], sp[3]};
        for (int i = t; i < a.np; i += kResThreads) res_point((a.k0 + i) * a.df, S[i], p, s);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            double v = s.v[i];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if ((t & 31) == 0) red[t >> 5][i] = v;
        }
        __syncthreads();
        if (t < 16) {
            double v = 0.0;
            for (int w = 0; w < kResThreads / 32; ++w) v += red[w][t];
            tot.v[t] = v;
        }
        __syncthreads();
    };
    // initial values (one thread, a pass over the band)
    if (t == 0) {
        int kp = 0;
        double B = S[0];
        for (int i = 1; i < a.np; ++i) {
            if (S[i] > S[kp]) kp = i;
            if (S[i] < B) B = S[i];
        }
        const double h = S[kp] - B, half = B + 0.5 * h;
        int lo = kp, hi = kp;
        while (lo > 0 && S[lo - 1] > half) --lo;
        while (hi < a.np - 1 && S[hi + 1] > half) ++hi;
        const double fl = (lo == 0) ? (a.k0 + lo) * a.df
                                    : (a.k0 + lo - 1) * a.df + (half - S[lo - 1]) / (S[lo] - S[lo - 1]) * a.df;
        const double fh = (hi == a.np - 1) ? (a.k0 + hi) * a.df
                                           : (a.k0 + hi) * a.df + (S[hi] - half) / (S[hi] - S[hi + 1]) * a.df;
        const double width = fmax(fh - fl, a.df);
        const double f0 = (a.k0 + kp) * a.df;
        const double Q = f0 / width;
        sp[0] = f0;
        sp[1] = Q;
        sp[2] = h / (Q * Q);
        sp[3] = B;
        s_ctl = 0;
    }
    __syncthreads();
    double p[4], chi2 = 0.0, lambda = a.lambda0, Hc[10], gc[4];
    int it = 0, st = 1;
    sums();
    if (t == 0) {
        for (int i = 0; i < 4; ++i) p[i] = sp[i];
        chi2 = (tot.v[15] > 0.0) ? INFINITY : tot.v[14];
        for (int i = 0; i < 10; ++i) Hc[i] = tot.v[i];
        for (int i = 0; i < 4; ++i) gc[i] = tot.v[10 + i];
        if (!(chi2 < INFINITY)) {
            st = 3;
            s_ctl = 1;
        }
    }
    __syncthreads();
    while (true) {
        // thread 0 proposes a trial point
        if (t == 0 && s_ctl == 0) {
            if (it >= a.max_iter) {
                s_ctl = 1;
            } else {
                ++it;
                double d[4];
                if (!res_solve(Hc, gc, lambda, d)) {
                    st = 2;
                    s_ctl = 1;
                } else {
                    for (int i = 0; i < 4; ++i) sp[i] = p[i] + d[i];
                }
            }
        }
        __syncthreads();
        if (s_ctl) break;
        sums();
        if (t == 0) {
            const double c2 = (tot.v[15] > 0.0) ? INFINITY : tot.v[14];
            if (!(c2 < INFINITY)) {
                lambda *= 10.0;
            } else if (fabs(c2 - chi2) <= a.tol * chi2) {
                if (c2 <= chi2) {
                    for (int i = 0; i < 4; ++i) p[i] = sp[i];
                    chi2 = c2;
                }
                st = 0;
                s_ctl = 1;
            } else if (c2 < chi2) {
                for (int i = 0; i < 4; ++i) p[i] = sp[i];
                chi2 = c2;
                for (int i = 0; i < 10; ++i) Hc[i] = tot.v[i];
                for (int i = 0; i < 4; ++i) gc[i] = tot.v[10 + i];
                lambda *= 0.1;
            } else {
                lambda *= 10.0;
            }
        }
        __syncthreads();
    }
    // standard errors from the sums at the result
    if (t == 0)
        for (int i = 0; i < 4; ++i) sp[i] = p[i];
    __syncthreads();
    sums();
    if (t == 0) {
        double dg[4] = {NAN, NAN, NAN, NAN};
        const bool inv = a.np > 4 && res_inv_diag(tot.v, dg);
        for (int i = 0; i < 4; ++i) {
            a.out[i] = p[i];
            a.out[4 + i] = inv ? sqrt(dg[i] * chi2 / (a.np - 4)) : NAN;
        }
        a.out[8] = chi2;
        a.out[9] = it;
        a.out[10] = st;
        a.out[11] = a.np;
    }
}

}  // namespace

}  // namespace cg

using namespace cg;

namespace {
cg_status psd_fail(cg_status st, const char* msg)
{
    cg::set_last_error(msg);
    return st;
}
cg_status psd_cuda_fail(cudaError_t e, const char* what)
{
    static thread_local char buf[256];
    std::snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
    cg::set_last_error(buf);
    return e == cudaErrorMemoryAllocation ? CG_ERR_NOMEM : CG_ERR_CUDA;
}
}  // namespace

cg_status cg_psd_create(int seg_len, cg_psd_t* out)
{
    if (!out) return psd_fail(CG_ERR_ARG, "out is NULL");
    *out = nullptr;
    const int L = seg_len / 2;
    void* fn = welch_ptr(L);
    if (seg_len % 2 != 0 || !fn) return psd_fail(CG_ERR_ARG, "seg_len must be 4096, 8192, 16384 or 32768");
    cg_psd_s* h = new cg_psd_s;
    cudaGetDevice(&h->device);
    h->L = L;
    const int M = seg_len;
    std::vector<float> w(M);
    double sw2 = 0.0;
    for (int n = 0; n < M; ++n) {
        const double v = 0.5 - 0.5 * std::cos(2.0 * M_PI * n / M);
        w[n] = static_cast<float>(v);
        sw2 += static_cast<double>(w[n]) * static_cast<double>(w[n]);   // the window the kernel applies
    }
    h->sum_w2 = sw2;
    std::vector<float2> tl(L), tm(L + 1);
    for (int m = 0; m < L; ++m) {
        const double ang = -2.0 * M_PI * m / L;
        tl[m] = make_float2(static_cast<float>(std::cos(ang)), static_cast<float>(std::sin(ang)));
    }
    for (int k = 0; k <= L; ++k) {
        const double ang = -2.0 * M_PI * k / M;
        tm[k] = make_float2(static_cast<float>(std::cos(ang)), static_cast<float>(std::sin(ang)));
    }
    int sms = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
    h->smem = sizeof(float2) * (static_cast<size_t>(L) + L / 16 + (L > 4096 ? 4096 : L) + 256);
    if (e == cudaSuccess) e = cg::raise_smem_limit(fn, h->smem);
    int occ = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, L / 16, h->smem);
    h->grid = sms * (occ > 0 ? occ : 1);
    if (e == cudaSuccess) e = cudaMalloc(&h->win, sizeof(float) * M);
    if (e == cudaSuccess) e = cudaMalloc(&h->twL, sizeof(float2) * L);
    if (e == cudaSuccess) e = cudaMalloc(&h->twM, sizeof(float2) * (L + 1));
    if (e == cudaSuccess) e = cudaMalloc(&h->part, sizeof(double) * (L + 1) * h->grid);
    if (e == cudaSuccess) e = cudaMemcpy(h->win, w.data(), sizeof(float) * M, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(h->twL, tl.data(), sizeof(float2) * L, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(h->twM, tm.data(), sizeof(float2) * (L + 1), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cg_psd_destroy(h);
        return psd_cuda_fail(e, "cg_psd_create");
    }
    *out = h;
    return CG_OK;
}

void cg_psd_destroy(cg_psd_t h)
{
    if (!h) return;
    cudaFree(h->win);
    cudaFree(h->twL);
    cudaFree(h->twM);
    cudaFree(h->part);
    delete h;
}

cg_status cg_psd_welch(cg_psd_t h, const float* x_dev, int64_t n, int64_t stride, double fs, double* psd_dev,
                       int64_t* n_segments, void* stream)
{
    if (!h || !x_dev || !psd_dev) return psd_fail(CG_ERR_ARG, "handle, x_dev and psd_dev are required");
    if (stride < 1) return psd_fail(CG_ERR_ARG, "stride must be >= 1");
    if (!(fs > 0.0) || !std::isfinite(fs)) return psd_fail(CG_ERR_ARG, "fs must be > 0");
    const int64_t M = 2LL * h->L;
    if (n < M) return psd_fail(CG_ERR_ARG, "series shorter than one segment");
    const int64_t K = (n - M) / h->L + 1;
    if (n_segments) *n_segments = K;
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    PsdArgs a{x_dev, stride, K, h->win, h->twL, h->twM, h->part};
    const int grid = static_cast<int>(K < h->grid ? K : h->grid);
    void* args[] = {&a};
    cudaError_t e = cudaLaunchKernel(welch_ptr(h->L), dim3(grid), dim3(h->L / 16), args, h->smem, s);
    if (e == cudaSuccess) {
        const double scale = 1.0 / (static_cast<double>(K) * fs * h->sum_w2);
        psd_reduce_kernel<<<(h->L + 1 + 255) / 256, 256, 0, s>>>(h->part, grid, h->L, scale, psd_dev);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return psd_cuda_fail(e, "cg_psd_welch");
    return CG_OK;
}

cg_status cg_resonance_fit(const double* psd_dev, int n_bins, double df, double f_lo, double f_hi, int max_iter,
                           double tol, double* out_dev, void* stream)
{
    if (!psd_dev || !out_dev) return psd_fail(CG_ERR_ARG, "psd_dev and out_dev are required");
    if (n_bins < 8 || !(df > 0.0) || !(f_hi > f_lo) || max_iter < 0 || !(tol >= 0.0))
        return psd_fail(CG_ERR_ARG, "need n_bins >= 8, df > 0, f_hi > f_lo, max_iter >= 0, tol >= 0");
    int k0 = static_cast<int>(std::ceil(f_lo / df));
    int k1 = static_cast<int>(std::floor(f_hi / df));
    if (k0 < 1) k0 = 1;                       // the model's f = 0 point carries no resonance information
    if (k1 > n_bins - 1) k1 = n_bins - 1;
    if (k1 - k0 + 1 < 8) return psd_fail(CG_ERR_ARG, "the band holds fewer than 8 bins");
    ResArgs a{psd_dev, k0, k1 - k0 + 1, df, max_iter, tol, 1e-3, out_dev};
    void* args[] = {&a};
    cudaError_t e = cudaLaunchKernel(reinterpret_cast<void*>(&resonance_fit_kernel), dim3(1), dim3(kResThreads),
                                     args, 0, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return psd_cuda_fail(e, "cg_resonance_fit");
    return CG_OK;
}
