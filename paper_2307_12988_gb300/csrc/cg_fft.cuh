// cg_fft.cuh -- shared-memory mixed-radix FFT pieces for the tooth readout.
//
// The paper transforms each 1 us row of samples with an FFT and reads the
// comb-tooth bins ("Data Capture and Processing"; Fig. 3 a->b).  Here a thread
// block transforms a batch of frames held in shared memory:
//   * a load stage turns the int16 samples of every frame into L complex
//     values: either the real-FFT packing z_n = x_{2n} + i x_{2n+1} (L = N/2),
//     or the coset fold z_n1 = W_N^{r n1} sum_{n2<M} x_{n1+L n2} W_M^{r n2}
//     (L = N/M), the first decimation-in-time stage of a radix-M transform
//     evaluated only at the output residue r mod M where the teeth are;
//   * Stockham autosort stages of radix 2,3,4,5,7,8,11,13 over L points;
//   * a readout stage evaluated only at the tooth bins (real-FFT split step, or
//     a direct read of the coset transform).
// Codelet constants are compile-time values of cos/sin(2 pi j / R) computed by
// a Taylor series in constexpr double arithmetic (below).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace cg {

// ---------------------------------------------------------------------------
// compile-time cos / sin of 2 pi j / R (Taylor series about 0 after reducing
// the angle to [-pi, pi]; 40 terms give full double accuracy there)
// ---------------------------------------------------------------------------
constexpr double kPiD = 3.14159265358979323846264338327950288;

constexpr double ce_cos_red(double x)
{
    double term = 1.0, sum = 1.0;
    for (int n = 1; n < 40; ++n) {
        term *= -x * x / (double)((2 * n - 1) * (2 * n));
        sum += term;
    }
    return sum;
}
constexpr double ce_sin_red(double x)
{
    double term = x, sum = x;
    for (int n = 1; n < 40; ++n) {
        term *= -x * x / (double)((2 * n) * (2 * n + 1));
        sum += term;
    }
    return sum;
}
// angle 2 pi j / R with j reduced into (-R/2, R/2]
constexpr double ce_angle(int j, int R)
{
    int jj = j % R;
    if (jj < 0) jj += R;
    if (2 * jj > R) jj -= R;
    return 2.0 * kPiD * (double)jj / (double)R;
}

template <int R>
struct RootTable {
    float c[R];
    float s[R];
    constexpr RootTable() : c(), s()
    {
        for (int j = 0; j < R; ++j) {
            c[j] = (float)ce_cos_red(ce_angle(j, R));
            s[j] = (float)ce_sin_red(ce_angle(j, R));
        }
    }
};

// ---------------------------------------------------------------------------
// complex helpers (float2 = re, im)
// ---------------------------------------------------------------------------
// (packed FP32x2 arithmetic: one instruction for both parts, each rounded as
// the scalar operation; a - b as fma(b, -1, a), rounded once like a - b)
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// multiply by -i
__device__ __forceinline__ float2 cmul_mi(float2 a) { return make_float2(a.y, -a.x); }
// |X| by the hardware's approximate square root (one instruction, within
// about an ulp: far inside the readout's 1e-5 of the reference), where
// sqrtf's correctly rounded sequence took most of the last stage's time
__device__ __forceinline__ float cabs_approx(float2 X)
{
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(fmaf(X.x, X.x, X.y * X.y)));
    return r;
}

// ---------------------------------------------------------------------------
// forward DFT codelets in registers: X[v] = sum_t a[t] exp(-2 pi i v t / R)
// ---------------------------------------------------------------------------
template <int R>
struct Dft;

template <>
struct Dft<2> {
    static __device__ __forceinline__ void run(float2 (&a)[2])
    {
        float2 t = a[1];
        a[1] = csub(a[0], t);
        a[0] = cadd(a[0], t);
    }
};

template <>
struct Dft<4> {
    static __device__ __forceinline__ void run(float2 (&a)[4])
    {
        float2 s02 = cadd(a[0], a[2]), d02 = csub(a[0], a[2]);
        float2 s13 = cadd(a[1], a[3]), d13 = cmul_mi(csub(a[1], a[3]));
        a[0] = cadd(s02, s13);
        a[2] = csub(s02, s13);
        a[1] = cadd(d02, d13);
        a[3] = csub(d02, d13);
    }
};

template <>
struct Dft<8> {
    static __device__ __forceinline__ void run(float2 (&a)[8])
    {
        float2 e[4] = {a[0], a[2], a[4], a[6]};
        float2 o[4] = {a[1], a[3], a[5], a[7]};
        Dft<4>::run(e);
        Dft<4>::run(o);
        constexpr float h = 0.70710678118654752440f;
        // W8^1 = (h, -h), W8^2 = -i, W8^3 = (-h, -h)
        float2 o1 = make_float2(h * (o[1].x + o[1].y), h * (o[1].y - o[1].x));
        float2 o2 = cmul_mi(o[2]);
        float2 o3 = make_float2(h * (o[3].y - o[3].x), -h * (o[3].x + o[3].y));
        a[0] = cadd(e[0], o[0]);
        a[4] = csub(e[0], o[0]);
        a[1] = cadd(e[1], o1);
        a[5] = csub(e[1], o1);
        a[2] = cadd(e[2], o2);
        a[6] = csub(e[2], o2);
        a[3] = cadd(e[3], o3);
        a[7] = csub(e[3], o3);
    }
};

// odd R: pair t with R-t.  With s_t = a_t + a_{R-t}, d_t = a_t - a_{R-t},
// P_v = a_0 + sum_t s_t cos(2 pi v t/R), Q_v = sum_t d_t sin(2 pi v t/R):
// X[v] = P_v - i Q_v and X[R-v] = P_v + i Q_v.
template <int R>
struct DftOdd {
    static __device__ __forceinline__ void run(float2 (&a)[R])
    {
        constexpr int H = (R - 1) / 2;
        constexpr RootTable<R> tab{};
        float2 s[H + 1], d[H + 1];
#pragma unroll
        for (int t = 1; t <= H; ++t) {
            s[t] = cadd(a[t], a[R - t]);
            d[t] = csub(a[t], a[R - t]);
        }
        float2 x0 = a[0];
#pragma unroll
        for (int t = 1; t <= H; ++t) x0 = cadd(x0, s[t]);
        float2 out[R];
        out[0] = x0;
#pragma unroll
        for (int v = 1; v <= H; ++v) {
            float2 P = a[0];
            float2 Q = make_float2(0.f, 0.f);
#pragma unroll
            for (int t = 1; t <= H; ++t) {
                const float c = tab.c[(v * t) % R];
                const float sn = tab.s[(v * t) % R];
                P = __ffma2_rn(s[t], make_float2(c, c), P);
                Q = __ffma2_rn(d[t], make_float2(sn, sn), Q);
            }
            out[v] = make_float2(P.x + Q.y, P.y - Q.x);
            out[R - v] = make_float2(P.x - Q.y, P.y + Q.x);
        }
#pragma unroll
        for (int t = 0; t < R; ++t) a[t] = out[t];
    }
};
template <> struct Dft<3> : DftOdd<3> {};
template <> struct Dft<5> : DftOdd<5> {};
template <> struct Dft<7> : DftOdd<7> {};
template <> struct Dft<11> : DftOdd<11> {};
template <> struct Dft<13> : DftOdd<13> {};

// composite R = R1 * R2 in registers (decimation in time, n = R2 n1 + n2,
// k = k1 + R1 k2):  X[k1 + R1 k2] =
//   sum_{n2} W_R2^{n2 k2} W_R^{n2 k1} sum_{n1} a[R2 n1 + n2] W_R1^{n1 k1}
template <int R1, int R2>
struct DftComposite {
    static constexpr int R = R1 * R2;
    static __device__ __forceinline__ void run(float2 (&a)[R])
    {
        constexpr RootTable<R> tab{};
        float2 B[R2][R1];
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2) {
            float2 v[R1];
#pragma unroll
            for (int n1 = 0; n1 < R1; ++n1) v[n1] = a[R2 * n1 + n2];
            Dft<R1>::run(v);
#pragma unroll
            for (int k1 = 0; k1 < R1; ++k1) {
                const int e = (n2 * k1) % R;
                if (e == 0) {
                    B[n2][k1] = v[k1];
                } else {
                    // W_R^e = cos(2 pi e/R) - i sin(2 pi e/R)
                    const float c = tab.c[e], s = tab.s[e];
                    B[n2][k1] = make_float2(fmaf(v[k1].x, c, v[k1].y * s), fmaf(v[k1].y, c, -v[k1].x * s));
                }
            }
        }
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) {
            float2 w[R2];
#pragma unroll
            for (int n2 = 0; n2 < R2; ++n2) w[n2] = B[n2][k1];
            Dft<R2>::run(w);
#pragma unroll
            for (int k2 = 0; k2 < R2; ++k2) a[k1 + R1 * k2] = w[k2];
        }
    }
};
template <> struct Dft<6> : DftComposite<2, 3> {};
template <> struct Dft<10> : DftComposite<2, 5> {};
template <> struct Dft<12> : DftComposite<4, 3> {};
template <> struct Dft<16> : DftComposite<4, 4> {};
template <> struct Dft<20> : DftComposite<4, 5> {};
template <> struct Dft<22> : DftComposite<2, 11> {};
template <> struct Dft<25> : DftComposite<5, 5> {};

// ---------------------------------------------------------------------------
// One Stockham stage of radix R over F frames in shared memory.
//   Ns = product of the radices of the earlier stages.
//   butterfly j < L/R of a frame: a[r] = in[j + r L/R] * W_{Ns R}^{r (j mod Ns)},
//   R-point DFT, out[(j / Ns) Ns R + (j mod Ns) + r Ns] = a[r].
// twL[m] = W_L^m; W_{Ns R}^{r k} = twL[r k L / (Ns R)].
// ---------------------------------------------------------------------------
template <int R>
__device__ __forceinline__ void stockham_stage(const float2* __restrict__ in, float2* __restrict__ out,
                                               int L, int Ns, int nf, int fstride,
                                               const float2* __restrict__ twL)
{
    const int per = L / R;
    const int total = nf * per;
    const int twstep = L / (Ns * R);
    for (int item = threadIdx.x; item < total; item += blockDim.x) {
        const int f = item / per;
        const int j = item - f * per;
        const float2* src = in + f * fstride;
        float2* dst = out + f * fstride;
        const int k = j % Ns;
        float2 a[R];
#pragma unroll
        for (int r = 0; r < R; ++r) a[r] = src[j + r * per];
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) a[r] = cmul(a[r], twL[r * k * twstep]);
        }
        Dft<R>::run(a);
        const int idx = (j - k) * R + k;   // (j / Ns) * Ns * R + k
#pragma unroll
        for (int r = 0; r < R; ++r) dst[idx + r * Ns] = a[r];
    }
}

__device__ __forceinline__ void stockham_dispatch(int R, const float2* in, float2* out, int L, int Ns,
                                                  int nf, int fstride, const float2* twL)
{
    switch (R) {
    case 2: stockham_stage<2>(in, out, L, Ns, nf, fstride, twL); break;
    case 3: stockham_stage<3>(in, out, L, Ns, nf, fstride, twL); break;
    case 4: stockham_stage<4>(in, out, L, Ns, nf, fstride, twL); break;
    case 5: stockham_stage<5>(in, out, L, Ns, nf, fstride, twL); break;
    case 7: stockham_stage<7>(in, out, L, Ns, nf, fstride, twL); break;
    case 8: stockham_stage<8>(in, out, L, Ns, nf, fstride, twL); break;
    case 11: stockham_stage<11>(in, out, L, Ns, nf, fstride, twL); break;
    case 13: stockham_stage<13>(in, out, L, Ns, nf, fstride, twL); break;
    default: break;
    }
}

}  // namespace cg
