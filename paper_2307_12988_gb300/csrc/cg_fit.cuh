// cg_fit.cuh -- initial guess and Levenberg-Marquardt fit of one normalised
// comb spectrum per group of G lanes (G = 32: one warp per frame).
//
// Paper ("Data Capture and Processing", fit paragraphs): every normalised
// optical spectrum is fit by Levenberg-Marquardt, at most 20 iterations,
// tolerance 1e-6; the initial value sets the iteration count (~4 typical).
// Model (this library): m(u) = B + A g^2 / ((u-c)^2 + g^2), fit on the
// normalised abscissa u = (x - x_mid) / x_scale.
//
// Per point, with d = u - c, q = 1 / (d^2 + g^2), L = g^2 q:
//   dm/dA = L, dm/dB = 1, dm/dc = 2A L d q, dm/dg = 2A L d^2 q / g,
// so with jc = L q d and jg = jc d the Jacobian columns are
//   (2A) jc, (2A/g) jg, L, 1
// and J^T J, J^T r need only 14 running sums, reduced over the group with
// shuffles.  Marquardt step: (H + lambda diag H) delta = J^T r, solved by a
// Cholesky factorisation of the Jacobi-scaled matrix S H S + lambda I.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace cg {

constexpr unsigned kFull = 0xffffffffu;

struct FitArgs {
    int64_t n;              // frames
    int T;                  // teeth
    const float* u;         // [T] normalised abscissa (global)
    const float* inv_ref;   // [T] 1 / reference (global)
    const int* outer_idx;   // [n_outer] teeth of the outer fifth
    int n_outer;
    float u_mid, du, span;  // normalised midpoint, spacing, span
    float x_mid, x_scale;   // x = x_mid + x_scale * u
    int max_iter;
    float tol, lambda0;
    const float* y;         // standalone fit: [n][T] normalised spectra, or null
    const float* amps_in;   // standalone fit when y is null: [n][T] magnitudes
    const float* p0;        // [n][4] user units, or null (moment init)
    float* params;          // [n][4]
    float* rss;             // [n] or null
    int16_t* iters;         // [n] or null
    int16_t* status;        // [n] or null
};

enum { kConverged = 0, kMaxIter = 1, kSingular = 2, kNonfinite = 3, kInitFlat = 0x10 };

template <int G>
__device__ __forceinline__ float gsum(float v)
{
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}
template <int G>
__device__ __forceinline__ float gmax(float v)
{
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(kFull, v, o));
    return v;
}

// 14 sums: LL, Ljc, Ljg, L, jcjc, jcjg, jc, jgjg, jg, Lr, jcr, jgr, r, rr
struct LmSums {
    float v[14];
};

// Transpose-style reduction of the 14 sums (padded to 16) over G lanes.  At
// split level l (xor offset G/2^(l+1)) every lane keeps one half of its
// current values and adds the partner's copy of that half, so the widths go
// 16 -> 8 -> 4 -> 2 -> 1 and each level moves half as many values as the
// last; offsets left over once one value per lane remains are plain
// butterflies.  A final gather gives every lane of the group all 14 sums.
constexpr int red_levels(int G) { return G >= 16 ? 4 : (G == 8 ? 3 : (G == 4 ? 2 : (G == 2 ? 1 : 0))); }
constexpr int red_owner(int idx, int G)
{
    int w = 16, lo = 0, bits = 0;
    for (int o = G / 2; o > 0 && w > 1; o >>= 1) {
        const int h = w / 2;
        if (idx >= lo + h) { bits |= o; lo += h; }
        w = h;
    }
    return bits;
}
constexpr int red_slot(int idx, int G)
{
    int w = 16, lo = 0;
    for (int o = G / 2; o > 0 && w > 1; o >>= 1) {
        const int h = w / 2;
        if (idx >= lo + h) lo += h;
        w = h;
    }
    return idx - lo;
}

template <int G>
__device__ __forceinline__ void reduce_sums(LmSums& S)
{
    constexpr int kLev = red_levels(G);
    float a[16];
#pragma unroll
    for (int i = 0; i < 14; ++i) a[i] = S.v[i];
    a[14] = 0.f;
    a[15] = 0.f;
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int l = 0; l < kLev; ++l) {
        const int o = G >> (l + 1);
        const int half = 8 >> l;
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const float send = upper ? a[i] : a[i + half];
            const float keep = upper ? a[i + half] : a[i];
            a[i] = keep + __shfl_xor_sync(kFull, send, o);
        }
    }
    constexpr int kWidth = 16 >> kLev;
#pragma unroll
    for (int o = G >> (kLev + 1); o > 0; o >>= 1) {
#pragma unroll
        for (int i = 0; i < kWidth; ++i) a[i] += __shfl_xor_sync(kFull, a[i], o);
    }
    const int gbase = lane & ~(G - 1);
#pragma unroll
    for (int idx = 0; idx < 14; ++idx)
        S.v[idx] = __shfl_sync(kFull, a[red_slot(idx, G)], gbase + red_owner(idx, G));
}

__device__ __forceinline__ float rcp_fast(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void accum_point(float u, float y, float c, float g2, float A, float B,
                                            LmSums& S)
{
    const float d = u - c;
    const float D = fmaf(d, d, g2);
    const float q = rcp_fast(D);
    const float L = g2 * q;
    // (y - B) is exact while y and B agree within a factor of two (Sterbenz),
    // so the residual carries one rounding instead of two
    const float r = fmaf(-A, L, y - B);
    const float t = L * q;
    const float jc = t * d;
    const float jg = jc * d;
    S.v[0] = fmaf(L, L, S.v[0]);
    S.v[1] = fmaf(L, jc, S.v[1]);
    S.v[2] = fmaf(L, jg, S.v[2]);
    S.v[3] += L;
    S.v[4] = fmaf(jc, jc, S.v[4]);
    S.v[5] = fmaf(jc, jg, S.v[5]);
    S.v[6] += jc;
    S.v[7] = fmaf(jg, jg, S.v[7]);
    S.v[8] += jg;
    S.v[9] = fmaf(L, r, S.v[9]);
    S.v[10] = fmaf(jc, r, S.v[10]);
    S.v[11] = fmaf(jg, r, S.v[11]);
    S.v[12] += r;
    S.v[13] = fmaf(r, r, S.v[13]);
}

// Normal equations in the order (c, g, A, B) from the sums at (g, A).
struct Normal {
    float H[10];   // cc cg cA cB gg gA gB AA AB BB
    float b[4];
};

__device__ __forceinline__ void make_normal(const LmSums& S, float g, float A, int T, Normal& N)
{
    const float ac = 2.0f * A;
    const float ag = 2.0f * A / g;
    N.H[0] = ac * ac * S.v[4];
    N.H[1] = ac * ag * S.v[5];
    N.H[2] = ac * S.v[1];
    N.H[3] = ac * S.v[6];
    N.H[4] = ag * ag * S.v[7];
    N.H[5] = ag * S.v[2];
    N.H[6] = ag * S.v[8];
    N.H[7] = S.v[0];
    N.H[8] = S.v[3];
    N.H[9] = (float)T;
    N.b[0] = ac * S.v[10];
    N.b[1] = ag * S.v[11];
    N.b[2] = S.v[9];
    N.b[3] = S.v[12];
}

// Solve (H + lambda diag H) delta = b; false when not positive definite.
__device__ __forceinline__ bool lm_solve4(const Normal& N, float lambda, float (&delta)[4])
{
    const float dH[4] = {N.H[0], N.H[4], N.H[7], N.H[9]};
    float s[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if (!(dH[i] > 0.0f) || !(dH[i] < INFINITY)) return false;
        s[i] = rsqrtf(dH[i]);
    }
    // scaled symmetric matrix M = S H S + lambda I (diagonal 1 + lambda)
    const float dg = 1.0f + lambda;
    float m10 = N.H[1] * s[1] * s[0];
    float m20 = N.H[2] * s[2] * s[0], m21 = N.H[5] * s[2] * s[1];
    float m30 = N.H[3] * s[3] * s[0], m31 = N.H[6] * s[3] * s[1], m32 = N.H[8] * s[3] * s[2];
    // Cholesky M = L L^T
    float l00 = dg;
    if (!(l00 > 0.f)) return false;
    l00 = sqrtf(l00);
    const float i00 = 1.0f / l00;
    const float l10 = m10 * i00, l20 = m20 * i00, l30 = m30 * i00;
    float l11 = dg - l10 * l10;
    if (!(l11 > 0.f)) return false;
    l11 = sqrtf(l11);
    const float i11 = 1.0f / l11;
    const float l21 = (m21 - l20 * l10) * i11;
    const float l31 = (m31 - l30 * l10) * i11;
    float l22 = dg - l20 * l20 - l21 * l21;
    if (!(l22 > 0.f)) return false;
    l22 = sqrtf(l22);
    const float i22 = 1.0f / l22;
    const float l32 = (m32 - l30 * l20 - l31 * l21) * i22;
    float l33 = dg - l30 * l30 - l31 * l31 - l32 * l32;
    if (!(l33 > 0.f)) return false;
    l33 = sqrtf(l33);
    const float i33 = 1.0f / l33;
    const float b0 = N.b[0] * s[0], b1 = N.b[1] * s[1], b2 = N.b[2] * s[2], b3 = N.b[3] * s[3];
    const float z0 = b0 * i00;
    const float z1 = (b1 - l10 * z0) * i11;
    const float z2 = (b2 - l20 * z0 - l21 * z1) * i22;
    const float z3 = (b3 - l30 * z0 - l31 * z1 - l32 * z2) * i33;
    const float u3 = z3 * i33;
    const float u2 = (z2 - l32 * u3) * i22;
    const float u1 = (z1 - l21 * u2 - l31 * u3) * i11;
    const float u0 = (z0 - l10 * u1 - l20 * u2 - l30 * u3) * i00;
    delta[0] = u0 * s[0];
    delta[1] = u1 * s[1];
    delta[2] = u2 * s[2];
    delta[3] = u3 * s[3];
    return true;
}

// --- throughput variants: approximate reciprocal / reciprocal square root ---
// (the step only has to point downhill; the fixed point is set by the sums)
__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void make_normal_fast(const LmSums& S, float g, float A, int T, Normal& N)
{
    const float ac = 2.0f * A;
    const float ag = ac * rcp_approx(g);
    N.H[0] = ac * ac * S.v[4];
    N.H[1] = ac * ag * S.v[5];
    N.H[2] = ac * S.v[1];
    N.H[3] = ac * S.v[6];
    N.H[4] = ag * ag * S.v[7];
    N.H[5] = ag * S.v[2];
    N.H[6] = ag * S.v[8];
    N.H[7] = S.v[0];
    N.H[8] = S.v[3];
    N.H[9] = static_cast<float>(T);
    N.b[0] = ac * S.v[10];
    N.b[1] = ag * S.v[11];
    N.b[2] = S.v[9];
    N.b[3] = S.v[12];
}

// ---------------------------------------------------------------------------
// The paper's Fano lineshape (c free; A, B boxed; q, gamma fixed):
//   e = (u - c) / gamma, F = (q + e)^2 / (1 + e^2), m = B + A F
//   dm/dc = -A F'(e) / gamma, F'(e) = 2 (q + e)(1 - q e) / (1 + e^2)^2,
//   dm/dA = F, dm/dB = 1.
// Sums: v0 jc jc, v1 jc F, v2 jc, v3 F F, v4 F, v5 jc r, v6 F r, v7 r,
// v13 r r (the 1.1 entry is the point count).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void accum_point_fano(float u, float y, float c, float inv_g, float q, float A, float B,
                                                 LmSums& S)
{
    const float e = (u - c) * inv_g;
    const float id = rcp_fast(fmaf(e, e, 1.0f));
    const float qe = q + e;
    const float F = qe * qe * id;
    const float r = fmaf(-A, F, y - B);
    const float jc = -2.0f * A * inv_g * qe * fmaf(-q, e, 1.0f) * id * id;
    S.v[0] = fmaf(jc, jc, S.v[0]);
    S.v[1] = fmaf(jc, F, S.v[1]);
    S.v[2] += jc;
    S.v[3] = fmaf(F, F, S.v[3]);
    S.v[4] += F;
    S.v[5] = fmaf(jc, r, S.v[5]);
    S.v[6] = fmaf(F, r, S.v[6]);
    S.v[7] += r;
    S.v[13] = fmaf(r, r, S.v[13]);
}

// Normal equations of (c, A, B) in H[0..5] = cc cA cB AA AB BB, b[0..2].
__device__ __forceinline__ void make_normal_fano(const LmSums& S, int T, Normal& N)
{
    N.H[0] = S.v[0];
    N.H[1] = S.v[1];
    N.H[2] = S.v[2];
    N.H[3] = S.v[3];
    N.H[4] = S.v[4];
    N.H[5] = static_cast<float>(T);
    N.b[0] = S.v[5];
    N.b[1] = S.v[6];
    N.b[2] = S.v[7];
}

// (H + lambda diag H) delta = b for the 3 Fano parameters: Jacobi-scaled
// Cholesky in R (float or double); false when not positive definite.  Bit 1
// (A) or 2 (B) of held keeps that parameter's delta at zero and decouples it
// from the others (the reduced system of an active bound).
template <class R>
__device__ __forceinline__ bool lm_solve3(const Normal& N, float lambda, int held, float (&delta)[3])
{
    const R h00 = N.H[0], h01 = N.H[1], h02 = N.H[2], h11 = N.H[3], h12 = N.H[4], h22 = N.H[5];
    if (!(h00 > R(0)) || !(h11 > R(0)) || !(h22 > R(0)) || !(h00 < R(INFINITY)) || !(h11 < R(INFINITY)))
        return false;
    const R s0 = R(1) / sqrt(h00), s1 = R(1) / sqrt(h11), s2 = R(1) / sqrt(h22);
    const R dg = R(1) + R(lambda);
    const bool hA = (held & 2) != 0, hB = (held & 4) != 0;
    const R m10 = hA ? R(0) : h01 * s1 * s0, m20 = hB ? R(0) : h02 * s2 * s0;
    const R m21 = (hA || hB) ? R(0) : h12 * s2 * s1;
    const R l00 = sqrt(dg);
    const R l10 = m10 / l00, l20 = m20 / l00;
    const R v11 = dg - l10 * l10;
    if (!(v11 > R(0))) return false;
    const R l11 = sqrt(v11);
    const R l21 = (m21 - l20 * l10) / l11;
    const R v22 = dg - l20 * l20 - l21 * l21;
    if (!(v22 > R(0))) return false;
    const R l22 = sqrt(v22);
    const R z0 = R(N.b[0]) * s0 / l00;
    const R z1 = ((hA ? R(0) : R(N.b[1]) * s1) - l10 * z0) / l11;
    const R z2 = ((hB ? R(0) : R(N.b[2]) * s2) - l20 * z0 - l21 * z1) / l22;
    const R u2 = z2 / l22;
    const R u1 = (z1 - l21 * u2) / l11;
    const R u0 = (z0 - l10 * u1 - l20 * u2) / l00;
    delta[0] = static_cast<float>(u0 * s0);
    delta[1] = static_cast<float>(u1 * s1);
    delta[2] = static_cast<float>(u2 * s2);
    return true;
}

// Cholesky of S H S + lambda I keeping only the inverse pivots (rsqrt).
__device__ __forceinline__ bool lm_solve4_fast(const Normal& N, float lambda, float (&delta)[4])
{
    const float dH[4] = {N.H[0], N.H[4], N.H[7], N.H[9]};
    float s[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if (!(dH[i] > 0.0f) || !(dH[i] < INFINITY)) return false;
        s[i] = rsqrtf(dH[i]);
    }
    const float dg = 1.0f + lambda;
    const float m10 = N.H[1] * s[1] * s[0];
    const float m20 = N.H[2] * s[2] * s[0], m21 = N.H[5] * s[2] * s[1];
    const float m30 = N.H[3] * s[3] * s[0], m31 = N.H[6] * s[3] * s[1], m32 = N.H[8] * s[3] * s[2];
    const float i00 = rsqrtf(dg);
    const float l10 = m10 * i00, l20 = m20 * i00, l30 = m30 * i00;
    const float v11 = fmaf(-l10, l10, dg);
    if (!(v11 > 0.f)) return false;
    const float i11 = rsqrtf(v11);
    const float l21 = fmaf(-l20, l10, m21) * i11;
    const float l31 = fmaf(-l30, l10, m31) * i11;
    const float v22 = fmaf(-l21, l21, fmaf(-l20, l20, dg));
    if (!(v22 > 0.f)) return false;
    const float i22 = rsqrtf(v22);
    const float l32 = fmaf(-l31, l21, fmaf(-l30, l20, m32)) * i22;
    const float v33 = fmaf(-l32, l32, fmaf(-l31, l31, fmaf(-l30, l30, dg)));
    if (!(v33 > 0.f)) return false;
    const float i33 = rsqrtf(v33);
    const float z0 = N.b[0] * s[0] * i00;
    const float z1 = fmaf(-l10, z0, N.b[1] * s[1]) * i11;
    const float z2 = fmaf(-l21, z1, fmaf(-l20, z0, N.b[2] * s[2])) * i22;
    const float z3 = fmaf(-l32, z2, fmaf(-l31, z1, fmaf(-l30, z0, N.b[3] * s[3]))) * i33;
    const float u3 = z3 * i33;
    const float u2 = fmaf(-l32, u3, z2) * i22;
    const float u1 = fmaf(-l31, u3, fmaf(-l21, u2, z1)) * i11;
    const float u0 = fmaf(-l30, u3, fmaf(-l20, u2, fmaf(-l10, u1, z0))) * i00;
    delta[0] = u0 * s[0];
    delta[1] = u1 * s[1];
    delta[2] = u2 * s[2];
    delta[3] = u3 * s[3];
    return true;
}

// 1/sqrt(v) in FP64 without division or square root (both are long software
// sequences at this part's FP64 rate): an FP32 seed (~23 correct bits)
// refined by one step of Newton's iteration r <- r (3 - v r^2) / 2, which
// doubles the correct bits to ~46 -- far beyond the FP32 step it produces.
__device__ __forceinline__ double rsqrt_f64(double v)
{
    const double r = static_cast<double>(rsqrtf(static_cast<float>(v)));
    return r * fma(-0.5 * v, r * r, 1.5);
}

// The same solve in FP64 (form with the split-precision tensor-core readout:
// the normal equations are formed in FP32, only the 4x4 solve is double).
// Only inverse pivots are needed, so the factorisation uses rsqrt_f64 alone.
__device__ __forceinline__ bool lm_solve4_f64(const Normal& N, float lambda, float (&delta)[4])
{
    const double h00 = N.H[0], h11 = N.H[4], h22 = N.H[7], h33 = N.H[9];
    if (!(h00 > 0.0) || !(h11 > 0.0) || !(h22 > 0.0) || !(h33 > 0.0)) return false;
    if (!(h00 < INFINITY) || !(h11 < INFINITY) || !(h22 < INFINITY) || !(h33 < INFINITY)) return false;
    const double s0 = rsqrt_f64(h00), s1 = rsqrt_f64(h11), s2 = rsqrt_f64(h22), s3 = rsqrt_f64(h33);
    const double dg = 1.0 + static_cast<double>(lambda);
    const double m10 = N.H[1] * s1 * s0;
    const double m20 = N.H[2] * s2 * s0, m21 = N.H[5] * s2 * s1;
    const double m30 = N.H[3] * s3 * s0, m31 = N.H[6] * s3 * s1, m32 = N.H[8] * s3 * s2;
    const double i00 = rsqrt_f64(dg);
    const double l10 = m10 * i00, l20 = m20 * i00, l30 = m30 * i00;
    const double v11 = fma(-l10, l10, dg);
    if (!(v11 > 0.0)) return false;
    const double i11 = rsqrt_f64(v11);
    const double l21 = fma(-l20, l10, m21) * i11, l31 = fma(-l30, l10, m31) * i11;
    const double v22 = fma(-l21, l21, fma(-l20, l20, dg));
    if (!(v22 > 0.0)) return false;
    const double i22 = rsqrt_f64(v22);
    const double l32 = fma(-l31, l21, fma(-l30, l20, m32)) * i22;
    const double v33 = fma(-l32, l32, fma(-l31, l31, fma(-l30, l30, dg)));
    if (!(v33 > 0.0)) return false;
    const double i33 = rsqrt_f64(v33);
    const double z0 = N.b[0] * s0 * i00;
    const double z1 = fma(-l10, z0, N.b[1] * s1) * i11;
    const double z2 = fma(-l21, z1, fma(-l20, z0, N.b[2] * s2)) * i22;
    const double z3 = fma(-l32, z2, fma(-l31, z1, fma(-l30, z0, N.b[3] * s3))) * i33;
    const double u3 = z3 * i33;
    const double u2 = fma(-l32, u3, z2) * i22;
    const double u1 = fma(-l31, u3, fma(-l21, u2, z1)) * i11;
    const double u0 = fma(-l30, u3, fma(-l20, u2, fma(-l10, u1, z0))) * i00;
    delta[0] = static_cast<float>(u0 * s0);
    delta[1] = static_cast<float>(u1 * s1);
    delta[2] = static_cast<float>(u2 * s2);
    delta[3] = static_cast<float>(u3 * s3);
    return true;
}

// Convergence test of the FP32 kernels.  chi^2 is evaluated in FP32: every
// residual carries a rounding error of about eps (|y| + |m|), so chi^2 itself
// is known only to about 2 eps Y sqrt(chi^2), Y ~ 2 (|A| + |B|) bounding
// |y| + |m|.  A trial whose change lies within three standard deviations of
// the difference of two such evaluations cannot be told from no change and
// counts as converged, as does a change within tol * chi^2 (the FP64 oracle
// needs only the latter).
__device__ __forceinline__ bool chi2_settled(float chi2_new, float chi2_old, float tol, float A, float B)
{
    const float Y = 2.0f * (fabsf(A) + fabsf(B));
    const float noise = 8.5f * 5.9604645e-8f * Y * sqrtf(chi2_old);
    return fabsf(chi2_new - chi2_old) <= fmaxf(tol * chi2_old, noise);
}

// Moment initial guess on the normalised abscissa (see the oracle for the
// reading): baseline = median of the outer fifth, centroid of the one-signed
// excess, amplitude = its extreme, width from area / (pi |A|).
template <int G>
__device__ __forceinline__ void moment_init(const float* ys, const float* us, const FitArgs& a,
                                            float (&p)[4], int& flag)
{
    const int gl = threadIdx.x & (G - 1);
    const int T = a.T;
    const int no = a.n_outer;
    // median of y over the outer set by rank counting (ties broken by index)
    const int rlo = (no - 1) >> 1, rhi = no >> 1;
    float vlo = 0.f, vhi = 0.f;
    for (int j = gl; j < no; j += G) {
        const float vj = ys[a.outer_idx[j]];
        int rank = 0;
        for (int i = 0; i < no; ++i) {
            const float vi = ys[a.outer_idx[i]];
            rank += (vi < vj) || (vi == vj && i < j);
        }
        if (rank == rlo) vlo += vj;
        if (rank == rhi) vhi += vj;
    }
    vlo = gsum<G>(vlo);
    vhi = gsum<G>(vhi);
    const float B0 = 0.5f * (vlo + vhi);
    // extreme deviation (first index on ties)
    float best = -1.f;
    int bestk = 0x7fffffff;
    for (int k = gl; k < T; k += G) {
        const float v = fabsf(ys[k] - B0);
        if (v > best) { best = v; bestk = k; }
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        const float ob = __shfl_xor_sync(kFull, best, o);
        const int ok = __shfl_xor_sync(kFull, bestk, o);
        if (ob > best || (ob == best && ok < bestk)) { best = ob; bestk = ok; }
    }
    float sgn = 1.0f;
    if (bestk >= 0 && bestk < T) sgn = (ys[bestk] - B0) >= 0.f ? 1.0f : -1.0f;
    float W = 0.f, Wu = 0.f, wmax = 0.f;
    for (int k = gl; k < T; k += G) {
        const float w = fmaxf(sgn * (ys[k] - B0), 0.f);
        W += w;
        Wu = fmaf(w, us[k], Wu);
        wmax = fmaxf(wmax, w);
    }
    W = gsum<G>(W);
    Wu = gsum<G>(Wu);
    wmax = gmax<G>(wmax);
    flag = 0;
    if (!(W > 0.f)) {
        p[0] = a.u_mid;
        p[1] = 0.5f * a.du;
        p[2] = 0.f;
        p[3] = B0;
        flag = kInitFlat;
        return;
    }
    const float A0 = sgn * wmax;
    float g0 = W * a.du / (3.14159265358979f * fabsf(A0));
    g0 = fminf(fmaxf(g0, 0.5f * a.du), 0.5f * a.span);
    p[0] = Wu / W;
    p[1] = g0;
    p[2] = A0;
    p[3] = B0;
}

// Full LM for the frame whose normalised spectrum is ys[0..T) (shared memory),
// executed by all G lanes of a group; every lane of the warp must call it
// (frames beyond n pass valid = false).  Results written by group lane 0.
template <int G>
__device__ __forceinline__ void fit_group(const float* ys, const float* us, const FitArgs& a,
                                          int64_t frame, bool valid)
{
    const int gl = threadIdx.x & (G - 1);
    const int T = a.T;
    float p[4];
    int flag = 0;
    if (a.p0 != nullptr) {
        float q[4] = {0.f, 1.f, 0.f, 0.f};
        if (valid) {
#pragma unroll
            for (int i = 0; i < 4; ++i) q[i] = a.p0[frame * 4 + i];
        }
        p[0] = (q[0] - a.x_mid) / a.x_scale;
        p[1] = q[1] / a.x_scale;
        p[2] = q[2];
        p[3] = q[3];
    } else {
        moment_init<G>(ys, us, a, p, flag);
    }

    LmSums S;
    Normal Nm;
    float lambda = a.lambda0;
    {
#pragma unroll
        for (int i = 0; i < 14; ++i) S.v[i] = 0.f;
        const float g2 = p[1] * p[1];
        for (int k = gl; k < T; k += G) accum_point(us[k], ys[k], p[0], g2, p[2], p[3], S);
        reduce_sums<G>(S);
        make_normal(S, p[1], p[2], T, Nm);
    }
    float chi2 = S.v[13];
    int status = kMaxIter;
    bool active = valid;
    if (!(chi2 < INFINITY)) {   // NaN or Inf
        status = kNonfinite;
        active = false;
    }
    if (a.max_iter <= 0) active = false;
    int it = 0;
    while (__any_sync(kFull, active)) {
        float delta[4] = {0.f, 0.f, 0.f, 0.f};
        const bool ok = lm_solve4(Nm, lambda, delta);
        if (active && !ok) {
            status = kSingular;
            active = false;
        }
        float pt[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) pt[i] = p[i] + delta[i];
        LmSums St;
#pragma unroll
        for (int i = 0; i < 14; ++i) St.v[i] = 0.f;
        const float g2 = pt[1] * pt[1];
        for (int k = gl; k < T; k += G) accum_point(us[k], ys[k], pt[0], g2, pt[2], pt[3], St);
        reduce_sums<G>(St);
        if (active) {
            ++it;
            const float chi2t = St.v[13];
            if (!(chi2t < INFINITY)) {
                lambda *= 10.0f;
            } else if (chi2_settled(chi2t, chi2, a.tol, p[2], p[3])) {
                if (chi2t <= chi2) {
#pragma unroll
                    for (int i = 0; i < 4; ++i) p[i] = pt[i];
                    chi2 = chi2t;
                }
                status = kConverged;
                active = false;
            } else if (chi2t < chi2) {
#pragma unroll
                for (int i = 0; i < 4; ++i) p[i] = pt[i];
                chi2 = chi2t;
                make_normal(St, pt[1], pt[2], T, Nm);
                lambda *= 0.1f;
            } else {
                lambda *= 10.0f;
            }
            if (active && it >= a.max_iter) active = false;
        }
    }
    if (valid && gl == 0) {
        float* po = a.params + frame * 4;
        po[0] = fmaf(a.x_scale, p[0], a.x_mid);
        po[1] = a.x_scale * fabsf(p[1]);
        po[2] = p[2];
        po[3] = p[3];
        if (a.rss) a.rss[frame] = chi2;
        if (a.iters) a.iters[frame] = (int16_t)it;
        if (a.status) a.status[frame] = (int16_t)(status | flag);
    }
}

}  // namespace cg
