/*
 * cg_oracle.c -- plain FP64 CPU oracle for the comb-spectrum readout and fit.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library path may call this file;
 * only the tests, the smoke check and the bench's CPU-baseline leg use it.
 * It shares no code, header, table or constant generator with the CUDA path.
 *
 * What it computes (arXiv 2307.12988, "Data Capture and Processing"):
 *   1. each digitised sample is taken as a real number (the paper casts the
 *      integer samples to floating point before any arithmetic);
 *   2. each frame of N consecutive samples is Fourier transformed; the method
 *      only ever reads the transform at the comb-tooth bins, so the oracle
 *      evaluates the DFT definition X_b = sum_n x_n exp(-2 pi i b n / N) by
 *      direct summation at exactly those bins (no FFT);
 *   3. the tooth magnitudes |X_b| are divided by a reference spectrum
 *      (the averaged cavity-free spectrum recorded at the start of a run);
 *   4. each normalised spectrum is fit by Levenberg-Marquardt (paper:
 *      "Data Capture and Processing", fit paragraph: at most 20 iterations,
 *      tolerance 1e-6) with the 4-parameter Lorentzian cavity model
 *      m(x) = B + A g^2 / ((x-c)^2 + g^2), parameters p = (c, g, A, B).
 *
 * Readings of points the paper leaves open (all stated once more in the
 * design notes of the repository):
 *   - "C2R-FFT" is read as the forward real-input transform, unnormalised,
 *     sign exp(-2 pi i b n / N); the readout quantity is the magnitude |X_b|.
 *   - bin of a tooth at signed frequency f: b = floor(|f| N / fs + 1/2),
 *     reduced mod N and folded into [0, N/2] (aliases land on N - b).
 *   - LM is the Marquardt (1963) form: solve (H + lambda diag H) d = J^T r
 *     with H = J^T J, lambda0 = 1e-3, /10 on a step that lowers chi^2,
 *     *10 on one that raises it; each trial step counts as one iteration;
 *     the fit stops as converged when a trial changes chi^2 by no more than
 *     tol * chi^2 (the lower of the two points is kept).
 *   - initial guess: moments of the spectrum about a baseline taken as the
 *     median of the outer fifth of the teeth; and the paper's own initial
 *     centre (or_median_*): the batch of spectra as a time x tooth image,
 *     a 7x7 median filter with mirrored edges, the lowest filtered value of
 *     each row.
 *
 * The paper's own lineshape (a Fano profile with the centre free, scale and
 * offset boxed to +-10 % of averages, asymmetry and width fixed) is the
 * second model here (or_fano_*), a box-constrained LM over (c, A, B).
 *
 * Parity: the DFT is pinned by closed forms (pure tone gives a N/2,
 * X_0 = sum x, X_{N/2} = alternating sum, Parseval) and by numpy's rfft;
 * the LM optimum by noise-free recovery, shift/scale/mirror invariants,
 * a brute-force variable-projection grid on tiny inputs and MINPACK's LM;
 * the Jacobian by central finite differences; the moment initial guess by a
 * hand-computed example.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* per-frame fit outcome (same numbering as the library's public header,
 * written out independently here) */
enum { OR_CONVERGED = 0, OR_MAX_ITER = 1, OR_SINGULAR = 2, OR_NONFINITE = 3 };
#define OR_INIT_FLAT 0x10

/* ------------------------------------------------------------------ */
/* Tooth -> DFT bin (reading: nearest bin, aliased into [0, N/2]).     */
/* ------------------------------------------------------------------ */
int or_tooth_bins(double fs, int N, int T, const double* f, int* bins)
{
    if (fs <= 0 || N < 2 || T < 1) return -1;
    for (int k = 0; k < T; ++k) {
        double pos = fabs(f[k]) * (double)N / fs;
        long long b = (long long)floor(pos + 0.5);
        b %= N;
        if (b > N / 2) b = N - b;
        bins[k] = (int)b;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Direct-sum DFT at selected bins (definition, no fast algorithm).    */
/* The phase index (b*n) mod N is reduced exactly in integers, and the */
/* table holds cos/sin(2 pi j / N) for j < N, evaluated by libm.        */
/* ------------------------------------------------------------------ */
static void make_table(int N, double* tc, double* ts)
{
    for (int j = 0; j < N; ++j) {
        double a = 2.0 * M_PI * (double)j / (double)N;
        tc[j] = cos(a);
        ts[j] = sin(a);
    }
}

static void dft_frame_i16(const int16_t* x, int N, int nb, const int* bins,
                          const double* tc, const double* ts, double* re, double* im)
{
    for (int q = 0; q < nb; ++q) {
        long long b = bins[q];
        double sr = 0.0, si = 0.0;
        for (int n = 0; n < N; ++n) {
            int j = (int)((b * (long long)n) % N);
            double v = (double)x[n];
            sr += v * tc[j];
            si -= v * ts[j];
        }
        re[q] = sr;
        im[q] = si;
    }
}

static void dft_frame_f64(const double* x, int N, int nb, const int* bins,
                          const double* tc, const double* ts, double* re, double* im)
{
    for (int q = 0; q < nb; ++q) {
        long long b = bins[q];
        double sr = 0.0, si = 0.0;
        for (int n = 0; n < N; ++n) {
            int j = (int)((b * (long long)n) % N);
            sr += x[n] * tc[j];
            si -= x[n] * ts[j];
        }
        re[q] = sr;
        im[q] = si;
    }
}

int or_dft_bins(const int16_t* x, int64_t n_frames, int N, int nb, const int* bins,
                double* re, double* im)
{
    double* tc = (double*)malloc(sizeof(double) * (size_t)N);
    double* ts = (double*)malloc(sizeof(double) * (size_t)N);
    if (!tc || !ts) { free(tc); free(ts); return -1; }
    make_table(N, tc, ts);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n_frames; ++i)
        dft_frame_i16(x + i * (int64_t)N, N, nb, bins, tc, ts, re + i * nb, im + i * nb);
    free(tc);
    free(ts);
    return 0;
}

int or_dft_bins_f64(const double* x, int64_t n_frames, int N, int nb, const int* bins,
                    double* re, double* im)
{
    double* tc = (double*)malloc(sizeof(double) * (size_t)N);
    double* ts = (double*)malloc(sizeof(double) * (size_t)N);
    if (!tc || !ts) { free(tc); free(ts); return -1; }
    make_table(N, tc, ts);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n_frames; ++i)
        dft_frame_f64(x + i * (int64_t)N, N, nb, bins, tc, ts, re + i * nb, im + i * nb);
    free(tc);
    free(ts);
    return 0;
}

/* Readout of one frame's tooth bins: amps_k = |X_{b_k}| (the magnitude, not
 * the power), y_k = amps_k / ref_k with ref indexed by tooth k, not by bin
 * (ref may be NULL: y not written). */
static void tooth_readout(const double* re, const double* im, int T, const double* ref,
                          double* amps, double* y)
{
    for (int k = 0; k < T; ++k) {
        double a = sqrt(re[k] * re[k] + im[k] * im[k]);
        amps[k] = a;
        if (ref && y) y[k] = a / ref[k];
    }
}

/* frames are int16 (x16) or FP64 (x64, for noise-free unquantised input);
 * exactly one of the two is given */
static int readout_any(const int16_t* x16, const double* x64, int64_t n_frames, int N, int T,
                       const int* bins, const double* ref, double* amps, double* y)
{
    double* tc = (double*)malloc(sizeof(double) * (size_t)N);
    double* ts = (double*)malloc(sizeof(double) * (size_t)N);
    if (!tc || !ts) { free(tc); free(ts); return -1; }
    make_table(N, tc, ts);
#pragma omp parallel
    {
        double* re = (double*)malloc(sizeof(double) * (size_t)T);
        double* im = (double*)malloc(sizeof(double) * (size_t)T);
#pragma omp for schedule(dynamic, 16)
        for (int64_t i = 0; i < n_frames; ++i) {
            if (x16)
                dft_frame_i16(x16 + i * (int64_t)N, N, T, bins, tc, ts, re, im);
            else
                dft_frame_f64(x64 + i * (int64_t)N, N, T, bins, tc, ts, re, im);
            tooth_readout(re, im, T, ref, amps + i * T, y ? y + i * T : NULL);
        }
        free(re);
        free(im);
    }
    free(tc);
    free(ts);
    return 0;
}

int or_readout(const int16_t* x, int64_t n_frames, int N, int T, const int* bins,
               const double* ref, double* amps, double* y)
{
    return readout_any(x, NULL, n_frames, N, T, bins, ref, amps, y);
}

int or_readout_f64(const double* x, int64_t n_frames, int N, int T, const int* bins,
                   const double* ref, double* amps, double* y)
{
    return readout_any(NULL, x, n_frames, N, T, bins, ref, amps, y);
}

/* reference spectrum: the mean (sum / count) over cavity-free frames of the
 * tooth magnitudes |X_{b_k}| -- a mean of magnitudes, not the magnitude of a
 * mean spectrum */
static int reference_any(const int16_t* x16, const double* x64, int64_t n_frames, int N, int T,
                         const int* bins, double* ref)
{
    if (n_frames < 1) return -1;
    double* amps = (double*)malloc(sizeof(double) * (size_t)n_frames * (size_t)T);
    if (!amps) return -1;
    if (readout_any(x16, x64, n_frames, N, T, bins, NULL, amps, NULL) != 0) { free(amps); return -1; }
    for (int k = 0; k < T; ++k) {
        double s = 0.0;
        for (int64_t i = 0; i < n_frames; ++i) s += amps[i * T + k];
        ref[k] = s / (double)n_frames;
    }
    free(amps);
    return 0;
}

int or_reference(const int16_t* x, int64_t n_frames, int N, int T, const int* bins, double* ref)
{
    return reference_any(x, NULL, n_frames, N, T, bins, ref);
}

int or_reference_f64(const double* x, int64_t n_frames, int N, int T, const int* bins, double* ref)
{
    return reference_any(NULL, x, n_frames, N, T, bins, ref);
}

/* ------------------------------------------------------------------ */
/* Lorentzian cavity model and its Jacobian.                           */
/*   D = (x-c)^2 + g^2, L = g^2 / D, m = B + A L                        */
/*   dm/dc = 2 A g^2 (x-c) / D^2     dm/dg = 2 A g (x-c)^2 / D^2         */
/*   dm/dA = L                        dm/dB = 1                          */
/* ------------------------------------------------------------------ */
void or_model(const double* x, int T, const double* p, double* m)
{
    double c = p[0], g = p[1], A = p[2], B = p[3];
    for (int k = 0; k < T; ++k) {
        double d = x[k] - c;
        double D = d * d + g * g;
        m[k] = B + A * (g * g) / D;
    }
}

void or_jacobian(const double* x, int T, const double* p, double* J)
{
    double c = p[0], g = p[1], A = p[2];
    for (int k = 0; k < T; ++k) {
        double d = x[k] - c;
        double D = d * d + g * g;
        double D2 = D * D;
        J[4 * k + 0] = 2.0 * A * g * g * d / D2;
        J[4 * k + 1] = 2.0 * A * g * d * d / D2;
        J[4 * k + 2] = g * g / D;
        J[4 * k + 3] = 1.0;
    }
}

/* chi^2, H = J^T J and grad = J^T r at p, with r = y - m */
static double lm_eval(const double* x, const double* y, int T, const double* p,
                      double H[4][4], double grad[4])
{
    double c = p[0], g = p[1], A = p[2], B = p[3];
    double chi2 = 0.0;
    for (int i = 0; i < 4; ++i) {
        grad[i] = 0.0;
        for (int j = 0; j < 4; ++j) H[i][j] = 0.0;
    }
    for (int k = 0; k < T; ++k) {
        double d = x[k] - c;
        double D = d * d + g * g;
        double D2 = D * D;
        double L = g * g / D;
        double r = y[k] - (B + A * L);
        double J[4];
        J[0] = 2.0 * A * g * g * d / D2;
        J[1] = 2.0 * A * g * d * d / D2;
        J[2] = L;
        J[3] = 1.0;
        chi2 += r * r;
        for (int i = 0; i < 4; ++i) {
            grad[i] += J[i] * r;
            for (int j = 0; j < 4; ++j) H[i][j] += J[i] * J[j];
        }
    }
    return chi2;
}

static double lm_chi2(const double* x, const double* y, int T, const double* p)
{
    double c = p[0], g = p[1], A = p[2], B = p[3];
    double chi2 = 0.0;
    for (int k = 0; k < T; ++k) {
        double d = x[k] - c;
        double r = y[k] - (B + A * (g * g) / (d * d + g * g));
        chi2 += r * r;
    }
    return chi2;
}

/* (H + lambda diag H) delta = grad, via Cholesky of the diagonally scaled
 * matrix S H S + lambda I with S = diag(H)^(-1/2) (an exact rewrite that
 * keeps parameters of very different units well conditioned).
 * Returns 0 on success, -1 when H is not positive definite. */
static int lm_solve(const double H[4][4], double lambda, const double grad[4], double delta[4])
{
    double s[4], M[4][4], b[4], Lc[4][4], z[4], u[4];
    for (int i = 0; i < 4; ++i) {
        if (!(H[i][i] > 0.0) || !isfinite(H[i][i])) return -1;
        s[i] = 1.0 / sqrt(H[i][i]);
    }
    for (int i = 0; i < 4; ++i) {
        for (int j = 0; j < 4; ++j) M[i][j] = H[i][j] * s[i] * s[j];
        M[i][i] = 1.0 + lambda;
        b[i] = grad[i] * s[i];
    }
    memset(Lc, 0, sizeof(Lc));
    for (int j = 0; j < 4; ++j) {
        double v = M[j][j];
        for (int q = 0; q < j; ++q) v -= Lc[j][q] * Lc[j][q];
        if (!(v > 0.0)) return -1;
        Lc[j][j] = sqrt(v);
        for (int i = j + 1; i < 4; ++i) {
            double w = M[i][j];
            for (int q = 0; q < j; ++q) w -= Lc[i][q] * Lc[j][q];
            Lc[i][j] = w / Lc[j][j];
        }
    }
    for (int i = 0; i < 4; ++i) {
        double v = b[i];
        for (int q = 0; q < i; ++q) v -= Lc[i][q] * z[q];
        z[i] = v / Lc[i][i];
    }
    for (int i = 3; i >= 0; --i) {
        double v = z[i];
        for (int q = i + 1; q < 4; ++q) v -= Lc[q][i] * u[q];
        u[i] = v / Lc[i][i];
    }
    for (int i = 0; i < 4; ++i) delta[i] = u[i] * s[i];
    return 0;
}

/* Levenberg-Marquardt fit of one spectrum.  On return p holds the fit
 * with g reported as |g|; rss is chi^2 at the returned p. */
void or_lm_fit(const double* y, const double* x, int T, const double* p0,
               int max_iter, double tol, double lambda0,
               double* p_out, double* rss, int* iters, int* status)
{
    double p[4], H[4][4], grad[4];
    for (int i = 0; i < 4; ++i) p[i] = p0[i];
    double lambda = lambda0;
    double chi2 = lm_eval(x, y, T, p, H, grad);
    int it = 0, st = OR_MAX_ITER;
    if (!isfinite(chi2)) {
        st = OR_NONFINITE;
    } else {
        while (it < max_iter) {
            double delta[4], pt[4], Ht[4][4], gt[4];
            ++it;
            if (lm_solve(H, lambda, grad, delta) != 0) { st = OR_SINGULAR; break; }
            for (int i = 0; i < 4; ++i) pt[i] = p[i] + delta[i];
            double chi2t = lm_eval(x, y, T, pt, Ht, gt);
            if (!isfinite(chi2t)) { lambda *= 10.0; continue; }
            if (fabs(chi2t - chi2) <= tol * chi2) {
                if (chi2t <= chi2) {
                    for (int i = 0; i < 4; ++i) p[i] = pt[i];
                    chi2 = chi2t;
                }
                st = OR_CONVERGED;
                break;
            }
            if (chi2t < chi2) {
                for (int i = 0; i < 4; ++i) {
                    p[i] = pt[i];
                    grad[i] = gt[i];
                    for (int j = 0; j < 4; ++j) H[i][j] = Ht[i][j];
                }
                chi2 = chi2t;
                lambda /= 10.0;
            } else {
                lambda *= 10.0;
            }
        }
    }
    for (int i = 0; i < 4; ++i) p_out[i] = p[i];
    p_out[1] = fabs(p_out[1]);
    *rss = lm_chi2(x, y, T, p_out);
    *iters = it;
    *status = st;
}

/* ------------------------------------------------------------------ */
/* Moment initial guess (reading of the paper's "reasonably chosen      */
/* starting parameters"; its 7x7 median-filter init is not used):       */
/*   outer set O: teeth whose distance from the span midpoint is at     */
/*     least the ceil(T/5)-th largest such distance (ties included);    */
/*   B0 = median of y over O;  d = y - B0;  s = sign of d at argmax|d|; */
/*   w = max(s d, 0);  c0 = sum w x / sum w;  A0 = s max w;             */
/*   g0 = sum w * dx / (pi |A0|), clamped to [dx/2, span/2],            */
/*   dx = span / (T-1).  sum w == 0 gives c0 = midpoint, A0 = 0 and     */
/*   the OR_INIT_FLAT flag.                                             */
/* ------------------------------------------------------------------ */
static int cmp_double(const void* a, const void* b)
{
    double u = *(const double*)a, v = *(const double*)b;
    return (u > v) - (u < v);
}

int or_moment_init(const double* y, const double* x, int T, double* p0)
{
    double xmin = x[0], xmax = x[0];
    for (int k = 1; k < T; ++k) {
        if (x[k] < xmin) xmin = x[k];
        if (x[k] > xmax) xmax = x[k];
    }
    double mid = 0.5 * (xmin + xmax);
    double span = xmax - xmin;
    double dx = span / (double)(T - 1);
    int n_o = (T + 4) / 5;

    double* dist = (double*)malloc(sizeof(double) * (size_t)T);
    double* sel = (double*)malloc(sizeof(double) * (size_t)T);
    for (int k = 0; k < T; ++k) dist[k] = fabs(x[k] - mid);
    memcpy(sel, dist, sizeof(double) * (size_t)T);
    qsort(sel, (size_t)T, sizeof(double), cmp_double);       /* ascending */
    double thresh = sel[T - n_o];                              /* n_o-th largest */
    int m = 0;
    for (int k = 0; k < T; ++k)
        if (dist[k] >= thresh) sel[m++] = y[k];
    qsort(sel, (size_t)m, sizeof(double), cmp_double);
    double B0 = (m % 2) ? sel[m / 2] : 0.5 * (sel[m / 2 - 1] + sel[m / 2]);
    free(dist);
    free(sel);

    int jstar = 0;
    double best = -1.0;
    for (int k = 0; k < T; ++k) {
        double a = fabs(y[k] - B0);
        if (a > best) { best = a; jstar = k; }
    }
    double s = (y[jstar] - B0) >= 0.0 ? 1.0 : -1.0;
    double W = 0.0, Wx = 0.0, wmax = 0.0;
    for (int k = 0; k < T; ++k) {
        double w = s * (y[k] - B0);
        if (w < 0.0) w = 0.0;
        W += w;
        Wx += w * x[k];
        if (w > wmax) wmax = w;
    }
    if (!(W > 0.0)) {
        p0[0] = mid;
        p0[1] = 0.5 * dx;
        p0[2] = 0.0;
        p0[3] = B0;
        return OR_INIT_FLAT;
    }
    double A0 = s * wmax;
    double g0 = W * dx / (M_PI * fabs(A0));
    if (g0 < 0.5 * dx) g0 = 0.5 * dx;
    if (g0 > 0.5 * span) g0 = 0.5 * span;
    p0[0] = Wx / W;
    p0[1] = g0;
    p0[2] = A0;
    p0[3] = B0;
    return 0;
}

/* Fit a batch of spectra y[n][T].  p0 == NULL: moment initial guess. */
void or_fit_batch(const double* y, int64_t n, const double* x, int T,
                  const double* p0, int max_iter, double tol, double lambda0,
                  double* init_out, double* params, double* rss, int* iters, int* status)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        double q0[4];
        int flag = 0;
        if (p0) {
            for (int j = 0; j < 4; ++j) q0[j] = p0[4 * i + j];
        } else {
            flag = or_moment_init(y + i * T, x, T, q0);
        }
        if (init_out)
            for (int j = 0; j < 4; ++j) init_out[4 * i + j] = q0[j];
        or_lm_fit(y + i * T, x, T, q0, max_iter, tol, lambda0,
                  params + 4 * i, rss + i, iters + i, status + i);
        status[i] |= flag;
    }
}

/* The whole per-frame path: readout, normalisation, moment init, LM. */
int or_process(const int16_t* frames, int64_t n, int N, int T, const int* bins,
               const double* ref, const double* x, int max_iter, double tol, double lambda0,
               double* amps, double* y, double* params, double* rss, int* iters, int* status)
{
    if (or_readout(frames, n, N, T, bins, ref, amps, y) != 0) return -1;
    or_fit_batch(y, n, x, T, NULL, max_iter, tol, lambda0, NULL, params, rss, iters, status);
    return 0;
}

/* Brute force for tiny inputs (variable projection): for each (c, g) on a
 * grid, the model is linear in (A, B), solved by 2x2 least squares; the
 * grid point of least chi^2 is returned with its (A, B) and chi^2. */
void or_grid_fit(const double* y, const double* x, int T,
                 const double* cgrid, int nc, const double* ggrid, int ng,
                 double* p_best, double* chi2_best)
{
    double best = INFINITY;
    for (int a = 0; a < nc; ++a) {
        for (int b = 0; b < ng; ++b) {
            double c = cgrid[a], g = ggrid[b];
            double sLL = 0, sL = 0, sLy = 0, sy = 0;
            for (int k = 0; k < T; ++k) {
                double d = x[k] - c;
                double L = g * g / (d * d + g * g);
                sLL += L * L;
                sL += L;
                sLy += L * y[k];
                sy += y[k];
            }
            double det = sLL * (double)T - sL * sL;
            if (!(fabs(det) > 0.0)) continue;
            double A = (sLy * (double)T - sL * sy) / det;
            double B = (sLL * sy - sL * sLy) / det;
            double q[4] = { c, g, A, B };
            double chi2 = lm_chi2(x, y, T, q);
            if (chi2 < best) {
                best = chi2;
                for (int j = 0; j < 4; ++j) p_best[j] = q[j];
            }
        }
    }
    *chi2_best = best;
}

/* ------------------------------------------------------------------ */
/* The paper's fitted lineshape: a Fano profile                       */
/* ("Data Capture and Processing", fit paragraph; Fano 1961)           */
/*   eps = (x - c) / gamma,   F = (q + eps)^2 / (1 + eps^2),           */
/*   m(x) = B + A F                                                    */
/* with the centre c free, the scale A and offset B held to a box      */
/* [lo, hi] of +-box around pre-computed averages (A_bar, B_bar), and  */
/* the asymmetry q and width gamma fixed.  Bounds: a parameter on a    */
/* bound whose gradient points outward is held out of the step (an     */
/* active set), the others take the reduced LM step, and the trial     */
/* point is clamped onto the box.  q = 0 gives the Lorentzian dip      */
/* B + A - A / (1 + eps^2).                                            */
/*   dm/dc = -A F'(eps) / gamma,  F'(eps) = 2 (q+eps)(1 - q eps)/(1+eps^2)^2 */
/*   dm/dA = F,                    dm/dB = 1                            */
/* ------------------------------------------------------------------ */
void or_fano_model(const double* x, int T, double q, double gamma, const double* p, double* m)
{
    for (int k = 0; k < T; ++k) {
        const double e = (x[k] - p[0]) / gamma;
        m[k] = p[2] + p[1] * (q + e) * (q + e) / (1.0 + e * e);
    }
}

/* Jacobian rows (dm/dc, dm/dA, dm/dB), p = (c, A, B) */
void or_fano_jacobian(const double* x, int T, double q, double gamma, const double* p, double* J)
{
    for (int k = 0; k < T; ++k) {
        const double e = (x[k] - p[0]) / gamma;
        const double d = 1.0 + e * e;
        J[3 * k + 0] = -p[1] * 2.0 * (q + e) * (1.0 - q * e) / (d * d) / gamma;
        J[3 * k + 1] = (q + e) * (q + e) / d;
        J[3 * k + 2] = 1.0;
    }
}

static double fano_eval(const double* x, const double* y, int T, double q, double gamma, const double* p,
                        double H[3][3], double grad[3])
{
    double chi2 = 0.0;
    double J[3];
    for (int i = 0; i < 3; ++i) {
        grad[i] = 0.0;
        for (int j = 0; j < 3; ++j) H[i][j] = 0.0;
    }
    for (int k = 0; k < T; ++k) {
        const double e = (x[k] - p[0]) / gamma;
        const double d = 1.0 + e * e;
        const double F = (q + e) * (q + e) / d;
        const double r = y[k] - (p[2] + p[1] * F);
        J[0] = -p[1] * 2.0 * (q + e) * (1.0 - q * e) / (d * d) / gamma;
        J[1] = F;
        J[2] = 1.0;
        chi2 += r * r;
        for (int i = 0; i < 3; ++i) {
            grad[i] += J[i] * r;
            for (int j = 0; j < 3; ++j) H[i][j] += J[i] * J[j];
        }
    }
    return chi2;
}

/* (H + lambda diag H) delta = grad for 3 parameters, Jacobi-scaled Cholesky;
 * a parameter whose bit is set in held keeps delta = 0 and drops out of the
 * system (its row and column are decoupled from the others). */
static int fano_solve(const double H[3][3], double lambda, const double grad[3], int held, double delta[3])
{
    double s[3], M[3][3], Lc[3][3], z[3], u[3];
    for (int i = 0; i < 3; ++i) {
        if (!(H[i][i] > 0.0) || !isfinite(H[i][i])) return -1;
        s[i] = 1.0 / sqrt(H[i][i]);
    }
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) M[i][j] = ((held >> i) & 1) || ((held >> j) & 1) ? 0.0 : H[i][j] * s[i] * s[j];
        M[i][i] = 1.0 + lambda;
    }
    memset(Lc, 0, sizeof(Lc));
    for (int j = 0; j < 3; ++j) {
        double v = M[j][j];
        for (int t = 0; t < j; ++t) v -= Lc[j][t] * Lc[j][t];
        if (!(v > 0.0)) return -1;
        Lc[j][j] = sqrt(v);
        for (int i = j + 1; i < 3; ++i) {
            double w = M[i][j];
            for (int t = 0; t < j; ++t) w -= Lc[i][t] * Lc[j][t];
            Lc[i][j] = w / Lc[j][j];
        }
    }
    for (int i = 0; i < 3; ++i) {
        double v = ((held >> i) & 1) ? 0.0 : grad[i] * s[i];
        for (int t = 0; t < i; ++t) v -= Lc[i][t] * z[t];
        z[i] = v / Lc[i][i];
    }
    for (int i = 2; i >= 0; --i) {
        double v = z[i];
        for (int t = i + 1; t < 3; ++t) v -= Lc[t][i] * u[t];
        u[i] = v / Lc[i][i];
    }
    for (int i = 0; i < 3; ++i) delta[i] = u[i] * s[i];
    return 0;
}

static double clampd(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* Box of +-box around avg (ordered whatever the sign of avg). */
static void fano_box(double avg, double box, double* lo, double* hi)
{
    const double a = avg * (1.0 - box), b = avg * (1.0 + box);
    *lo = a < b ? a : b;
    *hi = a < b ? b : a;
}

/* Initial guess: the centre at the lowest tooth (the paper's "lowest value"
 * reading) moved to where the profile's minimum lies, eps = -q, i.e.
 * c0 = x_min + q gamma; A and B at their averages. */
void or_fano_init(const double* y, const double* x, int T, double q, double gamma, double A_bar, double B_bar,
                  double* p0)
{
    int kmin = 0;
    for (int k = 1; k < T; ++k)
        if (y[k] < y[kmin]) kmin = k;
    p0[0] = x[kmin] + q * gamma;
    p0[1] = A_bar;
    p0[2] = B_bar;
}

/* Bit i set when parameter i sits on a bound of its box and the gradient
 * J^T (y - m) points out of the box there (moving it inward cannot lower
 * chi^2 to first order): it is held for this step. */
static int fano_held(const double p[3], const double grad[3], double Alo, double Ahi, double Blo, double Bhi)
{
    int h = 0;
    if ((p[1] <= Alo && grad[1] < 0.0) || (p[1] >= Ahi && grad[1] > 0.0)) h |= 2;
    if ((p[2] <= Blo && grad[2] < 0.0) || (p[2] >= Bhi && grad[2] > 0.0)) h |= 4;
    return h;
}

/* Box-constrained Levenberg-Marquardt of one spectrum, p = (c, A, B):
 * the parameters held by fano_held stay where they are, the others take the
 * damped step of the reduced system, and the trial point is clamped onto the
 * box; accept / reject, lambda and the stopping rule as in or_lm_fit. */
void or_fano_fit(const double* y, const double* x, int T, double q, double gamma, double A_bar, double B_bar,
                 double box, const double* p0, int max_iter, double tol, double lambda0, double* p_out,
                 double* rss, int* iters, int* status)
{
    double Alo, Ahi, Blo, Bhi;
    fano_box(A_bar, box, &Alo, &Ahi);
    fano_box(B_bar, box, &Blo, &Bhi);
    double p[3], H[3][3], grad[3];
    p[0] = p0[0];
    p[1] = clampd(p0[1], Alo, Ahi);
    p[2] = clampd(p0[2], Blo, Bhi);
    double lambda = lambda0;
    double chi2 = fano_eval(x, y, T, q, gamma, p, H, grad);
    int it = 0, st = OR_MAX_ITER;
    if (!isfinite(chi2)) {
        st = OR_NONFINITE;
    } else {
        while (it < max_iter) {
            double delta[3], pt[3], Ht[3][3], gt[3];
            ++it;
            if (fano_solve(H, lambda, grad, fano_held(p, grad, Alo, Ahi, Blo, Bhi), delta) != 0) {
                st = OR_SINGULAR;
                break;
            }
            pt[0] = p[0] + delta[0];
            pt[1] = clampd(p[1] + delta[1], Alo, Ahi);
            pt[2] = clampd(p[2] + delta[2], Blo, Bhi);
            const double chi2t = fano_eval(x, y, T, q, gamma, pt, Ht, gt);
            if (!isfinite(chi2t)) { lambda *= 10.0; continue; }
            if (fabs(chi2t - chi2) <= tol * chi2) {
                if (chi2t <= chi2) {
                    for (int i = 0; i < 3; ++i) p[i] = pt[i];
                    chi2 = chi2t;
                }
                st = OR_CONVERGED;
                break;
            }
            if (chi2t < chi2) {
                for (int i = 0; i < 3; ++i) p[i] = pt[i];
                chi2 = chi2t;
                memcpy(H, Ht, sizeof(H));
                memcpy(grad, gt, sizeof(grad));
                lambda *= 0.1;
            } else {
                lambda *= 10.0;
            }
        }
    }
    for (int i = 0; i < 3; ++i) p_out[i] = p[i];
    *rss = chi2;
    *iters = it;
    *status = st;
}

/* Batch: p0 == NULL takes or_fano_init. */
void or_fano_fit_batch(const double* y, int64_t n, const double* x, int T, double q, double gamma, double A_bar,
                       double B_bar, double box, const double* p0, int max_iter, double tol, double lambda0,
                       double* init_out, double* params, double* rss, int* iters, int* status)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        double q0[3];
        if (p0) {
            for (int j = 0; j < 3; ++j) q0[j] = p0[3 * i + j];
        } else {
            or_fano_init(y + i * T, x, T, q, gamma, A_bar, B_bar, q0);
        }
        if (init_out)
            for (int j = 0; j < 3; ++j) init_out[3 * i + j] = q0[j];
        or_fano_fit(y + i * T, x, T, q, gamma, A_bar, B_bar, box, q0, max_iter, tol, lambda0, params + 3 * i,
                    rss + i, iters + i, status + i);
    }
}

/* Brute force for tiny inputs: least chi^2 over a grid of centres with A
 * and B on grids inside their boxes. */
void or_fano_grid_fit(const double* y, const double* x, int T, double q, double gamma, const double* cgrid, int nc,
                      const double* Agrid, int nA, const double* Bgrid, int nB, double* p_best, double* chi2_best)
{
    double best = INFINITY;
    double* m = (double*)malloc(sizeof(double) * (size_t)T);
    if (!m) return;
    for (int a = 0; a < nc; ++a)
        for (int b = 0; b < nA; ++b)
            for (int c = 0; c < nB; ++c) {
                const double p[3] = { cgrid[a], Agrid[b], Bgrid[c] };
                or_fano_model(x, T, q, gamma, p, m);
                double chi2 = 0.0;
                for (int k = 0; k < T; ++k) chi2 += (y[k] - m[k]) * (y[k] - m[k]);
                if (chi2 < best) {
                    best = chi2;
                    for (int j = 0; j < 3; ++j) p_best[j] = p[j];
                }
            }
    free(m);
    *chi2_best = best;
}

/* ------------------------------------------------------------------ */
/* The paper's initial centre ("Data Capture and Processing", initial- */
/* value paragraph; Fig. 3c): the normalised spectra of a batch form   */
/* an image y[i][k] (frame i in time order, tooth k); a 2-D median     */
/* filter with a 7x7 footprint is applied, and the lowest value of     */
/* each filtered row gives the initial centre x_k (+ shift; the Fano   */
/* profile's minimum lies q gamma below its centre).                   */
/* Readings: the image edges are mirrored without repeating the edge   */
/* sample's neighbour -- index -1 maps to 0, -2 to 1, n to n-1 (the    */
/* "reflect" convention, d c b a | a b c d | d c b a, repeated for     */
/* images smaller than the footprint); the median of the 49 values is  */
/* the 25th smallest; ties in the row minimum go to the lowest tooth.  */
/* ------------------------------------------------------------------ */
static int64_t mirror_index(int64_t i, int64_t n)
{
    const int64_t period = 2 * n;
    int64_t j = i % period;
    if (j < 0) j += period;
    return j >= n ? period - 1 - j : j;
}

static double median49(double* v)
{
    for (int i = 1; i < 49; ++i) {          /* insertion sort */
        const double t = v[i];
        int j = i - 1;
        while (j >= 0 && v[j] > t) {
            v[j + 1] = v[j];
            --j;
        }
        v[j + 1] = t;
    }
    return v[24];
}

void or_median_filter7(const double* y, int64_t n, int T, double* out)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double v[49];
        for (int k = 0; k < T; ++k) {
            int m = 0;
            for (int di = -3; di <= 3; ++di)
                for (int dk = -3; dk <= 3; ++dk)
                    v[m++] = y[mirror_index(i + di, n) * T + mirror_index(k + dk, T)];
            out[i * T + k] = median49(v);
        }
    }
}

/* c0[i] = x[kmin[i]] + shift with kmin[i] the first tooth of the lowest
 * filtered value of row i; filtered (n x T) may be NULL. */
int or_median_init(const double* y, int64_t n, int T, const double* x, double shift, double* c0, int* kmin,
                   double* filtered)
{
    double* f = filtered ? filtered : (double*)malloc(sizeof(double) * (size_t)n * (size_t)T);
    if (!f) return -1;
    or_median_filter7(y, n, T, f);
    for (int64_t i = 0; i < n; ++i) {
        int best = 0;
        for (int k = 1; k < T; ++k)
            if (f[i * T + k] < f[i * T + best]) best = k;
        kmin[i] = best;
        c0[i] = x[best] + shift;
    }
    if (!filtered) free(f);
    return 0;
}
