// cg_api.cu -- the C ABI: plan construction and the plain-path entry points.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "cg_internal.h"

namespace {

thread_local std::string g_last_error;

cg_status fail(cg_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

cg_status cuda_fail(cudaError_t e, const char* what)
{
    return fail(e == cudaErrorMemoryAllocation ? CG_ERR_NOMEM : CG_ERR_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

constexpr double kTwoPi = 6.28318530717958647692528676655900577;

// radices of the shared-memory stages, largest first among powers of two
bool factorize(int L, std::vector<int>& out)
{
    out.clear();
    int r = L;
    while (r % 8 == 0 && r > 8) { out.push_back(8); r /= 8; }
    if (r == 8) { out.push_back(8); r = 1; }
    while (r % 4 == 0) { out.push_back(4); r /= 4; }
    while (r % 2 == 0) { out.push_back(2); r /= 2; }
    for (int q : {5, 3, 7, 11, 13})
        while (r % q == 0) { out.push_back(q); r /= q; }
    return r == 1 && static_cast<int>(out.size()) <= cg::kMaxStages;
}

// Choose the transform: the largest M | N (4 <= M, N/M >= 2) such that every
// tooth bin is congruent to +r or -r mod M, so the teeth are read from one
// L = N/M point transform of the folded frame; otherwise the real FFT through
// an N/2-point complex transform (N even) or the complex N-point one (M = 1).
void choose_fft(cg_plan_s* p)
{
    const int N = p->N;
    p->kind = CG_FFT_FULL;
    p->M = 2;
    p->r0 = 0;
    p->L = N / 2;
    std::vector<int> rad;
    if (p->opts.fft != CG_FFT_FULL) {
        for (int M = N / 2; M >= 4; --M) {
            if (N % M) continue;
            const int L = N / M;
            if (L < 2 || M > 4096) continue;
            const int r = p->bins[0] % M;
            bool ok = true;
            for (int b : p->bins) {
                const int q = b % M;
                if (q != r && q != (M - r) % M) { ok = false; break; }
            }
            if (!ok || !factorize(L, rad)) continue;
            p->kind = CG_FFT_COSET;
            p->M = M;
            p->r0 = r;
            p->L = L;
            p->radices = rad;
            return;
        }
    }
    if (N % 2 == 0 && factorize(N / 2, rad)) {
        p->radices = rad;
        return;
    }
    // odd N: complex transform of the real samples (a fold with M = 1)
    p->kind = CG_FFT_COSET;
    p->M = 1;
    p->r0 = 0;
    p->L = N;
    if (!factorize(N, rad)) p->radices.clear();
    else p->radices = rad;
}

int align16(int v) { return (v + 15) & ~15; }

template <typename T>
cudaError_t upload(T** dst, const std::vector<T>& src)
{
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(dst), sizeof(T) * std::max<size_t>(src.size(), 1));
    if (e != cudaSuccess) return e;
    if (!src.empty()) e = cudaMemcpy(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice);
    return e;
}

void free_tables(cg::DevTables& d)
{
    cudaFree(d.tw_L);
    cudaFree(d.tw_M);
    cudaFree(d.tw_n1);
    cudaFree(d.tw_b);
    cudaFree(d.zidx);
    cudaFree(d.inv_ref);
    cudaFree(d.u);
    cudaFree(d.outer_idx);
    cudaFree(d.ref_part);
    cudaFree(d.ref_out);
    cudaFree(d.tw_M5);
    cudaFree(d.tooth_of_m);
    cudaFree(d.fit_counter);
    cudaFree(d.gemm_W);
    cudaFree(d.fold_W);
    cudaFree(d.err);
    cudaFree(d.mlp_W);
    cudaFree(d.mlp_tab);
    cudaFree(d.fb_list);
    cudaFree(d.fb_count);
    cudaFree(d.median_cx);
    d = cg::DevTables{};
}

void free_plan(cg_plan_s* p)
{
    free_tables(p->d);
    if (p->s_read) cudaStreamDestroy(p->s_read);
    if (p->s_fit) cudaStreamDestroy(p->s_fit);
    for (cudaEvent_t e : {p->ev_fork, p->ev_read, p->ev_join_r, p->ev_join_f})
        if (e) cudaEventDestroy(e);
    for (const auto& t : p->timed) {
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    for (cudaEvent_t e : p->ev_pool) cudaEventDestroy(e);
    delete p;
}

// Throughput path: fast readout (N = 10 Q' with L = 10 Q) and the
// register-resident LM.  Chooses the batch size, shared-memory layout, lane
// group and launch grids; leaves fast_ok false when the geometry does not fit.
cudaError_t setup_fast(cg_plan_s* p, const std::vector<int>& zidx)
{
    p->fast_ok = false;
    const int N = p->N, T = p->T, L = p->L;
    if (p->kind != CG_FFT_COSET || p->M != 10 || L % 10 != 0) return cudaSuccess;
    const int Q = L / 10;
    if (!cg::fast_readout_ptr(Q)) return cudaSuccess;
    std::vector<int> tom(L, -1);
    for (int k = 0; k < T; ++k) {
        if (tom[zidx[k]] >= 0) return cudaSuccess;   // two teeth on one bin: generic path
        tom[zidx[k]] = k;
    }
    if (!p->fit_ok) return cudaSuccess;
    std::vector<float2> tw5(5);
    for (int j = 0; j < 5; ++j) {
        const double ang = -kTwoPi * static_cast<double>((p->r0 * j) % 10) / 10.0;
        tw5[j] = make_float2(static_cast<float>(std::cos(ang)), static_cast<float>(std::sin(ang)));
    }
    cudaError_t e;
    if ((e = upload(&p->d.tw_M5, tw5)) != cudaSuccess) return e;
    if ((e = upload(&p->d.tooth_of_m, tom)) != cudaSuccess) return e;
    // batch size and layout for samples of sb bytes: minimise idle thread
    // slots of the two transform stages (stage 1: 10 items per frame, cost
    // ~ 50 Q; stage 2: Q items, cost ~ 200); at most ~52 KiB of shared
    // memory per block keeps four blocks per SM
    auto layout = [&](int sb, cg::FastArgs& a, void* fn, int& grid) -> cudaError_t {
        int bestF = 2;
        double best = 1e30;
        for (int F = 2; F <= 32; ++F) {
            const int bytes = sb * N * F + 32 + 8 * L * F;
            if (bytes > 52 * 1024) break;
            const double cost =
                (std::ceil(10.0 * F / 128.0) * 50.0 * Q + std::ceil(double(Q) * F / 128.0) * 200.0) / F;
            if (cost < best - 1e-9) { best = cost; bestF = F; }
        }
        // frames per block measured best on GB300 for the instantiated
        // transforms (occupancy and lane use trade against each other, which
        // the idle-slot model above does not see): 10^6 paper-rate frames
        // take 0.525 ms at F = 8 vs 0.547 ms at the model's 11; 8-bit
        // 2200-sample frames 0.996 vs 1.08 ms; wide frames 0.624 vs 0.662 ms
        struct Measured { int Q, sb, F; };
        static const Measured kMeasured[] = {{10, 2, 12}, {11, 2, 8}, {22, 1, 8}, {25, 2, 5}};
        for (const Measured& mf : kMeasured)
            if (mf.Q == Q && mf.sb == sb && sb * N * mf.F + 32 + 8 * L * mf.F <= 52 * 1024) bestF = mf.F;
        a.N = N;
        a.T = T;
        a.F = bestF;
        a.pair_isign = (p->r0 & 1) ? -1 : 1;
        int off = 0;
        a.sm_twL = off; off = align16(off + 8 * L);
        a.sm_twN = off; off = align16(off + 8 * L);
        a.sm_tom = off; off = align16(off + 4 * L);
        a.sm_iref = off; off = align16(off + 4 * T);
        a.sm_u = 0;
        a.sm_raw = off; off = align16(off + sb * N * bestF + 32);
        a.sm_Y = off; off = align16(off + 8 * L * bestF);
        a.sm_amps = 0;
        a.sm_y = 0;
        a.sm_total = off;
        a.twL = p->d.tw_L;
        a.twN = p->d.tw_n1;
        a.twM = p->d.tw_M5;
        a.tooth_of_m = p->d.tooth_of_m;
        a.inv_ref = p->d.inv_ref;
        a.u = p->d.u;
        cudaError_t e2 = cg::raise_smem_limit(fn, a.sm_total);
        if (e2 != cudaSuccess) return e2;
        int occ = 0;
        if ((e2 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, 128, a.sm_total)) != cudaSuccess) return e2;
        grid = p->num_sms * occ;
        return cudaSuccess;
    };
    if ((e = layout(2, p->fa, cg::fast_readout_ptr(Q), p->grid_fast)) != cudaSuccess) return e;
    if (p->grid_fast < 1) return cudaSuccess;
    p->Q = Q;
    p->fast_ok = true;
    if (void* fr8 = cg::fast_readout_ptr(Q, 1)) {
        // int8 samples: the staging takes half the bytes, so more frames per block
        if ((e = layout(1, p->fa8, fr8, p->grid_fast8)) != cudaSuccess) return e;
        p->fast_i8_ok = p->grid_fast8 >= 1;
    }
    return cudaSuccess;
}

// Initial-guess and register/shared-memory LM kernels of the throughput
// path, its streams and events.  They need only the teeth (T, abscissa,
// outer set), so any readout can feed them.  Leaves fit_ok false when T is
// beyond what the kernels were instantiated for.
cudaError_t setup_fit_kernels(cg_plan_s* p)
{
    p->fit_ok = false;
    const int T = p->T;
    // LM lanes per frame (measured on GB300).  FP32 solve: one lane per frame
    // for small T (no reductions), two lanes for T <= 100 (twice the resident
    // frames at one shuffle level), else four (eight beyond the instantiated
    // point counts).  FP64 solve: the solve's long dependent FP64 chain runs
    // once per lane group, so fewer lanes per frame (more frames per warp)
    // win: one lane for T <= 100, else four.
    int G = p->opts.lanes_per_frame;
    if (G == 0) {
        if (p->solve_f64)
            G = T <= 100 ? 1 : 4;
        else
            G = T <= 48 ? 1 : (T <= 100 ? 2 : 4);
    }
    const int model = p->opts.model;
    if (model == CG_MODEL_FANO && G == 1) G = 2;   // the Fano fit runs in the register-resident kernel
    bool exact = false;
    int ppl = cg::fit2_ppl(G, T, &exact, model);
    while (ppl == 0 && G < 32 && !p->opts.lanes_per_frame) ppl = cg::fit2_ppl(G *= 2, T, &exact, model);
    if (ppl == 0) return cudaSuccess;
    const int npad = cg::init_npad(p->n_outer);
    if (npad == 0) return cudaSuccess;
    // lane-per-frame initial guess: tables + 4 warps x 32 staged rows
    cg::InitArgs& ia = p->ia;
    ia.T = T;
    ia.row_stride = T | 1;
    ia.n_outer = p->n_outer;
    ia.inv_ref = p->d.inv_ref;
    ia.u = p->d.u;
    ia.outer_idx = p->d.outer_idx;
    ia.u_mid = p->u_mid;
    ia.du = p->du;
    ia.span = p->span;
    ia.x_mid = static_cast<float>(p->x_mid);
    ia.x_scale = static_cast<float>(p->x_scale);
    p->init_npad = npad;
    // tables, 2 mbarriers and 2 x 32 staged rows per warp (4 warps)
    p->init_smem = 4 * ((2 * T + p->n_outer + 3) & ~3) + 8 * 2 * 4 + 4 * 4 * 2 * 32 * ia.row_stride;
    cudaError_t e;
    int occ = 0;
    void* ff = cg::fit2_ptr(G, ppl, exact, model);
    const size_t fsm = cg::fit2_smem(G, T, model);
    if ((e = cg::raise_smem_limit(ff, static_cast<int>(fsm))) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ff, cg::fit2_threads(G), fsm)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&p->d.fit_counter, sizeof(unsigned long long))) != cudaSuccess) return e;
    if (occ < 1) return cudaSuccess;
    p->grid_fit2 = p->num_sms * occ;
    if (!p->d.err) {
        if ((e = cudaMalloc(&p->d.err, sizeof(int))) != cudaSuccess) return e;
        if ((e = cudaMemset(p->d.err, 0, sizeof(int))) != cudaSuccess) return e;
    }
    void* fi = cg::init_ptr(npad, p->n_outer);
    if ((e = cg::raise_smem_limit(fi, p->init_smem)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fi, 128, p->init_smem)) != cudaSuccess) return e;
    if (occ < 1) return cudaSuccess;
    p->grid_init = p->num_sms * occ;
    p->ppl_exact = exact;
    if ((e = cudaStreamCreateWithFlags(&p->s_read, cudaStreamNonBlocking)) != cudaSuccess) return e;
    if ((e = cudaStreamCreateWithFlags(&p->s_fit, cudaStreamNonBlocking)) != cudaSuccess) return e;
    for (cudaEvent_t* ev : {&p->ev_fork, &p->ev_read, &p->ev_join_r, &p->ev_join_f})
        if ((e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming)) != cudaSuccess) return e;
    p->G2 = G;
    p->PPL = ppl;
    // lanes per frame left to the library: the shared-memory kernel where it
    // is instantiated
    if (p->opts.lanes_per_frame == 0 && (e = cg::setup_fit3(p)) != cudaSuccess) return e;
    // 0: the whole call is one chunk (one launch per kernel; measured fastest
    // for large calls, since each kernel then has frames enough for every SM)
    p->chunk = p->opts.chunk_frames ? p->opts.chunk_frames : (int64_t(1) << 40);
    p->fit_ok = true;
    return cudaSuccess;
}

std::vector<float> inv_ref_of(const std::vector<double>& ref)
{
    std::vector<float> v(ref.size());
    for (size_t i = 0; i < ref.size(); ++i) v[i] = static_cast<float>(1.0 / ref[i]);
    return v;
}

}  // namespace

void cg::set_last_error(const char* msg) { g_last_error = msg ? msg : ""; }

cudaError_t cg::raise_smem_limit(const void* fn, int bytes)
{
    static std::mutex mu;
    std::lock_guard<std::mutex> lk(mu);
    cudaFuncAttributes at;
    cudaError_t e = cudaFuncGetAttributes(&at, fn);
    if (e != cudaSuccess) return e;
    if (at.maxDynamicSharedSizeBytes >= bytes) return cudaSuccess;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

namespace {

// runs launch(); with the plan's timing on, brackets it by two CUDA events
// recorded on the stream the kernel is launched on
template <class F>
cudaError_t timed(cg_plan_s* p, int stage, cudaStream_t s, F&& launch)
{
    if (!p->timing) return launch();
    cudaEvent_t ev[2];
    for (cudaEvent_t& x : ev) {
        if (!p->ev_pool.empty()) {
            x = p->ev_pool.back();
            p->ev_pool.pop_back();
        } else if (cudaError_t r = cudaEventCreate(&x); r != cudaSuccess) {
            return r;
        }
    }
    cudaError_t e = cudaEventRecord(ev[0], s);
    if (e == cudaSuccess) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], s);
    p->timed.push_back({stage, ev[0], ev[1]});
    return e;
}

}  // namespace

extern "C" {

void cg_opts_default(cg_opts* o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->readout = CG_READOUT_FFT;
    o->fft = CG_FFT_AUTO;
    o->init = CG_INIT_MOMENT;
    o->max_iter = 20;
    o->tol = 1e-6;
    o->lambda0 = 1e-3;
    o->lanes_per_frame = 0;
    o->path = CG_PATH_AUTO;
    o->chunk_frames = 0;
    o->sample_bits = 16;
    o->solve_f64 = -1;
    o->model = CG_MODEL_LORENTZ;
    o->fano_box = 0.1;
}

const char* cg_status_string(cg_status s)
{
    switch (s) {
    case CG_OK: return "ok";
    case CG_ERR_ARG: return "invalid argument";
    case CG_ERR_CUDA: return "CUDA error";
    case CG_ERR_NOMEM: return "out of memory";
    case CG_ERR_TOOTH_RANGE: return "tooth out of range";
    case CG_ERR_OVERFLOW: return "ring buffer overflow";
    case CG_ERR_TIMEOUT: return "timeout";
    case CG_ERR_DEVICE_CHECK: return "device-side check failed";
    case CG_ERR_UNSUPPORTED: return "unsupported";
    case CG_ERR_STATE: return "invalid state";
    }
    return "unknown status";
}

const char* cg_last_error(void) { return g_last_error.c_str(); }

int cg_version(void) { return CG_VERSION; }

cg_status cg_plan(cg_plan_t* out, double fs, int N, int T, const double* tooth_freqs,
                  const double* tooth_x, const double* ref, const cg_opts* opts)
{
    g_last_error.clear();
    if (!out) return fail(CG_ERR_ARG, "plan pointer is NULL");
    *out = nullptr;
    if (!(fs > 0.0) || !std::isfinite(fs)) return fail(CG_ERR_ARG, "sample_rate must be > 0");
    if (N < cg::kMinN || N > cg::kMaxN) return fail(CG_ERR_ARG, "frame_len %d outside [%d, %d]", N, cg::kMinN, cg::kMaxN);
    if (T < cg::kMinT || T > cg::kMaxT) return fail(CG_ERR_ARG, "n_teeth %d outside [%d, %d]", T, cg::kMinT, cg::kMaxT);
    if (!tooth_freqs) return fail(CG_ERR_ARG, "tooth_freqs is NULL");
    cg_opts o;
    cg_opts_default(&o);
    if (opts) o = *opts;
    if (o.max_iter < 0 || o.max_iter > 32767) return fail(CG_ERR_ARG, "max_iter outside [0, 32767]");
    if (!(o.tol >= 0.0) || !(o.lambda0 > 0.0)) return fail(CG_ERR_ARG, "tol must be >= 0 and lambda0 > 0");
    if (o.lanes_per_frame != 0 && o.lanes_per_frame != 1 && o.lanes_per_frame != 2 &&
        o.lanes_per_frame != 4 && o.lanes_per_frame != 8 && o.lanes_per_frame != 16 &&
        o.lanes_per_frame != 32)
        return fail(CG_ERR_ARG, "lanes_per_frame must be 0, 1, 2, 4, 8, 16 or 32");
    if (o.path < CG_PATH_AUTO || o.path > CG_PATH_PIPELINE) return fail(CG_ERR_ARG, "path must be a CG_PATH_* value");
    if (o.chunk_frames < 0) return fail(CG_ERR_ARG, "chunk_frames must be >= 0");
    if (o.readout != CG_READOUT_FFT && o.readout != CG_READOUT_GEMM_SPLIT && o.readout != CG_READOUT_FOLD_GEMM)
        return fail(CG_ERR_ARG, "readout must be CG_READOUT_FFT, CG_READOUT_GEMM_SPLIT or CG_READOUT_FOLD_GEMM");
    if (o.sample_bits != 12 && o.sample_bits != 16) return fail(CG_ERR_ARG, "sample_bits must be 12 or 16");
    if (o.solve_f64 < -1 || o.solve_f64 > 1) return fail(CG_ERR_ARG, "solve_f64 must be -1, 0 or 1");
    if (o.init != CG_INIT_MOMENT && o.init != CG_INIT_MLP && o.init != CG_INIT_MEDIAN)
        return fail(CG_ERR_ARG, "init must be CG_INIT_MOMENT, CG_INIT_MLP or CG_INIT_MEDIAN");
    if (o.polish_iter < 0 || o.polish_iter > 32767) return fail(CG_ERR_ARG, "polish_iter outside [0, 32767]");
    if (o.polish_iter == 0) o.polish_iter = 2;
    if (o.model != CG_MODEL_LORENTZ && o.model != CG_MODEL_FANO)
        return fail(CG_ERR_ARG, "model must be CG_MODEL_LORENTZ or CG_MODEL_FANO");
    if (o.model == CG_MODEL_FANO) {
        if (!(o.fano_gamma > 0.0) || !std::isfinite(o.fano_gamma)) return fail(CG_ERR_ARG, "fano_gamma must be > 0");
        if (!(o.fano_A != 0.0) || !std::isfinite(o.fano_A) || !std::isfinite(o.fano_B) || !std::isfinite(o.fano_q))
            return fail(CG_ERR_ARG, "fano_A (nonzero), fano_B and fano_q must be finite");
        if (!(o.fano_box >= 0.0) || !(o.fano_box < 1.0)) return fail(CG_ERR_ARG, "fano_box must be in [0, 1)");
        if (o.init == CG_INIT_MLP)
            return fail(CG_ERR_UNSUPPORTED, "the Fano model takes the lowest-tooth or median-filter initial centre "
                                            "(init CG_INIT_MOMENT or CG_INIT_MEDIAN)");
    }
    for (size_t i = 0; i < sizeof(o.reserved) / sizeof(o.reserved[0]); ++i)
        if (o.reserved[i] != 0) return fail(CG_ERR_ARG, "reserved option fields must be zero");

    auto* p = new cg_plan_s();
    p->fs = fs;
    p->N = N;
    p->T = T;
    p->opts = o;
    p->bins.resize(T);
    p->x.resize(T);
    p->ref.assign(T, 1.0);
    for (int k = 0; k < T; ++k) {
        const double f = tooth_freqs[k];
        if (!std::isfinite(f)) { delete p; return fail(CG_ERR_ARG, "tooth_freqs[%d] is not finite", k); }
        const double pos = std::fabs(f) * static_cast<double>(N) / fs;
        if (pos > 1e15) { delete p; return fail(CG_ERR_TOOTH_RANGE, "tooth %d far beyond the sample rate", k); }
        long long b = static_cast<long long>(std::floor(pos + 0.5)) % N;
        if (b > N / 2) b = N - b;
        p->bins[k] = static_cast<int>(b);
        p->x[k] = tooth_x ? tooth_x[k] : f;
        if (!std::isfinite(p->x[k])) { delete p; return fail(CG_ERR_ARG, "tooth_x[%d] is not finite", k); }
        if (ref) {
            if (!(ref[k] > 0.0) || !std::isfinite(ref[k])) { delete p; return fail(CG_ERR_ARG, "ref_spectrum[%d] must be > 0", k); }
            p->ref[k] = ref[k];
        }
    }
    for (int i = 0; i < T; ++i)
        for (int j = i + 1; j < T; ++j)
            if (p->bins[i] == p->bins[j]) ++p->n_collisions;

    // abscissa normalisation u = (x - x_mid) / x_scale, x_scale = mean spacing
    const double xmin = *std::min_element(p->x.begin(), p->x.end());
    const double xmax = *std::max_element(p->x.begin(), p->x.end());
    if (!(xmax > xmin)) { delete p; return fail(CG_ERR_ARG, "tooth_x values must not all be equal"); }
    p->x_mid = 0.5 * (xmin + xmax);
    p->x_scale = (xmax - xmin) / static_cast<double>(T - 1);
    std::vector<float> u(T);
    for (int k = 0; k < T; ++k) u[k] = static_cast<float>((p->x[k] - p->x_mid) / p->x_scale);
    p->u_mid = 0.0f;
    p->du = 1.0f;
    p->span = static_cast<float>(T - 1);
    // outer fifth of the teeth by distance from the span midpoint (ties kept)
    {
        std::vector<double> dist(T);
        for (int k = 0; k < T; ++k) dist[k] = std::fabs(p->x[k] - p->x_mid);
        std::vector<double> s = dist;
        std::sort(s.begin(), s.end());
        const int no = (T + 4) / 5;
        const double thr = s[T - no];
        std::vector<int> idx;
        for (int k = 0; k < T; ++k)
            if (dist[k] >= thr) idx.push_back(k);
        p->n_outer = static_cast<int>(idx.size());
        cudaError_t e = cudaGetDevice(&p->device);
        if (e != cudaSuccess) { delete p; return cuda_fail(e, "cudaGetDevice"); }
        e = upload(&p->d.outer_idx, idx);
        if (e != cudaSuccess) { free_tables(p->d); delete p; return cuda_fail(e, "outer index upload"); }
    }
    cudaError_t e = cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device);
    if (e != cudaSuccess) { free_tables(p->d); delete p; return cuda_fail(e, "SM count"); }

    choose_fft(p);
    if (p->radices.empty()) {
        free_tables(p->d);
        delete p;
        return fail(CG_ERR_UNSUPPORTED, "frame_len %d: transform length is not a product of 2,3,5,7,11,13", N);
    }
    // the fused / split kernels take groups of 4..32 lanes (1 and 2 exist only
    // in the pipelined fit)
    p->G = o.lanes_per_frame >= 4 ? o.lanes_per_frame : 8;

    // twiddles (FP64 on the host, rounded to FP32)
    const int L = p->L, M = p->M;
    std::vector<float2> twL(L), twM(std::max(M, 1)), twn1(L), twb(T);
    for (int m = 0; m < L; ++m) {
        const double a = -kTwoPi * static_cast<double>(m) / L;
        twL[m] = make_float2(static_cast<float>(std::cos(a)), static_cast<float>(std::sin(a)));
    }
    std::vector<int> zidx(T);
    if (p->kind == CG_FFT_COSET) {
        for (int n2 = 0; n2 < M; ++n2) {
            const double a = -kTwoPi * static_cast<double>((static_cast<long long>(p->r0) * n2) % M) / M;
            twM[n2] = make_float2(static_cast<float>(std::cos(a)), static_cast<float>(std::sin(a)));
        }
        for (int n1 = 0; n1 < L; ++n1) {
            const double a = -kTwoPi * static_cast<double>((static_cast<long long>(p->r0) * n1) % N) / N;
            twn1[n1] = make_float2(static_cast<float>(std::cos(a)), static_cast<float>(std::sin(a)));
        }
        for (int k = 0; k < T; ++k) {
            const int b = p->bins[k];
            int m;
            if (((b - p->r0) % M + M) % M == 0) m = (b - p->r0) / M;
            else m = (N - b - p->r0) / M;   // conjugate-symmetric partner N - b
            zidx[k] = ((m % L) + L) % L;
        }
    } else {
        for (int k = 0; k < T; ++k) {
            const int b = p->bins[k];
            const double a = -kTwoPi * static_cast<double>(b) / N;
            twb[k] = make_float2(static_cast<float>(std::cos(a)), static_cast<float>(std::sin(a)));
            zidx[k] = b;
        }
    }

    // batch size and shared-memory layout
    cg::ReadoutArgs& ra = p->ra;
    ra.N = N;
    ra.T = T;
    ra.L = L;
    ra.M = M;
    ra.r0 = p->r0;
    ra.kind = p->kind;
    ra.nst = static_cast<int>(p->radices.size());
    for (int s = 0; s < cg::kMaxStages; ++s) ra.radix[s] = s < ra.nst ? p->radices[s] : 1;
    ra.fstride = L;
    ra.ystride = T;
    int tables = 0;
    ra.sm_twL = tables; tables = align16(tables + 8 * L);
    ra.sm_twM = tables; tables = align16(tables + 8 * std::max(M, 1));
    ra.sm_twn1 = tables; tables = align16(tables + 8 * L);
    ra.sm_twb = tables; tables = align16(tables + 8 * T);
    ra.sm_zidx = tables; tables = align16(tables + 4 * T);
    ra.sm_iref = tables; tables = align16(tables + 4 * T);
    ra.sm_u = tables; tables = align16(tables + 4 * T);
    ra.sm_acc = tables; tables = align16(tables + 8 * T);
    const int per_frame = 2 * N + 2 * 8 * ra.fstride + 4 * ra.ystride;
    const int budget = 100 * 1024;
    int F = (budget - tables) / per_frame;
    F = std::max(1, std::min(F, 64));
    ra.F = F;
    p->F = F;
    ra.sm_raw = tables;
    int off = align16(tables + 2 * N * F + 32);
    ra.sm_a = off; off = align16(off + 8 * ra.fstride * F);
    ra.sm_b = off; off = align16(off + 8 * ra.fstride * F);
    ra.sm_y = off; off = align16(off + 4 * ra.ystride * F);
    ra.sm_total = off;
    if (ra.sm_total > 227 * 1024) {
        free_tables(p->d);
        delete p;
        return fail(CG_ERR_UNSUPPORTED, "frame_len %d needs %d bytes of shared memory", N, ra.sm_total);
    }

    std::vector<float> iref = inv_ref_of(p->ref);
    if ((e = upload(&p->d.tw_L, twL)) != cudaSuccess || (e = upload(&p->d.tw_M, twM)) != cudaSuccess ||
        (e = upload(&p->d.tw_n1, twn1)) != cudaSuccess || (e = upload(&p->d.tw_b, twb)) != cudaSuccess ||
        (e = upload(&p->d.zidx, zidx)) != cudaSuccess || (e = upload(&p->d.inv_ref, iref)) != cudaSuccess ||
        (e = upload(&p->d.u, u)) != cudaSuccess) {
        free_tables(p->d);
        delete p;
        return cuda_fail(e, "table upload");
    }
    ra.tw_L = p->d.tw_L;
    ra.tw_M = p->d.tw_M;
    ra.tw_n1 = p->d.tw_n1;
    ra.tw_b = p->d.tw_b;
    ra.zidx = p->d.zidx;
    ra.inv_ref = p->d.inv_ref;
    ra.u = p->d.u;

    if ((e = cg::configure_kernels(p)) != cudaSuccess) {
        free_tables(p->d);
        delete p;
        return cuda_fail(e, "kernel configuration");
    }
    p->d.ref_part_rows = p->grid_readout;
    if ((e = cudaMalloc(&p->d.ref_part, sizeof(double) * static_cast<size_t>(p->d.ref_part_rows) * T)) != cudaSuccess ||
        (e = cudaMalloc(&p->d.ref_out, sizeof(double) * T)) != cudaSuccess) {
        free_tables(p->d);
        delete p;
        return cuda_fail(e, "reference scratch");
    }
    p->solve_f64 = (o.solve_f64 == -1) ? (o.readout == CG_READOUT_GEMM_SPLIT ? 1 : 0) : o.solve_f64;
    if (o.readout == CG_READOUT_GEMM_SPLIT) {
        p->gemm_split_x = (o.sample_bits == 12) ? 0 : 1;
        if ((e = cg::setup_gemm(p)) != cudaSuccess) {
            free_plan(p);
            return cuda_fail(e, "tensor-core readout set-up");
        }
    }
    if ((e = setup_fit_kernels(p)) != cudaSuccess) {
        free_plan(p);
        return cuda_fail(e, "fit kernel set-up");
    }
    if (o.readout == CG_READOUT_GEMM_SPLIT && !p->fit_ok) {
        free_plan(p);
        return fail(CG_ERR_UNSUPPORTED, "n_teeth %d: no fit kernel for the tensor-core readout", T);
    }
    if ((e = setup_fast(p, zidx)) != cudaSuccess) {
        free_plan(p);
        return cuda_fail(e, "throughput path set-up");
    }
    if ((e = cg::setup_pow2(p)) != cudaSuccess) {
        free_plan(p);
        return cuda_fail(e, "power-of-two readout set-up");
    }
    if (o.readout == CG_READOUT_FOLD_GEMM) {
        if ((e = cg::setup_fold(p, zidx)) != cudaSuccess) {
            free_plan(p);
            return cuda_fail(e, "folded tensor-core readout set-up");
        }
        if (!p->fold_ok || !p->fit_ok) {
            free_plan(p);
            return fail(CG_ERR_UNSUPPORTED,
                        "the folded tensor-core readout needs a radix-10 coset geometry with even L = N / 10, "
                        "n_teeth <= 128 and the fit kernels");
        }
    }
    if (o.model == CG_MODEL_FANO && !p->fit_ok) {
        free_plan(p);
        return fail(CG_ERR_UNSUPPORTED, "no Fano fit kernel for this n_teeth and lanes_per_frame");
    }
    if (o.init == CG_INIT_MEDIAN) {
        // the median-filter guess writes x_k + shift (the Fano profile's
        // minimum lies q gamma below its centre)
        const double shift = o.model == CG_MODEL_FANO ? o.fano_q * o.fano_gamma : 0.0;
        std::vector<float> cx(T);
        for (int k = 0; k < T; ++k) cx[k] = static_cast<float>(p->x[k] + shift);
        if ((e = upload(&p->d.median_cx, cx)) != cudaSuccess || (e = cg::setup_median(p)) != cudaSuccess) {
            free_plan(p);
            return cuda_fail(e, "median-filter initial guess set-up");
        }
        if (!p->median_ok || !p->fit_ok) {
            free_plan(p);
            return fail(CG_ERR_UNSUPPORTED, "the median-filter initial guess needs the fit kernels");
        }
    }
    if (o.init == CG_INIT_MLP && (!p->fit_ok || T > 256)) {
        free_plan(p);
        return fail(CG_ERR_UNSUPPORTED, "the learned initial guess needs the fit kernels and n_teeth <= 256");
    }
    // the allocation-free reference entry point's set-up (address lookup and
    // module loads), so that its calls neither allocate nor load anything
    if ((e = cg::bind_noalloc_scratch(p)) != cudaSuccess || (e = cg::preload_reference_kernels(p)) != cudaSuccess) {
        free_plan(p);
        return cuda_fail(e, "allocation-free scratch set-up");
    }
    *out = p;
    return CG_OK;
}

void cg_plan_destroy(cg_plan_t p)
{
    if (!p) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(p->device);
    cudaDeviceSynchronize();
    free_plan(p);
    cudaSetDevice(prev);
}

cg_status cg_plan_describe(cg_plan_t p, cg_plan_info* info, int* bins_host)
{
    if (!p || !info) return fail(CG_ERR_ARG, "plan or info is NULL");
    std::memset(info, 0, sizeof(*info));
    info->frame_len = p->N;
    info->n_teeth = p->T;
    info->fft_kind = p->kind;
    info->coset_modulus = p->M;
    info->coset_residue = p->r0;
    info->fft_len = p->L;
    info->n_radices = static_cast<int>(p->radices.size());
    for (int i = 0; i < info->n_radices && i < 8; ++i) info->radices[i] = p->radices[i];
    info->frames_per_cta = p->F;
    info->lanes_per_frame = p->G;
    info->n_collisions = p->n_collisions;
    info->path = (p->opts.path == CG_PATH_AUTO) ? (p->fit_ok ? CG_PATH_PIPELINE : CG_PATH_FUSED)
               : (p->opts.path == CG_PATH_PIPELINE && !p->fit_ok) ? CG_PATH_FUSED : p->opts.path;
    if (p->opts.readout != CG_READOUT_FFT || p->opts.init != CG_INIT_MOMENT || p->opts.model == CG_MODEL_FANO)
        info->path = CG_PATH_PIPELINE;
    if (info->path == CG_PATH_PIPELINE) info->lanes_per_frame = p->fit3_ok ? p->fit3_G : p->G2;
    if (bins_host) std::memcpy(bins_host, p->bins.data(), sizeof(int) * p->T);
    return CG_OK;
}

cg_status cg_set_reference(cg_plan_t p, const double* ref)
{
    if (!p || !ref) return fail(CG_ERR_ARG, "plan or ref is NULL");
    for (int k = 0; k < p->T; ++k)
        if (!(ref[k] > 0.0) || !std::isfinite(ref[k])) return fail(CG_ERR_ARG, "ref_spectrum[%d] must be > 0", k);
    p->ref.assign(ref, ref + p->T);
    std::vector<float> iref = inv_ref_of(p->ref);
    cudaError_t e = cudaMemcpy(p->d.inv_ref, iref.data(), sizeof(float) * p->T, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "reference upload");
    return CG_OK;
}

static cg_status check_frames(const cg_plan_s* p, const int16_t* frames, int64_t n)
{
    if (!p) return fail(CG_ERR_ARG, "plan is NULL");
    if (n < 0) return fail(CG_ERR_ARG, "n_frames < 0");
    if (n > 0 && !frames) return fail(CG_ERR_ARG, "frames_dev is NULL");
    if (reinterpret_cast<uintptr_t>(frames) & 1) return fail(CG_ERR_ARG, "frames_dev must be 2-byte aligned");
    if (n > (int64_t(1) << 40) / p->N) return fail(CG_ERR_ARG, "n_frames too large");
    return CG_OK;
}

static cg_status check_frames_i8(const cg_plan_s* p, const int8_t* frames, int64_t n)
{
    if (!p) return fail(CG_ERR_ARG, "plan is NULL");
    if (n < 0) return fail(CG_ERR_ARG, "n_frames < 0");
    if (n > 0 && !frames) return fail(CG_ERR_ARG, "frames_dev is NULL");
    if (n > (int64_t(1) << 40) / p->N) return fail(CG_ERR_ARG, "n_frames too large");
    if (!p->fast_i8_ok || p->opts.readout != CG_READOUT_FFT)
        return fail(CG_ERR_UNSUPPORTED,
                    "8-bit samples are read out by the pruned comb transform only (N = 2200 with every tooth "
                    "bin at +-r mod 10, readout CG_READOUT_FFT)");
    return CG_OK;
}

// The whole path for int16 (sbytes = 2) or int8 (sbytes = 1) frames.
static cg_status process_impl(cg_plan_t p, const void* frames, int sbytes, int64_t n, float* amps, float* y,
                              float* params, float* rss, int16_t* iters, int16_t* status, void* stream)
{
    if (n == 0) return CG_OK;
    if (!amps || !params) return fail(CG_ERR_ARG, "amps_dev and params_dev are required");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    const bool gemm = p->opts.readout == CG_READOUT_GEMM_SPLIT;
    const bool mlp = p->opts.init == CG_INIT_MLP;
    // both comb readouts read sample pairs as 32-bit words (frames 4-byte
    // aligned); otherwise the pipeline reads out with the general transform
    const bool aligned4 = !(reinterpret_cast<uintptr_t>(frames) & 3);
    const int16_t* frames16 = static_cast<const int16_t*>(frames);   // the non-pipeline paths (int16 only)
    const bool fold = p->opts.readout == CG_READOUT_FOLD_GEMM && p->fold_ok && aligned4;
    if (mlp && !p->mlp_ok) return fail(CG_ERR_STATE, "init is CG_INIT_MLP but no network is loaded (cg_mlp_load)");
    int path = p->opts.path;
    if (path == CG_PATH_AUTO) path = p->fit_ok ? CG_PATH_PIPELINE : CG_PATH_FUSED;
    if (path == CG_PATH_PIPELINE && !p->fit_ok) path = CG_PATH_FUSED;
    // tensor-core readouts or learned guess: readout, then guess and fit kernels
    const bool fano = p->opts.model == CG_MODEL_FANO;
    const bool median = p->opts.init == CG_INIT_MEDIAN;
    if (p->opts.readout != CG_READOUT_FFT || mlp || sbytes == 1 || fano || median) path = CG_PATH_PIPELINE;
    const bool fast = !gemm && !fold && p->fast_ok && aligned4;
    const bool pow2 = !gemm && !fold && !fast && p->pow2_ok && aligned4;
    if (path == CG_PATH_PIPELINE) {
        const int64_t cmax = n < p->chunk ? n : p->chunk;
        if (mlp && p->d.fb_cap < cmax) {
            // frames left by the polish of one chunk (grows, never shrinks)
            cudaFree(p->d.fb_list);
            p->d.fb_list = nullptr;
            p->d.fb_cap = 0;
            if ((e = cudaMalloc(&p->d.fb_list, sizeof(int) * cmax)) != cudaSuccess) return cuda_fail(e, "fallback list");
            if (!p->d.fb_count && (e = cudaMalloc(&p->d.fb_count, sizeof(int))) != cudaSuccess)
                return cuda_fail(e, "fallback count");
            p->d.fb_cap = cmax;
        }
        // fork onto the plan's two streams; chunk c is read out (and its
        // initial guess made) on s_read while chunk c-1 is fitted on s_fit; the
        // guess goes to params and its flag to status, where the fit reads them
        e = cudaEventRecord(p->ev_fork, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(p->s_read, p->ev_fork, 0);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(p->s_fit, p->ev_fork, 0);
        // the median filter runs over the call's whole time x tooth image
        const int64_t chunk = median ? n : p->chunk;
        for (int64_t c0 = 0; c0 < n && e == cudaSuccess; c0 += chunk) {
            const int64_t m = (n - c0) < chunk ? (n - c0) : chunk;
            const int64_t T = p->T;
            const char* fb = static_cast<const char*>(frames) + c0 * p->N * sbytes;
            const int16_t* fc = reinterpret_cast<const int16_t*>(fb);
            float* ac = amps + c0 * T;
            float* yc = y ? y + c0 * T : nullptr;
            float* pc = params + c0 * 4;
            float* rc = rss ? rss + c0 : nullptr;
            int16_t* ic = iters ? iters + c0 : nullptr;
            int16_t* sc = status ? status + c0 : nullptr;
            e = timed(p, CG_STAGE_READOUT, p->s_read, [&] {
                if (sbytes == 1)
                    return cg::launch_fast_readout_i8(p, reinterpret_cast<const int8_t*>(fb), m, ac, yc, p->s_read);
                return gemm   ? cg::launch_gemm_readout(p, fc, m, ac, yc, p->s_read)
                       : fold ? cg::launch_fold_readout(p, fc, m, ac, yc, p->s_read)
                       : fast ? cg::launch_fast_readout(p, fc, m, ac, yc, p->s_read)
                       : pow2 ? cg::launch_pow2_readout(p, fc, m, ac, yc, p->s_read)
                              : cg::launch_readout(p, fc, m, ac, yc, p->s_read);
            });
            if (e == cudaSuccess && mlp)
                e = timed(p, CG_STAGE_MLP, p->s_read, [&] { return cg::launch_mlp(p, yc, ac, m, pc, sc, p->s_read); });
            else if (e == cudaSuccess && !fano)
                e = timed(p, CG_STAGE_INIT, p->s_read,
                          [&] { return cg::launch_init(p, yc, ac, m, pc, sc, p->s_read, nullptr, nullptr); });
            if (e == cudaSuccess && median)   // the centre of the guess from the filtered image
                e = timed(p, CG_STAGE_MEDIAN, p->s_read,
                          [&] { return cg::launch_median(p, yc, ac, m, pc, p->s_read); });
            if (e == cudaSuccess) e = cudaEventRecord(p->ev_read, p->s_read);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(p->s_fit, p->ev_read, 0);
            if (e == cudaSuccess && mlp) {
                // polish steps from the learned guess; frames that do not
                // converge are listed and refit by the full LM from the moment
                // guess
                cg::FitLaunch pol;
                pol.max_iter = p->opts.polish_iter < p->opts.max_iter ? p->opts.polish_iter : p->opts.max_iter;
                pol.fb_list = p->d.fb_list;
                pol.fb_count = p->d.fb_count;
                e = cudaMemsetAsync(p->d.fb_count, 0, sizeof(int), p->s_fit);
                if (e == cudaSuccess)
                    e = timed(p, CG_STAGE_FIT, p->s_fit, [&] {
                        return cg::launch_fit2(p, yc, ac, m, pc, sc, pc, rc, ic, sc, p->s_fit, pol);
                    });
                if (e == cudaSuccess)
                    e = timed(p, CG_STAGE_FALLBACK, p->s_fit, [&] {
                        return cg::launch_init(p, yc, ac, m, pc, sc, p->s_fit, p->d.fb_list, p->d.fb_count);
                    });
                cg::FitLaunch fb;
                fb.list = p->d.fb_list;
                fb.list_n = p->d.fb_count;
                fb.iters_base = pol.max_iter;
                fb.status_or = CG_FIT_FALLBACK;
                if (e == cudaSuccess)
                    e = timed(p, CG_STAGE_FALLBACK, p->s_fit, [&] {
                        return cg::launch_fit2(p, yc, ac, m, pc, sc, pc, rc, ic, sc, p->s_fit, fb);
                    });
            } else if (e == cudaSuccess) {
                // the Fano fit reads a given centre only from the median filter
                const float* p0 = (fano && !median) ? nullptr : pc;
                const int16_t* fl = fano ? nullptr : sc;
                e = timed(p, CG_STAGE_FIT, p->s_fit,
                          [&] { return cg::launch_fit2(p, yc, ac, m, p0, fl, pc, rc, ic, sc, p->s_fit); });
            }
        }
        if (e == cudaSuccess) e = cudaEventRecord(p->ev_join_r, p->s_read);
        if (e == cudaSuccess) e = cudaEventRecord(p->ev_join_f, p->s_fit);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, p->ev_join_r, 0);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, p->ev_join_f, 0);
    } else if (path == CG_PATH_FUSED) {
        e = timed(p, CG_STAGE_FUSED, s,
                  [&] { return cg::launch_fused(p, frames16, n, amps, y, params, rss, iters, status, s); });
    } else {
        e = timed(p, CG_STAGE_READOUT, s, [&] { return cg::launch_readout(p, frames16, n, amps, y, s); });
        // without y_dev the fit reads the magnitudes and applies the reference itself
        if (e == cudaSuccess)
            e = timed(p, CG_STAGE_FIT, s,
                      [&] { return cg::launch_fit(p, y, amps, n, nullptr, params, rss, iters, status, s); });
    }
    if (e != cudaSuccess) return cuda_fail(e, "cg_process launch");
    return CG_OK;
}

cg_status cg_process(cg_plan_t p, const int16_t* frames, int64_t n, float* amps, float* y,
                     float* params, float* rss, int16_t* iters, int16_t* status, void* stream)
{
    cg_status st = check_frames(p, frames, n);
    if (st != CG_OK) return st;
    return process_impl(p, frames, 2, n, amps, y, params, rss, iters, status, stream);
}

cg_status cg_process_i8(cg_plan_t p, const int8_t* frames, int64_t n, float* amps, float* y,
                        float* params, float* rss, int16_t* iters, int16_t* status, void* stream)
{
    cg_status st = check_frames_i8(p, frames, n);
    if (st != CG_OK) return st;
    return process_impl(p, frames, 1, n, amps, y, params, rss, iters, status, stream);
}

cg_status cg_readout_i8(cg_plan_t p, const int8_t* frames, int64_t n, float* amps, float* y, void* stream)
{
    cg_status st = check_frames_i8(p, frames, n);
    if (st != CG_OK) return st;
    if (n == 0) return CG_OK;
    if (!amps && !y) return fail(CG_ERR_ARG, "amps_dev and y_dev are both NULL");
    const cudaError_t e = cg::launch_fast_readout_i8(p, frames, n, amps, y, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "cg_readout_i8 launch");
    return CG_OK;
}

cg_status cg_readout(cg_plan_t p, const int16_t* frames, int64_t n, float* amps, float* y, void* stream)
{
    cg_status st = check_frames(p, frames, n);
    if (st != CG_OK) return st;
    if (n == 0) return CG_OK;
    if (!amps && !y) return fail(CG_ERR_ARG, "amps_dev and y_dev are both NULL");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    const bool aligned4 = !(reinterpret_cast<uintptr_t>(frames) & 3);
    if (p->opts.readout == CG_READOUT_GEMM_SPLIT)
        e = cg::launch_gemm_readout(p, frames, n, amps, y, s);
    else if (p->opts.readout == CG_READOUT_FOLD_GEMM && p->fold_ok && aligned4)
        e = cg::launch_fold_readout(p, frames, n, amps, y, s);
    else if (p->fast_ok && (p->opts.path == CG_PATH_AUTO || p->opts.path == CG_PATH_PIPELINE) && aligned4)
        e = cg::launch_fast_readout(p, frames, n, amps, y, s);
    else if (p->pow2_ok && (p->opts.path == CG_PATH_AUTO || p->opts.path == CG_PATH_PIPELINE) && aligned4)
        e = cg::launch_pow2_readout(p, frames, n, amps, y, s);
    else
        e = cg::launch_readout(p, frames, n, amps, y, s);
    if (e != cudaSuccess) return cuda_fail(e, "cg_readout launch");
    return CG_OK;
}

cg_status cg_fit(cg_plan_t p, const float* y, int64_t n, const float* p0, float* params, float* rss,
                 int16_t* iters, int16_t* status, void* stream)
{
    if (!p) return fail(CG_ERR_ARG, "plan is NULL");
    if (n < 0) return fail(CG_ERR_ARG, "n < 0");
    if (n == 0) return CG_OK;
    if (!y || !params) return fail(CG_ERR_ARG, "y_dev and params_dev are required");
    cudaError_t e = cudaSuccess;
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool fano = p->opts.model == CG_MODEL_FANO;
    if (p->opts.init == CG_INIT_MEDIAN && !p0) {
        // guess in params (Lorentzian: moments, then the filtered centre), then the fit from it
        if (!fano) e = cg::launch_init(p, y, nullptr, n, params, status, s, nullptr, nullptr);
        if (e == cudaSuccess) e = cg::launch_median(p, y, nullptr, n, params, s);
        if (e == cudaSuccess)
            e = cg::launch_fit2(p, y, nullptr, n, params, fano ? nullptr : status, params, rss, iters, status, s);
    } else if (fano) {   // the Fano fit makes its own guess; p0 is not read
        e = cg::launch_fit2(p, y, nullptr, n, nullptr, nullptr, params, rss, iters, status, s);
    } else {
        e = cg::launch_fit(p, y, nullptr, n, p0, params, rss, iters, status, s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "cg_fit launch");
    return CG_OK;
}

cg_status cg_reference_accumulate(cg_plan_t p, const int16_t* frames, int64_t n, double* ref_host,
                                  void* stream)
{
    cg_status st = check_frames(p, frames, n);
    if (st != CG_OK) return st;
    if (n < 1) return fail(CG_ERR_ARG, "need at least one reference frame");
    if (!ref_host) return fail(CG_ERR_ARG, "ref_host is NULL");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cg::launch_reference(p, frames, n, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ref_host, p->d.ref_out, sizeof(double) * p->T, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "cg_reference_accumulate");
    return CG_OK;
}

}  // extern "C"

extern "C" cg_status cg_check_device(cg_plan_t p)
{
    if (!p) return fail(CG_ERR_ARG, "plan is NULL");
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != p->device) cudaSetDevice(p->device);
    cudaError_t e = cudaDeviceSynchronize();
    int word = 0;
    if (e == cudaSuccess && p->d.err) e = cudaMemcpy(&word, p->d.err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && word != 0) e = cudaMemset(p->d.err, 0, sizeof(int));
    if (prev >= 0 && prev != p->device) cudaSetDevice(prev);
    if (e != cudaSuccess) return cuda_fail(e, "cg_check_device");
    if (word != 0) return fail(CG_ERR_DEVICE_CHECK, "a kernel's bounded wait ran out (code %d)", word);
    return CG_OK;
}

extern "C" cg_status cg_mlp_load(cg_plan_t p, const void* blob, size_t bytes)
{
    if (!p || !blob) return fail(CG_ERR_ARG, "plan or blob is NULL");
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != p->device) cudaSetDevice(p->device);
    cudaError_t e = cudaDeviceSynchronize();
    const char* why = nullptr;
    if (e == cudaSuccess) e = cg::setup_mlp(p, static_cast<const unsigned char*>(blob), bytes, &why);
    if (prev >= 0 && prev != p->device) cudaSetDevice(prev);
    if (why) {
        p->mlp_ok = false;
        return fail(e == cudaErrorInvalidValue ? CG_ERR_ARG : CG_ERR_CUDA, "cg_mlp_load: %s", why);
    }
    if (e != cudaSuccess) {
        p->mlp_ok = false;
        return cuda_fail(e, "cg_mlp_load");
    }
    return CG_OK;
}

extern "C" cg_status cg_mlp_infer(cg_plan_t p, const float* y, int64_t n, float* p0, void* stream)
{
    if (!p) return fail(CG_ERR_ARG, "plan is NULL");
    if (n < 0) return fail(CG_ERR_ARG, "n < 0");
    if (!p->mlp_ok) return fail(CG_ERR_STATE, "no network is loaded (cg_mlp_load)");
    if (n == 0) return CG_OK;
    if (!y || !p0) return fail(CG_ERR_ARG, "y_dev and p0_dev are required");
    cudaError_t e = cg::launch_mlp(p, y, nullptr, n, p0, nullptr, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "cg_mlp_infer launch");
    return CG_OK;
}

extern "C" cg_status cg_timing_enable(cg_plan_t p, int enable)
{
    if (!p) return fail(CG_ERR_ARG, "plan is NULL");
    p->timing = enable != 0;
    return CG_OK;
}

extern "C" cg_status cg_timing_collect(cg_plan_t p, double* ms, int64_t* launches)
{
    if (!p) return fail(CG_ERR_ARG, "plan is NULL");
    double acc[CG_N_STAGES] = {0};
    int64_t cnt[CG_N_STAGES] = {0};
    cudaError_t e = cudaSuccess;
    for (const auto& t : p->timed) {
        if (e == cudaSuccess) e = cudaEventSynchronize(t.b);
        float v = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&v, t.a, t.b);
        if (e == cudaSuccess && t.stage >= 0 && t.stage < CG_N_STAGES) {
            acc[t.stage] += v;
            cnt[t.stage] += 1;
        }
        p->ev_pool.push_back(t.a);
        p->ev_pool.push_back(t.b);
    }
    p->timed.clear();
    if (e != cudaSuccess) return cuda_fail(e, "cg_timing_collect");
    for (int i = 0; i < CG_N_STAGES; ++i) {
        if (ms) ms[i] = acc[i];
        if (launches) launches[i] = cnt[i];
    }
    return CG_OK;
}
