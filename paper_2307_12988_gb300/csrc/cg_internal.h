// cg_internal.h -- plan layout and kernel argument blocks shared by the
// library's translation units (not part of the public ABI).
#pragma once
#include <cstdint>
#include <string>
#include <vector>
#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/combgpu.h"
#include "cg_fit.cuh"

namespace cg {

constexpr int kMaxStages = 8;
constexpr int kMinN = 8;
constexpr int kMaxN = 16384;
constexpr int kMinT = 5;
constexpr int kMaxT = 1024;
constexpr int kThreads = 256;

// Arguments of the readout kernels (cast -> shared-memory FFT -> tooth read).
struct ReadoutArgs {
    const int16_t* frames;
    int64_t n_frames;
    int N, T, L, M, r0, kind, nst;
    int radix[kMaxStages];
    int F;            // frames per batch of one thread block
    int fstride;      // complex elements per frame in the work buffers
    int ystride;      // floats per frame of the shared normalised spectra
    const float2* tw_L;    // [L]  W_L^m
    const float2* tw_M;    // [M]  W_M^{r n2}        (coset)
    const float2* tw_n1;   // [L]  W_N^{r n1}        (coset)
    const float2* tw_b;    // [T]  W_N^{b_k}         (full)
    const int* zidx;       // [T]  coset: m_k; full: b_k
    const float* inv_ref;  // [T]
    const float* u;        // [T]  normalised abscissa (fused fit)
    float* amps;           // [n][T] or null
    float* y;              // [n][T] or null
    double* ref_part;      // reference mode: per-block partial sums [grid][T]
    // shared-memory layout (byte offsets)
    int sm_twL, sm_twM, sm_twn1, sm_twb, sm_zidx, sm_iref, sm_u;
    int sm_raw, sm_a, sm_b, sm_y, sm_acc, sm_total;
};

// Arguments of the fast readout (comb geometries, N = 10 P Q).
struct FastArgs {
    const void* frames;      // int16 or int8 samples (the kernel's instantiation)
    int64_t n_frames;
    int N, T, F;
    int pair_isign;          // (-1)^r: sign pairing x_j with x_{j+5} in the fold
    const float2* twL;       // [L]  W_L^m
    const float2* twN;       // [L]  W_N^{r n1}
    const float2* twM;       // [5]  W_10^{r j}
    const int* tooth_of_m;   // [L]  tooth reading Z[m], or -1
    const float* inv_ref;    // [T]
    const float* u;          // [T]
    float* amps;             // [n][T] or null
    float* y;                // [n][T] or null
    int sm_twL, sm_twN, sm_tom, sm_iref, sm_u, sm_raw, sm_Y, sm_amps, sm_y, sm_total;
};

// Arguments of the lane-per-frame moment initial guess.
struct InitArgs {
    int64_t n;
    int T;
    int row_stride;          // odd row stride of the staged spectra
    int n_outer;
    const float* y;          // [n][T] normalised, or null
    const float* amps;       // [n][T] magnitudes when y is null
    const float* inv_ref;    // [T]
    const float* u;          // [T]
    const int* outer_idx;    // [n_outer]
    float u_mid, du, span, x_mid, x_scale;
    float* p0_out;           // [n][4] abscissa units
    int16_t* flag_out;       // [n] or null
    const int* list;         // task i is frame list[i] (fallback pass), or null
    const int* list_n;       // device count of list entries, or null
    int bulk;                // 1: whole 32-row tasks arrive by bulk copies (T odd)
    int* err;                // device error word (a bulk copy that never landed)
};

// Arguments of the register-resident LM kernel.
struct Fit2Args {
    int64_t n;
    int T;
    int task;                // frames per warp task
    int row_stride;          // odd stride of the lane-per-frame spectrum slots
    int solve_f64;           // 1: the 4x4 normal equations are solved in FP64
    unsigned long long* counter;  // next task (zeroed before the launch)
    const float* y;          // [n][T] normalised, or null
    const float* amps;       // [n][T] magnitudes when y is null
    const float* inv_ref;    // [T]
    const float* u;          // [T]
    const float* p0;         // [n][4] starting parameters (abscissa units)
    const int16_t* flags_in; // [n] initial-guess flags or null
    float x_mid, x_scale;
    int max_iter;
    float tol, lambda0;
    float* params;
    float* rss;
    int16_t* iters;
    int16_t* status;
    // learned-guess polish and its fallback
    const int* list;         // task i is frame list[i], or null (task i is frame i)
    const int* list_n;       // device count of list entries (read at start), or null
    int* fb_list;            // frames that end without converging are appended, or null
    int* fb_count;
    int iters_base;          // added to the reported iteration count
    int status_or;           // OR-ed into the reported status
    // the Fano lineshape (model 1), on the normalised abscissa: asymmetry q,
    // width g (fixed), the lowest-tooth shift q g, the boxes of A and B and
    // their averages (the starting values)
    float fano_q, fano_g, fano_inv_g, fano_shift;
    float fano_A0, fano_B0, fano_Alo, fano_Ahi, fano_Blo, fano_Bhi;
    // rows of the y / amps buffer (the shared-memory kernel's copies stay inside it)
    int64_t n_rows;
    int* err;                // device error word (a row copy that never landed)
};

// Arguments of the learned initial-guess inference kernel (cg_mlp_tc.cu).
struct MlpArgs {
    const float* y;          // [n][T] normalised, or null
    const float* amps;       // [n][T] magnitudes when y is null
    const float* inv_ref;    // [T]
    int64_t n;
    int T, nkb;              // teeth, K blocks of 64 of the first layer
    const float* tab;        // FP32 tables at the kMlpTab* offsets
    float x_mid, g_lo, g_hi; // fallback centre; clamp of |g| (abscissa units)
    float* p0;               // [n][4]
    int16_t* flags;          // [n] or null
    int stages;
    int* err;
};
constexpr char kMlpMagic[9] = "CGMLP001";
constexpr int kMlpHeaderBytes = 24;
constexpr int kMlpTabB1 = 0, kMlpTabB2 = 256, kMlpTabW3 = 512, kMlpTabB3 = 1536, kMlpTabOutMean = 1540,
              kMlpTabOutScale = 1544, kMlpTabIn = 1548;

// Arguments of the split-precision DFT-at-teeth GEMM readout.
struct GemmArgs {
    const int16_t* frames;
    int64_t n;
    int N, T;
    int nkb;                 // K blocks of 64 samples
    int ntile;               // output columns per tile (2 per tooth), multiple of 16
    int n_ctiles;            // column tiles (block b: frame tile b / n_ctiles, column tile b % n_ctiles)
    int nrows_total;         // rows of one (hi or lo) half of the twiddle matrix
    int tmem_cols;           // TMEM columns allocated per block (n_acc * acc_cols)
    int acc_cols;            // columns of one accumulator
    int n_acc;               // accumulators the K blocks alternate over
    int stages;              // pipeline depth
    int vec8;                // frames 8-byte aligned and N % 4 == 0
    const float* inv_ref;
    float* amps;
    float* y;
    int* err;                // set to nonzero by a block whose bounded wait ran out
};

// Arguments of the folded DFT-at-teeth readout on the tensor cores
// (cg_fold_gemm.cu): the radix-10 coset fold on the CUDA cores, then the
// L-point DFT at the teeth as a split-precision product on the tensor cores.
struct FoldArgs {
    const int16_t* frames;
    int64_t n;
    int N, T, L;
    int nkb;                 // K blocks of 32 FP16 elements (16 fold outputs, Re/Im)
    int ntile;               // output columns (2 per tooth), multiple of 16, <= 256
    int acc_stride;          // TMEM columns between the two accumulators
    int tmem_cols;           // TMEM columns allocated per block
    int stages;              // A ring stages
    float c1, s1, c2, s2;    // W_10^(r j) for j = 1, 2
    float z_scale;           // fold outputs are scaled by this power of two before FP16
    float out_scale;         // 1 / z_scale, applied to |X|
    const float2* twN;       // [L] W_N^(r m)
    const float* inv_ref;    // [T]
    float* amps;             // [n][T] or null
    float* y;                // [n][T] or null
    int* err;
    // shared-memory layout (byte offsets from the 1024-byte-aligned base)
    int sm_W, sm_A, sm_stage, sm_tw, sm_iref, sm_bar, sm_total;
};

// Arguments of the median-filter initial centre (cg_median.cu).
struct MedianArgs {
    const float* y;          // [n][T] or null (then amps x inv_ref)
    const float* amps;       // [n][T]
    const float* inv_ref;    // [T]
    const float* cx;         // [T] x_k + shift, abscissa units
    float* params;           // [n][4]: c0 into column 0
    int64_t n;
    int T, S, R;             // teeth, shared row stride ((T + 6) | 1), rows per block
    int sm_key, sm_raw, sm_total;   // shared-memory layout
};

struct DevTables {
    void* gemm_W = nullptr;       // [2][rows][Kpad] FP16 twiddles (hi, lo)
    void* fold_W = nullptr;       // [2][ntile][Kpad] FP16 twiddles of the folded readout
    int* err = nullptr;           // device-side error word
    float2* tw_M5 = nullptr;
    int* tooth_of_m = nullptr;
    float2* tw_L = nullptr;
    float2* tw_M = nullptr;
    float2* tw_n1 = nullptr;
    float2* tw_b = nullptr;
    int* zidx = nullptr;
    float* inv_ref = nullptr;
    float* u = nullptr;
    int* outer_idx = nullptr;
    double* ref_part = nullptr;   // [ref_part_rows][T]
    double* ref_out = nullptr;    // [T]
    int ref_part_rows = 0;
    unsigned long long* fit_counter = nullptr;   // dynamic task counter of the fit kernels
    void* mlp_W = nullptr;        // [512][256] BF16 weights of the learned guess
    float* mlp_tab = nullptr;     // its FP32 tables
    int* fb_list = nullptr;       // [fb_cap] frames left by the polish
    int* fb_count = nullptr;      // [1]
    int64_t fb_cap = 0;
    float* median_cx = nullptr;   // [T] x_k + shift of the median-filter guess
};

}  // namespace cg

struct cg_plan_s {
    int device = 0;
    int num_sms = 0;
    double fs = 0;
    int N = 0, T = 0;
    cg_opts opts{};
    std::vector<int> bins;
    std::vector<double> x, ref;
    double x_mid = 0, x_scale = 1;
    int kind = CG_FFT_FULL, M = 2, r0 = 0, L = 0;
    std::vector<int> radices;
    int F = 1;               // frames per batch
    int G = 8;               // lanes per frame
    int n_collisions = 0;
    int n_outer = 0;
    float u_mid = 0, du = 1, span = 1;
    cg::DevTables d;
    int grid_readout = 0, grid_fused = 0, grid_fit = 0;
    cg::ReadoutArgs ra{};
    // throughput path (fast readout + register-resident LM over chunks)
    bool fit_ok = false;     // init + fit kernels of the throughput path configured
    bool fast_ok = false;    // geometry admits the fast readout
    bool fast_i8_ok = false; // ... and an int8 instantiation exists for it
    cg::FastArgs fa8{};      // its batch size and layout
    int grid_fast8 = 0;
    // split-precision GEMM readout
    CUtensorMap gemm_map{};
    int gemm_split_x = 1, gemm_smem = 0, gemm_ntiles = 0;
    bool median_ok = false;  // median-filter initial centre configured
    cg::MedianArgs med{};
    int grid_median = 0;
    bool pow2_ok = false;    // power-of-two full-transform readout configured
    cg::ReadoutArgs pa{};
    int grid_pow2 = 0;
    bool fold_ok = false;    // folded tensor-core readout configured
    CUtensorMap fold_map{};
    cg::FoldArgs fo{};
    int grid_fold = 0;
    int fold_sign = 1;       // (-1)^r of the coset fold
    bool gemm_ring = false;  // decoupled-ring kernel (12-bit samples, NT <= 256)
    int gemm_halves = 1, gemm_ring_stages = 0, gemm_ring_smem = 0;
    int solve_f64 = 0;
    cg::GemmArgs ga{};
    int Q = 0;               // L = 10 Q
    bool fit3_ok = false;    // shared-memory LM kernel (cg_fit3.cu) configured
    int fit3_G = 0, fit3_warps = 0, fit3_smem = 0, grid_fit3 = 0;
    int G2 = 4;              // LM lanes per frame of the register-resident fit
    int PPL = 0;             // LM points per lane
    bool ppl_exact = false;  // PPL == ceil(T / G2)
    int grid_fast = 0, grid_fit2 = 0, grid_init = 0;
    int init_npad = 0, init_smem = 0;
    cg::InitArgs ia{};
    int64_t chunk = 0;       // frames per pipelined chunk
    cg::FastArgs fa{};
    cudaStream_t s_read = nullptr, s_fit = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_read = nullptr, ev_join_r = nullptr, ev_join_f = nullptr;
    // learned initial guess
    bool mlp_ok = false;
    CUtensorMap mlp_map{};
    int mlp_smem = 0;
    cg::MlpArgs ma{};
    // device address of the allocation-free reference scratch (set by cg_plan)
    double* noalloc_scratch = nullptr;
    // per-kernel timing
    bool timing = false;
    struct TimedLaunch {
        int stage;
        cudaEvent_t a, b;
    };
    std::vector<TimedLaunch> timed;
    std::vector<cudaEvent_t> ev_pool;
};

namespace cg {

// launchers (cg_kernels.cu)
cudaError_t configure_kernels(cg_plan_s* p);
cudaError_t launch_readout(const cg_plan_s* p, const int16_t* frames, int64_t n, float* amps,
                           float* y, cudaStream_t s);
cudaError_t launch_fused(const cg_plan_s* p, const int16_t* frames, int64_t n, float* amps,
                         float* y, float* params, float* rss, int16_t* iters, int16_t* status,
                         cudaStream_t s);
cudaError_t launch_fit(const cg_plan_s* p, const float* y, const float* amps, int64_t n,
                       const float* p0, float* params, float* rss, int16_t* iters,
                       int16_t* status, cudaStream_t s);
cudaError_t launch_reference(const cg_plan_s* p, const int16_t* frames, int64_t n, cudaStream_t s);
// reference accumulation with caller-chosen scratch (max_rows partial rows of
// T doubles) and output (T doubles), both device memory
cudaError_t launch_reference_into(const cg_plan_s* p, const int16_t* frames, int64_t n,
                                  double* part, int max_rows, double* out, cudaStream_t s);
// loads the reference-accumulation kernels of the plan's lane count (no launch)
cudaError_t preload_reference_kernels(const cg_plan_s* p);
// looks up the allocation-free scratch array on the plan's device (which must
// be current) and keeps its address in the plan
cudaError_t bind_noalloc_scratch(cg_plan_s* p);

FitArgs make_fit_args(const cg_plan_s* p);

// throughput path (cg_fast.cu)
void* fast_readout_ptr(int Q, int sample_bytes = 2);
void* init_ptr(int npad, int n_outer);
int init_npad(int n_outer);
void* fit2_ptr(int G, int PPL, bool exact, int model);
int fit2_ppl(int G, int T, bool* exact, int model);
int fit2_threads(int G);
void* fit1_ptr();   // lane-per-frame LM kernel (cg_fit1.cu)
size_t fit2_smem(int G, int T, int model);
cudaError_t launch_fast_readout_i8(const cg_plan_s* p, const int8_t* frames, int64_t n, float* amps, float* y,
                                   cudaStream_t s);
cudaError_t launch_fast_readout(const cg_plan_s* p, const int16_t* frames, int64_t n, float* amps,
                                float* y, cudaStream_t s);
// options of a fit launch beyond the plan's: polish cap, frame list, fallback list
struct FitLaunch {
    int max_iter = -1;           // -1: the plan's
    const int* list = nullptr;
    const int* list_n = nullptr;
    int* fb_list = nullptr;
    int* fb_count = nullptr;
    int iters_base = 0;
    int status_or = 0;
};
cudaError_t launch_init(const cg_plan_s* p, const float* y, const float* amps, int64_t n,
                        float* p0_out, int16_t* flag_out, cudaStream_t s, const int* list,
                        const int* list_n);
cudaError_t launch_fit2(const cg_plan_s* p, const float* y, const float* amps, int64_t n,
                        const float* p0, const int16_t* flags_in, float* params, float* rss,
                        int16_t* iters, int16_t* status, cudaStream_t s,
                        const FitLaunch& fl = FitLaunch());
// the shared-memory LM kernel: set-up at plan creation, launch with the
// arguments launch_fit2 prepared
cudaError_t setup_fit3(cg_plan_s* p);
cudaError_t launch_fit3(const cg_plan_s* p, Fit2Args a, cudaStream_t s);

// learned initial guess (cg_mlp_tc.cu)
cudaError_t setup_mlp(cg_plan_s* p, const unsigned char* blob, size_t bytes, const char** why);
cudaError_t launch_mlp(const cg_plan_s* p, const float* y, const float* amps, int64_t n, float* p0,
                       int16_t* flags, cudaStream_t s);

// power-of-two full-transform readout (cg_pow2.cu)
cudaError_t setup_median(cg_plan_s* p);
cudaError_t launch_median(const cg_plan_s* p, const float* y, const float* amps, int64_t n, float* params,
                          cudaStream_t s);
cudaError_t setup_pow2(cg_plan_s* p);
cudaError_t launch_pow2_readout(const cg_plan_s* p, const int16_t* frames, int64_t n, float* amps, float* y,
                                cudaStream_t s);

// folded DFT-at-teeth readout on the tensor cores (cg_fold_gemm.cu)
cudaError_t setup_fold(cg_plan_s* p, const std::vector<int>& zidx);
cudaError_t launch_fold_readout(const cg_plan_s* p, const int16_t* frames, int64_t n, float* amps, float* y,
                                cudaStream_t s);

// split-precision GEMM readout (cg_gemm.cu)
cudaError_t setup_gemm(cg_plan_s* p);
cudaError_t launch_gemm_readout(const cg_plan_s* p, const int16_t* frames, int64_t n, float* amps, float* y,
                                cudaStream_t s);

// sets the thread-local text returned by cg_last_error()
void set_last_error(const char* msg);

// Raises (never lowers) a kernel's dynamic shared-memory limit.  The limit
// belongs to the function on the device, so every plan shares it: one plan
// must not shrink what another plan's launches need.
cudaError_t raise_smem_limit(const void* fn, int bytes);

}  // namespace cg
