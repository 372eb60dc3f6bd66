/*
 * combgpu.h -- C ABI of the GB300 comb-spectrum readout and fitting library.
 *
 * The library turns digitised self-heterodyne comb interferograms into fitted
 * cavity parameters, following arXiv 2307.12988 ("Data Capture and
 * Processing"): integer samples are cast to floating point on the GPU, each
 * frame is Fourier transformed, the comb-tooth bins are read out, divided by
 * an averaged reference spectrum, and each normalised spectrum is fit by
 * Levenberg-Marquardt.  The paper fits a Fano line with gpufit; this library
 * fits the 4-parameter Lorentzian cavity mode
 *     m(x) = B + A g^2 / ((x - c)^2 + g^2),   p = (c, g, A, B),
 * g being the half width at half maximum, in the units of the tooth abscissa.
 *
 * Conventions shared by every entry point:
 *   - Every call returns a cg_status; no exception or signal crosses the ABI.
 *     cg_last_error() gives a thread-local description of the last failure.
 *   - Pointers named *_dev are CUDA device pointers owned by the caller; the
 *     library never frees or retains them after the call returns.  Pointers
 *     named *_host are host memory, read or written before the call returns
 *     unless stated otherwise.
 *   - Work is enqueued asynchronously on the caller's CUDA stream
 *     (`cuda_stream`, a cudaStream_t; NULL = the legacy default stream).
 *   - A plan belongs to the device that was current when it was made; use it
 *     from one host thread at a time.
 *   - Arrays are row-major: frames [n][N] int16, per-tooth outputs [n][T],
 *     parameters [n][4] in the order (c, g, A, B).
 */
#ifndef COMBGPU_H
#define COMBGPU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CG_VERSION 100

typedef enum cg_status {
    CG_OK = 0,
    CG_ERR_ARG = 1,           /* invalid argument (NULL, size, alignment) */
    CG_ERR_CUDA = 2,          /* a CUDA runtime call failed */
    CG_ERR_NOMEM = 3,         /* device or host allocation failed */
    CG_ERR_TOOTH_RANGE = 4,   /* a tooth lies outside [0, fs/2] after aliasing rules */
    CG_ERR_OVERFLOW = 5,      /* streaming ring overflowed (frames dropped) */
    CG_ERR_TIMEOUT = 6,       /* a bounded wait ran out */
    CG_ERR_DEVICE_CHECK = 7,  /* a kernel's own check failed */
    CG_ERR_UNSUPPORTED = 8,   /* geometry or option not supported */
    CG_ERR_STATE = 9          /* call not valid in the object's current state */
} cg_status;

/* Per-frame fit outcome, written to status_dev (int16). */
#define CG_FIT_CONVERGED 0    /* a trial step changed chi^2 by <= tol * chi^2 */
#define CG_FIT_MAX_ITER 1     /* max_iter trial steps without convergence */
#define CG_FIT_SINGULAR 2     /* J^T J not positive definite */
#define CG_FIT_NONFINITE 3    /* the spectrum or chi^2 at the start is not finite */
#define CG_FIT_INIT_FLAT 0x10 /* flag: moment initial guess saw a flat spectrum */
#define CG_FIT_FALLBACK 0x20  /* flag: the learned initial guess and its polish steps
                                 did not converge; the frame was refit by the full LM
                                 from the moment initial guess */

/* Tooth readout.  FFT: the pruned (coset) or general shared-memory transform
   on the CUDA cores.  GEMM_SPLIT: X at the tooth bins as one dense product
   [frames x N] . [N x 2 teeth] on the tensor cores (FP16 samples, FP16 hi + lo
   twiddles, FP32 accumulation).  FOLD_GEMM: radix-10 coset geometries only
   (N = 10 L, L even, every tooth bin = +-r mod 10, at most 128 teeth): each
   frame is folded to L complex values on the CUDA cores, then the L-point DFT
   at the teeth is a split-precision (hi + lo) product on the tensor cores;
   frames that are not 4-byte aligned are read out by the general transform. */
enum { CG_READOUT_FFT = 0, CG_READOUT_GEMM_SPLIT = 1, CG_READOUT_FOLD_GEMM = 2 };
enum { CG_FFT_AUTO = 0, CG_FFT_FULL = 1, CG_FFT_COSET = 2 };
/* Initial guess.  MOMENT: moments of the spectrum (Lorentzian) or the
   lowest tooth (Fano).  MLP: the learned network (Lorentzian only).  MEDIAN
   (the paper's, "Data Capture and Processing"): the frames of one
   cg_process / cg_fit call form a time x tooth image (teeth in plan order);
   a 7x7 median filter with mirrored edges (index -1 -> 0, n -> n - 1) is
   applied and the lowest filtered value of each row gives the centre (first
   tooth on ties; plus q gamma for the Fano profile); the Lorentzian's other
   parameters come from the moments.  A MEDIAN call is processed as one
   chunk (chunk_frames is ignored), since every row's filter reads three
   rows on either side. */
enum { CG_INIT_MOMENT = 0, CG_INIT_MLP = 1, CG_INIT_MEDIAN = 2 };
/* Fitted lineshape.  LORENTZ: m = B + A g^2 / ((x - c)^2 + g^2), all four
   parameters free.  FANO (the paper's fit, "Data Capture and Processing"):
   m = B + A (q + e)^2 / (1 + e^2), e = (x - c) / gamma, with the centre c
   free, the scale A and offset B held to fano_box (e.g. 0.1 = +-10 %) around
   the pre-computed averages fano_A, fano_B, the asymmetry q and width gamma
   fixed.  Bounds: A or B on a bound with the gradient pointing outward is
   held out of that LM step (active set), the others take the reduced step,
   and the trial point is clamped onto the box.  The initial centre
   is the lowest tooth moved by q gamma (where the profile's minimum lies).
   params_dev then holds (c, gamma, A, B).  A Fano plan refuses init =
   CG_INIT_MLP (CG_ERR_UNSUPPORTED), runs its fit in two or more lanes per
   frame, and cg_plan fails with CG_ERR_UNSUPPORTED when no Fano kernel
   covers n_teeth at the requested lanes_per_frame. */
enum { CG_MODEL_LORENTZ = 0, CG_MODEL_FANO = 1 };
/* Kernel arrangement of cg_process. */
enum {
    CG_PATH_AUTO = 0,      /* PIPELINE when the fit kernels cover n_teeth, else FUSED */
    CG_PATH_FUSED = 1,     /* one kernel: readout and fit per thread block */
    CG_PATH_SPLIT = 2,     /* a readout kernel, then a fit kernel */
    CG_PATH_PIPELINE = 3   /* readout kernel (the pruned comb transform when the
                              geometry admits it and the frames are 4-byte
                              aligned, else the general transform), then the
                              initial-guess and fit kernels, over chunks on two
                              plan-owned streams */
};

/* Options of a plan.  Fill with cg_opts_default() and change what you need. */
typedef struct cg_opts {
    int readout;          /* CG_READOUT_FFT (default), CG_READOUT_GEMM_SPLIT or
                             CG_READOUT_FOLD_GEMM */
    int fft;              /* CG_FFT_AUTO: coset-pruned transform when every tooth bin
                             lies in one residue pair +-r mod M (M | N), else full */
    int init;             /* CG_INIT_MOMENT (default), CG_INIT_MLP or CG_INIT_MEDIAN */
    int max_iter;         /* LM trial steps per frame; paper: 20 */
    double tol;           /* relative chi^2 change for convergence; paper: 1e-6 */
    double lambda0;       /* initial Marquardt damping; 1e-3 */
    int lanes_per_frame;  /* LM lanes cooperating on one frame: 4, 8, 16 or 32
                             (32 = one warp per frame); 0 = library default */
    int path;             /* CG_PATH_* (default CG_PATH_AUTO) */
    int chunk_frames;     /* frames per pipelined chunk; 0 = the whole call */
    int sample_bits;      /* GEMM readout: 12 = samples lie in [-2048, 2047] and are
                             exact in FP16 (two products per step); 16 (default) =
                             full int16, split into 256 hi + lo (four products) */
    int solve_f64;        /* -1 (default): FP64 4x4 LM solve with the GEMM readout,
                             FP32 otherwise; 0: FP32; 1: FP64 */
    int polish_iter;      /* CG_INIT_MLP: LM trial steps from the learned initial
                             guess before a frame falls back to the full LM from
                             the moment guess; 0 = 2 */
    int model;            /* CG_MODEL_LORENTZ (default) or CG_MODEL_FANO (pipeline
                             path, moment-free: the Fano fit makes its own guess) */
    int reserved[3];      /* must be zero */
    double fano_q;        /* CG_MODEL_FANO: asymmetry q (fixed) */
    double fano_gamma;    /* CG_MODEL_FANO: width gamma in abscissa units (fixed, > 0) */
    double fano_A;        /* CG_MODEL_FANO: average scale A (box centre, != 0) */
    double fano_B;        /* CG_MODEL_FANO: average offset B (box centre) */
    double fano_box;      /* CG_MODEL_FANO: relative half-width of the A and B boxes (>= 0) */
} cg_opts;

typedef struct cg_plan_s* cg_plan_t;

/* Summary of what a plan decided (for logging and tests). */
typedef struct cg_plan_info {
    int frame_len;        /* N */
    int n_teeth;          /* T */
    int fft_kind;         /* CG_FFT_FULL or CG_FFT_COSET */
    int coset_modulus;    /* M (coset transform) or 2 (full real transform) */
    int coset_residue;    /* r (coset transform) */
    int fft_len;          /* complex transform length L = N / M */
    int n_radices;        /* number of shared-memory FFT stages */
    int radices[8];
    int frames_per_cta;   /* frames one thread block transforms at a time */
    int lanes_per_frame;  /* LM lanes per frame */
    int n_collisions;     /* pairs of teeth that read the same bin */
    int path;             /* CG_PATH_* that cg_process takes for aligned frames */
} cg_plan_info;

/* Fill *opts with the defaults (FFT readout, moment init, 20 iterations,
 * tol 1e-6, lambda0 1e-3, CG_PATH_AUTO).  opts must not be NULL. */
void cg_opts_default(cg_opts* opts);

/*
 * cg_plan -- precompute everything that depends on the instrument geometry
 * (paper, "Data Capture and Processing": frames of N samples, tooth bins
 * "selected and mapped" into the optical spectrum, a pre-calculated average
 * reference spectrum).
 *   sample_rate   digitiser rate fs in Hz (> 0)
 *   frame_len     N samples per frame, 8 <= N <= 16384
 *   n_teeth       T teeth read out, 5 <= T <= 1024
 *   tooth_freqs   host [T]: signed RF frequency of each tooth in Hz; its bin is
 *                 floor(|f| N / fs + 1/2) reduced mod N and folded into [0, N/2]
 *   tooth_x       host [T] or NULL: fit abscissa of each tooth (e.g. optical
 *                 offset in Hz); NULL uses tooth_freqs
 *   ref_spectrum  host [T] or NULL: mean |X| of cavity-free frames per tooth
 *                 (must be > 0); NULL means 1 (y equals the raw magnitudes)
 *   opts          NULL for defaults
 * All host arrays are copied.  On success *plan owns device memory until
 * cg_plan_destroy.  Errors: CG_ERR_ARG, CG_ERR_UNSUPPORTED (N not a product of
 * radices 2,3,5,7,11,13), CG_ERR_NOMEM, CG_ERR_CUDA.
 */
cg_status cg_plan(cg_plan_t* plan, double sample_rate, int frame_len, int n_teeth,
                  const double* tooth_freqs, const double* tooth_x,
                  const double* ref_spectrum, const cg_opts* opts);

/* Release a plan (NULL is ignored).  Synchronises the plan's device first. */
void cg_plan_destroy(cg_plan_t plan);

/* Describe a plan; bins_host (may be NULL) receives the T folded bins. */
cg_status cg_plan_describe(cg_plan_t plan, cg_plan_info* info, int* bins_host);

/* Replace the reference spectrum (host [T], every value > 0). */
cg_status cg_set_reference(cg_plan_t plan, const double* ref_spectrum);

/*
 * cg_process -- the whole per-frame path on n_frames frames resident on the
 * device: cast, transform, tooth readout, normalisation, initial guess and
 * LM fit (paper, "Data Capture and Processing", both paragraphs on the fit).
 *   frames_dev   int16 [n_frames][N], 2-byte aligned (16-byte alignment is
 *                faster); samples are read as signed integers
 *   amps_dev     float [n_frames][T]: |X_b| at each tooth (required)
 *   y_dev        float [n_frames][T] or NULL: amps / reference
 *   params_dev   float [n_frames][4]: (c, g, A, B), g >= 0, abscissa units
 *   rss_dev      float [n_frames] or NULL: sum of squared residuals of y
 *   iters_dev    int16 [n_frames] or NULL: LM trial steps taken
 *   status_dev   int16 [n_frames] or NULL: CG_FIT_* outcome | flags
 * n_frames == 0 is a no-op.  Asynchronous on cuda_stream.
 */
cg_status cg_process(cg_plan_t plan, const int16_t* frames_dev, int64_t n_frames,
                     float* amps_dev, float* y_dev, float* params_dev, float* rss_dev,
                     int16_t* iters_dev, int16_t* status_dev, void* cuda_stream);

/*
 * cg_readout -- only the cast, transform and tooth readout (with
 * normalisation when y_dev is not NULL) of cg_process.
 */
cg_status cg_readout(cg_plan_t plan, const int16_t* frames_dev, int64_t n_frames,
                     float* amps_dev, float* y_dev, void* cuda_stream);

/*
 * cg_process_i8, cg_readout_i8 -- the same with 8-bit samples (int8, two's
 * complement; the paper's digitiser format: "Experimental Setup", 8-bit at
 * 2.2 GS/s).  frames_dev is int8 [n_frames][frame_len], any byte alignment.
 * Supported where the pruned comb readout applies to an 8-bit frame of
 * N = 2200 samples (every tooth bin at +-r mod 10, L = 220), with readout
 * CG_READOUT_FFT; otherwise CG_ERR_UNSUPPORTED.  Results equal, bit for bit,
 * those of cg_process / cg_readout on the same samples widened to int16.
 * The path is always CG_PATH_PIPELINE.
 */
cg_status cg_process_i8(cg_plan_t plan, const int8_t* frames_dev, int64_t n_frames,
                        float* amps_dev, float* y_dev, float* params_dev, float* rss_dev,
                        int16_t* iters_dev, int16_t* status_dev, void* cuda_stream);
cg_status cg_readout_i8(cg_plan_t plan, const int8_t* frames_dev, int64_t n_frames,
                        float* amps_dev, float* y_dev, void* cuda_stream);

/*
 * cg_fit -- only the initial guess and LM fit of cg_process, on normalised
 * spectra y_dev float [n][T].  p0_dev float [n][4] (abscissa units) or NULL
 * for the plan's initial guess: the moments (CG_INIT_MOMENT), or the median
 * filter over the call's n spectra as one time x tooth image
 * (CG_INIT_MEDIAN); with CG_MODEL_FANO p0_dev is not read (the lowest tooth,
 * or the median filter's centre).  Outputs as in cg_process.
 */
cg_status cg_fit(cg_plan_t plan, const float* y_dev, int64_t n, const float* p0_dev,
                 float* params_dev, float* rss_dev, int16_t* iters_dev,
                 int16_t* status_dev, void* cuda_stream);

/*
 * cg_reference_accumulate -- the averaged cavity-free reference spectrum that
 * each spectrum is divided by ("Data Capture and Processing"; recorded once,
 * before the measurement): ref_host[k] = mean over the n cavity-free
 * frames of |X_{b_k}|, accumulated in FP64 on the device.  Blocks until the
 * result is in ref_host (double [T]).  Does not change the plan's reference.
 */
cg_status cg_reference_accumulate(cg_plan_t plan, const int16_t* frames_dev, int64_t n,
                                  double* ref_host, void* cuda_stream);

/*
 * cg_reference_accumulate_noalloc -- the same average as
 * cg_reference_accumulate, for callers that cannot allocate device memory at
 * the moment they need it: a real-time acquisition loop that must never
 * wait on the allocator, a process whose device memory is held by a pool it
 * does not own, or a host application that lends the library only a stream
 * and buffers.  The paper has no counterpart; this is a convenience of the
 * library's interface.
 *   frames_dev  int16 [n][N] cavity-free frames in device memory of the
 *               plan's device, n >= 1
 *   ref_dev     double [n_teeth] in device memory of the plan's device,
 *               8-byte aligned: receives mean |X_{b_k}| (the caller owns it)
 * Allocates nothing and calls no allocating routine.  Its scratch is one array
 * of 32768 doubles (256 KiB) compiled into the library, present on every GPU
 * that loads it until the process exits; each call uses at most
 * floor(32768 / n_teeth) thread blocks, and a plan whose n_teeth exceeds
 * 32768 would be rejected with CG_ERR_ARG.  Every call shares that array:
 * two calls whose work overlaps on the GPU (other streams, other threads)
 * race and give wrong results, so serialise them.  Each call writes every
 * scratch value it reads, so nothing needs clearing between calls.  The
 * set-up is done by cg_plan, which may allocate: with the plan's device
 * current it looks up the array's device address (cudaGetSymbolAddress),
 * which also loads the array onto the device, loads the accumulation
 * kernels, and keeps the address in the plan; this entry point only reads
 * it.  Pointers that are not device memory of the plan's device are
 * refused (CG_ERR_ARG) before any launch.  Asynchronous on cuda_stream;
 * errors: CG_ERR_ARG, CG_ERR_UNSUPPORTED, CG_ERR_CUDA.
 */
cg_status cg_reference_accumulate_noalloc(cg_plan_t plan, const int16_t* frames_dev,
                                          int64_t n, double* ref_dev, void* cuda_stream);

/*
 * cg_check_device -- synchronise the plan's device and report (then clear)
 * the plan's device-side error word.  Kernels never trap: a kernel whose
 * bounded wait on a pipeline barrier runs out records the event there,
 * unwinds and leaves its outputs unwritten.  Returns CG_OK or
 * CG_ERR_DEVICE_CHECK (or CG_ERR_CUDA if the synchronisation fails).
 */
cg_status cg_check_device(cg_plan_t plan);

/*
 * Per-kernel timing (diagnostics).  While enabled, cg_process records a pair
 * of CUDA events around every kernel it launches, on the stream it launches
 * that kernel on.  cg_timing_collect waits for the recorded events, returns
 * the summed milliseconds and launch counts per stage since the last collect
 * (ms_host, launches_host: arrays of CG_N_STAGES, either may be NULL) and
 * forgets them.  Enabling costs two event records per launch.
 */
enum {
    CG_STAGE_READOUT = 0,   /* cast + transform + tooth readout (FFT or GEMM) */
    CG_STAGE_INIT = 1,      /* moment initial guess */
    CG_STAGE_MLP = 2,       /* learned initial guess */
    CG_STAGE_FIT = 3,       /* LM (full, or the polish steps after the MLP) */
    CG_STAGE_FALLBACK = 4,  /* moment guess + full LM of frames the polish left */
    CG_STAGE_FUSED = 5,     /* single-kernel path */
    CG_STAGE_MEDIAN = 6,    /* median-filter initial centre */
    CG_N_STAGES = 8
};
cg_status cg_timing_enable(cg_plan_t plan, int enable);
cg_status cg_timing_collect(cg_plan_t plan, double* ms_host, int64_t* launches_host);

/*
 * cg_fp32_peak -- measured FP32 fused multiply-add throughput of the current
 * device, the denominator of the LM kernels' ALU roofline (a diagnostic; the
 * paper has no counterpart).  Launches, on cuda_stream, one warm-up and then
 * reps timed launches of a kernel whose threads each run 16 independent
 * chains a <- a m + c (packed = 1: 8 chains of FP32x2 pairs, one instruction
 * per two fused multiply-adds), 4 blocks of 256 threads per SM, and writes
 * 2 x fused multiply-adds / elapsed time (CUDA events) to *tflops_host in
 * TFLOP/s.  Blocks until done.  Allocates no device memory.  Errors:
 * CG_ERR_ARG (packed not 0 or 1, reps < 1, NULL output), CG_ERR_CUDA.
 */
cg_status cg_fp32_peak(int packed, int reps, double* tflops_host, void* cuda_stream);

/*
 * ---- Learned initial guess -------------------------------------------------
 * A multilayer perceptron n_in -> H -> H -> n_out with tanh-form GELU hidden
 * activations (z/2 (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3)))) and a linear
 * output maps a normalised spectrum to the LM starting point, so that the LM
 * only polishes (the paper notes that the iteration count depends on the
 * initial parameters; it seeds them from filtered data instead).
 *
 * Training object (cg_mlp_t): FP32 master parameters, gradients and Adam
 * moments on the current device, trained by the library's own kernels.  Flat
 * parameter order: W1 [H][n_in], b1 [H], W2 [H][H], b2 [H], W3 [n_out][H],
 * b3 [n_out], row-major.  Inputs and targets given to the training calls are
 * already standardised by the caller; the standardisation vectors travel in
 * the saved blob and are applied by cg_mlp_load's inference kernel.
 */
typedef struct cg_mlp_s* cg_mlp_t;

/* Number of parameters of an (n_in, n_hidden, n_out) network. */
int64_t cg_mlp_param_count(int n_in, int n_hidden, int n_out);

/*
 * cg_mlp_create -- allocate a network for batches of up to max_batch rows.
 * 1 <= n_in, n_hidden <= 1024; 1 <= n_out <= 16; 1 <= max_batch <= 1<<20.
 * Weights are drawn uniformly from +-1/sqrt(fan_in) by a counter-based hash
 * (SplitMix64) of (seed, parameter index); biases are zero; Adam state zero.
 */
cg_status cg_mlp_create(cg_mlp_t* mlp, int n_in, int n_hidden, int n_out, int max_batch,
                        uint64_t seed);
void cg_mlp_destroy(cg_mlp_t mlp);

/* Copy the parameters to / from host float [count]; count must equal
 * cg_mlp_param_count.  set_params also clears the Adam state. Synchronous.
 * get_params (and cg_mlp_save) return CG_ERR_TIMEOUT when a matrix-product
 * block of an earlier asynchronous call gave up a bounded wait (its outputs,
 * and everything computed from them, are then invalid); the flag is cleared. */
cg_status cg_mlp_get_params(cg_mlp_t mlp, float* params_host, int64_t count);
cg_status cg_mlp_set_params(cg_mlp_t mlp, const float* params_host, int64_t count);

/* FP32 forward pass: x_dev float [n][n_in] -> out_dev float [n][n_out]
 * (any n >= 0; processed in slices of max_batch).  Asynchronous. */
cg_status cg_mlp_forward(cg_mlp_t mlp, const float* x_dev, int64_t n, float* out_dev,
                         void* cuda_stream);

/*
 * cg_mlp_backward -- loss L = mean over rows and outputs of (out - t)^2 and
 * its gradient for one batch (1 <= n <= max_batch): x_dev [n][n_in], t_dev
 * [n][n_out].  The gradient stays in the object for cg_mlp_adam; grad_dev
 * (float [param_count]) and loss_dev (float [1]) receive copies when not NULL.
 * Deterministic: no atomics, fixed summation order.  Asynchronous.
 */
cg_status cg_mlp_backward(cg_mlp_t mlp, const float* x_dev, const float* t_dev, int64_t n,
                          float* loss_dev, float* grad_dev, void* cuda_stream);

/* One Adam step (Kingma & Ba 2015) on the stored gradient, bias-corrected,
 * step counter kept in the object.  Asynchronous. */
cg_status cg_mlp_adam(cg_mlp_t mlp, float lr, float beta1, float beta2, float eps,
                      void* cuda_stream);

/*
 * cg_mlp_train_epoch -- minibatch loop on the device: for each batch b of
 * `batch` rows (the last may be shorter) gathers rows perm_dev[b*batch ...]
 * of x_dev / t_dev, runs cg_mlp_backward and cg_mlp_adam(lr, 0.9, 0.999,
 * 1e-8).  perm_dev int32 [n] (a permutation of 0..n-1 chosen by the caller;
 * an entry outside [0, n) contributes a zero row);
 * losses_dev float [ceil(n / batch)] or NULL receives each batch's loss.
 * 1 <= batch <= max_batch.  Asynchronous.
 */
cg_status cg_mlp_train_epoch(cg_mlp_t mlp, const float* x_dev, const float* t_dev, int64_t n,
                             const int32_t* perm_dev, int batch, float lr, float* losses_dev,
                             void* cuda_stream);

/* Standardisation stored with the network (host arrays): the network's input
 * is (y - in_mean) * in_scale, its output o maps to o * out_scale + out_mean. */
cg_status cg_mlp_set_norm(cg_mlp_t mlp, const float* in_mean, const float* in_scale,
                          const float* out_mean, const float* out_scale);

/*
 * cg_mlp_save -- serialise (synchronous) into blob_host of capacity bytes:
 * header "CGMLP001", int32 n_in, n_hidden, n_out, 0, then float in_mean[n_in],
 * in_scale[n_in], out_mean[n_out], out_scale[n_out], params[param_count],
 * little-endian.  *bytes_out receives the size (call with blob_host NULL to
 * ask for it).
 */
cg_status cg_mlp_save(cg_mlp_t mlp, void* blob_host, size_t capacity, size_t* bytes_out);

/*
 * cg_mlp_load -- give a plan the learned initial guess from a blob written by
 * cg_mlp_save.  The network must have n_in == n_teeth (inputs in the plan's
 * tooth order), n_hidden == 256, n_out == 4 with outputs (c, g, A, B) in
 * abscissa units.  Weights are stored on the device in BF16 for the
 * tensor-core inference kernel (FP32 accumulation); biases and the output
 * layer stay FP32.  Required before cg_process with init = CG_INIT_MLP.
 * Errors: CG_ERR_ARG (malformed blob, shape mismatch), CG_ERR_CUDA.
 */
cg_status cg_mlp_load(cg_plan_t plan, const void* blob_host, size_t bytes);

/*
 * cg_mlp_infer -- only the learned initial guess of cg_process: y_dev float
 * [n][T] normalised spectra -> p0_dev float [n][4] (c, g, A, B) in abscissa
 * units, g clamped to [dx/2, span/2] as the moment guess is.  Asynchronous.
 * CG_ERR_STATE if no network is loaded.
 */
cg_status cg_mlp_infer(cg_plan_t plan, const float* y_dev, int64_t n, float* p0_dev,
                       void* cuda_stream);

/*
 * ---- Streaming ---------------------------------------------------------------
 * The paper's acquisition loop ("Data Capture and Processing"): the digitiser
 * fills a ring buffer on the host while the GPU processes earlier batches;
 * batches finish out of order and are sorted back into time order; the
 * production rate must not exceed the consumption rate, or the ring
 * overflows.  Here a server (one scheduler thread per GPU) serves several
 * instrument streams, each with its own plan (geometry), pinned host ring and
 * result queue:
 *   - continuous batching: whenever a stream has a batch of frames waiting
 *     (or its oldest frame has waited max_delay) and one of its device batch
 *     buffers is free, the batch is copied to the device and processed on its
 *     own CUDA stream, overlapping other batches and other streams;
 *   - admission by device memory: a stream's batch buffers (frames, outputs)
 *     are granted from the server's budget; a stream that does not fit waits,
 *     with its ring still accepting frames, until memory is returned;
 *   - running averages on the device: FP64 means of y_k and of the fit
 *     parameters over consecutive windows of avg_window frames;
 *   - results are handed out in push order with their latency (result time
 *     minus arrival time), whose p50 / p99 the stream reports.
 * A frame's ring slot is reused only after its result has been polled, so a
 * consumer that does not keep up makes cg_stream_push overflow.
 * No call waits without a bound: every wait takes a timeout and returns
 * CG_ERR_TIMEOUT when it runs out.
 */
typedef struct cg_server_s* cg_server_t;
typedef struct cg_stream_s* cg_stream_t;

typedef struct cg_result {
    uint64_t seq;         /* sequence number: first_seq of its push + index */
    double t_arrival;     /* arrival time (cg_clock seconds) given at push */
    double t_done;        /* time its result became available to cg_stream_poll */
    float params[4];      /* (c, g, A, B) as cg_process */
    float rss;
    int16_t iters;
    int16_t status;
} cg_result;

typedef struct cg_stream_stats_t {
    int64_t frames_pushed;    /* accepted into the ring */
    int64_t frames_dropped;   /* rejected by cg_stream_push (overflow) */
    int64_t frames_done;      /* results produced */
    int64_t frames_polled;    /* results taken by cg_stream_poll */
    int64_t batches;          /* batches processed */
    double latency_p50_s;     /* over every result so far (1 % bins) */
    double latency_p99_s;
    double latency_max_s;
    double input_bytes_per_s; /* frame bytes processed / (last result - first push) */
    int admitted;             /* 1 once device memory was granted */
    int64_t window_index;     /* last completed running-average window, -1 if none */
    int64_t window_frames;    /* frames averaged in it (converged fits only) */
} cg_stream_stats_t;

/* Seconds on the library's monotonic clock (the time base of t_arrival). */
double cg_clock(void);

/*
 * cg_server_create -- scheduler for the current device.  device_budget_bytes
 * bounds the batch buffers of all its streams together (> 0).
 */
cg_status cg_server_create(cg_server_t* server, size_t device_budget_bytes);

/* Stop the scheduler (destroying any stream still open) and free everything. */
cg_status cg_server_destroy(cg_server_t server);

/*
 * Host-side fault injection for tests (no GPU fault is ever provoked):
 *   CG_INJECT_THROTTLE_S: the scheduler sleeps value seconds before each batch
 *                         launch (a consumer slower than the producer);
 *   CG_INJECT_HOLD:       value != 0 holds back every completed batch (a stalled
 *                         pipeline), 0 releases them;
 *   CG_INJECT_FAIL_LAUNCH: the next value batch launches fail as if the launch
 *                         call had returned an error; the stream enters its
 *                         error state (CG_ERR_CUDA).
 */
enum { CG_INJECT_THROTTLE_S = 1, CG_INJECT_HOLD = 2, CG_INJECT_FAIL_LAUNCH = 3 };
cg_status cg_server_inject(cg_server_t server, int what, double value);

/*
 * cg_stream_create -- an instrument stream on a server.
 *   plan          geometry and options (not owned; must outlive the stream and
 *                 is used only by the scheduler thread while the stream lives);
 *                 each batch is one cg_process call, so with CG_INIT_MEDIAN the
 *                 median filter's image is the batch
 *   ring_bytes    pinned host ring for the stream's frames (>= 2 batches)
 *   batch_frames  frames per batch (>= 1)
 *   max_delay_s   a partial batch is launched once its oldest frame has waited
 *                 this long (>= 0)
 *   avg_window    frames per running-average window (>= 1)
 * Admission needs 2 batch buffers within the server's remaining budget; up to
 * 4 are used when the budget allows.  Errors: CG_ERR_ARG, CG_ERR_NOMEM (pinned
 * ring), CG_ERR_UNSUPPORTED (2 batch buffers exceed the whole budget).
 */
cg_status cg_stream_create(cg_stream_t* stream, cg_server_t server, cg_plan_t plan,
                           size_t ring_bytes, int batch_frames, double max_delay_s,
                           int64_t avg_window);

/*
 * cg_stream_push -- copy n frames (host int16 [n][N]) into the ring.  If the
 * ring lacks room for all n, none is taken: CG_ERR_OVERFLOW, and the n frames
 * count as dropped.  t_arrival < 0 stamps cg_clock().  Thread-safe against
 * cg_stream_poll; one pushing thread per stream.
 */
cg_status cg_stream_push(cg_stream_t stream, const int16_t* frames_host, int64_t n,
                         uint64_t first_seq, double t_arrival);

/*
 * cg_stream_poll -- take up to cap results in push order: recs (host
 * cg_result [cap]) and, if amps_host is not NULL, their tooth magnitudes
 * (host float [cap][T]).  Waits up to timeout_s for the first result; *n_out
 * = 0 and CG_ERR_TIMEOUT if none came.  Returns the stream's error status if it
 * entered its error state.
 */
cg_status cg_stream_poll(cg_stream_t stream, cg_result* recs, float* amps_host, int64_t cap,
                         int64_t* n_out, double timeout_s);

/* Launch the frames still waiting and wait (up to timeout_s) until every
 * pushed frame has a result ready to poll. */
cg_status cg_stream_flush(cg_stream_t stream, double timeout_s);

cg_status cg_stream_stats(cg_stream_t stream, cg_stream_stats_t* stats);

/*
 * cg_stream_window -- means of the last completed running-average window:
 * mean_y_host double [T] (y = |X| / reference) and mean_params_host double [4],
 * over the window's frames whose fit converged.  *index = -1 if no window has
 * completed yet.  Any output pointer may be NULL.
 */
cg_status cg_stream_window(cg_stream_t stream, int64_t* index, int64_t* count,
                           double* mean_y_host, double* mean_params_host);

/* Wait (bounded) for the stream's batches, free its ring and buffers and
 * return its device memory to the server. */
cg_status cg_stream_destroy(cg_stream_t stream);

/* Text of a status code (static storage). */
const char* cg_status_string(cg_status status);

/* Thread-local description of the last failure on this thread ("" if none). */
const char* cg_last_error(void);

/* CG_VERSION of the loaded library. */
int cg_version(void);

/*
 * ---- Displacement PSD and mechanical resonance ---------------------------
 * Paper, "Experimental Results" and Fig. 6: the series of fitted cavity
 * positions is turned into a power spectral density for several averaging
 * times, and the accelerometer's mechanical resonance frequency f0 and
 * quality factor Q are fitted to it.
 *
 * cg_psd_create -- tables and scratch for Welch PSDs with segments of
 *   seg_len samples (4096, 8192, 16384 or 32768) on the current device.
 *   Errors: CG_ERR_ARG (seg_len), CG_ERR_NOMEM / CG_ERR_CUDA.
 * cg_psd_welch -- one-sided density of the series x_dev[i * stride],
 *   i < n (float, device memory; e.g. the centre column of cg_process's
 *   params with stride 4): segments of seg_len samples advanced by seg_len/2
 *   (only complete segments), segment mean removed, periodic Hann window
 *   w_n = 1/2 - 1/2 cos(2 pi n / seg_len), mean |rfft|^2 over the segments,
 *   doubled except at DC and seg_len/2, divided by fs sum w^2.  psd_dev:
 *   double [seg_len/2 + 1] (device), bin k at k fs / seg_len.  *n_segments
 *   (host, may be NULL) receives the number of segments.  Asynchronous on
 *   cuda_stream.  Errors: CG_ERR_ARG (NULL pointers, stride < 1, fs <= 0,
 *   n < seg_len).  The transform runs in FP32, the averages in FP64.
 * cg_resonance_fit -- fits S(f) = A f0^4 / ((f0^2 - f^2)^2 + (f f0/Q)^2) + B
 *   to ln psd over the bins k with f_lo <= k df <= f_hi (k >= 1; at least 8
 *   bins), FP64 Levenberg-Marquardt (at most max_iter steps; converged when a
 *   step changes chi^2 by no more than tol chi^2; tol 1e-12 is a fine
 *   default), initial values from the band (largest bin, smallest bin, the
 *   width at half height).  out_dev: double [12] (device) = f0, Q, A, B, their
 *   standard errors (from diag(H^-1) chi^2 / (n - 4)), chi^2, steps, status
 *   (0 converged, 1 step limit, 2 singular, 3 non-finite), bins used.
 *   Asynchronous.  Errors: CG_ERR_ARG.
 */
typedef struct cg_psd_s* cg_psd_t;
cg_status cg_psd_create(int seg_len, cg_psd_t* out);
void cg_psd_destroy(cg_psd_t psd);
cg_status cg_psd_welch(cg_psd_t psd, const float* x_dev, int64_t n, int64_t stride, double fs,
                       double* psd_dev, int64_t* n_segments, void* cuda_stream);
cg_status cg_resonance_fit(const double* psd_dev, int n_bins, double df, double f_lo, double f_hi,
                           int max_iter, double tol, double* out_dev, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* COMBGPU_H */
