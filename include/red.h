/*
 * red.h -- C-ABI of libred: RED (REgularization by Denoising) solved by the fixed-point
 * iteration and accelerated by vector extrapolation, on one GB300 GPU (sm_103a).
 *
 * Method: Hong, Romano, Elad, "Acceleration of RED via Vector Extrapolation".
 *   objective       E(x) = ||Hx - y||^2 / (2 sigma^2) + (alpha/2) x^T (x - f(x))   Eq. (4)
 *   FP step         x_{k+1} = [H^T H / sigma^2 + alpha I]^{-1}
 *                             [H^T y / sigma^2 + alpha f(x_k)]                      Eq. (7)
 *   extrapolation   x_(m,kappa) = sum_i gamma_i x_{m+i}, sum gamma_i = 1            Eq. (11)
 *                   MPE (Algorithm 1), RRE (Eq. (19)); cycling (Algorithm 3)
 *
 * Conventions for every entry point:
 *   - Images are single-channel, row-major, contiguous, height x width, values on the
 *     [0, 255] scale. Element type is float32 unless a config's `storage` says otherwise.
 *   - "dev" pointers are CUDA device pointers owned by the caller; "host" pointers are
 *     host memory owned by the caller. The library never frees caller memory.
 *   - `stream` is a cudaStream_t passed as an opaque pointer (NULL = legacy default
 *     stream). Calls enqueue work on it and return without waiting, except where stated.
 *   - Every function returns red_status and never throws. On failure the handle is left
 *     usable unless the status is RED_ECUDA (a CUDA error; the context may be lost).
 *     red_last_error() gives a message for the calling thread's last failure.
 *   - A red_problem or red_batch handle is not thread-safe; a red_server is.
 */
#ifndef RED_H
#define RED_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct red_problem_s *red_problem;
typedef struct red_batch_s *red_batch;
typedef struct red_server_s *red_server;

typedef enum {
  RED_OK = 0,
  RED_EINVAL = 1,          /* bad argument (null handle, unsupported size, ...)          */
  RED_ENOMEM = 2,          /* device or host allocation failed                           */
  RED_ECUDA = 3,           /* a CUDA runtime call failed                                 */
  RED_EVE_BREAKDOWN = 4,   /* informational: an extrapolation did not exist; the output */
                           /* is still valid (the last FP iterate was used instead)      */
  RED_ENOT_CONVERGED = 5,  /* informational: the FP-call budget ran out before rel_tol  */
  RED_ETIMEOUT = 6,        /* red_wait timed out, or a bounded device wait gave up       */
  RED_EBUSY = 7,           /* red_poll: the request is still running                     */
  RED_EUNSUPPORTED = 8     /* valid but not supported by this build (e.g. patch != 5)    */
} red_status;

typedef enum { RED_DEBLUR = 0, RED_SR = 1 } red_task;

/* Extrapolation method (Sec. III-B): MPE (Algorithm 1), RRE (Eq. (19)), SVD-MPE (gamma from
 * the right singular vector of R for its smallest singular value). */
typedef enum { RED_VE_NONE = 0, RED_VE_MPE = 1, RED_VE_RRE = 2, RED_VE_SVDMPE = 3 } red_ve;

/* Storage type of images and iterates; arithmetic is always FP32, the extrapolation
 * Gram matrix exact-product with double-float sums and the gamma solve double-float (MPE,
 * RRE) or FP64 (SVD-MPE). */
typedef enum { RED_F32 = 0, RED_BF16 = 1, RED_F16 = 2 } red_dtype;

/* Baseline map that Algorithm 3 cycles (one denoiser call per step, Sec. IV):
 *   RED_BASE_FP: the fixed-point step of Eq. (7);
 *   RED_BASE_SD: the fixed-step steepest descent x - mu grad E(x) on Eq. (5) (the
 *                baseline of SD-MPE, Sec. IV-A/B). */
typedef enum { RED_BASE_FP = 0, RED_BASE_SD = 1 } red_baseline;

typedef struct {
  int task;              /* red_task                                                    */
  int height, width;     /* image (high-resolution) size; each must be 2^a * 3^b, width  */
                         /* even, 8 <= size <= 2048                                      */
  int scale;             /* 1 for deblurring; the decimation factor for SR (LR size is  */
                         /* floor(height/scale) x floor(width/scale), samples at 0,s,.) */
  const float *psf;      /* host, psf_h x psf_w row-major taps, copied at creation;      */
  int psf_h, psf_w;      /* odd sizes; the centre tap ((psf_h-1)/2, (psf_w-1)/2) is the  */
                         /* origin of the circular convolution                           */
  double sigma;          /* noise standard deviation of Eq. (1)                          */
  double alpha;          /* RED weight alpha of Eq. (4)                                  */
  int nlm_patch;         /* non-local-means patch side (5 supported)                    */
  int nlm_search;        /* search window side (11 supported)                           */
  double nlm_h;          /* NLM filtering parameter h (weights exp(-d/h^2), d the mean  */
                         /* squared patch difference)                                    */
  int ve;                /* red_ve                                                      */
  int ve_k;              /* FP steps per cycle = columns of U = kappa + 1 (1..12)        */
  int ve_m;              /* lead-in FP steps per cycle before the stored window (0..64)  */
  int cg_iters;          /* CG iterations per FP step for SR (0..1000; default 20)       */
  int storage;           /* red_dtype of the iterate history (F32, BF16 or F16)          */
  int baseline;          /* red_baseline (default RED_BASE_FP)                           */
  double sd_mu;          /* SD step size mu (RED_BASE_SD); 0 selects                     */
                         /* 1 / (max |K(w)|^2 / sigma^2 + alpha), K the PSF spectrum     */
  int ve_freeze;         /* cycling with frozen gamma (Sec. III-C remark): 0 = every     */
                         /* cycle solves for gamma; n >= 1 = after n successful          */
                         /* extrapolations, later cycles run ve_m + ve_k - 1 steps and   */
                         /* combine with the last gamma (needs ve_m + ve_k >= 2)         */
  double ve_stop_tol;    /* extrapolation ended by its own criterion, then baseline steps */
                         /* (the "additional iterations after terminating the VE" remark  */
                         /* of Sec. III-C): at the first FP step whose relative change is  */
                         /* below ve_stop_tol, that cycle takes no extrapolation and every */
                         /* later step is a plain baseline step, until rel_tol or the      */
                         /* budget; 0 = never (full cycling). Needs ve != RED_VE_NONE and  */
                         /* ve_freeze = 0                                                  */
} red_config;

typedef struct {
  int fp_calls;          /* FP steps = denoiser calls made                               */
  int ve_steps;          /* extrapolations attempted                                     */
  int ve_breakdowns;     /* extrapolations that did not exist (Sec. III-B remark)        */
  int converged;         /* 1 if rel_tol was met, 0 if the budget ran out                */
  double rel_change;     /* ||x_{i+1} - x_i|| / ||x_i|| of the last FP step              */
  double sum_abs_gamma;  /* sum |gamma_i| of the last extrapolation, Eq. (21)            */
  double ms_total;       /* wall time of the call (red_solve*) or request (server)       */
} red_stats;

/* Fills `cfg` with the defaults used by the paper's deblurring experiments (Sec. IV-A):
 * NLM 5x5 / 11x11 / h = 10, alpha = 0.02, RRE with ve_k = 5, ve_m = 0, cg_iters = 20,
 * the FP baseline, no frozen gamma. */
void red_config_default(red_config *cfg);

/* ----------------------------------------------------------------------------------- */
/* Problems                                                                             */
/* ----------------------------------------------------------------------------------- */

/* Creates a problem (Eq. (1): y = H x + e) and precomputes its per-problem constants:
 * for deblurring the Fourier-domain solve of Eq. (7) (footnote: block-circulant H), for
 * SR the right-hand side H^T y / sigma^2. y_dev: device float32, LR size for SR, image
 * size otherwise; read during the call's stream work only. Allocates all device memory
 * the problem needs (iterate history, spectra, CG vectors). Errors: RED_EINVAL for bad
 * sizes/parameters, RED_EUNSUPPORTED, RED_ENOMEM, RED_ECUDA. */
red_status red_create_problem(const red_config *cfg, const void *y_dev, void *stream,
                              red_problem *out);

/* Replaces the observation y of an existing problem (same config) and recomputes the
 * constants. y may be host (y_is_host = 1, float32, copied through the stream) or device
 * memory. Lets a caller reuse one problem's memory for a stream of observations. */
red_status red_set_observation(red_problem p, const void *y, int y_is_host, void *stream);

red_status red_destroy_problem(red_problem p);

/* One FP step, Eq. (7): x_out = [H^T H/sigma^2 + alpha I]^{-1}[H^T y/sigma^2 + alpha f(x_in)]
 * (or, with baseline RED_BASE_SD, the steepest-descent step x_in - mu grad E(x_in) of Eq. (5)).
 * x_in_dev, x_out_dev: device float32 images, distinct, 8-byte aligned (RED_EINVAL
 * otherwise). */
red_status red_fp_step(red_problem p, const void *x_in_dev, void *x_out_dev, void *stream);

/* The denoiser alone: f_dev = f(x_dev), pixelwise non-local means (the role of f in
 * Eq. (3)); device float32 images. */
red_status red_denoise(red_problem p, const void *x_dev, void *f_dev, void *stream);

/* One extrapolation (Algorithm 1 with the problem's ve method: MPE, RRE Eq. (19) or SVD-MPE) from
 * n_vec = kappa + 2 device float32 iterates xs_dev[0..n_vec) (x_m .. x_{m+kappa+1}), host
 * array of device pointers, 3 <= n_vec <= 13. Writes x_(m,kappa) to x_out_dev (may alias
 * xs_dev[0]). If gamma_host is non-null the call synchronises the stream and copies the
 * kappa + 1 weights gamma_i (double) there. Returns RED_EVE_BREAKDOWN (x_out = the last
 * iterate) when the extrapolation does not exist. */
red_status red_ve_extrapolate(red_problem p, const void *const *xs_dev, int n_vec,
                              void *x_out_dev, double *gamma_host, void *stream);

/* Allocation-free extrapolation. The paper has no counterpart: this is the extrapolation
 * of red_ve_extrapolate for a caller that holds iterates of its own fixed-point
 * iteration and cannot allocate device memory at the call site: cudaMalloc and cudaFree
 * synchronise the whole device (stalling every other stream of a serving process), and a
 * process whose device memory is reserved up front by another allocator has no room for
 * a problem's buffers. No problem handle is needed and nothing is allocated: the Gram
 * partial sums, xi, gamma and the status live in one file-scope device array of
 * 624 KiB + 320 bytes per device (1024 rows of 78 partial sums, enough for any n).
 *   xs_dev:  host array of n_vec device pointers to float32 vectors x_m .. x_{m+kappa+1},
 *            each of n elements, 3 <= n_vec <= 13 (any alignment; 16-byte aligned
 *            vectors take the vectorised path).
 *   n:       elements per vector, 1 <= n <= 2^31 - 1; larger n returns RED_EINVAL.
 *   method:  RED_VE_MPE (Algorithm 1), RED_VE_RRE (Eq. (19)) or RED_VE_SVDMPE.
 *   x_out_dev: device float32, n elements, may alias xs_dev[0]; on RED_EVE_BREAKDOWN it
 *            holds the last iterate.
 *   gamma_host: null, or room for kappa + 1 doubles.
 * The first call on each device looks up the array's address (with that device current)
 * and should come before any stream capture. The call zeroes the status block, launches
 * three kernels on `stream` and synchronises it. All calls on one device share the one
 * array: calls that overlap in time (other streams or host threads) race and must be
 * serialised by the caller. Errors: RED_EINVAL (arguments, size), RED_ECUDA. */
red_status red_ve_extrapolate_static(const void *const *xs_dev, int n_vec, int64_t n,
                                     int method, void *x_out_dev, double *gamma_host,
                                     void *stream);

/* Full solve, Algorithm 3: cycles of ve_m + ve_k FP steps followed by one extrapolation
 * (plain FP iteration when ve = RED_VE_NONE), until the relative change of an FP step is
 * below rel_tol or max_fp_calls FP steps were made; x_out is that last FP iterate.
 * x0_dev, x_out_dev: device float32. Synchronises the stream (termination is read back
 * at most once per cycle). `stats` may be null. Returns RED_OK, or RED_ENOT_CONVERGED
 * when rel_tol > 0 and the budget ran out first. */
red_status red_solve(red_problem p, const void *x0_dev, int max_fp_calls, double rel_tol,
                     void *x_out_dev, red_stats *stats, void *stream);

/* Evaluates the objective E(x) of Eq. (4) at a device float32 image, 8-byte aligned (one
 * denoiser call); synchronises the stream. */
red_status red_objective(red_problem p, const void *x_dev, double *e_host, void *stream);

/* ----------------------------------------------------------------------------------- */
/* Batches: many problems (any mix of sizes and tasks, same ve/ve_k/ve_m) solved        */
/* together, one kernel launch per phase over all problems, cycles replayed as CUDA     */
/* graphs, launch shapes chosen by the autotuner.                                       */
/* ----------------------------------------------------------------------------------- */

/* Groups n problems (host array of handles) into a batch. The problems must outlive the
 * batch and must not be used on their own while it exists. Tunes launch shapes on first
 * solve unless the tuning cache (env RED_TUNE_CACHE) already has them. */
red_status red_batch_create(const red_problem *problems, int n, red_batch *out);
red_status red_batch_destroy(red_batch b);

/* Solves every problem of the batch (Algorithm 3 each, as red_solve). x0_dev[i] and
 * x_out_dev[i] are device float32 images of problem i (host arrays of n pointers).
 * stats may be null or an array of n. Synchronises the stream. */
red_status red_batch_solve(red_batch b, const void *const *x0_dev, int max_fp_calls,
                           double rel_tol, void *const *x_out_dev, red_stats *stats,
                           void *stream);

/* As red_batch_solve, but x0 and x_out are HOST float32 images (pinned or pageable);
 * the host-to-device and device-to-host copies run on `stream` inside the call. If
 * y_host is non-null it also uploads each problem's observation y_host[i] (LR-sized for
 * SR) and recomputes its constants first, with the same result as red_set_observation;
 * the deblurring problems' constants (the half spectrum of y, then C and G of Eq. (7)) are
 * formed for the whole batch in three launches. */
red_status red_batch_solve_host(red_batch b, const float *const *y_host,
                                const float *const *x0_host, int max_fp_calls,
                                double rel_tol, float *const *x_out_host, red_stats *stats,
                                void *stream);

/* Kernel phases of a cycle, for red_batch_phase_ms. */
typedef enum {
  RED_PHASE_NLM = 0,      /* the denoiser f over all problems                           */
  RED_PHASE_FFT = 1,      /* the Fourier-domain solve (row, column, row passes)          */
  RED_PHASE_CG = 2,       /* the super-resolution CG solve                               */
  RED_PHASE_GRAM = 3,     /* G = U^T U and, in its last CTA per problem, gamma           */
  RED_PHASE_VESOLVE = 4,  /* gamma from G (runs inside the Gram launch: no launches)      */
  RED_PHASE_COMBINE = 5   /* x_(m,kappa) from gamma                                      */
} red_phase;

/* Diagnostics. With timing enabled, solves launch their cycles directly (not as a graph)
 * and record CUDA events around every kernel phase; red_batch_phase_ms then reports the
 * mean device time of one launch of `phase` over the most recent solve (and how many
 * launches that mean covers; launches of problems that had already terminated are
 * included). Call between solves. */
red_status red_batch_set_phase_timing(red_batch b, int enable);
red_status red_batch_phase_ms(red_batch b, int phase, double *avg_ms, int *launches);

/* Writes a one-line JSON description of the batch's launch shapes (as chosen by the
 * autotuner on the first solve) into buf (NUL-terminated, truncated to len). */
red_status red_batch_describe(red_batch b, char *buf, size_t len);

/* ----------------------------------------------------------------------------------- */
/* Serving: a request loop that continuously batches RED solves of different sizes and  */
/* tasks as they arrive. Requests are admitted while their device footprint fits in     */
/* hbm_budget_bytes and a slot is free; each running request keeps its iterate history  */
/* and constants on the device. Requests of one task, size class and extrapolation     */
/* setting share launches and advance one Algorithm 3 cycle at a time on their own      */
/* stream; finished requests are retired after each cycle, freeing room for waiting     */
/* ones. A request's result does not depend on the others in flight. All server         */
/* functions are thread-safe.                                                           */
/* ----------------------------------------------------------------------------------- */

red_status red_server_create(size_t hbm_budget_bytes, int max_slots, red_server *out);

/* Queues a request. cfg and the host PSF are copied. y_host: host float32 observation
 * (copied before return). x_out_host: host float32 image that receives the result; it
 * must stay valid until red_poll/red_wait reports completion. x0 = y for deblurring and
 * the pixel-replicated upsampling of y for SR. */
red_status red_submit(red_server s, const red_config *cfg, const float *y_host,
                      float *x_out_host, int max_fp_calls, double rel_tol,
                      uint64_t *ticket);

/* RED_EBUSY while the request runs; its status (RED_OK / RED_ENOT_CONVERGED / error)
 * once finished. `stats` (may be null) is filled when finished. */
red_status red_poll(red_server s, uint64_t ticket, red_stats *stats);

/* Blocks until the request finishes or timeout_ms passes (RED_ETIMEOUT); timeout_ms < 0
 * waits without limit. */
red_status red_wait(red_server s, uint64_t ticket, int timeout_ms, red_stats *stats);

/* Stops the scheduler after draining admitted requests; waiting requests are failed. */
red_status red_server_destroy(red_server s);

/* ----------------------------------------------------------------------------------- */

const char *red_status_string(red_status st);
const char *red_last_error(void);

/* Bytes of device memory a problem with this config allocates (admission accounting). */
red_status red_problem_footprint(const red_config *cfg, size_t *bytes);

/* Measures the throughput of the arithmetic units the hot path is bound by, in lane
 * operations per second over the whole device: FP32 FMA (the NLM's arithmetic), the
 * ex2.approx special function (its weights), FP64 FMA (the SVD-MPE solve) and packed
 * FP32 FMA (fma.rn.f32x2, two lane operations per instruction), each by independent
 * dependency chains on every SM (a few ms; synchronises the stream). No counterpart in the
 * paper: it puts measured peaks beside the derived ones of the roofline. */
red_status red_measure_peaks(double *fp32_fma_lane_ops, double *ex2_lane_ops,
                             double *fp64_fma_lane_ops, double *fp32x2_fma_lane_ops,
                             void *stream);

/* Number of kernel launches this library has issued in this process (for accounting). */
uint64_t red_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* RED_H */
