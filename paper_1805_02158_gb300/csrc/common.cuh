// Internal declarations shared by the libred translation units (not part of the C-ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <string>
#include <vector>

namespace red {

constexpr int kMaxK = 12;                       // largest ve_k (columns of U)
constexpr int kMaxPairs = kMaxK * (kMaxK + 1) / 2;
constexpr int kGramChunk = 2048;                // pixels per Gram / combine work unit
constexpr int kNlmR = 6;                        // output rows per NLM thread
constexpr int kNlmTW = 60;                      // output columns per NLM warp (64 - 4 halo)

constexpr double kRankTol = 1e-12;              // rank-loss threshold on r_jj^2 / ||u_j||^2
constexpr double kSumTol = 1e-12;               // MPE existence: |sum c| > tol * sum |c|

enum Task { kDeblur = 0, kSR = 1 };
enum Ve { kVeNone = 0, kVeMpe = 1, kVeRre = 2, kVeSvdMpe = 3 };
enum Baseline { kBaseFP = 0, kBaseSD = 1 };   // the map Algorithm 3 cycles

// Per-problem termination state, device resident; written by the step kernels.
struct ProbState {
  int done;            // 1 once the solve of this problem has terminated
  int calls;           // FP steps taken
  int final_slot;      // ring slot holding the result once done
  int converged;       // 1 if terminated by the relative-change test
  int ve_steps;
  int ve_breakdowns;
  int max_calls;
  int ve_status;       // last extrapolation: 0 ok, 1 breakdown
  double tol;
  double rel_change;
  double sum_abs_gamma;
  unsigned int counter;   // arrival counter for last-block reductions
  unsigned int counter2;
  // cycling with frozen gamma (ProbDev::ve_freeze > 0)
  int ve_ok;           // extrapolations that succeeded
  int frozen;          // 1 once ve_ok reached ve_freeze: later cycles reuse xi
  int solved;          // 1 between a gamma solve and the combine that uses it
  int frozen_steps;    // combines with the frozen xi
  // extrapolation ended by the relative-change criterion (red_config::ve_stop_tol)
  double ve_stop_tol;  // 0: never
  int ve_off;          // 1 from the first FP step whose relative change was below it
};

// Step size of the steepest-descent baseline: mu = 1 / (max |K(w)|^2 / sigma^2 + alpha)
// unless the config gives one. Written by the set-up kernels, read by the step kernels.
struct SdParams {
  double mu;               // FP64 (the spectral constants are formed in FP64)
  float mu_f;              // mu and mu * alpha in FP32 (the step epilogues)
  float mu_alpha_f;
  unsigned int kmax_bits;  // bits of max |K(w)|^2 as a float (non-negative floats order
                           // as unsigned integers, so atomicMax on the bits takes the max)
  unsigned int pad;
};

// Everything a kernel needs to know about one problem. Plain data, copied to device
// tables; one table per launch group (single problem or batch).
struct ProbDev {
  int H, W, M, Wh, N;     // image size; M = W/2; Wh = M + 1; N = H*W
  int slot_stride;        // elements between ring slots (multiple of 64)
  int task, scale, lh, lw;
  int storage;            // StoreType of the ring: 0 = f32, 1 = bf16, 2 = f16
  int nslots;
  int n_row_items;        // CTAs of one row-FFT launch for this problem
  int n_chunks;           // Gram / combine work units
  int kh, kw;             // SR blur size
  int cg_iters;
  int ve_k;
  int ve_method;
  int baseline;           // Baseline: FP step of Eq. (7) or SD step on Eq. (5)
  int ve_freeze;          // 0, or freeze gamma after this many successful extrapolations
  float inv_sigma2, alpha;
  double inv_sigma2_d, alpha_d;   // the same in FP64 (the per-problem spectral constants)
  float nlm_k;            // NLM prescale sqrt(log2(e) / (P^2 h^2))
  void *ring;             // nslots * slot_stride elements (float, bf16 or half)
  float *f;               // denoiser output, N
  const float *y;         // the observation (deblur: H x W; SR: lh x lw)
  float2 *spec;           // H x Wh half spectrum workspace (deblur)
  const float2 *Kh;       // H x Wh: K, the PSF spectrum (for H x in the objective)
  const float2 *Cc;       // H x Wh: conj(K) Y / (sigma^2 D) / (H W)
  const float *Gg;        // H x Wh: alpha / D / (H W)
  const float2 *tw_m;     // e^{-2 pi i t / M}, t < M
  const float2 *tw_w;     // e^{-2 pi i t / W}, t <= M
  const float2 *tw_h;     // e^{-2 pi i t / H}, t < H
  float2 *row_stats;      // H partial sums (sum d^2, sum x^2) of one FP step
  // SR
  const float *b0;        // H^T y / sigma^2 (N)
  float *cg_x, *cg_r, *cg_p, *cg_ap, *cg_z;   // CG vectors; z is LR sized
  const float *psf;       // kh x kw taps
  // steepest descent (baseline kBaseSD): the step size, set up on the device
  struct SdParams *sd;
  // extrapolation
  float2 *gram_part;      // n_chunks x kMaxPairs double-float (hi, lo) partial sums
  double *ve_coef;        // kMaxK: xi_j of Algorithm 1 step 3 (difference form), + gamma
  double *gamma;          // kMaxK
  ProbState *st;
};

struct Item {             // one CTA's work unit
  int prob;
  int a, b, c;
};

// Which ring slots a launch reads and writes, or explicit pointers (single-problem calls).
struct StepArgs {
  int src, dst;           // ring slots
  const void *src_ptr;    // if non-null: read this instead of slot src (f32)
  float *dst_ptr;         // if non-null: write this instead of slot dst (f32)
  int update_state;       // 1: batched solve step (skip done problems, count calls)
  int skip_frozen;        // 1: the last step of a full cycle (skipped by frozen problems)
};

struct VeArgs {
  int slots[kMaxK + 1];   // ring slots of x_m .. x_{m+k}
  const float *ptrs[kMaxK + 1];  // explicit vectors (single-problem call) or null
  float *out_ptr;         // explicit output or null
  int out_slot;
  int nvec;               // k + 1
  int update_state;
  int skip_frozen;        // 1: Gram and gamma solve are skipped by frozen problems
};

// ---- host-side launch helpers (defined in the .cu files) -------------------------------
struct LaunchCfg {
  int nlm_wy = 4;          // warps per NLM CTA (one 60 x kNlmR warp tile each)
  int nlm_occ = 4;         // resident NLM CTAs per SM the register budget allows (3 or 4)
  int fft_rows = 0;        // rows per row-FFT CTA (0 = auto from the row length)
  int fft_cols = 0;        // columns per column-FFT CTA (0 = auto from the column length)
  int sr_cluster = 8;      // CTAs per super-resolution cluster (one cluster per problem)
  int fft_cluster = 16;    // CTAs per cluster of the fused Fourier solve (0: three passes)
};

// NLM over the items: reads slot sa.src (or sa.src_ptr), writes f_override (if non-null) or
// each problem's f buffer.
cudaError_t launch_nlm(const ProbDev *d_probs, const Item *d_items, int n_items, int wy,
                       StepArgs sa, int src_type, cudaStream_t s, float *f_override, int occ);
// FFT launches: items carry (prob, first row/col, count). tw_cap = largest transform
// length in the launch (M for rows, H for columns); buf_cap = largest per-item buffer
// (rows * M, or cols * (H + 1)) in complex elements.
// step: null for transforms of a given image (set-up, objective); the FP step's slots
// otherwise (an SD problem's step transforms x_k instead of f).
cudaError_t launch_fft_r2c(const ProbDev *d_probs, const Item *d_items, int n_items,
                           int tw_cap, int buf_cap, const float *src_override,
                           float2 *dst_override, int skip_done, cudaStream_t s,
                           const StepArgs *step = nullptr);
cudaError_t launch_fft_cols(const ProbDev *d_probs, const Item *d_items, int n_items,
                            int tw_cap, int buf_cap, int mode, float2 *spec_override,
                            int skip_done, cudaStream_t s);
cudaError_t launch_fft_c2r(const ProbDev *d_probs, const Item *d_items, int n_items,
                           int tw_cap, int buf_cap, StepArgs sa, cudaStream_t s);
// sd: null for the FP solve's C and G, else the SD step's constants with its step size.
cudaError_t launch_spectral_constants(const ProbDev *d_prob, const float2 *k_hat,
                                      const float2 *y_hat, float2 *Cc, float *Gg, int n,
                                      double inv_sigma2, double alpha, double inv_hw,
                                      cudaStream_t s, const SdParams *sd = nullptr);
// The SD step size of one problem into P->sd: max |K(w)|^2 over the H x (W/2 + 1) half
// spectrum by direct evaluation of the PSF's DFT, then mu (mu_given > 0 overrides).
cudaError_t launch_sd_step_size(const ProbDev *d_prob, const float *psf, int kh, int kw, int H,
                                int W, double inv_sigma2, double alpha, double mu_given,
                                SdParams *sd, cudaStream_t s);
// G = U^T U per chunk, then (the last chunk of each problem) the gamma solve.
cudaError_t launch_gram(const ProbDev *d_probs, const Item *d_items, int n_items,
                        const VeArgs &va, cudaStream_t s);
cudaError_t launch_combine(const ProbDev *d_probs, const Item *d_items, int n_items,
                           const VeArgs &va, cudaStream_t s);
cudaError_t launch_copy_slots(const ProbDev *d_probs, const Item *d_items, int n_items,
                              int mode, int slot, float *const *d_ptrs, cudaStream_t s);
cudaError_t launch_convert_to_slot(const ProbDev *d_prob, const float *src, int slot,
                                   cudaStream_t s);
cudaError_t launch_fetch_slot(const ProbDev *d_prob, int slot, float *dst, cudaStream_t s);
cudaError_t launch_sr_rhs(const ProbDev *d_prob, const float *y, cudaStream_t s);
// Shared-memory extents (4-byte words) of the super-resolution CG kernel.
struct SrCaps {
  int taps = 0;      // kh * kw
  int rows = 0;      // row-window entries of a band (band rows + kh - 1)
  int zrows = 0;     // LR rows of z kept by a band
  int cols = 0;      // W + kw - 1
  int zfloats = 0;   // zrows * lw
  int band = 0;      // pixels of the largest band
  int band_ext = 0;  // pixels of the largest band with kh - 1 halo rows on each side
  int spec737 = 1;   // every problem has a 7x7 PSF and scale 3 (specialised kernel)
  int resident = 0;  // the band's CG vectors are kept in shared memory
  int resident_off = 0;   // (set at launch) word offset of the resident vectors
};
void sr_caps(int H, int W, int scale, int kh, int kw, int ncta, SrCaps *c);
int sr_smem_bytes(const SrCaps &c, int resident);
cudaError_t launch_sr_step(const ProbDev *d_probs, const int *d_sr_probs, int n_sr,
                           int cluster, const SrCaps &caps, StepArgs sa, cudaStream_t s);
cudaError_t launch_objective(const ProbDev *d_prob, const float *x, const float *hx,
                             const float *y, const float *f, double *out, cudaStream_t s);

// Cluster solve (one cluster per deblurring problem, spectrum in shared memory).
void fft_cluster_caps(int H, int W, int ncta, int *a_elems, int *buf_elems, int *cg_elems);
int fft_cluster_smem(int tw_cap_m, int tw_cap_h, int a_cap, int buf_cap, int cg_cap);
// Shared memory per CTA of the cluster solve up to which two CTAs fit on an SM (the C/G
// staging is dropped above it, so the 16-CTA clusters of every problem stay resident).
constexpr int kClusterSmemTwoPerSm = 112 * 1024;
cudaError_t fft_cluster_prepare(int smem, int ncta);
// C and G of every deblurring problem listed (one item per 256 frequencies of a problem:
// {prob, first frequency}), from its K and the half spectrum of y in its spec buffer.
cudaError_t launch_spectral_constants_items(const ProbDev *d_probs, const Item *d_items,
                                            int n_items, cudaStream_t s);
// Flag of launch_fft_r2c's `skip_done` word: transform each problem's observation y.
constexpr int kFftSrcY = 4;
int fft_cluster_max_active(int ncta, int smem);
cudaError_t launch_fft_solve_cluster(const ProbDev *d_probs, const int *d_list, int n, int ncta,
                                     int tw_cap_m, int tw_cap_h, int a_cap, int buf_cap,
                                     int cg_cap, StepArgs sa, cudaStream_t s);
int fft_smem_rows(int tw_cap, int buf_cap);
int fft_smem_cols(int tw_cap, int buf_cap);

void count_launches(uint64_t n);
cudaError_t fft_prepare(int row_tw_cap, int row_buf_cap, int col_tw_cap, int col_buf_cap);
cudaError_t sr_prepare(int cluster, int smem);
int sr_max_active_clusters(int cluster, int smem, int spec737);
cudaError_t nlm_prepare(int wy);

// NLM work items of one image (nlm.cu).
void nlm_items(int prob, int H, int W, std::vector<Item> &out);

// ---- small device helpers ---------------------------------------------------------------
// Division by a run-time invariant d < 2^16 for numerators t < 2^16: q = hi32(t * m) with
// m = floor(2^32 / d) + 1 (exact in that range; d = 1 handled separately). Every index
// divided with it is below 2^16 (image sides <= 2048, <= 16 sequences per FFT CTA).
struct FastDiv {
  uint32_t d, m;
  __device__ __forceinline__ explicit FastDiv(int dd)
      : d((uint32_t)dd), m(dd > 1 ? 0xFFFFFFFFu / (uint32_t)dd + 1u : 0u) {}
  __device__ __forceinline__ int div(int t) const { return d == 1 ? t : (int)__umulhi((uint32_t)t, m); }
  __device__ __forceinline__ void divmod(int t, int &q, int &r) const {
    q = div(t);
    r = t - q * (int)d;
  }
};

// Stride of one transform sequence of length n in shared memory: one pad slot per 16
// elements, rounded up to odd (bank-conflict-free strided and transposed accesses).
__host__ __device__ __forceinline__ int fft_seq_stride(int n) { return (n + (n >> 4)) | 1; }

__host__ __device__ __forceinline__ int mirror_index(int i, int n) {
  // half-sample symmetric reflection into [0, n), period 2n
  int p = 2 * n;
  i %= p;
  if (i < 0) i += p;
  return i < n ? i : p - 1 - i;
}

// Storage types of the iterate ring (ProbDev::storage): kStoreF32, kStoreBF16, kStoreF16.
// Arithmetic is FP32 in every case; a 16-bit type only changes how iterates are kept.
enum StoreType { kStoreF32 = 0, kStoreBF16 = 1, kStoreF16 = 2 };

__host__ __device__ __forceinline__ int store_bytes(int type) { return type ? 2 : 4; }

__device__ __forceinline__ float load_img(const void *base, long idx, int type) {
  if (type == kStoreBF16) return __bfloat162float(reinterpret_cast<const __nv_bfloat16 *>(base)[idx]);
  if (type == kStoreF16) return __half2float(reinterpret_cast<const __half *>(base)[idx]);
  return reinterpret_cast<const float *>(base)[idx];
}

__device__ __forceinline__ void store_img(void *base, long idx, float v, int type) {
  if (type == kStoreBF16)
    reinterpret_cast<__nv_bfloat16 *>(base)[idx] = __float2bfloat16_rn(v);
  else if (type == kStoreF16)
    reinterpret_cast<__half *>(base)[idx] = __float2half_rn(v);
  else
    reinterpret_cast<float *>(base)[idx] = v;
}

// The value a store of v in `type` keeps (round to nearest even).
__device__ __forceinline__ float round_to_storage(float v, int type) {
  if (type == kStoreBF16) return __bfloat162float(__float2bfloat16_rn(v));
  if (type == kStoreF16) return __half2float(__float2half_rn(v));
  return v;
}

}  // namespace red
