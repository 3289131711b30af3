// Host-side internals of libred shared by api.cu, batch.cu and server.cpp.
#pragma once

#include <cuda_runtime.h>

#include <memory>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"
#include "red.h"

namespace red {

struct Fail {
  red_status st;
  std::string msg;
};

void set_error(const std::string &m);

#define CUDA_OK(expr)                                                                    \
  do {                                                                                   \
    cudaError_t _e = (expr);                                                             \
    if (_e != cudaSuccess)                                                               \
      throw ::red::Fail{RED_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)};  \
  } while (0)

#define CHECK_ARG(cond, msg)                                \
  do {                                                      \
    if (!(cond)) throw ::red::Fail{RED_EINVAL, (msg)};      \
  } while (0)

template <class F>
red_status guarded(F &&f) {
  try {
    return f();
  } catch (const Fail &e) {
    set_error(e.msg);
    return e.st;
  } catch (const std::bad_alloc &) {
    set_error("host allocation failed");
    return RED_ENOMEM;
  } catch (const std::exception &e) {
    set_error(e.what());
    return RED_ECUDA;
  } catch (...) {
    set_error("unexpected exception");
    return RED_ECUDA;
  }
}

struct Layout {
  size_t ring, f, spec, kh, cc, gg, row_stats, gram, coef, gamma, state, y, tmp, b0, cx, cr,
      cp, cap, cz, psf, obj, sd, total;
};

// Work-item lists of one launch group (one problem, or a batch) for one launch shape.
struct Plan {
  LaunchCfg lc;
  Item *d_items = nullptr;
  int *d_sr = nullptr;
  int *d_fused = nullptr;     // deblurring problems solved by the cluster kernel
  int n_fused = 0, fused_ncta = 0, fused_tw_m = 0, fused_tw_h = 0, fused_a = 0, fused_buf = 0;
  int fused_cg = 0;           // C/G values staged per CTA (0: read from global memory)
  int n_nlm = 0, n_rows = 0, n_cols = 0, n_chunks = 0, n_sr = 0;
  int off_nlm = 0, off_rows = 0, off_cols = 0, off_chunks = 0;
  int row_tw_cap = 0, row_buf_cap = 0, col_tw_cap = 0, col_buf_cap = 0;
  SrCaps sr_cap;              // shared-memory extents of the super-resolution CG launch
  std::vector<int> n_row_items;
  // Device lists are reused when large enough; with a stream the uploads are ordered on it
  // (no device-wide synchronisation), otherwise they are synchronous.
  size_t items_cap = 0, sr_cap_n = 0, fused_cap = 0;
  void build(const std::vector<ProbDev> &pds, const LaunchCfg &cfg, cudaStream_t stream = nullptr,
             bool async = false);
  void release();
  ~Plan() { release(); }
};

// One operation of the cycle of Algorithm 3: an FP step src -> dst (kind 0) or an
// extrapolation from `slots` into `out` (kind 1). skip_frozen: the step, or the Gram and
// gamma solve of the extrapolation, is skipped by problems whose gamma is frozen.
struct CycleOp {
  int kind;
  int src, dst;
  std::vector<int> slots;
  int out;
  int skip_frozen;
};

void launch_fp_step(const ProbDev *d_probs, const Plan &pl, StepArgs sa, int src_type,
                    cudaStream_t s);
void launch_ve(const ProbDev *d_probs, int n_probs, const Plan &pl, const VeArgs &va,
               cudaStream_t s);
void launch_fft_solve(const ProbDev *d_probs, const Plan &pl, StepArgs sa, cudaStream_t s);
std::vector<CycleOp> cycle_ops(int ve, int k, int m, int freeze);
void prepare_launch_attrs(const Plan &pl);
int fft_cluster_override();   // RED_FFT_CLUSTER, or -1 when unset
int sr_cluster_override();    // RED_SR_CLUSTER (8, 10, 12 or 16), or -1 when unset
void nlm_shape_override(int *wy, int *occ);   // RED_NLM_SHAPE=<w>,<o>; unchanged when unset

}  // namespace red

struct red_batch_s;

struct red_problem_s {
  red_config cfg{};
  std::vector<float> psf;
  red::Layout L{};
  red::ProbDev pd{};
  void *block = nullptr;
  red::ProbDev *d_pd = nullptr;
  red::Plan plan;                // FP steps of this problem alone
  red::Plan plan3;               // three-pass Fourier items (set-up, objective)
  red::LaunchCfg lc;
  char *h_pinned = nullptr;     // 4 KB pinned staging
  red_batch_s *own_batch = nullptr;
  std::vector<float> psf_pad;   // host source of the PSF-spectrum upload (kept alive)
  bool khat_ready = false;
  bool sd_ready = false;        // SD step size computed (it depends on the PSF only)
  ~red_problem_s();
};

struct red_batch_s {
  std::vector<red_problem_s *> probs;
  int ve = 0, k = 1, m = 0, freeze = 0;
  std::vector<red::ProbDev> pds;
  red::ProbDev *d_pds = nullptr;
  red::ProbState *d_states = nullptr;
  red::ProbState *h_states = nullptr;   // pinned
  float **d_ptrs = nullptr;
  float **h_ptrs = nullptr;             // pinned
  red::Plan plan;
  red::LaunchCfg lc;
  bool ready = false;
  // observation-dependent set-up of all deblurring problems at once (host-buffer solves):
  // three-pass Fourier items over every problem, and one constants item per 256 frequencies
  red::Plan pre;
  red::Item *d_pre_const = nullptr;
  int n_pre_const = 0;
  bool pre_ready = false;
  std::vector<red::CycleOp> ops;
  int fp_per_cycle = 1;
  cudaGraphExec_t graph = nullptr;
  uint64_t graph_kernels = 0;
  cudaStream_t cap_stream = nullptr;
  std::string tune_key;
  bool phase_timing = false;
  struct PhaseEv { int phase; cudaEvent_t a, b; };
  std::vector<PhaseEv> phase_events;     // launch order within one solve
  size_t phase_next = 0;                 // events used by the current / last solve
  ~red_batch_s();
};

namespace red {
void problem_upload_pd(red_problem_s *P);
void problem_precompute(red_problem_s *P, cudaStream_t s);
red_status batch_solve_impl(red_batch_s *b, const void *const *x0, int max_calls, double tol,
                            void *const *xout, red_stats *stats, cudaStream_t s);
red_batch_s *batch_new(const red_problem *problems, int n);
}  // namespace red
