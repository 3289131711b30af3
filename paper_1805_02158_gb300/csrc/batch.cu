// Batched solves (Algorithm 3 for many problems at once), cycles replayed as CUDA graphs,
// and the launch-shape autotuner.
//
// A batch owns a device table of problem descriptors and per-problem termination states.
// Every phase of a cycle is one launch over all problems (work lists of tiles, rows,
// columns, chunks; one cluster per super-resolution problem). Problems that have
// terminated skip their work inside the kernels, so the host only reads the states back
// once per cycle (or never, for a fixed FP-call budget) and a cycle is a fixed sequence
// of launches on fixed ring slots, captured once as a CUDA graph and replayed.
//
// Autotuner: the launch shapes (NLM CTA height, rows per row-FFT CTA, columns per
// column-FFT CTA, CTAs per super-resolution cluster) only change how fixed work units
// are grouped into CTAs, never a pixel's arithmetic, so every candidate gives bitwise the
// same result. Candidates are timed with CUDA events on the batch's own buffers; the
// choice is cached per process and, if RED_TUNE_CACHE names a file, across processes.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <functional>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "common.cuh"
#include "red.h"
#include "runtime.h"

using namespace red;

red_batch_s::~red_batch_s() {
  for (auto &e : phase_events) {
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  if (graph) cudaGraphExecDestroy(graph);
  if (cap_stream) cudaStreamDestroy(cap_stream);
  plan.release();
  pre.release();
  if (d_pre_const) cudaFree(d_pre_const);
  if (d_pds) cudaFree(d_pds);
  if (d_states) cudaFree(d_states);
  if (d_ptrs) cudaFree(d_ptrs);
  if (h_states) cudaFreeHost(h_states);
  if (h_ptrs) cudaFreeHost(h_ptrs);
}

namespace red {

namespace {

std::mutex g_tune_mu;
std::map<std::string, LaunchCfg> g_tune_mem;

bool tune_lookup(const std::string &key, LaunchCfg &out) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune_mem.find(key);
  if (it != g_tune_mem.end()) {
    out = it->second;
    return true;
  }
  const char *path = std::getenv("RED_TUNE_CACHE");
  if (!path || !*path) return false;
  std::ifstream in(path);
  std::string line;
  while (std::getline(in, line)) {
    std::istringstream ss(line);
    std::string k;
    LaunchCfg c;
    if (ss >> k >> c.nlm_wy >> c.nlm_occ >> c.fft_rows >> c.fft_cols >> c.sr_cluster >> c.fft_cluster &&
        k == key) {
      g_tune_mem[key] = c;
      out = c;
      return true;
    }
  }
  return false;
}

void tune_store(const std::string &key, const LaunchCfg &c) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_mem[key] = c;
  const char *path = std::getenv("RED_TUNE_CACHE");
  if (!path || !*path) return;
  std::ofstream out(path, std::ios::app);
  out << key << " " << c.nlm_wy << " " << c.nlm_occ << " " << c.fft_rows << " " << c.fft_cols << " " << c.sr_cluster
      << " " << c.fft_cluster << "\n";
}

std::string tune_key(const red_batch_s *b) {
  std::vector<std::string> parts;
  for (auto *p : b->probs) {
    std::ostringstream o;
    o << p->cfg.task << "x" << p->cfg.height << "x" << p->cfg.width << "s" << p->cfg.storage;
    parts.push_back(o.str());
  }
  std::sort(parts.begin(), parts.end());
  std::ostringstream key;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop;
  cudaGetDeviceProperties(&prop, dev);
  key << "v7|sm" << prop.major << prop.minor << "x" << prop.multiProcessorCount << "|";
  for (size_t i = 0; i < parts.size(); ++i) key << (i ? "," : "") << parts[i];
  std::string k = key.str();
  std::replace(k.begin(), k.end(), ' ', '_');
  return k;
}

void upload_pds(red_batch_s *b) {
  for (size_t i = 0; i < b->pds.size(); ++i) {
    b->pds[i].n_row_items = b->plan.n_row_items[i];
    b->pds[i].st = b->d_states + i;
  }
  CUDA_OK(cudaMemcpy(b->d_pds, b->pds.data(), sizeof(ProbDev) * b->pds.size(),
                     cudaMemcpyHostToDevice));
  prepare_launch_attrs(b->plan);
}

float time_ms(cudaStream_t s, int reps, const std::function<void()> &fn) {
  cudaEvent_t e0, e1;
  CUDA_OK(cudaEventCreate(&e0));
  CUDA_OK(cudaEventCreate(&e1));
  fn();  // warm-up
  CUDA_OK(cudaEventRecord(e0, s));
  for (int i = 0; i < reps; ++i) fn();
  CUDA_OK(cudaEventRecord(e1, s));
  CUDA_OK(cudaEventSynchronize(e1));
  float ms = 0.f;
  CUDA_OK(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ms / reps;
}

// Coordinate-wise search over the launch-shape knobs, each timed on the batch.
LaunchCfg autotune(red_batch_s *b, cudaStream_t s) {
  LaunchCfg best;
  const int n = (int)b->probs.size();
  StepArgs sa{0, 1, nullptr, nullptr, 0};
  const int reps = 5;
  auto rebuild = [&](const LaunchCfg &c) {
    b->plan.build(b->pds, c);
    upload_pds(b);
  };
  // NLM warps per CTA and register budget. The shapes are within a few per cent of each
  // other, so every candidate is timed in three interleaved rounds and its best round
  // counts: a clock still ramping up, or one stray delay, does not decide the choice.
  {
    struct Cand {
      int occ, wy;
      float t;
    };
    std::vector<Cand> cands;
    for (int occ : {4, 3})
      for (int wy : {1, 2, 4}) cands.push_back({occ, wy, 1e30f});
    LaunchCfg c = best;
    for (int round = 0; round < 3; ++round)
      for (auto &cd : cands) {
        c.nlm_wy = cd.wy;
        c.nlm_occ = cd.occ;
        rebuild(c);
        const float t = time_ms(s, 2 * reps, [&] {
          CUDA_OK(launch_nlm(b->d_pds, b->plan.d_items + b->plan.off_nlm, b->plan.n_nlm, cd.wy, sa,
                             0, s, nullptr, cd.occ));
        });
        cd.t = std::min(cd.t, t);
      }
    float bt = 1e30f;
    for (const auto &cd : cands)
      if (cd.t < bt) {
        bt = cd.t;
        best.nlm_wy = cd.wy;
        best.nlm_occ = cd.occ;
      }
  }
  bool has_deblur = false, has_sr = false;
  for (auto *p : b->probs) (p->cfg.task == RED_DEBLUR ? has_deblur : has_sr) = true;
  if (has_deblur) {
    // fused cluster solve (0 = three passes for every problem)
    float bt = 1e30f;
    LaunchCfg c = best;
    for (int q : {16, 8, 4, 0}) {
      c.fft_cluster = q;
      if (q > 0) {
        int ac = 0, bc = 0, cgc = 0, tm = 0, th = 0, aa = 0, bb = 0;
        for (auto *p : b->probs)
          if (p->cfg.task == RED_DEBLUR) {
            fft_cluster_caps(p->pd.H, p->pd.W, q, &ac, &bc, &cgc);
            tm = std::max(tm, p->pd.M); th = std::max(th, p->pd.H);
            aa = std::max(aa, ac); bb = std::max(bb, bc);
          }
        const int smem = std::min(fft_cluster_smem(tm, th, aa, bb, 0), 220 * 1024);
        if (fft_cluster_prepare(smem, q) != cudaSuccess || fft_cluster_max_active(q, smem) < 1) {
          cudaGetLastError();
          continue;
        }
      }
      rebuild(c);
      const Plan &pl = b->plan;
      const float t = time_ms(s, reps, [&] { launch_fft_solve(b->d_pds, pl, sa, s); });
      if (t < bt) { bt = t; best.fft_cluster = q; }
    }
    bt = 1e30f;
    c = best;
    for (int r : {0, 2, 4, 8, 16}) {
      c.fft_rows = r;
      rebuild(c);
      const Plan &pl = b->plan;
      const float t = time_ms(s, reps, [&] {
        CUDA_OK(launch_fft_r2c(b->d_pds, pl.d_items + pl.off_rows, pl.n_rows, pl.row_tw_cap,
                               pl.row_buf_cap, nullptr, nullptr, 0, s));
        CUDA_OK(launch_fft_c2r(b->d_pds, pl.d_items + pl.off_rows, pl.n_rows, pl.row_tw_cap,
                               pl.row_buf_cap, sa, s));
      });
      if (t < bt) { bt = t; best.fft_rows = r; }
    }
    bt = 1e30f;
    c = best;
    for (int q : {0, 2, 4, 8}) {
      c.fft_cols = q;
      rebuild(c);
      const Plan &pl = b->plan;
      const float t = time_ms(s, reps, [&] {
        CUDA_OK(launch_fft_cols(b->d_pds, pl.d_items + pl.off_cols, pl.n_cols, pl.col_tw_cap,
                                pl.col_buf_cap, 1, nullptr, 0, s));
      });
      if (t < bt) { bt = t; best.fft_cols = q; }
    }
  }
  if (has_sr) {
    float bt = 1e30f;
    LaunchCfg c = best;
    // 8 and 16 CTAs per problem, and the sizes between them: with one CTA per SM a
    // cluster must fit in one GPC, so which sizes pack best depends on the batch
    for (int cl : {8, 10, 12, 16}) {
      c.sr_cluster = cl;
      rebuild(c);
      const Plan &pl = b->plan;
      if (pl.lc.sr_cluster != cl) continue;   // the plan had to change it
      prepare_launch_attrs(pl);
      const float t = time_ms(s, 1, [&] {
        CUDA_OK(launch_sr_step(b->d_pds, pl.d_sr, pl.n_sr, cl, pl.sr_cap, sa, s));
      });
      if (t < bt) { bt = t; best.sr_cluster = cl; }
    }
  }
  (void)n;
  return best;
}

// Phase timing: events are created once per (cycle, op, phase) of a solve and recorded
// around the phase's launches; with timing on, cycles are launched directly (no graph),
// so every launch of the solve keeps its own event pair.
struct PhaseScope {
  red_batch_s *b;
  cudaStream_t s;
  size_t &next;
  void begin(int phase) {
    if (!b->phase_timing) return;
    if (next >= b->phase_events.size()) {
      red_batch_s::PhaseEv e{phase, nullptr, nullptr};
      CUDA_OK(cudaEventCreate(&e.a));
      CUDA_OK(cudaEventCreate(&e.b));
      b->phase_events.push_back(e);
    }
    CUDA_OK(cudaEventRecord(b->phase_events[next].a, s));
  }
  void end() {
    if (!b->phase_timing) return;
    CUDA_OK(cudaEventRecord(b->phase_events[next].b, s));
    ++next;
  }
};

void enqueue_cycle(red_batch_s *b, cudaStream_t s) {
  const int n = (int)b->probs.size();
  const Plan &pl = b->plan;
  PhaseScope ps{b, s, b->phase_next};
  for (const CycleOp &op : b->ops) {
    if (op.kind == 0) {
      StepArgs sa{op.src, op.dst, nullptr, nullptr, 1, op.skip_frozen};
      ps.begin(RED_PHASE_NLM);
      CUDA_OK(launch_nlm(b->d_pds, pl.d_items + pl.off_nlm, pl.n_nlm, pl.lc.nlm_wy, sa, 0, s,
                         nullptr, pl.lc.nlm_occ));
      ps.end();
      if (pl.n_rows || pl.n_fused) {
        ps.begin(RED_PHASE_FFT);
        launch_fft_solve(b->d_pds, pl, sa, s);
        ps.end();
      }
      if (pl.n_sr) {
        ps.begin(RED_PHASE_CG);
        CUDA_OK(launch_sr_step(b->d_pds, pl.d_sr, pl.n_sr, pl.lc.sr_cluster, pl.sr_cap, sa, s));
        ps.end();
      }
    } else {
      VeArgs va{};
      for (size_t i = 0; i < op.slots.size(); ++i) va.slots[i] = op.slots[i];
      va.nvec = (int)op.slots.size();
      va.out_slot = op.out;
      va.update_state = 1;
      va.skip_frozen = op.skip_frozen;
      ps.begin(RED_PHASE_GRAM);
      CUDA_OK(launch_gram(b->d_pds, pl.d_items + pl.off_chunks, pl.n_chunks, va, s));
      ps.end();
      ps.begin(RED_PHASE_COMBINE);
      VeArgs vc = va;
      vc.skip_frozen = 0;   // frozen problems combine with their stored xi
      CUDA_OK(launch_combine(b->d_pds, pl.d_items + pl.off_chunks, pl.n_chunks, vc, s));
      ps.end();
    }
  }
}

void ensure_ready(red_batch_s *b, cudaStream_t s) {
  if (!b->ready) {
    LaunchCfg c;
    if (!tune_lookup(b->tune_key, c)) {
      c = autotune(b, s);
      tune_store(b->tune_key, c);
    }
    if (fft_cluster_override() >= 0) c.fft_cluster = fft_cluster_override();
    if (sr_cluster_override() > 0) c.sr_cluster = sr_cluster_override();
    nlm_shape_override(&c.nlm_wy, &c.nlm_occ);
    b->lc = c;
    b->plan.build(b->pds, c);
    upload_pds(b);
    if (b->graph) {
      cudaGraphExecDestroy(b->graph);
      b->graph = nullptr;
    }
    b->ready = true;
  }
  const char *ng = std::getenv("RED_NO_GRAPHS");
  if (!b->graph && !b->phase_timing && !(ng && *ng == '1')) {
    if (!b->cap_stream) CUDA_OK(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
    const uint64_t before = red_kernel_launches();
    CUDA_OK(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeRelaxed));
    try {
      enqueue_cycle(b, b->cap_stream);
    } catch (...) {
      cudaGraph_t g;
      cudaStreamEndCapture(b->cap_stream, &g);
      if (g) cudaGraphDestroy(g);
      throw;
    }
    cudaGraph_t g = nullptr;
    CUDA_OK(cudaStreamEndCapture(b->cap_stream, &g));
    b->graph_kernels = red_kernel_launches() - before;
    count_launches((uint64_t)0 - b->graph_kernels);   // captured, not yet executed
    cudaError_t e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    CUDA_OK(e);
  }
}

void run_cycle(red_batch_s *b, cudaStream_t s) {
  if (b->graph) {
    CUDA_OK(cudaGraphLaunch(b->graph, s));
    count_launches(b->graph_kernels);
  } else {
    enqueue_cycle(b, s);
  }
}

}  // namespace

red_batch_s *batch_new(const red_problem *problems, int n) {
  CHECK_ARG(problems != nullptr && n >= 1, "empty batch");
  std::unique_ptr<red_batch_s> b(new red_batch_s());
  for (int i = 0; i < n; ++i) {
    CHECK_ARG(problems[i] != nullptr, "null problem in batch");
    b->probs.push_back(problems[i]);
  }
  const red_config &c0 = b->probs[0]->cfg;
  b->ve = c0.ve;
  b->k = c0.ve_k;
  b->m = c0.ve_m;
  b->freeze = c0.ve_freeze;
  for (auto *p : b->probs)
    CHECK_ARG(p->cfg.ve == b->ve && p->cfg.ve_k == b->k && p->cfg.ve_m == b->m &&
                  p->cfg.ve_freeze == b->freeze,
              "all problems of a batch need the same ve, ve_k, ve_m and ve_freeze");
  for (auto *p : b->probs) b->pds.push_back(p->pd);
  CUDA_OK(cudaMalloc(&b->d_pds, sizeof(ProbDev) * n));
  CUDA_OK(cudaMalloc(&b->d_states, sizeof(ProbState) * n));
  CUDA_OK(cudaMemset(b->d_states, 0, sizeof(ProbState) * n));
  CUDA_OK(cudaMalloc(&b->d_ptrs, sizeof(float *) * 2 * n));
  CUDA_OK(cudaMallocHost(&b->h_states, sizeof(ProbState) * n));
  CUDA_OK(cudaMallocHost(&b->h_ptrs, sizeof(float *) * 2 * n));
  b->ops = cycle_ops(b->ve, b->k, b->m, b->freeze);
  b->fp_per_cycle = 0;
  for (auto &op : b->ops) b->fp_per_cycle += op.kind == 0;
  b->tune_key = tune_key(b.get());
  return b.release();
}

red_status batch_solve_impl(red_batch_s *b, const void *const *x0, int max_calls, double tol,
                            void *const *xout, red_stats *stats, cudaStream_t s) {
  CHECK_ARG(b && x0 && xout, "null argument");
  CHECK_ARG(max_calls >= 0, "max_fp_calls must be >= 0");
  const auto t0 = std::chrono::steady_clock::now();
  const int n = (int)b->probs.size();
  for (int i = 0; i < n; ++i) CHECK_ARG(x0[i] && xout[i], "null image pointer");
  ensure_ready(b, s);
  for (int i = 0; i < n; ++i) {
    b->h_ptrs[i] = const_cast<float *>(static_cast<const float *>(x0[i]));
    b->h_ptrs[n + i] = static_cast<float *>(xout[i]);
    ProbState &st = b->h_states[i];
    std::memset(&st, 0, sizeof(st));
    st.max_calls = max_calls;
    st.tol = tol;
    st.ve_stop_tol = b->probs[i]->cfg.ve_stop_tol;
    st.done = max_calls <= 0 ? 1 : 0;
  }
  CUDA_OK(cudaMemcpyAsync(b->d_ptrs, b->h_ptrs, sizeof(float *) * 2 * n, cudaMemcpyHostToDevice, s));
  CUDA_OK(cudaMemcpyAsync(b->d_states, b->h_states, sizeof(ProbState) * n, cudaMemcpyHostToDevice, s));
  CUDA_OK(launch_copy_slots(b->d_pds, b->plan.d_items + b->plan.off_chunks, b->plan.n_chunks, 0, 0,
                            b->d_ptrs, s));
  b->phase_next = 0;
  // a frozen cycle makes one FP step fewer: the budget may need more cycles than the
  // full-cycle count, after which the states are read back every cycle
  const int full_cycles = max_calls <= 0 ? 0 : (max_calls + b->fp_per_cycle - 1) / b->fp_per_cycle;
  const int min_steps = b->freeze > 0 ? b->fp_per_cycle - 1 : b->fp_per_cycle;
  const int max_cycles = max_calls <= 0 ? 0 : (max_calls + min_steps - 1) / min_steps;
  for (int c = 0; c < max_cycles; ++c) {
    run_cycle(b, s);
    if ((tol > 0.0 || c + 1 >= full_cycles) && c + 1 < max_cycles) {
      CUDA_OK(cudaMemcpyAsync(b->h_states, b->d_states, sizeof(ProbState) * n, cudaMemcpyDeviceToHost, s));
      CUDA_OK(cudaStreamSynchronize(s));
      bool all = true;
      for (int i = 0; i < n; ++i) all = all && b->h_states[i].done;
      if (all) break;
    }
  }
  CUDA_OK(launch_copy_slots(b->d_pds, b->plan.d_items + b->plan.off_chunks, b->plan.n_chunks, 1, 0,
                            b->d_ptrs + n, s));
  CUDA_OK(cudaMemcpyAsync(b->h_states, b->d_states, sizeof(ProbState) * n, cudaMemcpyDeviceToHost, s));
  CUDA_OK(cudaStreamSynchronize(s));
  const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  red_status ret = RED_OK;
  for (int i = 0; i < n; ++i) {
    const ProbState &st = b->h_states[i];
    if (tol > 0.0 && !st.converged) ret = RED_ENOT_CONVERGED;
    if (stats) {
      stats[i].fp_calls = st.calls;
      stats[i].ve_steps = st.ve_steps;
      stats[i].ve_breakdowns = st.ve_breakdowns;
      stats[i].converged = st.converged;
      stats[i].rel_change = st.rel_change;
      stats[i].sum_abs_gamma = st.sum_abs_gamma;
      stats[i].ms_total = ms;
    }
  }
  return ret;
}

}  // namespace red

extern "C" {

red_status red_batch_create(const red_problem *problems, int n, red_batch *out) {
  return guarded([&] {
    CHECK_ARG(out != nullptr, "null output");
    *out = batch_new(problems, n);
    return RED_OK;
  });
}

red_status red_batch_destroy(red_batch b) {
  return guarded([&] {
    delete b;
    return RED_OK;
  });
}

red_status red_batch_solve(red_batch b, const void *const *x0_dev, int max_fp_calls,
                           double rel_tol, void *const *x_out_dev, red_stats *stats,
                           void *stream) {
  return guarded([&] {
    return batch_solve_impl(b, x0_dev, max_fp_calls, rel_tol, x_out_dev, stats,
                            static_cast<cudaStream_t>(stream));
  });
}

red_status red_batch_set_phase_timing(red_batch b, int enable) {
  return guarded([&] {
    CHECK_ARG(b != nullptr, "null batch");
    if (b->phase_timing != (enable != 0)) {
      b->phase_timing = enable != 0;
      if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
      }
    }
    return RED_OK;
  });
}

red_status red_batch_phase_ms(red_batch b, int phase, double *avg_ms, int *launches) {
  return guarded([&] {
    CHECK_ARG(b != nullptr && avg_ms != nullptr, "null argument");
    double sum = 0.0;
    int cnt = 0;
    for (size_t i = 0; i < b->phase_next && i < b->phase_events.size(); ++i) {
      const auto &e = b->phase_events[i];
      if (e.phase != phase) continue;
      float ms = 0.f;
      CUDA_OK(cudaEventElapsedTime(&ms, e.a, e.b));
      sum += ms;
      ++cnt;
    }
    *avg_ms = cnt ? sum / cnt : 0.0;
    if (launches) *launches = cnt;
    return RED_OK;
  });
}

red_status red_batch_describe(red_batch b, char *buf, size_t len) {
  return guarded([&] {
    CHECK_ARG(b != nullptr && buf != nullptr && len > 0, "null argument");
    const Plan &pl = b->plan;
    const LaunchCfg &c = b->lc;
    std::ostringstream o;
    o << "{\"tuned\": " << (b->ready ? "true" : "false") << ", \"nlm_warps_per_cta\": " << c.nlm_wy
      << ", \"nlm_ctas_per_sm\": " << c.nlm_occ
      << ", \"nlm_ctas\": " << pl.n_nlm << ", \"fft_cluster\": " << pl.fused_ncta
      << ", \"fft_cluster_problems\": " << pl.n_fused << ", \"fft_row_ctas\": " << pl.n_rows
      << ", \"fft_col_ctas\": " << pl.n_cols << ", \"sr_cluster\": " << c.sr_cluster
      << ", \"sr_problems\": " << pl.n_sr << ", \"chunk_ctas\": " << pl.n_chunks
      << ", \"graph\": " << (b->graph ? "true" : "false") << ", \"graph_kernels_per_cycle\": "
      << b->graph_kernels << "}";
    const std::string s = o.str();
    const size_t n = std::min(len - 1, s.size());
    std::memcpy(buf, s.data(), n);
    buf[n] = 0;
    return RED_OK;
  });
}

red_status red_solve(red_problem p, const void *x0_dev, int max_fp_calls, double rel_tol,
                     void *x_out_dev, red_stats *stats, void *stream) {
  return guarded([&] {
    CHECK_ARG(p != nullptr, "null problem");
    if (!p->own_batch) {
      red_problem one = p;
      p->own_batch = batch_new(&one, 1);
    }
    const void *x0[1] = {x0_dev};
    void *xo[1] = {x_out_dev};
    return batch_solve_impl(p->own_batch, x0, max_fp_calls, rel_tol, xo, stats,
                            static_cast<cudaStream_t>(stream));
  });
}

// The set-up that depends on y (Eq. (7): the half spectrum of y, then C and G) for every
// deblurring problem of the batch in three launches (rows, columns, constants) instead of
// three per problem; the same arithmetic, item for item, as problem_precompute. The PSF
// spectrum (and an SD problem's step size) comes from the problem's creation; where one is
// missing, every problem takes the per-problem set-up. SR problems form b0 on their own.
static void batch_precompute(red_batch_s *b, cudaStream_t s) {
  bool ready = true;
  for (auto *p : b->probs)
    if (p->cfg.task == RED_DEBLUR &&
        (!p->khat_ready || (p->cfg.baseline == RED_BASE_SD && !p->sd_ready)))
      ready = false;
  if (!ready) {
    for (auto *p : b->probs) problem_precompute(p, s);
    return;
  }
  if (!b->pre_ready) {
    LaunchCfg three = b->lc;
    three.fft_cluster = 0;   // every deblurring problem on the three-pass items
    b->pre.build(b->pds, three);
    std::vector<Item> ci;
    for (int i = 0; i < (int)b->pds.size(); ++i)
      if (b->pds[i].task == kDeblur)
        for (int f = 0; f < b->pds[i].H * b->pds[i].Wh; f += 256) ci.push_back({i, f, 0, 0});
    if (!ci.empty()) {
      CUDA_OK(cudaMalloc(&b->d_pre_const, ci.size() * sizeof(Item)));
      CUDA_OK(cudaMemcpy(b->d_pre_const, ci.data(), ci.size() * sizeof(Item), cudaMemcpyHostToDevice));
    }
    b->n_pre_const = (int)ci.size();
    b->pre_ready = true;
  }
  const Plan &pl = b->pre;
  prepare_launch_attrs(pl);
  CUDA_OK(launch_fft_r2c(b->d_pds, pl.d_items + pl.off_rows, pl.n_rows, pl.row_tw_cap,
                         pl.row_buf_cap, nullptr, nullptr, kFftSrcY, s));
  CUDA_OK(launch_fft_cols(b->d_pds, pl.d_items + pl.off_cols, pl.n_cols, pl.col_tw_cap,
                          pl.col_buf_cap, 0, nullptr, 0, s));
  CUDA_OK(launch_spectral_constants_items(b->d_pds, b->d_pre_const, b->n_pre_const, s));
  for (auto *p : b->probs)
    if (p->cfg.task != RED_DEBLUR) problem_precompute(p, s);
}

red_status red_batch_solve_host(red_batch b, const float *const *y_host,
                                const float *const *x0_host, int max_fp_calls, double rel_tol,
                                float *const *x_out_host, red_stats *stats, void *stream) {
  return guarded([&] {
    CHECK_ARG(b && x0_host && x_out_host, "null argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int n = (int)b->probs.size();
    std::vector<const void *> x0(n);
    std::vector<void *> xo(n);
    for (int i = 0; i < n; ++i) {
      red_problem_s *p = b->probs[i];
      char *blk = static_cast<char *>(p->block);
      if (y_host) {
        CHECK_ARG(y_host[i] != nullptr, "null y");
        const size_t ny = (size_t)p->pd.lh * p->pd.lw;
        CUDA_OK(cudaMemcpyAsync(blk + p->L.y, y_host[i], ny * 4, cudaMemcpyHostToDevice, s));
      }
      // stage x0 in the problem's scratch buffer; the result comes back through it too
      float *tmp = reinterpret_cast<float *>(blk + p->L.tmp);
      CUDA_OK(cudaMemcpyAsync(tmp, x0_host[i], (size_t)p->pd.N * 4, cudaMemcpyHostToDevice, s));
      x0[i] = tmp;
      xo[i] = tmp;
    }
    if (y_host) batch_precompute(b, s);
    red_status st = batch_solve_impl(b, x0.data(), max_fp_calls, rel_tol, xo.data(), stats, s);
    for (int i = 0; i < n; ++i) {
      red_problem_s *p = b->probs[i];
      CUDA_OK(cudaMemcpyAsync(x_out_host[i], xo[i], (size_t)p->pd.N * 4, cudaMemcpyDeviceToHost, s));
    }
    CUDA_OK(cudaStreamSynchronize(s));
    return st;
  });
}

}  // extern "C"
