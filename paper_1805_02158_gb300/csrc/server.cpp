// Serving loop: continuous batching of RED solves (Algorithm 3 per request) of different
// sizes and tasks, admitted by device-memory footprint.
//
// One scheduler thread owns the GPU work. Requests are grouped by task, size class and
// extrapolation settings (ve, ve_k, ve_m); every group has its own stream and advances one cycle of
// Algorithm 3 at a time, independently of the other groups, so a deblurring group is not
// held back by the slower super-resolution CG of another. The loop
//   1. admits waiting requests (FIFO) while a slot is free and the request's device
//      footprint fits in the budget: it takes an idle problem of the same shape and
//      physics from the pool (or creates one), uploads y, recomputes the constants,
//      writes x0 into ring slot 0 and arms the request's termination state;
//   2. for every group whose cycle in flight has completed: reads the termination states
//      (copied back at the end of the cycle), returns finished results to host memory
//      and puts their problems back in the pool, freeing the slot;
//   3. for every idle group with running requests (new ones included): launches one
//      cycle (ve_m + ve_k FP steps and one extrapolation; one launch per phase over the
//      group's requests; requests that meet rel_tol or their budget stop on the device)
//      and the copy of the termination states, then records the group's event.
// Every running request starts each cycle from ring slot 0, so newly admitted and running
// requests share the same launches. A request's arithmetic never depends on the other
// requests in flight (fixed per-problem work decomposition, no cross-problem reductions),
// so its result is the same alone and in the mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <iomanip>
#include <map>
#include <memory>
#include <mutex>
#include <sstream>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"
#include "red.h"
#include "runtime.h"

using namespace red;

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t ticket = 0;
  red_config cfg{};
  std::vector<float> psf;
  std::vector<float> y;
  float *x_out = nullptr;
  int max_calls = 0;
  double tol = 0.0;
  size_t footprint = 0;
  std::string key;        // shape + physics: problems with the same key are reusable
  std::string group;      // (ve, ve_k, ve_m): requests that can share launches
  red_status status = RED_EBUSY;
  bool finished = false;
  red_stats stats{};
  Clock::time_point t_submit, t_admit, t_done;
  red_problem_s *prob = nullptr;   // set at admission: a pooled problem, or null (create)
};

std::string key_of(const red_config &c, const std::vector<float> &psf) {
  std::ostringstream o;
  // sigma, alpha and h printed so that they round-trip, and every PSF tap by its raw bits:
  // equal keys mean equal physics (no hash, so no collisions)
  o << std::setprecision(17);
  o << c.task << "|" << c.height << "x" << c.width << "|" << c.scale << "|" << c.psf_h << "x"
    << c.psf_w << "|" << c.sigma << "|" << c.alpha << "|" << c.nlm_h << "|" << c.ve << "|"
    << c.ve_k << "|" << c.ve_m << "|" << c.cg_iters << "|" << c.storage << "|" << c.baseline
    << "|" << c.sd_mu << "|" << c.ve_freeze << "|" << std::hex;
  for (float v : psf) {
    uint32_t u;
    std::memcpy(&u, &v, 4);
    o << std::setw(8) << std::setfill('0') << u;
  }
  return o.str();
}

// Requests of one task, extrapolation setting and size class share launches; small images
// are not paced by the FP steps of large ones (classes: up to 256^2, up to 512^2, larger).
std::string group_of(const red_config &c) {
  const long n = (long)c.height * c.width;
  const int size_class = n <= 256L * 256 ? 0 : (n <= 512L * 512 ? 1 : 2);
  std::ostringstream o;
  o << c.task << "|" << size_class << "|" << c.ve << "|" << c.ve_k << "|" << c.ve_m << "|"
    << c.ve_freeze;
  return o.str();
}

}  // namespace

struct red_server_s {
  size_t budget = 0;
  int max_slots = 1;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Request>> waiting;
  std::map<uint64_t, std::shared_ptr<Request>> all;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::thread th;
  // scheduler-thread state
  cudaStream_t stream = nullptr;
  size_t used = 0;                                       // bytes of allocated problems
  std::map<std::string, std::vector<red_problem_s *>> pool;
  std::map<std::string, size_t> pool_bytes;
  std::vector<std::shared_ptr<Request>> running;
  struct Group {                                         // requests sharing launches
    int ve = 0, k = 1, m = 0, freeze = 0;
    std::vector<red_problem_s *> members;                // as of the last table build
    red::Plan plan;
    std::vector<red::ProbDev> pds;
    red::ProbDev *d_pds = nullptr;
    int pds_cap = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;                          // end of the cycle in flight
    bool busy = false;
    std::vector<std::shared_ptr<Request>> inflight;      // requests of that cycle
    ProbState *h_states = nullptr;                       // pinned, one per inflight request
    int states_cap = 0;
  };
  std::map<std::string, std::unique_ptr<Group>> groups;
  float *d_stage = nullptr;                              // y / x0 staging (largest image)
  size_t stage_elems = 0;
  std::string sticky_error;
};

namespace {

void finish(red_server_s *S, const std::shared_ptr<Request> &r, red_status st) {
  std::lock_guard<std::mutex> lk(S->mu);
  r->status = st;
  r->finished = true;
  r->t_done = Clock::now();
  r->stats.ms_total = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
  S->cv_done.notify_all();
}

void ensure_stage(red_server_s *S, size_t elems) {
  if (elems <= S->stage_elems) return;
  if (S->d_stage) cudaFree(S->d_stage);
  S->d_stage = nullptr;
  CUDA_OK(cudaMalloc(&S->d_stage, elems * 4));
  S->stage_elems = elems;
}

// Frees idle pooled problems until `need` more bytes fit (largest first).
bool make_room(red_server_s *S, size_t need) {
  while (S->used + need > S->budget) {
    std::string best;
    size_t bb = 0;
    for (auto &kv : S->pool)
      if (!kv.second.empty() && S->pool_bytes[kv.first] > bb) {
        bb = S->pool_bytes[kv.first];
        best = kv.first;
      }
    if (best.empty()) return false;
    red_problem_s *p = S->pool[best].back();
    S->pool[best].pop_back();
    S->used -= bb;
    // a group whose last build included p must rebuild (its address may be reused)
    for (auto &kv : S->groups)
      if (std::find(kv.second->members.begin(), kv.second->members.end(), p) !=
          kv.second->members.end())
        kv.second->members.clear();
    delete p;
  }
  return true;
}

// Takes an idle problem for r (or creates one), loads y and x0, arms its state.
void admit(red_server_s *S, const std::shared_ptr<Request> &r) {
  cudaStream_t s = S->stream;
  const int H = r->cfg.height, W = r->cfg.width;
  const int lh = r->cfg.task == RED_SR ? H / r->cfg.scale : H;
  const int lw = r->cfg.task == RED_SR ? W / r->cfg.scale : W;
  ensure_stage(S, (size_t)H * W);
  CUDA_OK(cudaMemcpyAsync(S->d_stage, r->y.data(), (size_t)lh * lw * 4, cudaMemcpyHostToDevice, s));
  red_problem_s *P = r->prob;
  if (P) {
    red_status st = red_set_observation(P, S->d_stage, 0, s);
    if (st != RED_OK) throw Fail{st, red_last_error()};
  } else {
    // the bytes were reserved (S->used) when the request was admitted
    red_config c = r->cfg;
    c.psf = r->psf.data();
    red_problem out = nullptr;
    red_status st = red_create_problem(&c, S->d_stage, s, &out);
    if (st != RED_OK) {
      S->used -= r->footprint;
      throw Fail{st, red_last_error()};
    }
    P = out;
  }
  r->prob = P;
  // x0 = y for deblurring; pixel replication of y, edge-extended, for SR
  std::vector<float> x0;
  const float *x0p = r->y.data();
  if (r->cfg.task == RED_SR) {
    x0.resize((size_t)H * W);
    const int sc = r->cfg.scale;
    for (int i = 0; i < H; ++i)
      for (int j = 0; j < W; ++j) {
        const int li = std::min(i / sc, lh - 1), lj = std::min(j / sc, lw - 1);
        x0[(size_t)i * W + j] = r->y[(size_t)li * lw + lj];
      }
    x0p = x0.data();
  }
  char *blk = static_cast<char *>(P->block);
  if (P->pd.storage == 0) {
    CUDA_OK(cudaMemcpyAsync(blk + P->L.ring, x0p, (size_t)H * W * 4, cudaMemcpyHostToDevice, s));
  } else {
    // 16-bit history (bf16 or f16): stage through f32 and convert with the copy kernel
    CUDA_OK(cudaMemcpyAsync(blk + P->L.tmp, x0p, (size_t)H * W * 4, cudaMemcpyHostToDevice, s));
    CUDA_OK(launch_convert_to_slot(P->d_pd, reinterpret_cast<float *>(blk + P->L.tmp), 0, s));
  }
  ProbState st{};
  st.max_calls = r->max_calls;
  st.tol = r->tol;
  st.ve_stop_tol = r->cfg.ve_stop_tol;
  st.done = r->max_calls <= 0 ? 1 : 0;
  CUDA_OK(cudaMemcpyAsync(blk + P->L.state, &st, sizeof(st), cudaMemcpyHostToDevice, s));
  // the x0 host vector must outlive the copy
  CUDA_OK(cudaStreamSynchronize(s));
  r->t_admit = Clock::now();
  // the observation now lives on the device: a finished request keeps only its status and
  // statistics on the host
  std::vector<float>().swap(r->y);
  std::vector<float>().swap(r->psf);
}

// Launches one cycle of Algorithm 3 for the group's running requests on the group's
// stream, then the copy of their termination states and the group's event. The work
// lists and descriptor table are rebuilt (in stream order, buffers reused) only when the
// membership changed.
void launch_group_cycle(red_server_s::Group &g, std::vector<std::shared_ptr<Request>> members) {
  cudaStream_t s = g.stream;
  const int n = (int)members.size();
  std::vector<red_problem_s *> probs;
  for (auto &r : members) probs.push_back(r->prob);
  if (probs != g.members) {
    g.pds.clear();
    for (auto *p : probs) g.pds.push_back(p->pd);   // st = the problem's own state
    // fixed launch shapes, so that a request's arithmetic (its reduction orders included)
    // does not depend on which other requests share the launches
    LaunchCfg lc;
    lc.sr_cluster = 16;
    g.plan.build(g.pds, lc, s, true);
    for (int i = 0; i < n; ++i) g.pds[i].n_row_items = g.plan.n_row_items[i];
    if (n > g.pds_cap) {
      if (g.d_pds) cudaFree(g.d_pds);
      g.d_pds = nullptr;
      CUDA_OK(cudaMalloc(&g.d_pds, sizeof(ProbDev) * n));
      g.pds_cap = n;
    }
    CUDA_OK(cudaMemcpyAsync(g.d_pds, g.pds.data(), sizeof(ProbDev) * n, cudaMemcpyHostToDevice, s));
    prepare_launch_attrs(g.plan);
    g.members = probs;
  }
  for (const CycleOp &op : cycle_ops(g.ve, g.k, g.m, g.freeze)) {
    if (op.kind == 0) {
      StepArgs sa{op.src, op.dst, nullptr, nullptr, 1, op.skip_frozen};
      launch_fp_step(g.d_pds, g.plan, sa, 0, s);
    } else {
      VeArgs va{};
      for (size_t i = 0; i < op.slots.size(); ++i) va.slots[i] = op.slots[i];
      va.nvec = (int)op.slots.size();
      va.out_slot = op.out;
      va.update_state = 1;
      va.skip_frozen = op.skip_frozen;
      launch_ve(g.d_pds, n, g.plan, va, s);
    }
  }
  if (n > g.states_cap) {
    if (g.h_states) cudaFreeHost(g.h_states);
    g.h_states = nullptr;
    CUDA_OK(cudaMallocHost(&g.h_states, sizeof(ProbState) * n));
    g.states_cap = n;
  }
  for (int i = 0; i < n; ++i) {
    red_problem_s *P = probs[i];
    CUDA_OK(cudaMemcpyAsync(g.h_states + i, static_cast<char *>(P->block) + P->L.state,
                            sizeof(ProbState), cudaMemcpyDeviceToHost, s));
  }
  CUDA_OK(cudaEventRecord(g.done, s));
  g.inflight = std::move(members);
  g.busy = true;
}

// The group's cycle has completed: finished requests get their result and release their
// slot; the others stay running.
void complete_group_cycle(red_server_s *S, red_server_s::Group &g) {
  g.busy = false;
  std::vector<std::shared_ptr<Request>> done;
  for (size_t i = 0; i < g.inflight.size(); ++i) {
    auto &r = g.inflight[i];
    const ProbState &st = g.h_states[i];
    if (!st.done) continue;
    red_problem_s *P = r->prob;
    CUDA_OK(launch_fetch_slot(P->d_pd, st.final_slot,
                              reinterpret_cast<float *>(static_cast<char *>(P->block) + P->L.tmp),
                              g.stream));
    CUDA_OK(cudaMemcpyAsync(r->x_out, static_cast<char *>(P->block) + P->L.tmp,
                            (size_t)P->pd.N * 4, cudaMemcpyDeviceToHost, g.stream));
    CUDA_OK(cudaStreamSynchronize(g.stream));
    r->stats.fp_calls = st.calls;
    r->stats.ve_steps = st.ve_steps;
    r->stats.ve_breakdowns = st.ve_breakdowns;
    r->stats.converged = st.converged;
    r->stats.rel_change = st.rel_change;
    r->stats.sum_abs_gamma = st.sum_abs_gamma;
    done.push_back(r);
  }
  g.inflight.clear();
  for (auto &r : done) {
    S->pool[r->key].push_back(r->prob);
    r->prob = nullptr;
    S->running.erase(std::find(S->running.begin(), S->running.end(), r));
    finish(S, r, (r->tol > 0.0 && !r->stats.converged) ? RED_ENOT_CONVERGED : RED_OK);
  }
}

void release_group(red_server_s::Group &g) {
  if (g.stream) cudaStreamSynchronize(g.stream);
  g.plan.release();
  if (g.d_pds) cudaFree(g.d_pds);
  if (g.h_states) cudaFreeHost(g.h_states);
  if (g.done) cudaEventDestroy(g.done);
  if (g.stream) cudaStreamDestroy(g.stream);
  g = red_server_s::Group();
}

red_server_s::Group &group_for(red_server_s *S, const Request &r) {
  auto &g = S->groups[r.group];
  if (!g) {
    g.reset(new red_server_s::Group());
    g->ve = r.cfg.ve;
    g->k = r.cfg.ve_k;
    g->m = r.cfg.ve_m;
    g->freeze = r.cfg.ve_freeze;
    CUDA_OK(cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking));
    CUDA_OK(cudaEventCreateWithFlags(&g->done, cudaEventDisableTiming));
  }
  return *g;
}

void scheduler(red_server_s *S) {
  cudaSetDevice(S->device);
  while (true) {
    std::vector<std::shared_ptr<Request>> to_admit;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      if (S->running.empty() && S->waiting.empty()) {
        if (S->stop) break;
        S->cv_work.wait_for(lk, std::chrono::milliseconds(50));
        continue;
      }
      if (S->stop) {
        for (auto &r : S->waiting) {
          r->status = RED_ETIMEOUT;
          r->finished = true;
        }
        S->waiting.clear();
        S->cv_done.notify_all();
      }
      // FIFO admission by slots and device footprint
      // (an idle problem of the same key is taken now, so that make_room cannot free it
      // for a later request; a new problem's bytes are reserved now)
      while (!S->waiting.empty() &&
             (int)(S->running.size() + to_admit.size()) < S->max_slots) {
        auto r = S->waiting.front();
        auto &idle = S->pool[r->key];
        if (!idle.empty()) {
          r->prob = idle.back();
          idle.pop_back();
        } else {
          if (!make_room(S, r->footprint)) break;
          S->used += r->footprint;
          S->pool_bytes[r->key] = r->footprint;
        }
        S->waiting.pop_front();
        to_admit.push_back(r);
      }
    }
    bool progressed = !to_admit.empty();
    try {
      for (auto &r : to_admit) {
        try {
          admit(S, r);
          S->running.push_back(r);
        } catch (const Fail &e) {
          if (r->prob) {   // a pooled problem whose observation upload failed
            S->used -= S->pool_bytes[r->key];
            delete r->prob;
            r->prob = nullptr;
          }
          r->stats = red_stats{};
          finish(S, r, e.st);
        }
      }
      // completed cycles
      for (auto &kv : S->groups) {
        auto &g = *kv.second;
        if (!g.busy) continue;
        const cudaError_t q = cudaEventQuery(g.done);
        if (q == cudaErrorNotReady) continue;
        CUDA_OK(q);
        complete_group_cycle(S, g);
        progressed = true;
      }
      // next cycles of idle groups (newly admitted requests join here)
      std::map<std::string, std::vector<std::shared_ptr<Request>>> members;
      for (auto &r : S->running) members[r->group].push_back(r);
      for (auto &kv : members) {
        auto &g = group_for(S, *kv.second.front());
        if (g.busy) continue;
        launch_group_cycle(g, kv.second);
        progressed = true;
      }
    } catch (const Fail &e) {
      S->sticky_error = e.msg;
      for (auto &kv : S->groups)
        if (kv.second->stream) cudaStreamSynchronize(kv.second->stream);
      for (auto &r : S->running) {
        if (r->prob) {
          delete r->prob;
          r->prob = nullptr;
        }
        finish(S, r, e.st);
      }
      S->running.clear();
      S->used = 0;
      for (auto &kv : S->pool)
        for (auto *p : kv.second) delete p;
      S->pool.clear();
      for (auto &kv : S->groups) release_group(*kv.second);
      S->groups.clear();
      continue;
    }
    if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

}  // namespace

extern "C" {

red_status red_server_create(size_t hbm_budget_bytes, int max_slots, red_server *out) {
  return guarded([&] {
    CHECK_ARG(out != nullptr, "null output");
    CHECK_ARG(max_slots >= 1 && hbm_budget_bytes > 0, "need max_slots >= 1 and a budget");
    std::unique_ptr<red_server_s> S(new red_server_s());
    S->budget = hbm_budget_bytes;
    S->max_slots = max_slots;
    CUDA_OK(cudaGetDevice(&S->device));
    CUDA_OK(cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking));
    red_server_s *raw = S.get();
    S->th = std::thread([raw] { scheduler(raw); });
    *out = S.release();
    return RED_OK;
  });
}

red_status red_submit(red_server s, const red_config *cfg, const float *y_host, float *x_out_host,
                      int max_fp_calls, double rel_tol, uint64_t *ticket) {
  return guarded([&] {
    CHECK_ARG(s && cfg && y_host && x_out_host && ticket, "null argument");
    CHECK_ARG(max_fp_calls >= 0, "max_fp_calls must be >= 0");
    size_t fp = 0;
    red_status st = red_problem_footprint(cfg, &fp);
    if (st != RED_OK) return st;
    if (fp > s->budget) throw Fail{RED_ENOMEM, "request footprint exceeds the server budget"};
    auto r = std::make_shared<Request>();
    r->cfg = *cfg;
    r->psf.assign(cfg->psf, cfg->psf + (size_t)cfg->psf_h * cfg->psf_w);
    r->cfg.psf = nullptr;
    const size_t ny = cfg->task == RED_SR
                          ? (size_t)(cfg->height / cfg->scale) * (cfg->width / cfg->scale)
                          : (size_t)cfg->height * cfg->width;
    r->y.assign(y_host, y_host + ny);
    r->x_out = x_out_host;
    r->max_calls = max_fp_calls;
    r->tol = rel_tol;
    r->footprint = fp;
    r->key = key_of(r->cfg, r->psf);
    r->group = group_of(r->cfg);
    r->t_submit = Clock::now();
    {
      std::lock_guard<std::mutex> lk(s->mu);
      CHECK_ARG(!s->stop, "server is shutting down");
      r->ticket = s->next_ticket++;
      s->all[r->ticket] = r;
      s->waiting.push_back(r);
    }
    s->cv_work.notify_one();
    *ticket = r->ticket;
    return RED_OK;
  });
}

red_status red_poll(red_server s, uint64_t ticket, red_stats *stats) {
  return guarded([&] {
    CHECK_ARG(s != nullptr, "null server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    CHECK_ARG(it != s->all.end(), "unknown ticket");
    if (!it->second->finished) return RED_EBUSY;
    if (stats) *stats = it->second->stats;
    return it->second->status;
  });
}

red_status red_wait(red_server s, uint64_t ticket, int timeout_ms, red_stats *stats) {
  return guarded([&] {
    CHECK_ARG(s != nullptr, "null server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    CHECK_ARG(it != s->all.end(), "unknown ticket");
    auto r = it->second;
    auto pred = [&] { return r->finished; };
    if (timeout_ms < 0) {
      s->cv_done.wait(lk, pred);
    } else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred)) {
      return RED_ETIMEOUT;
    }
    if (stats) *stats = r->stats;
    return r->status;
  });
}

red_status red_server_destroy(red_server s) {
  return guarded([&] {
    if (!s) return RED_OK;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->th.joinable()) s->th.join();
    for (auto &kv : s->pool)
      for (auto *p : kv.second) delete p;
    for (auto &kv : s->groups) release_group(*kv.second);
    if (s->d_stage) cudaFree(s->d_stage);
    if (s->stream) cudaStreamDestroy(s->stream);
    delete s;
    return RED_OK;
  });
}

}  // extern "C"
