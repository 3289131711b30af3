// Host runtime of libred: problems, launch plans, batched solves (Algorithm 3) with cycles
// replayed as CUDA graphs, the launch-shape autotuner, and the C-ABI entry points.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <new>
#include <sstream>
#include <string>
#include <vector>

#include "common.cuh"
#include "red.h"
#include "runtime.h"

namespace red {

static std::atomic<uint64_t> g_launches{0};
void count_launches(uint64_t n) { g_launches += n; }

thread_local std::string g_err;
void set_error(const std::string &m) { g_err = m; }

// ---------------------------------------------------------------------------------------
// twiddle tables: e^{-2 pi i t / n}, t = 0..n (n + 1 entries), computed in double
// ---------------------------------------------------------------------------------------
static std::mutex g_tw_mu;
static std::map<int, float2 *> g_tw;

static const float2 *twiddles(int n) {
  std::lock_guard<std::mutex> lk(g_tw_mu);
  auto it = g_tw.find(n);
  if (it != g_tw.end()) return it->second;
  std::vector<float2> h(n + 1);
  const double two_pi = 6.283185307179586476925286766559;
  for (int t = 0; t <= n; ++t) {
    const double a = -two_pi * (double)t / (double)n;
    h[t] = make_float2((float)std::cos(a), (float)std::sin(a));
  }
  float2 *d = nullptr;
  CUDA_OK(cudaMalloc(&d, sizeof(float2) * (n + 1)));
  CUDA_OK(cudaMemcpy(d, h.data(), sizeof(float2) * (n + 1), cudaMemcpyHostToDevice));
  g_tw[n] = d;
  return d;
}

static bool is_2a3b(int n) {
  if (n < 1) return false;
  while (n % 2 == 0) n /= 2;
  while (n % 3 == 0) n /= 3;
  return n == 1;
}

// ---------------------------------------------------------------------------------------
// memory layout of one problem
// ---------------------------------------------------------------------------------------
struct Carve {
  size_t off = 0;
  size_t take(size_t bytes) {
    const size_t o = off;
    off += (bytes + 255) & ~size_t(255);
    return o;
  }
};

static Layout layout_for(const red_config &c, int nslots, int slot_stride) {
  Layout L{};
  Carve cv;
  const size_t N = (size_t)c.height * c.width;
  const size_t esz = c.storage == RED_F32 ? 4 : 2;
  const size_t Wh = (size_t)c.width / 2 + 1;
  const size_t nchunks = (N + kGramChunk - 1) / kGramChunk;
  const bool sr = c.task == RED_SR;
  const size_t lh = sr ? c.height / c.scale : c.height, lw = sr ? c.width / c.scale : c.width;
  L.ring = cv.take((size_t)nslots * slot_stride * esz);
  L.f = cv.take(N * 4);
  L.spec = sr ? 0 : cv.take((size_t)c.height * Wh * 8);
  L.kh = sr ? 0 : cv.take((size_t)c.height * Wh * 8);
  L.cc = sr ? 0 : cv.take((size_t)c.height * Wh * 8);
  L.gg = sr ? 0 : cv.take((size_t)c.height * Wh * 4);
  L.row_stats = cv.take((size_t)std::max(c.height, 32) * 8);   // rows, or cluster CTAs
  L.gram = cv.take(nchunks * kMaxPairs * 8);
  L.coef = cv.take(kMaxK * 8);
  L.gamma = cv.take(kMaxK * 8);
  L.state = cv.take(sizeof(ProbState));
  L.y = cv.take(lh * lw * 4);
  L.tmp = cv.take(N * 4);
  L.b0 = sr ? cv.take(N * 4) : 0;
  L.cx = sr ? cv.take(N * 4) : 0;
  L.cr = sr ? cv.take(N * 4) : 0;
  L.cp = sr ? cv.take(N * 4) : 0;
  L.cap = sr ? cv.take(N * 4) : 0;
  L.cz = sr ? cv.take(lh * lw * 4) : 0;
  L.psf = cv.take((size_t)c.psf_h * c.psf_w * 4);
  L.obj = cv.take(4 * 8);
  L.sd = cv.take(sizeof(SdParams));
  L.total = cv.off;
  return L;
}

static int nslots_for(const red_config &c) { return c.ve == RED_VE_NONE ? 2 : c.ve_k + 2; }
static int slot_stride_for(const red_config &c) {
  const size_t N = (size_t)c.height * c.width;
  return (int)((N + 63) / 64 * 64);
}

static void validate(const red_config *c) {
  CHECK_ARG(c != nullptr, "null config");
  CHECK_ARG(c->task == RED_DEBLUR || c->task == RED_SR, "task must be RED_DEBLUR or RED_SR");
  CHECK_ARG(c->height >= 8 && c->height <= 2048 && c->width >= 8 && c->width <= 2048,
            "image sides must be in [8, 2048]");
  CHECK_ARG(is_2a3b(c->height) && is_2a3b(c->width) && c->width % 2 == 0,
            "image sides must be 2^a 3^b and the width even");
  CHECK_ARG(c->psf != nullptr && c->psf_h >= 1 && c->psf_w >= 1 && (c->psf_h & 1) && (c->psf_w & 1),
            "psf must be given with odd sizes");
  CHECK_ARG(c->psf_h <= c->height && c->psf_w <= c->width, "psf larger than the image");
  CHECK_ARG(c->sigma > 0 && c->alpha > 0 && c->nlm_h > 0, "sigma, alpha and nlm_h must be > 0");
  if (c->task == RED_DEBLUR) CHECK_ARG(c->scale == 1, "deblurring needs scale 1");
  if (c->task == RED_SR) CHECK_ARG(c->scale >= 2 && c->height / c->scale >= 1 && c->width / c->scale >= 1,
                                   "super-resolution needs scale >= 2");
  CHECK_ARG(c->ve >= RED_VE_NONE && c->ve <= RED_VE_SVDMPE, "bad ve method");
  CHECK_ARG(c->ve_k >= 1 && c->ve_k <= kMaxK, "ve_k must be in [1, 12]");
  CHECK_ARG(c->ve_m >= 0 && c->ve_m <= 64, "ve_m must be in [0, 64]");
  CHECK_ARG(c->cg_iters >= 0 && c->cg_iters <= 1000, "cg_iters must be in [0, 1000]");
  if (c->nlm_patch != 5 || c->nlm_search != 11)
    throw Fail{RED_EUNSUPPORTED, "only 5x5 patches and 11x11 search windows are supported"};
  CHECK_ARG(c->storage == RED_F32 || c->storage == RED_BF16 || c->storage == RED_F16,
            "storage must be RED_F32, RED_BF16 or RED_F16");
  CHECK_ARG(c->baseline == RED_BASE_FP || c->baseline == RED_BASE_SD,
            "baseline must be RED_BASE_FP or RED_BASE_SD");
  CHECK_ARG(c->sd_mu >= 0.0 && std::isfinite(c->sd_mu), "sd_mu must be finite and >= 0");
  CHECK_ARG(c->ve_freeze >= 0, "ve_freeze must be >= 0");
  if (c->ve_freeze > 0) {
    CHECK_ARG(c->ve != RED_VE_NONE, "ve_freeze needs an extrapolation method");
    // a frozen cycle runs ve_m + ve_k - 1 baseline steps: at least one
    CHECK_ARG(c->ve_m + c->ve_k >= 2, "ve_freeze needs ve_m + ve_k >= 2");
  }
  CHECK_ARG(c->ve_stop_tol >= 0.0 && std::isfinite(c->ve_stop_tol),
            "ve_stop_tol must be finite and >= 0");
  if (c->ve_stop_tol > 0.0) {
    CHECK_ARG(c->ve != RED_VE_NONE, "ve_stop_tol needs an extrapolation method");
    // a frozen cycle has no last iterate to carry on from
    CHECK_ARG(c->ve_freeze == 0, "ve_stop_tol and ve_freeze do not combine");
  }
}

// ---------------------------------------------------------------------------------------
// plans: work-item lists for a set of problems under one launch configuration
// ---------------------------------------------------------------------------------------
static int auto_rows(int M) { return std::max(1, std::min(16, 2048 / M)); }
static int auto_cols(int H) {
  const int budget = 200 * 1024 / 8;
  return std::max(1, std::min(16, (budget - H) / (2 * fft_seq_stride(H))));
}

// Whether the device runs clusters of `ncta` CTAs with the cluster solve's largest
// shared-memory footprint (checked once per size).
static bool cluster_ok(int ncta) {
  static std::mutex mu;
  static std::map<int, bool> known;
  std::lock_guard<std::mutex> lk(mu);
  auto it = known.find(ncta);
  if (it != known.end()) return it->second;
  const int smem = 220 * 1024;
  bool ok = fft_cluster_prepare(smem, ncta) == cudaSuccess && fft_cluster_max_active(ncta, smem) >= 1;
  cudaGetLastError();
  known[ncta] = ok;
  return ok;
}

// RED_FFT_CLUSTER=<n> forces the cluster size of the fused Fourier solve (0: three passes).
int fft_cluster_override() {
  const char *e = std::getenv("RED_FFT_CLUSTER");
  return (e && *e) ? std::atoi(e) : -1;
}

// RED_SR_CLUSTER=<n> forces the cluster size of the super-resolution CG solve (8, 10, 12
// or 16).
int sr_cluster_override() {
  const char *e = std::getenv("RED_SR_CLUSTER");
  const int v = (e && *e) ? std::atoi(e) : -1;
  return (v == 8 || v == 10 || v == 12 || v == 16) ? v : -1;
}

// RED_NLM_SHAPE=<w>,<o> forces the NLM launch shape: w warp tiles per CTA (1, 2 or 4) at
// the register budget of o resident CTAs per SM (3 or 4). Other values are ignored.
void nlm_shape_override(int *wy, int *occ) {
  const char *e = std::getenv("RED_NLM_SHAPE");
  int w = 0, o = 0;
  if (!e || std::sscanf(e, "%d,%d", &w, &o) != 2) return;
  if ((w == 1 || w == 2 || w == 4) && (o == 3 || o == 4)) {
    *wy = w;
    *occ = o;
  }
}

void Plan::build(const std::vector<ProbDev> &pds, const LaunchCfg &cfg, cudaStream_t stream,
                 bool async) {
  if (!async) release();
  lc = cfg;
  if (lc.fft_cluster > 0 && !cluster_ok(lc.fft_cluster)) lc.fft_cluster = 0;
  std::vector<Item> nlm, rows, cols, chunks;
  std::vector<int> sr, fused;
  row_tw_cap = row_buf_cap = col_tw_cap = col_buf_cap = 0;
  fused_ncta = lc.fft_cluster;
  fused_tw_m = fused_tw_h = fused_a = fused_buf = fused_cg = 0;
  const int smem_limit = 220 * 1024;
  n_row_items.assign(pds.size(), 0);
  for (int p = 0; p < (int)pds.size(); ++p) {
    const ProbDev &d = pds[p];
    nlm_items(p, d.H, d.W, nlm);
    bool to_cluster = false;
    if (d.task == kDeblur && fused_ncta > 0) {
      int ac = 0, bc = 0, cgc = 0;
      fft_cluster_caps(d.H, d.W, fused_ncta, &ac, &bc, &cgc);
      const int tm = std::max(fused_tw_m, d.M), th = std::max(fused_tw_h, d.H);
      const int aa = std::max(fused_a, ac), bb = std::max(fused_buf, bc);
      if (fft_cluster_smem(tm, th, aa, bb, 0) <= smem_limit) {
        fused_tw_m = tm;
        fused_tw_h = th;
        fused_a = aa;
        fused_buf = bb;
        fused_cg = std::max(fused_cg, cgc);
        fused.push_back(p);
        to_cluster = true;
      }
    }
    if (d.task == kDeblur && !to_cluster) {
      const int rpi = lc.fft_rows > 0 ? lc.fft_rows : auto_rows(d.M);
      int cnt = 0;
      for (int r0 = 0; r0 < d.H; r0 += rpi, ++cnt) rows.push_back({p, r0, rpi, 0});
      n_row_items[p] = cnt;
      row_tw_cap = std::max(row_tw_cap, d.M);
      row_buf_cap = std::max(row_buf_cap, std::min(rpi, d.H) * fft_seq_stride(d.M));
      const int cpi = lc.fft_cols > 0 ? std::min(lc.fft_cols, auto_cols(d.H)) : auto_cols(d.H);
      for (int c0 = 0; c0 < d.Wh; c0 += cpi) cols.push_back({p, c0, cpi, 0});
      col_tw_cap = std::max(col_tw_cap, d.H);
      col_buf_cap = std::max(col_buf_cap, std::min(cpi, d.Wh) * fft_seq_stride(d.H));
    } else if (d.task == kSR) {
      sr.push_back(p);
    }
    for (int c = 0; c < d.n_chunks; ++c) chunks.push_back({p, c, 0, 0});
  }
  // stage C and G in shared memory only while two CTAs still fit on an SM
  if (fused_cg && fft_cluster_smem(fused_tw_m, fused_tw_h, fused_a, fused_buf, fused_cg) >
                      kClusterSmemTwoPerSm)
    fused_cg = 0;
  n_nlm = (int)nlm.size();
  n_rows = (int)rows.size();
  n_cols = (int)cols.size();
  n_chunks = (int)chunks.size();
  n_sr = (int)sr.size();
  off_nlm = 0;
  off_rows = off_nlm + n_nlm;
  off_cols = off_rows + n_rows;
  off_chunks = off_cols + n_cols;
  std::vector<Item> all;
  all.reserve(off_chunks + n_chunks);
  all.insert(all.end(), nlm.begin(), nlm.end());
  all.insert(all.end(), rows.begin(), rows.end());
  all.insert(all.end(), cols.begin(), cols.end());
  all.insert(all.end(), chunks.begin(), chunks.end());
  // device lists: grown when needed, uploaded synchronously or in stream order
  auto upload = [&](auto *&dev, size_t &cap, const auto &host) {
    using T = typename std::decay<decltype(host[0])>::type;
    const size_t n = std::max<size_t>(1, host.size());
    if (!dev || cap < n) {
      if (dev) cudaFree(dev);
      dev = nullptr;
      CUDA_OK(cudaMalloc(&dev, sizeof(T) * n));
      cap = n;
    }
    if (host.empty()) return;
    if (async)
      CUDA_OK(cudaMemcpyAsync(dev, host.data(), sizeof(T) * host.size(), cudaMemcpyHostToDevice, stream));
    else
      CUDA_OK(cudaMemcpy(dev, host.data(), sizeof(T) * host.size(), cudaMemcpyHostToDevice));
  };
  upload(d_items, items_cap, all);

  if (n_sr) upload(d_sr, sr_cap_n, sr);
  sr_cap = SrCaps{};
  if (n_sr) {
    // shared memory of the CG kernel grows with the band height: wide images need the
    // larger cluster
    auto caps_for = [&](int ncta) {
      SrCaps m;
      for (int p : sr) {
        const ProbDev &d = pds[p];
        SrCaps c;
        sr_caps(d.H, d.W, d.scale, d.kh, d.kw, ncta, &c);
        m.taps = std::max(m.taps, c.taps);
        m.rows = std::max(m.rows, c.rows);
        m.zrows = std::max(m.zrows, c.zrows);
        m.cols = std::max(m.cols, c.cols);
        m.zfloats = std::max(m.zfloats, c.zfloats);
        m.band = std::max(m.band, c.band);
        m.band_ext = std::max(m.band_ext, c.band_ext);
        m.spec737 = m.spec737 && c.spec737;
      }
      return m;
    };
    const int sr_limit = 227 * 1024;
    if (lc.sr_cluster < 1 || lc.sr_cluster > 16) lc.sr_cluster = 8;
    sr_cap = caps_for(lc.sr_cluster);
    if (sr_smem_bytes(sr_cap, 0) > sr_limit && lc.sr_cluster < 16) {
      lc.sr_cluster = 16;
      sr_cap = caps_for(16);
    }
    if (sr_smem_bytes(sr_cap, 0) > sr_limit)
      throw Fail{RED_EUNSUPPORTED, "super-resolution image too large for the CG kernel's shared memory"};
    const int sp = sr_cap.spec737;
    const int act0 = sr_max_active_clusters(lc.sr_cluster, sr_smem_bytes(sr_cap, 0), sp);
    if (act0 < 1) throw Fail{RED_EUNSUPPORTED, "the CG kernel's cluster does not fit on this device"};
    // the band's vectors in shared memory when they fit and as many clusters stay resident
    // as the launch needs
    const int smem1 = sr_smem_bytes(sr_cap, 1);
    sr_cap.resident = (smem1 <= sr_limit &&
                       sr_max_active_clusters(lc.sr_cluster, smem1, sp) >= std::min(n_sr, act0)) ? 1 : 0;
  }
  n_fused = (int)fused.size();
  if (n_fused) upload(d_fused, fused_cap, fused);
}

void prepare_launch_attrs(const Plan &pl) {
  CUDA_OK(nlm_prepare(pl.lc.nlm_wy));
  if (pl.n_fused)
    CUDA_OK(fft_cluster_prepare(fft_cluster_smem(pl.fused_tw_m, pl.fused_tw_h, pl.fused_a, pl.fused_buf,
                                                 pl.fused_cg),
                                pl.fused_ncta));
  if (pl.n_rows) CUDA_OK(fft_prepare(pl.row_tw_cap, pl.row_buf_cap, pl.col_tw_cap, pl.col_buf_cap));
  if (pl.n_sr) CUDA_OK(sr_prepare(pl.lc.sr_cluster, sr_smem_bytes(pl.sr_cap, pl.sr_cap.resident)));
}

void Plan::release() {
  if (d_items) cudaFree(d_items);

  if (d_sr) cudaFree(d_sr);
  if (d_fused) cudaFree(d_fused);
  d_items = nullptr;
  d_sr = nullptr;
  d_fused = nullptr;
  items_cap = sr_cap_n = fused_cap = 0;
  n_fused = 0;
}

// The Fourier-domain solve of one FP step for every deblurring problem of a plan.
void launch_fft_solve(const ProbDev *d_probs, const Plan &pl, StepArgs sa, cudaStream_t s) {
  if (pl.n_fused)
    CUDA_OK(launch_fft_solve_cluster(d_probs, pl.d_fused, pl.n_fused, pl.fused_ncta, pl.fused_tw_m,
                                     pl.fused_tw_h, pl.fused_a, pl.fused_buf, pl.fused_cg, sa, s));
  if (pl.n_rows) {
    const int skip = (sa.update_state ? 1 : 0) | (sa.skip_frozen ? 2 : 0);
    CUDA_OK(launch_fft_r2c(d_probs, pl.d_items + pl.off_rows, pl.n_rows, pl.row_tw_cap,
                           pl.row_buf_cap, nullptr, nullptr, skip, s, &sa));
    CUDA_OK(launch_fft_cols(d_probs, pl.d_items + pl.off_cols, pl.n_cols, pl.col_tw_cap,
                            pl.col_buf_cap, 1, nullptr, skip, s));
    CUDA_OK(launch_fft_c2r(d_probs, pl.d_items + pl.off_rows, pl.n_rows, pl.row_tw_cap,
                           pl.row_buf_cap, sa, s));
  }
}

// One FP step (Eq. (7)) over every problem of a plan.
void launch_fp_step(const ProbDev *d_probs, const Plan &pl, StepArgs sa, int src_type, cudaStream_t s) {
  CUDA_OK(launch_nlm(d_probs, pl.d_items + pl.off_nlm, pl.n_nlm, pl.lc.nlm_wy, sa, src_type, s,
                     nullptr, pl.lc.nlm_occ));
  launch_fft_solve(d_probs, pl, sa, s);
  if (pl.n_sr) CUDA_OK(launch_sr_step(d_probs, pl.d_sr, pl.n_sr, pl.lc.sr_cluster, pl.sr_cap, sa, s));
}

// One extrapolation (Algorithm 1 / RRE) over every problem of a plan.
void launch_ve(const ProbDev *d_probs, int n_probs, const Plan &pl, const VeArgs &va, cudaStream_t s) {
  CUDA_OK(launch_gram(d_probs, pl.d_items + pl.off_chunks, pl.n_chunks, va, s));
  VeArgs vc = va;
  vc.skip_frozen = 0;   // frozen problems combine with their stored xi
  CUDA_OK(launch_combine(d_probs, pl.d_items + pl.off_chunks, pl.n_chunks, vc, s));
}

// The cycle of Algorithm 3 as a list of operations on ring slots. With freeze > 0 (cycling
// with frozen gamma) the last FP step of the window and the Gram and gamma solve are marked
// to be skipped by problems whose gamma is frozen: for them the same launches run a cycle
// of m + k - 1 steps and a combine of x_m .. x_{m+k-1} with the stored xi.
std::vector<CycleOp> cycle_ops(int ve, int k, int m, int freeze) {
  std::vector<CycleOp> ops;
  if (ve == RED_VE_NONE) {
    for (int i = 0; i < 10; ++i) ops.push_back({0, i % 2, (i + 1) % 2, {}, 0, 0});
    return ops;
  }
  for (int i = 0; i < m; ++i) ops.push_back({0, i % 2, (i + 1) % 2, {}, 0, 0});
  const int base = m % 2;   // slot of x_m
  for (int j = 0; j < k; ++j)
    ops.push_back({0, base + j, base + j + 1, {}, 0, (freeze > 0 && j == k - 1) ? 1 : 0});
  CycleOp v{1, 0, 0, {}, 0, freeze > 0 ? 1 : 0};
  for (int j = 0; j <= k; ++j) v.slots.push_back(base + j);
  v.out = 0;
  ops.push_back(v);
  return ops;
}

}  // namespace red

using namespace red;

// ---------------------------------------------------------------------------------------
// problem
// ---------------------------------------------------------------------------------------
red_problem_s::~red_problem_s() {
  if (own_batch) delete own_batch;
  plan.release();
  plan3.release();
  if (d_pd) cudaFree(d_pd);
  if (block) cudaFree(block);
  if (h_pinned) cudaFreeHost(h_pinned);
}

static void fill_prob_dev(red_problem_s *P) {
  const red_config &c = P->cfg;
  ProbDev &d = P->pd;
  std::memset(&d, 0, sizeof(d));
  d.H = c.height;
  d.W = c.width;
  d.M = c.width / 2;
  d.Wh = d.M + 1;
  d.N = c.height * c.width;
  d.slot_stride = slot_stride_for(c);
  d.task = c.task;
  d.scale = c.task == RED_SR ? c.scale : 1;
  d.lh = c.height / d.scale;
  d.lw = c.width / d.scale;
  d.storage = c.storage == RED_BF16 ? kStoreBF16 : (c.storage == RED_F16 ? kStoreF16 : kStoreF32);
  d.nslots = nslots_for(c);
  d.n_chunks = (d.N + kGramChunk - 1) / kGramChunk;
  d.kh = c.psf_h;
  d.kw = c.psf_w;
  d.cg_iters = c.cg_iters;
  d.ve_k = c.ve_k;
  d.ve_method = c.ve;
  d.baseline = c.baseline == RED_BASE_SD ? kBaseSD : kBaseFP;
  d.ve_freeze = c.ve_freeze;
  d.inv_sigma2 = (float)(1.0 / (c.sigma * c.sigma));
  d.alpha = (float)c.alpha;
  d.inv_sigma2_d = 1.0 / (c.sigma * c.sigma);
  d.alpha_d = c.alpha;
  d.nlm_k = (float)std::sqrt(1.4426950408889634074 / (25.0 * c.nlm_h * c.nlm_h));
  char *b = static_cast<char *>(P->block);
  const Layout &L = P->L;
  d.ring = b + L.ring;
  d.f = reinterpret_cast<float *>(b + L.f);
  d.y = reinterpret_cast<const float *>(b + L.y);
  if (c.task == RED_DEBLUR) {
    d.spec = reinterpret_cast<float2 *>(b + L.spec);
    d.Kh = reinterpret_cast<const float2 *>(b + L.kh);
    d.Cc = reinterpret_cast<const float2 *>(b + L.cc);
    d.Gg = reinterpret_cast<const float *>(b + L.gg);
    d.tw_m = twiddles(d.M);
    d.tw_w = twiddles(d.W);
    d.tw_h = twiddles(d.H);
  } else {
    d.b0 = reinterpret_cast<const float *>(b + L.b0);
    d.cg_x = reinterpret_cast<float *>(b + L.cx);
    d.cg_r = reinterpret_cast<float *>(b + L.cr);
    d.cg_p = reinterpret_cast<float *>(b + L.cp);
    d.cg_ap = reinterpret_cast<float *>(b + L.cap);
    d.cg_z = reinterpret_cast<float *>(b + L.cz);
  }
  d.psf = reinterpret_cast<const float *>(b + L.psf);
  d.sd = reinterpret_cast<SdParams *>(b + L.sd);
  d.row_stats = reinterpret_cast<float2 *>(b + L.row_stats);
  d.gram_part = reinterpret_cast<float2 *>(b + L.gram);
  d.ve_coef = reinterpret_cast<double *>(b + L.coef);
  d.gamma = reinterpret_cast<double *>(b + L.gamma);
  d.st = reinterpret_cast<ProbState *>(b + L.state);
}

void red::problem_upload_pd(red_problem_s *P) {
  std::vector<ProbDev> one{P->pd};
  P->plan.build(one, P->lc);
  LaunchCfg three = P->lc;
  three.fft_cluster = 0;
  P->plan3.build(one, three);
  P->pd.n_row_items = P->plan3.n_row_items[0];
  CUDA_OK(cudaMemcpy(P->d_pd, &P->pd, sizeof(ProbDev), cudaMemcpyHostToDevice));
  prepare_launch_attrs(P->plan);
  prepare_launch_attrs(P->plan3);
}

// Per-problem constants from y (Eq. (7)): deblurring C, G (the PSF spectrum K once per
// problem), super-resolution b0 = H^T y / sigma^2. Reads the problem's copy of y.
void red::problem_precompute(red_problem_s *P, cudaStream_t s) {
  const red_config &c = P->cfg;
  ProbDev &d = P->pd;
  char *b = static_cast<char *>(P->block);
  float *y = reinterpret_cast<float *>(b + P->L.y);
  const bool sd = c.baseline == RED_BASE_SD;
  if (sd && !P->sd_ready) {
    // the SD step size depends on the PSF and the physics only (once per problem)
    CUDA_OK(launch_sd_step_size(P->d_pd, d.psf, c.psf_h, c.psf_w, d.H, d.W,
                                1.0 / (c.sigma * c.sigma), c.alpha, c.sd_mu, d.sd, s));
    P->sd_ready = true;
  }
  if (c.task == RED_DEBLUR) {
    const Plan &pl = P->plan3;
    float2 *kh = const_cast<float2 *>(d.Kh);
    if (!P->khat_ready) {
      // circularly centred, zero-padded PSF, then K = FFT2 of it
      P->psf_pad.assign((size_t)d.N, 0.f);
      const int c1 = (c.psf_h - 1) / 2, c2 = (c.psf_w - 1) / 2;
      for (int i = 0; i < c.psf_h; ++i)
        for (int j = 0; j < c.psf_w; ++j) {
          const int r = ((i - c1) % d.H + d.H) % d.H, q = ((j - c2) % d.W + d.W) % d.W;
          P->psf_pad[(size_t)r * d.W + q] += P->psf[(size_t)i * c.psf_w + j];
        }
      float *tmp = reinterpret_cast<float *>(b + P->L.tmp);
      CUDA_OK(cudaMemcpyAsync(tmp, P->psf_pad.data(), sizeof(float) * d.N, cudaMemcpyHostToDevice, s));
      CUDA_OK(launch_fft_r2c(P->d_pd, pl.d_items + pl.off_rows, pl.n_rows, pl.row_tw_cap,
                             pl.row_buf_cap, tmp, kh, 0, s));
      CUDA_OK(launch_fft_cols(P->d_pd, pl.d_items + pl.off_cols, pl.n_cols, pl.col_tw_cap,
                              pl.col_buf_cap, 0, kh, 0, s));
      P->khat_ready = true;
    }
    CUDA_OK(launch_fft_r2c(P->d_pd, pl.d_items + pl.off_rows, pl.n_rows, pl.row_tw_cap,
                           pl.row_buf_cap, y, d.spec, 0, s));
    CUDA_OK(launch_fft_cols(P->d_pd, pl.d_items + pl.off_cols, pl.n_cols, pl.col_tw_cap,
                            pl.col_buf_cap, 0, d.spec, 0, s));
    CUDA_OK(launch_spectral_constants(P->d_pd, d.Kh, d.spec, const_cast<float2 *>(d.Cc),
                                      const_cast<float *>(d.Gg), d.H * d.Wh,
                                      d.inv_sigma2_d, d.alpha_d,
                                      1.0 / ((double)d.H * d.W), s, sd ? d.sd : nullptr));
  } else {
    CUDA_OK(launch_sr_rhs(P->d_pd, y, s));
  }
}

extern "C" {

void red_config_default(red_config *c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->task = RED_DEBLUR;
  c->scale = 1;
  c->sigma = 1.4142135623730951;
  c->alpha = 0.02;
  c->nlm_patch = 5;
  c->nlm_search = 11;
  c->nlm_h = 10.0;
  c->ve = RED_VE_RRE;
  c->ve_k = 5;
  c->ve_m = 0;
  c->cg_iters = 20;
  c->storage = RED_F32;
}

red_status red_problem_footprint(const red_config *cfg, size_t *bytes) {
  return guarded([&] {
    validate(cfg);
    CHECK_ARG(bytes != nullptr, "null output");
    *bytes = layout_for(*cfg, nslots_for(*cfg), slot_stride_for(*cfg)).total;
    return RED_OK;
  });
}

red_status red_create_problem(const red_config *cfg, const void *y_dev, void *stream,
                              red_problem *out) {
  return guarded([&] {
    validate(cfg);
    CHECK_ARG(out != nullptr && y_dev != nullptr, "null argument");
    *out = nullptr;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::unique_ptr<red_problem_s> P(new red_problem_s());
    P->cfg = *cfg;
    P->psf.assign(cfg->psf, cfg->psf + (size_t)cfg->psf_h * cfg->psf_w);
    P->cfg.psf = nullptr;
    P->L = layout_for(*cfg, nslots_for(*cfg), slot_stride_for(*cfg));
    if (cudaMalloc(&P->block, P->L.total) != cudaSuccess) {
      cudaGetLastError();
      P->block = nullptr;
      throw Fail{RED_ENOMEM, "device allocation of " + std::to_string(P->L.total) + " bytes failed"};
    }
    CUDA_OK(cudaMemsetAsync(P->block, 0, P->L.total, s));
    CUDA_OK(cudaMalloc(&P->d_pd, sizeof(ProbDev)));
    CUDA_OK(cudaMallocHost(&P->h_pinned, 4096));
    fill_prob_dev(P.get());
    if (fft_cluster_override() >= 0) P->lc.fft_cluster = fft_cluster_override();
    if (sr_cluster_override() > 0) P->lc.sr_cluster = sr_cluster_override();
    nlm_shape_override(&P->lc.nlm_wy, &P->lc.nlm_occ);
    problem_upload_pd(P.get());
    char *b = static_cast<char *>(P->block);
    CUDA_OK(cudaMemcpyAsync(b + P->L.psf, P->psf.data(), sizeof(float) * P->psf.size(),
                            cudaMemcpyHostToDevice, s));
    const size_t ny = (size_t)P->pd.lh * P->pd.lw;
    CUDA_OK(cudaMemcpyAsync(b + P->L.y, y_dev, ny * 4, cudaMemcpyDeviceToDevice, s));
    problem_precompute(P.get(), s);
    *out = P.release();
    return RED_OK;
  });
}

red_status red_set_observation(red_problem p, const void *y, int y_is_host, void *stream) {
  return guarded([&] {
    CHECK_ARG(p != nullptr && y != nullptr, "null argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t ny = (size_t)p->pd.lh * p->pd.lw;
    char *b = static_cast<char *>(p->block);
    CHECK_ARG(y != b + p->L.y, "y must not be the problem's own buffer");
    CUDA_OK(cudaMemcpyAsync(b + p->L.y, y, ny * 4,
                            y_is_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
    problem_precompute(p, s);
    return RED_OK;
  });
}

red_status red_destroy_problem(red_problem p) {
  return guarded([&] {
    if (p) delete p;
    return RED_OK;
  });
}

red_status red_denoise(red_problem p, const void *x_dev, void *f_dev, void *stream) {
  return guarded([&] {
    CHECK_ARG(p && x_dev && f_dev, "null argument");
    StepArgs sa{0, 0, x_dev, nullptr, 0};
    CUDA_OK(launch_nlm(p->d_pd, p->plan.d_items + p->plan.off_nlm, p->plan.n_nlm,
                       p->plan.lc.nlm_wy, sa, 0, static_cast<cudaStream_t>(stream),
                       static_cast<float *>(f_dev), p->plan.lc.nlm_occ));
    return RED_OK;
  });
}

static bool aligned8(const void *ptr) { return (reinterpret_cast<uintptr_t>(ptr) & 7) == 0; }

red_status red_fp_step(red_problem p, const void *x_in_dev, void *x_out_dev, void *stream) {
  return guarded([&] {
    CHECK_ARG(p && x_in_dev && x_out_dev, "null argument");
    CHECK_ARG(x_in_dev != x_out_dev, "x_in and x_out must be distinct buffers");
    CHECK_ARG(aligned8(x_in_dev) && aligned8(x_out_dev), "x_in and x_out must be 8-byte aligned");
    StepArgs sa{0, 0, x_in_dev, static_cast<float *>(x_out_dev), 0};
    launch_fp_step(p->d_pd, p->plan, sa, 0, static_cast<cudaStream_t>(stream));
    return RED_OK;
  });
}

red_status red_ve_extrapolate(red_problem p, const void *const *xs_dev, int n_vec,
                              void *x_out_dev, double *gamma_host, void *stream) {
  return guarded([&] {
    CHECK_ARG(p && xs_dev && x_out_dev, "null argument");
    CHECK_ARG(n_vec >= 3 && n_vec <= kMaxK + 1, "n_vec must be in [3, 13]");
    CHECK_ARG(p->cfg.ve == RED_VE_MPE || p->cfg.ve == RED_VE_RRE || p->cfg.ve == RED_VE_SVDMPE,
              "the problem's ve method must be MPE, RRE or SVD-MPE");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    VeArgs va{};
    for (int i = 0; i < n_vec; ++i) {
      CHECK_ARG(xs_dev[i] != nullptr, "null vector");
      va.ptrs[i] = static_cast<const float *>(xs_dev[i]);
    }
    va.out_ptr = static_cast<float *>(x_out_dev);
    va.nvec = n_vec;
    va.update_state = 0;
    launch_ve(p->d_pd, 1, p->plan, va, s);
    char *b = static_cast<char *>(p->block);
    double *hg = reinterpret_cast<double *>(p->h_pinned);
    CUDA_OK(cudaMemcpyAsync(hg, b + p->L.gamma, kMaxK * 8, cudaMemcpyDeviceToHost, s));
    ProbState *hs = reinterpret_cast<ProbState *>(p->h_pinned + 1024);
    CUDA_OK(cudaMemcpyAsync(hs, b + p->L.state, sizeof(ProbState), cudaMemcpyDeviceToHost, s));
    CUDA_OK(cudaStreamSynchronize(s));
    if (hs->ve_status) return RED_EVE_BREAKDOWN;
    if (gamma_host)
      for (int i = 0; i < n_vec - 1; ++i) gamma_host[i] = hg[i];
    return RED_OK;
  });
}

red_status red_objective(red_problem p, const void *x_dev, double *e_host, void *stream) {
  return guarded([&] {
    CHECK_ARG(p && x_dev && e_host, "null argument");
    CHECK_ARG(aligned8(x_dev), "x must be 8-byte aligned");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const float *x = static_cast<const float *>(x_dev);
    char *b = static_cast<char *>(p->block);
    float *tmp = reinterpret_cast<float *>(b + p->L.tmp);
    const float *y = reinterpret_cast<const float *>(b + p->L.y);
    double *obj = reinterpret_cast<double *>(b + p->L.obj);
    // f(x) into the problem's f buffer
    StepArgs sa{0, 0, x, nullptr, 0};
    CUDA_OK(launch_nlm(p->d_pd, p->plan.d_items + p->plan.off_nlm, p->plan.n_nlm,
                       p->plan.lc.nlm_wy, sa, 0, s, nullptr, p->plan.lc.nlm_occ));
    const float *hx = nullptr;
    if (p->cfg.task == RED_DEBLUR) {
      const Plan &pl = p->plan3;
      CUDA_OK(launch_fft_r2c(p->d_pd, pl.d_items + pl.off_rows, pl.n_rows, pl.row_tw_cap,
                             pl.row_buf_cap, x, nullptr, 0, s));
      CUDA_OK(launch_fft_cols(p->d_pd, pl.d_items + pl.off_cols, pl.n_cols, pl.col_tw_cap,
                              pl.col_buf_cap, 2, nullptr, 0, s));
      StepArgs sb{0, 0, x, tmp, 0};
      CUDA_OK(launch_fft_c2r(p->d_pd, pl.d_items + pl.off_rows, pl.n_rows, pl.row_tw_cap,
                             pl.row_buf_cap, sb, s));
      hx = tmp;
    }
    CUDA_OK(launch_objective(p->d_pd, x, hx, y, p->pd.f, obj, s));
    double *h = reinterpret_cast<double *>(p->h_pinned + 2048);
    CUDA_OK(cudaMemcpyAsync(h, obj, 16, cudaMemcpyDeviceToHost, s));
    CUDA_OK(cudaStreamSynchronize(s));
    const double s2 = p->cfg.sigma * p->cfg.sigma;
    *e_host = h[0] / (2.0 * s2) + 0.5 * p->cfg.alpha * h[1];
    return RED_OK;
  });
}

const char *red_status_string(red_status st) {
  switch (st) {
    case RED_OK: return "ok";
    case RED_EINVAL: return "invalid argument";
    case RED_ENOMEM: return "out of memory";
    case RED_ECUDA: return "CUDA error";
    case RED_EVE_BREAKDOWN: return "extrapolation breakdown (last FP iterate used)";
    case RED_ENOT_CONVERGED: return "FP-call budget exhausted before the tolerance";
    case RED_ETIMEOUT: return "timed out";
    case RED_EBUSY: return "busy";
    case RED_EUNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

const char *red_last_error(void) { return g_err.c_str(); }

uint64_t red_kernel_launches(void) { return g_launches.load(); }

}  // extern "C"
