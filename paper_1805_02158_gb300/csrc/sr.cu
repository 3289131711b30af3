// Super-resolution linear solve of the FP step (Eq. (7), footnote: iterative methods
// for a general H). H = S B: B a circular blur (kh x kw taps), S keeps every scale-th
// pixel from index 0. The system
//     (B^T S^T S B / sigma^2 + alpha I) x = B^T S^T y / sigma^2 + alpha f(x_k)
// is solved by textbook conjugate gradients, cg_iters iterations, warm-started at x_k,
// residual formed afresh from b - A x_k (same sequence as the FP64 oracle).
//
// GB300 mapping: one thread-block cluster per problem (8 or 16 CTAs, autotuned). CTA q
// owns a band of HR rows. A p = B^T S^T z / sigma^2 + alpha p with z = S B p needs, for
// the band, the LR rows of z whose samples the adjoint blur of the band touches; each CTA
// keeps exactly those rows of z (its own and a halo of at most ceil(kh/s) rows) in shared
// memory. z is never formed from p: since p_{i+1} = r_{i+1} + beta p_i and S B is linear,
//     z_{i+1} = S B r_{i+1} + beta z_i,
// and r_{i+1} is final in every band once the r.r reduction's cluster barrier has passed.
// So one CG iteration is
//     A p (band, from shared z)  ->  p.Ap      [cluster barrier 1]
//     x += a p, r -= a Ap (band)  ->  r.r      [cluster barrier 2]
//     z = S B r + beta z (band + halo rows of r); p = r + beta p is folded into the next
//     adjoint pass
// with two barriers. The adjoint pass for the 7x7 / x3 workload gives each lane s
// consecutive columns, which together use every tap of a sampled row once (other extents:
// lanes take columns of one residue mod s). Dot products: each warp's partial goes to
// shared memory; after the barrier every warp reads all partials of the cluster through
// distributed shared memory and sums them in one fixed order, so all CTAs hold identical
// alpha and beta (no atomics). When the band's x, r, p, Ap fit in shared memory they live
// there and the halo rows of r are read from the neighbouring CTAs' shared memory, so an
// iteration touches no global memory; otherwise they stay in global memory (L2 resident)
// and every loop batches its loads.
#include <cooperative_groups.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace red {

namespace {

// 512 threads, one CTA per SM (the 128-register budget): against 256-thread CTAs, the same
// on nine 256^2 problems (where the SMs are full either way) and 7-9 % more solves/s when
// serving, whose SR groups are small enough for a 16-CTA cluster to take 16 SMs.
constexpr int kSrThreads = 512;
constexpr int kSrWarps = kSrThreads / 32;
constexpr int kSrMaxCluster = 16;
constexpr unsigned kFullMask = 0xffffffffu;

__device__ __forceinline__ int wrap1(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// out(u,v) = (B^T S^T z)(u,v) for HR pixel (u,v), z an LR image in global memory
// (the right-hand side B^T S^T y; once per observation).
__device__ __forceinline__ float apply_btst(const ProbDev *P, const float *z, int u, int v) {
  const int H = P->H, W = P->W, s = P->scale, lh = P->lh, lw = P->lw, kh = P->kh, kw = P->kw;
  const int c1 = (kh - 1) / 2, c2 = (kw - 1) / 2;
  float acc = 0.f;
  for (int a = 0; a < kh; ++a) {
    const int R = ((u + a - c1) % H + H) % H;
    if (R % s != 0 || R / s >= lh) continue;
    const float *zr = z + (long)(R / s) * lw;
    const float *taps = P->psf + a * kw;
    for (int b = 0; b < kw; ++b) {
      const int C = ((v + b - c2) % W + W) % W;
      if (C % s != 0 || C / s >= lw) continue;
      acc = fmaf(taps[b], zr[C / s], acc);
    }
  }
  return acc;
}

// Shared-memory tables of one CTA.
struct SrBand {
  int H, W, s, lh, lw, kh, kw, c1, c2;
  int r0, nb;            // HR rows [r0, r0 + nb)
  int T;                 // rowmap entries: unwrapped rows r0 - c1 + t, t < T = nb + kh - 1
  int nz;                // z rows kept
  int vlo, vhi;          // interior columns of the adjoint pass (no wrap, all samples valid)
  const float *taps;     // kh * kw
  const int *rowmap;     // t -> z row index, or -1
  const int *lrow;       // z row index -> LR row
  const int *zt;         // z row index -> its row-window entry t (HR row r0 - c1 + t)
  const int *colmap;     // c < W + kw - 1: LR column of wrapped HR column c - c2, or -1
  float *z;              // nz x lw
};

// Deterministic sum over the cluster of one float per warp (all warps get the result):
// each lane adds a fixed subset in a fixed order, then a fixed xor tree. FP32 only (the
// FP64 units of this part are a small fraction of the FP32 ones, and the CG scalars are
// FP32 quantities).
__device__ __forceinline__ float cluster_total(cg::cluster_group &cl, float *slot, float v, int ncta) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(kFullMask, v, off);
  if (lane == 0) slot[warp] = v;
  cl.sync();
  constexpr int kPer = kSrMaxCluster * kSrWarps / 32;
  float got[kPer];
  const int n = ncta * kSrWarps;
#pragma unroll
  for (int t = 0; t < kPer; ++t) {
    const int i = lane + 32 * t;
    got[t] = i < n ? *cl.map_shared_rank(slot + (i % kSrWarps), i / kSrWarps) : 0.f;
  }
  float acc = 0.f;
#pragma unroll
  for (int t = 0; t < kPer; ++t) acc += got[t];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(kFullMask, acc, off);
  return acc;
}

// Compile-time kernel extents where known (the x3 / 7x7 workload), else the runtime ones.
template <int KH, int KW, int S>
struct SrDims {
  int kh, kw, s;
  __device__ __forceinline__ explicit SrDims(const SrBand &g)
      : kh(KH ? KH : g.kh), kw(KW ? KW : g.kw), s(S ? S : g.s) {}
};

// acc += sum_b taps[b] row[w0 - b] (no wrap), kw taps.
template <int KW>
__device__ __forceinline__ float row_taps(const float *ta, const float *row, int w0, int kw, float acc) {
  if constexpr (KW > 0) {
#pragma unroll
    for (int b = 0; b < KW; ++b) acc = fmaf(ta[b], row[w0 - b], acc);
  } else {
    for (int b = 0; b < kw; ++b) acc = fmaf(ta[b], row[w0 - b], acc);
  }
  return acc;
}

// z (rows kept by the band) = S B v, or S B v + beta z when accumulate. rowp(k, li, a) gives
// the row of v that tap row a of z row k (LR row li) reads: in global memory, or in the
// band's halo-extended copy in shared memory.
template <int KH, int KW, int S, class RowP>
__device__ void band_sb(const SrBand &g, RowP &&rowp, float beta, bool accumulate) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const SrDims<KH, KW, S> d(g);
  const int W = g.W, c2 = g.c2;
  constexpr int kRowsMax = KH > 0 ? KH : 1;
  for (int k = warp; k < g.nz; k += kSrWarps) {
    const int li = g.lrow[k];
    float *zr = g.z + (long)k * g.lw;
    const float *rows[kRowsMax];
    if constexpr (KH > 0) {
#pragma unroll
      for (int a = 0; a < KH; ++a) rows[a] = rowp(k, li, a);
    }
    for (int j = lane; j < g.lw; j += 32) {
      const int w0 = d.s * j + c2;                 // HR column of tap b = 0
      const bool inner = (w0 - (d.kw - 1) >= 0) && (w0 <= W - 1);
      float acc = 0.f;
      if constexpr (KH > 0) {
        if (inner) {
#pragma unroll
          for (int a = 0; a < KH; ++a) acc = row_taps<KW>(g.taps + a * d.kw, rows[a], w0, d.kw, acc);
        } else {
#pragma unroll
          for (int a = 0; a < KH; ++a) {
            const float *ta = g.taps + a * d.kw;
            for (int b = 0; b < d.kw; ++b) acc = fmaf(ta[b], rows[a][wrap1(w0 - b, W)], acc);
          }
        }
      } else {
        for (int a = 0; a < d.kh; ++a) {
          const float *row = rowp(k, li, a);
          const float *ta = g.taps + a * d.kw;
          if (inner) {
            acc = row_taps<KW>(ta, row, w0, d.kw, acc);
          } else {
            for (int b = 0; b < d.kw; ++b) acc = fmaf(ta[b], row[wrap1(w0 - b, W)], acc);
          }
        }
      }
      zr[j] = accumulate ? fmaf(beta, zr[j], acc) : acc;
    }
  }
}

// acc += sum_t ta[t s] zr[t] over the column taps b = b0 + t s < kw of one residue.
template <int KW, int S>
__device__ __forceinline__ float col_taps(const float *ta, const float *zr, int b0, int kw, int s,
                                          float acc) {
  if constexpr (KW > 0 && S > 0) {
#pragma unroll
    for (int t = 0; t < (KW + S - 1) / S; ++t)
      if (b0 + t * S < KW) acc = fmaf(ta[t * S], zr[t], acc);
  } else {
    for (int t = 0; b0 + t * s < kw; ++t) acc = fmaf(ta[t * s], zr[t], acc);
  }
  return acc;
}

// For every pixel of the band: epi(e, l, (B^T S^T z)(e)), e the image index, l = e - r0 W.
// Lanes take columns of one residue mod s (any extents).
template <int KH, int KW, int S, class Epi>
__device__ __forceinline__ void band_adjoint_residue(const SrBand &g, Epi &&epi) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const SrDims<KH, KW, S> d(g);
  const int W = g.W, c2 = g.c2, lw = g.lw;
  // interior: warp item = (row, residue ph of the column mod s); the row's sampled taps
  // and the residue's column taps are the same for every lane
  if (g.vhi >= g.vlo) {
    for (int it = warp; it < g.nb * d.s; it += kSrWarps) {
      const int ul = it / d.s, ph = it - ul * d.s;
      const int qlo = (g.vlo - ph + d.s - 1) / d.s;                 // vlo >= c2 >= 0
      const int qhi = g.vhi >= ph ? (g.vhi - ph) / d.s : -1;
      if (qlo > qhi) continue;
      const int b0 = (c2 - ph + d.s) % d.s;                         // c2 - ph > -s
      const int d0 = (ph + b0 - c2) / d.s;                          // exact
      const long rowbase = (long)(g.r0 + ul) * W;
      const int lbase = ul * W;
      if constexpr (KH > 0) {
        int zoff[KH];   // offset in z of tap row a's sampled LR row, or -1
#pragma unroll
        for (int a = 0; a < KH; ++a) {
          const int zk = g.rowmap[ul + a];
          zoff[a] = zk >= 0 ? zk * lw : -1;
        }
        for (int q = qlo + lane; q <= qhi; q += 32) {
          float acc = 0.f;
#pragma unroll
          for (int a = 0; a < KH; ++a)
            if (zoff[a] >= 0)
              acc = col_taps<KW, S>(g.taps + a * d.kw + b0, g.z + zoff[a] + d0 + q, b0, d.kw, d.s, acc);
          epi(rowbase + d.s * q + ph, lbase + d.s * q + ph, acc);
        }
      } else {
        for (int q = qlo + lane; q <= qhi; q += 32) {
          float acc = 0.f;
          for (int a = 0; a < d.kh; ++a) {
            const int zk = g.rowmap[ul + a];
            if (zk >= 0)
              acc = col_taps<KW, S>(g.taps + a * d.kw + b0, g.z + zk * lw + d0 + q, b0, d.kw, d.s, acc);
          }
          epi(rowbase + d.s * q + ph, lbase + d.s * q + ph, acc);
        }
      }
    }
  }
  // edge columns (wrap-around or past the last LR sample): every tap checked
  const int nle = g.vhi >= g.vlo ? g.vlo : W;
  const int ne = g.vhi >= g.vlo ? g.vlo + (W - 1 - g.vhi) : W;
  for (int idx = threadIdx.x; idx < g.nb * ne; idx += kSrThreads) {
    const int ul = idx / ne, ei = idx - ul * ne;
    const int v = ei < nle ? ei : g.vhi + 1 + (ei - nle);
    float acc = 0.f;
    for (int a = 0; a < d.kh; ++a) {
      const int zk = g.rowmap[ul + a];
      if (zk < 0) continue;
      const float *zr = g.z + (long)zk * lw;
      const float *ta = g.taps + a * d.kw;
      for (int b = 0; b < d.kw; ++b) {
        const int cj = g.colmap[v + b];
        if (cj >= 0) acc = fmaf(ta[b], zr[cj], acc);
      }
    }
    epi((long)(g.r0 + ul) * W + v, ul * W + v, acc);
  }
}


__host__ __device__ constexpr int floor_div(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

// The same for compile-time extents: a lane takes S consecutive columns S q .. S q + S - 1,
// which together use every tap of a sampled row once and LR columns q + DMIN .. q + DMAX.
template <int KH, int KW, int S, class Epi>
__device__ __forceinline__ void band_adjoint_blocked(const SrBand &g, Epi &&epi) {
  constexpr int C2 = (KW - 1) / 2;
  constexpr int DMIN = floor_div(-C2, S), DMAX = floor_div(S - 1 + KW - 1 - C2, S);
  constexpr int ND = DMAX - DMIN + 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int W = g.W, lw = g.lw;
  // groups whose S columns are all interior
  const int glo = (g.vlo + S - 1) / S;
  const int ghi = g.vhi >= S - 1 ? (g.vhi - (S - 1)) / S : -1;
  for (int ul = warp; ul < g.nb; ul += kSrWarps) {
    int zoff[KH];
#pragma unroll
    for (int a = 0; a < KH; ++a) {
      const int zk = g.rowmap[ul + a];
      zoff[a] = zk >= 0 ? zk * lw : -1;
    }
    const long rowbase = (long)(g.r0 + ul) * W;
    const int lbase = ul * W;
    for (int q = glo + lane; q <= ghi; q += 32) {
      float acc[S];
#pragma unroll
      for (int ph = 0; ph < S; ++ph) acc[ph] = 0.f;
#pragma unroll
      for (int a = 0; a < KH; ++a) {
        if (zoff[a] < 0) continue;
        const float *zr = g.z + zoff[a] + q;
        float zv[ND];
#pragma unroll
        for (int i = 0; i < ND; ++i) zv[i] = zr[DMIN + i];
        const float *ta = g.taps + a * KW;
#pragma unroll
        for (int b = 0; b < KW; ++b) {
          const float t = ta[b];
#pragma unroll
          for (int ph = 0; ph < S; ++ph)
            if ((ph + b - C2 - DMIN * S) % S == 0)
              acc[ph] = fmaf(t, zv[floor_div(ph + b - C2, S) - DMIN], acc[ph]);
        }
      }
#pragma unroll
      for (int ph = 0; ph < S; ++ph) epi(rowbase + S * q + ph, lbase + S * q + ph, acc[ph]);
    }
  }
  // the remaining columns, every tap checked
  const int nle = ghi >= glo ? S * glo : W;
  const int ne = ghi >= glo ? nle + (W - S * (ghi + 1)) : W;
  for (int idx = threadIdx.x; idx < g.nb * ne; idx += kSrThreads) {
    const int ul = idx / ne, ei = idx - ul * ne;
    const int v = ei < nle ? ei : S * (ghi + 1) + (ei - nle);
    float acc = 0.f;
    for (int a = 0; a < KH; ++a) {
      const int zk = g.rowmap[ul + a];
      if (zk < 0) continue;
      const float *zr = g.z + (long)zk * lw;
      const float *ta = g.taps + a * KW;
#pragma unroll
      for (int b = 0; b < KW; ++b) {
        const int cj = g.colmap[v + b];
        if (cj >= 0) acc = fmaf(ta[b], zr[cj], acc);
      }
    }
    epi((long)(g.r0 + ul) * W + v, ul * W + v, acc);
  }
}

template <int KH, int KW, int S, class Epi>
__device__ __forceinline__ void band_adjoint(const SrBand &g, Epi &&epi) {
  if constexpr (KH > 0 && KW > 0 && S > 0)
    band_adjoint_blocked<KH, KW, S>(g, epi);
  else
    band_adjoint_residue<KH, KW, S>(g, epi);
}

// Shared memory (4-byte words): taps | rowmap | lrow | zt | colmap | z | 2 x per-warp
// partials | (resident bands only) x and r with kh - 1 halo rows on each side, p, Ap. The caps are maxima over the launch's
// problems (sr_caps on the host). When the band's vectors do not fit (large images) they
// stay in global memory and every loop batches its loads.
template <int KH, int KW, int S>
__global__ void __launch_bounds__(kSrThreads, 1)
k_sr_step(const ProbDev *__restrict__ probs, const int *__restrict__ sr_list, StepArgs sa,
          SrCaps caps, int resident) {
  extern __shared__ float sm_sr[];
  __shared__ int nz_sh;
  __shared__ float part_d[kSrWarps], part_x[kSrWarps];
  __shared__ float2 cl_stats[16];   // on rank 0: every CTA's (sum d^2, sum x^2), by rank
  __shared__ int band_start[kSrMaxCluster + 1];   // first HR row of every CTA's band, and H
  cg::cluster_group cl = cg::this_cluster();
  const int rank = cl.block_rank();
  const int ncta = cl.num_blocks();
  const ProbDev *P = probs + sr_list[blockIdx.x / ncta];
  if (sa.update_state && P->st->done) return;   // uniform over the cluster
  if (sa.skip_frozen && P->st->frozen) return;
  const int tid = threadIdx.x;

  SrBand g;
  g.H = P->H; g.W = P->W; g.s = P->scale; g.lh = P->lh; g.lw = P->lw; g.kh = P->kh; g.kw = P->kw;
  g.c1 = (g.kh - 1) / 2;
  g.c2 = (g.kw - 1) / 2;
  g.r0 = (int)((long)rank * g.H / ncta);
  g.nb = (int)((long)(rank + 1) * g.H / ncta) - g.r0;
  g.T = g.nb + g.kh - 1;
  g.vlo = g.c2;
  g.vhi = min(g.W - 1, g.s * (g.lw - 1)) - (g.kw - 1 - g.c2);
  float *taps = sm_sr;
  int *rowmap = reinterpret_cast<int *>(taps + caps.taps);
  int *lrow = rowmap + caps.rows;
  int *zt = lrow + caps.zrows;
  int *colmap = zt + caps.zrows;
  g.z = reinterpret_cast<float *>(colmap + caps.cols);
  float *slot_a = g.z + caps.zfloats;
  float *slot_b = slot_a + kSrWarps;
  g.taps = taps;
  g.rowmap = rowmap;
  g.lrow = lrow;
  g.zt = zt;
  g.colmap = colmap;

  for (int q = tid; q <= ncta; q += kSrThreads) band_start[q] = (int)((long)q * g.H / ncta);
  for (int i = tid; i < g.kh * g.kw; i += kSrThreads) taps[i] = P->psf[i];
  for (int t = tid; t < g.T; t += kSrThreads) {
    const int R = wrap1(g.r0 - g.c1 + t, g.H);
    rowmap[t] = (R % g.s == 0 && R / g.s < g.lh) ? R / g.s : -1;
  }
  for (int c = tid; c < g.W + g.kw - 1; c += kSrThreads) {
    const int C = wrap1(c - g.c2, g.W);
    colmap[c] = (C % g.s == 0 && C / g.s < g.lw) ? C / g.s : -1;
  }
  __syncthreads();
  if (tid == 0) {   // compact the sampled rows (T is at most a few hundred)
    int nz = 0;
    for (int t = 0; t < g.T; ++t)
      if (rowmap[t] >= 0) {
        lrow[nz] = rowmap[t];
        zt[nz] = t;
        rowmap[t] = nz++;
      }
    nz_sh = nz;
  }
  __syncthreads();
  g.nz = nz_sh;

  const float alpha = P->alpha, is2 = P->inv_sigma2;
  const long e0 = (long)g.r0 * g.W;
  const int nl = g.nb * g.W;                    // pixels of the band
  float *r_g = P->cg_r;                         // r in global memory (non-resident bands)
  const int hw = g.kh - 1;                      // halo rows of the resident copies of x, r
  // band vectors, indexed by the band-local pixel index
  float *xs, *rs, *ps, *aps;
  float *xh = nullptr, *rh = nullptr;           // resident: [hw halo | band | hw halo] rows
  if (resident) {
    xh = sm_sr + caps.resident_off;             // 16-byte aligned
    rh = xh + caps.band_ext;
    ps = rh + caps.band_ext;
    aps = ps + caps.band;
    xs = xh + (long)hw * g.W;
    rs = rh + (long)hw * g.W;
  } else {
    xs = P->cg_x + e0;
    rs = r_g + e0;
    ps = P->cg_p + e0;
    aps = P->cg_ap + e0;
  }
  const float *f = P->f, *b0 = P->b0;
  const int esz = store_bytes(P->storage);
  const void *xin = sa.src_ptr ? sa.src_ptr
                               : static_cast<const char *>(P->ring) + (size_t)sa.src * P->slot_stride * esz;
  const int in_type = sa.src_ptr ? kStoreF32 : P->storage;
  constexpr int kU = 4;   // elements per thread per batch of independent loads

  // x = x_k (warm start) into the band and global memory (S B x reads the halo rows)
  for (int l0 = tid; l0 < nl; l0 += kU * kSrThreads) {
    float v[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int l = l0 + u * kSrThreads;
      if (l < nl) v[u] = load_img(xin, e0 + l, in_type);
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int l = l0 + u * kSrThreads;
      if (l < nl) xs[l] = v[u];
    }
  }
  cl.sync();
  // Rows of x or r read by S B: resident bands copy the hw rows above and below the band
  // from the owning CTAs' shared memory (distributed shared memory) into their extended
  // copy, which then holds HR row r0 - hw + t at row t, wrapped; otherwise global memory.
  auto owner = [&](int R) {
    int q = (int)((long)R * ncta / g.H);
    while (q + 1 < ncta && (int)((long)(q + 1) * g.H / ncta) <= R) ++q;
    while (q > 0 && (int)((long)q * g.H / ncta) > R) --q;
    return q;
  };
  auto fill_halo = [&](float *ext, float *band_local) {
    const int warp = tid >> 5, lane = tid & 31;
    for (int hr = warp; hr < 2 * hw; hr += kSrWarps) {
      const int t = hr < hw ? hr : g.nb + hr;
      const int R = wrap1(g.r0 - hw + t, g.H);
      const int q = owner(R);
      const float *src = cl.map_shared_rank(band_local, q) +
                         (long)(R - (int)((long)q * g.H / ncta)) * g.W;
      float *dst = ext + (long)t * g.W;
      if ((g.W & 3) == 0) {   // rows start on 16-byte boundaries
        const float4 *s4 = reinterpret_cast<const float4 *>(src);
        float4 *d4 = reinterpret_cast<float4 *>(dst);
        const int n4 = g.W >> 2;
        for (int c0 = lane; c0 < n4; c0 += 4 * 32) {
          float4 v[4];
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (c0 + 32 * u < n4) v[u] = s4[c0 + 32 * u];
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (c0 + 32 * u < n4) d4[c0 + 32 * u] = v[u];
        }
      } else {
        for (int c0 = lane; c0 < g.W; c0 += 8 * 32) {
          float v[8];
#pragma unroll
          for (int u = 0; u < 8; ++u)
            if (c0 + 32 * u < g.W) v[u] = src[c0 + 32 * u];
#pragma unroll
          for (int u = 0; u < 8; ++u)
            if (c0 + 32 * u < g.W) dst[c0 + 32 * u] = v[u];
        }
      }
    }
  };
  // Inside the CG loop the halo rows of r are pushed instead: each CTA stores the rows of
  // its band that lie in other CTAs' halos straight into their extended copies (rows of a
  // band belong to exactly one CTA, so each halo row has one writer); the cluster barrier
  // of the r.r reduction that follows makes them visible, and no CTA waits on remote loads.
  // A halo is overwritten only after the p.Ap barrier of the same iteration, which every
  // CTA reaches after its last read of the previous r.
  auto push_halo = [&](float *ext, const float *band_local) {
    const int warp = tid >> 5, lane = tid & 31;
    for (int job = warp; job < ncta * 2 * hw; job += kSrWarps) {
      const int q = job / (2 * hw), hr = job - q * (2 * hw);
      const int r0q = band_start[q];
      const int nbq = band_start[q + 1] - r0q;
      const int t = hr < hw ? hr : nbq + hr;
      const int R = wrap1(r0q - hw + t, g.H);
      if (R < g.r0 || R >= g.r0 + g.nb) continue;   // a row of another band
      const float *src = band_local + (long)(R - g.r0) * g.W;
      float *dst = cl.map_shared_rank(ext, q) + (long)t * g.W;
      if ((g.W & 3) == 0) {
        const float4 *s4 = reinterpret_cast<const float4 *>(src);
        float4 *d4 = reinterpret_cast<float4 *>(dst);
        for (int c = lane; c < (g.W >> 2); c += 32) d4[c] = s4[c];
      } else {
        for (int c = lane; c < g.W; c += 32) dst[c] = src[c];
      }
    }
  };
  auto x_row = [&](int k, int li, int a) -> const float * {
    if (resident) return xh + (long)(zt[k] - a + hw) * g.W;
    return P->cg_x + (long)wrap1(g.s * li - a + g.c1, g.H) * g.W;
  };
  auto r_row = [&](int k, int li, int a) -> const float * {
    if (resident) return rh + (long)(zt[k] - a + hw) * g.W;
    return r_g + (long)wrap1(g.s * li - a + g.c1, g.H) * g.W;
  };
  if (resident) {
    fill_halo(xh, xs);
    __syncthreads();
  }
  band_sb<KH, KW, S>(g, x_row, 0.f, false);
  __syncthreads();
  float dot = 0.f;
  // r = b - A x, p = r
  band_adjoint<KH, KW, S>(g, [&](long e, int l, float acc) {
    const float ax = fmaf(acc, is2, alpha * xs[l]);
    const float rv = fmaf(alpha, f[e], b0[e]) - ax;
    rs[l] = rv;
    ps[l] = rv;
    dot = fmaf(rv, rv, dot);
  });
  // Steepest-descent baseline (SD-MPE, Sec. IV): the step x - mu grad E(x) of Eq. (5) is
  // x + mu r with r = b0 + alpha f - A x the residual just formed; no CG iterations.
  const bool sd_step = P->baseline == kBaseSD;   // uniform over the cluster
  if (sd_step) {
    const float mu = P->sd->mu_f;
    __syncthreads();
    for (int l = tid; l < nl; l += kSrThreads) xs[l] = fmaf(mu, rs[l], xs[l]);
  }
  float rr = sd_step ? 0.f : cluster_total(cl, slot_b, dot, ncta);
  if (!sd_step) {
    if (resident) {
      fill_halo(rh, rs);
      __syncthreads();
    }
    band_sb<KH, KW, S>(g, r_row, 0.f, false);   // z = S B p, p = r
    __syncthreads();
  }

  float beta = 0.f;   // p = r + beta p is applied in the adjoint pass (p = r at first)
  for (int it = 0; it < (sd_step ? 0 : P->cg_iters); ++it) {
    if (rr == 0.f) break;
    dot = 0.f;
    band_adjoint<KH, KW, S>(g, [&](long e, int l, float acc) {
      const float pv = fmaf(beta, ps[l], rs[l]);
      ps[l] = pv;
      const float apv = fmaf(acc, is2, alpha * pv);
      aps[l] = apv;
      dot = fmaf(pv, apv, dot);
    });
    const float pap = cluster_total(cl, slot_a, dot, ncta);
    if (pap <= 0.f) break;
    const float a = rr / pap;
    dot = 0.f;
    for (int l0 = tid; l0 < nl; l0 += kU * kSrThreads) {
      float pv[kU], av[kU], rv[kU], xv[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int l = l0 + u * kSrThreads;
        if (l < nl) {
          pv[u] = ps[l];
          av[u] = aps[l];
          rv[u] = rs[l];
          xv[u] = xs[l];
        }
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int l = l0 + u * kSrThreads;
        if (l < nl) {
          xs[l] = fmaf(a, pv[u], xv[u]);
          const float rn = fmaf(-a, av[u], rv[u]);
          rs[l] = rn;
          dot = fmaf(rn, rn, dot);
        }
      }
    }
    // the last iteration's r, beta and z = S B p are not used: x_{k+1} is final
    if (it + 1 == P->cg_iters) break;
    if (resident) {
      __syncthreads();          // the band's new r is complete in shared memory
      push_halo(rh, rs);
    }
    const float rr_new = cluster_total(cl, slot_b, dot, ncta);
    beta = rr_new / rr;
    rr = rr_new;
    band_sb<KH, KW, S>(g, r_row, beta, true);   // z = S B r + beta z = S B p
    __syncthreads();
  }
  cl.sync();   // every CTA has finished its remote reads of the last reduction's partials

  // x_{k+1} -> destination, statistics against x_k
  void *dst_ring = static_cast<char *>(P->ring) + (size_t)sa.dst * P->slot_stride * esz;
  float sd = 0.f, sx = 0.f;
  for (int l0 = tid; l0 < nl; l0 += kU * kSrThreads) {
    float xv[kU], xo[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int l = l0 + u * kSrThreads;
      if (l < nl) {
        xv[u] = xs[l];
        xo[u] = load_img(xin, e0 + l, in_type);
      }
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int l = l0 + u * kSrThreads;
      if (l < nl) {
        float v = xv[u];
        if (sa.dst_ptr) {
          sa.dst_ptr[e0 + l] = v;
        } else {
          store_img(dst_ring, e0 + l, v, P->storage);
          v = round_to_storage(v, P->storage);
        }
        sd = fmaf(v - xo[u], v - xo[u], sd);
        sx = fmaf(xo[u], xo[u], sx);
      }
    }
  }
  if (!sa.update_state) return;   // uniform over the cluster (a launch argument)
  // CTA sums (fixed order) into rank 0's shared memory; after a cluster barrier rank 0 sums
  // them in rank order and runs the termination test (no GPU-scope fence, no atomic)
  const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    sd += __shfl_xor_sync(kFullMask, sd, off);
    sx += __shfl_xor_sync(kFullMask, sx, off);
  }
  if (lane == 0) {
    part_d[warp] = sd;
    part_x[warp] = sx;
  }
  __syncthreads();
  if (tid == 0) {
    float td = 0.f, tx = 0.f;
    for (int w = 0; w < kSrWarps; ++w) {
      td += part_d[w];
      tx += part_x[w];
    }
    cl.map_shared_rank(cl_stats, 0)[rank] = make_float2(td, tx);
  }
  cl.sync();
  if (rank == 0 && tid == 0) {
    double tsd = 0.0, tsx = 0.0;
    for (int q = 0; q < ncta; ++q) {
      tsd += (double)cl_stats[q].x;
      tsx += (double)cl_stats[q].y;
    }
    ProbState *st = P->st;
    const double rel = tsx > 0.0 ? sqrt(tsd / tsx) : (tsd > 0.0 ? INFINITY : 0.0);
    st->rel_change = rel;
    st->calls += 1;
    if (rel < st->ve_stop_tol) st->ve_off = 1;   // extrapolation ends, baseline steps follow
    if (rel < st->tol || st->calls >= st->max_calls) {
      st->done = 1;
      st->converged = rel < st->tol ? 1 : 0;
      st->final_slot = sa.dst;
    }
  }
}
// b0 = B^T S^T y / sigma^2
__global__ void k_sr_rhs(const ProbDev *__restrict__ P, const float *__restrict__ y) {
  const long n = (long)P->H * P->W;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
    const int u = (int)(e / P->W), v = (int)(e % P->W);
    const_cast<float *>(P->b0)[e] = apply_btst(P, y, u, v) * P->inv_sigma2;
  }
}

// Terms of the objective Eq. (4): out[0] = ||H x - y||^2, out[1] = x^T (x - f).
// hx: H x for deblurring (full size) or null for SR (computed here from the taps).
// One CTA, fixed-order reduction (measurement only, not on the solve path).
__global__ void k_objective(const ProbDev *__restrict__ P, const float *__restrict__ x,
                            const float *__restrict__ hx, const float *__restrict__ y,
                            const float *__restrict__ f, double *out) {
  __shared__ double sa[1024 / 32], sb[1024 / 32];
  double a = 0.0, b = 0.0;
  const long n = (long)P->H * P->W;
  for (long e = threadIdx.x; e < n; e += blockDim.x) b += (double)x[e] * ((double)x[e] - (double)f[e]);
  if (hx) {
    for (long e = threadIdx.x; e < n; e += blockDim.x) {
      const double d = (double)hx[e] - (double)y[e];
      a += d * d;
    }
  } else {
    const int H = P->H, W = P->W, s = P->scale, lh = P->lh, lw = P->lw, kh = P->kh, kw = P->kw;
    const int c1 = (kh - 1) / 2, c2 = (kw - 1) / 2;
    for (long t = threadIdx.x; t < (long)lh * lw; t += blockDim.x) {
      const int i = (int)(t / lw), j = (int)(t % lw);
      double acc = 0.0;
      for (int aa = 0; aa < kh; ++aa)
        for (int bb = 0; bb < kw; ++bb) {
          const int rr = ((s * i - (aa - c1)) % H + H) % H, cc = ((s * j - (bb - c2)) % W + W) % W;
          acc += (double)P->psf[aa * kw + bb] * (double)x[(long)rr * W + cc];
        }
      const double d = acc - (double)y[t];
      a += d * d;
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int off = 16; off > 0; off >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, off);
    b += __shfl_xor_sync(0xffffffffu, b, off);
  }
  if (lane == 0) { sa[warp] = a; sb[warp] = b; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ta = 0.0, tb = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { ta += sa[w]; tb += sb[w]; }
    out[0] = ta;
    out[1] = tb;
  }
}

}  // namespace

cudaError_t launch_sr_rhs(const ProbDev *d_prob, const float *y, cudaStream_t s) {
  k_sr_rhs<<<304, 256, 0, s>>>(d_prob, y);
  count_launches(1);
  return cudaGetLastError();
}

// Shared-memory caps of one problem for a cluster of ncta CTAs (exact: the row windows
// of every band are scanned as the kernel does).
void sr_caps(int H, int W, int scale, int kh, int kw, int ncta, SrCaps *c) {
  const int lh = H / scale, lw = W / scale, c1 = (kh - 1) / 2, c2 = (kw - 1) / 2;
  (void)c2;
  SrCaps o{};
  o.spec737 = (kh == 7 && kw == 7 && scale == 3) ? 1 : 0;
  o.taps = kh * kw;
  o.cols = W + kw - 1;
  for (int q = 0; q < ncta; ++q) {
    const int r0 = (int)((long)q * H / ncta), nb = (int)((long)(q + 1) * H / ncta) - r0;
    const int T = nb + kh - 1;
    int nz = 0;
    for (int t = 0; t < T; ++t) {
      int R = r0 - c1 + t;
      R = R < 0 ? R + H : (R >= H ? R - H : R);
      if (R % scale == 0 && R / scale < lh) ++nz;
    }
    o.rows = std::max(o.rows, T);
    o.band = std::max(o.band, (nb * W + 3) & ~3);
    o.band_ext = std::max(o.band_ext, ((nb + 2 * (kh - 1)) * W + 3) & ~3);
    o.zrows = std::max(o.zrows, nz);
    o.zfloats = std::max(o.zfloats, nz * lw);
  }
  *c = o;
}

static int sr_base_words(const SrCaps &c) {
  return (c.taps + c.rows + 2 * c.zrows + c.cols + c.zfloats + 2 * kSrWarps + 3) & ~3;
}

int sr_smem_bytes(const SrCaps &c, int resident) {
  return 4 * (sr_base_words(c) + (resident ? 2 * c.band_ext + 2 * c.band : 0));
}

using SrKernel = void (*)(const ProbDev *, const int *, StepArgs, SrCaps, int);

// The instantiations: 7x7 taps at scale 3, and any extents.
static SrKernel sr_kernel(int spec737) {
  if (spec737) return k_sr_step<7, 7, 3>;
  return k_sr_step<0, 0, 0>;
}

// The dynamic shared-memory limit of a kernel only ever grows (high-water mark): launches
// of other problem sets, possibly still in flight on other streams, keep their room.
cudaError_t sr_prepare(int cluster, int smem) {
  static std::mutex mu;
  static int high_water = 0;
  static bool non_portable = false;
  std::lock_guard<std::mutex> lk(mu);
  for (const void *fn : {(const void *)k_sr_step<7, 7, 3>, (const void *)k_sr_step<0, 0, 0>}) {
    cudaError_t e = cudaSuccess;
    if (cluster > 8 && !non_portable)
      e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e == cudaSuccess && smem > high_water)
      e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
  }
  if (cluster > 8) non_portable = true;
  high_water = std::max(high_water, smem);
  return cudaSuccess;
}

int sr_max_active_clusters(int cluster, int smem, int spec737) {
  if (sr_prepare(cluster, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cluster);
  cfg.blockDim = dim3(kSrThreads);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, (const void *)sr_kernel(spec737), &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

cudaError_t launch_sr_step(const ProbDev *d_probs, const int *d_sr_probs, int n_sr, int cluster,
                           const SrCaps &caps, StepArgs sa, cudaStream_t s) {
  if (n_sr <= 0) return cudaSuccess;
  if (cluster < 1 || cluster > kSrMaxCluster) return cudaErrorInvalidValue;
  SrCaps c = caps;
  c.resident_off = sr_base_words(caps);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(n_sr * cluster);
  cfg.blockDim = dim3(kSrThreads);
  cfg.dynamicSmemBytes = sr_smem_bytes(caps, caps.resident);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, sr_kernel(caps.spec737), d_probs, d_sr_probs, sa,
                                     c, caps.resident);
  count_launches(1);
  return e;
}

cudaError_t launch_objective(const ProbDev *d_prob, const float *x, const float *hx,
                             const float *y, const float *f, double *out, cudaStream_t s) {
  k_objective<<<1, 1024, 0, s>>>(d_prob, x, hx, y, f, out);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace red
