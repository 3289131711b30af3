// Super-resolution linear solve of the FP step (Eq. (7), footnote: iterative methods
// for a general H). H = S B: B a circular blur (kh x kw taps), S keeps every scale-th
// pixel from index 0. The system
//     (B^T S^T S B / sigma^2 + alpha I) x = B^T S^T y / sigma^2 + alpha f(x_k)
// is solved by textbook conjugate gradients, cg_iters iterations, warm-started at x_k,
// residual formed afresh from b - A x_k (same sequence as the FP64 oracle).
//
// GB300 mapping: one thread-block cluster per problem (8 CTAs by default). Each CTA owns
// a band of image rows (and the low-resolution rows whose samples fall in it). The
// operator is applied as two fused passes per iteration,
//     z = S B p             (LR samples of the band; kh*kw taps each)
//     A p = B^T S^T z / sigma^2 + alpha p   (each HR pixel gathers the ~(kh/s)(kw/s)
//                                            LR samples its adjoint blur touches)
// with the vectors in global memory (L2 resident) and the dot products exchanged through
// distributed shared memory: every CTA writes its partial, and after a cluster barrier
// every CTA sums all partials in rank order, so all CTAs hold the same alpha/beta with no
// atomics and a fixed reduction order. Cluster barriers are hardware barriers.
#include <cooperative_groups.h>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace red {

namespace {

constexpr int kSrThreads = 256;

// Block-wide sum of a float (fixed order); all threads get the result.
__device__ float block_sum(float v, float *scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  __syncthreads();
  if (lane == 0) scratch[warp] = v;
  __syncthreads();
  float t = 0.f;
  const int nw = blockDim.x >> 5;
  for (int w = 0; w < nw; ++w) t += scratch[w];
  return t;
}

// Sum over the cluster's CTAs of each CTA's `part` (shared variable), rank order.
__device__ double cluster_sum(cg::cluster_group &cl, float *part) {
  double s = 0.0;
  const int n = cl.num_blocks();
  for (int r = 0; r < n; ++r) s += (double)*cl.map_shared_rank(part, r);
  return s;
}

// z = S B v on LR rows [i0, i1)
__device__ void apply_sb(const ProbDev *P, const float *v, float *z, int i0, int i1) {
  const int H = P->H, W = P->W, s = P->scale, lw = P->lw, kh = P->kh, kw = P->kw;
  const int c1 = (kh - 1) / 2, c2 = (kw - 1) / 2;
  const int n = (i1 - i0) * lw;
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    const int i = i0 + t / lw, j = t % lw;
    const int u = s * i, w = s * j;
    float acc = 0.f;
    for (int a = 0; a < kh; ++a) {
      const int rr = ((u - (a - c1)) % H + H) % H;
      const float *row = v + (long)rr * W;
      const float *taps = P->psf + a * kw;
      for (int b = 0; b < kw; ++b) {
        const int cc = ((w - (b - c2)) % W + W) % W;
        acc = fmaf(taps[b], row[cc], acc);
      }
    }
    z[(long)i * lw + j] = acc;
  }
}

// out(u,v) = (B^T S^T z)(u,v) for HR pixel (u,v)
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

__global__ void __launch_bounds__(kSrThreads)
k_sr_step(const ProbDev *__restrict__ probs, const int *__restrict__ sr_list, StepArgs sa) {
  __shared__ float scratch[32];
  __shared__ float part_a, part_b, part_c, part_d, part_e;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = cl.block_rank();
  const int ncta = cl.num_blocks();
  const ProbDev *P = probs + sr_list[blockIdx.x / ncta];
  if (sa.update_state && P->st->done) return;   // uniform over the cluster

  const int H = P->H, W = P->W, s = P->scale, lh = P->lh;
  const int rb0 = (int)((long)rank * H / ncta), rb1 = (int)((long)(rank + 1) * H / ncta);
  const int i0 = min(lh, (rb0 + s - 1) / s), i1 = min(lh, (rb1 + s - 1) / s);
  const long e0 = (long)rb0 * W, e1 = (long)rb1 * W;
  const float alpha = P->alpha, is2 = P->inv_sigma2;
  float *x = P->cg_x, *r = P->cg_r, *p = P->cg_p, *ap = P->cg_ap, *z = P->cg_z;
  const float *f = P->f, *b0 = P->b0;

  const int esz = P->storage ? 2 : 4;
  const void *xin = sa.src_ptr ? sa.src_ptr
                               : static_cast<const char *>(P->ring) + (size_t)sa.src * P->slot_stride * esz;
  const int in_bf16 = sa.src_ptr ? 0 : P->storage;

  // x = x_k (warm start)
  for (long e = e0 + threadIdx.x; e < e1; e += blockDim.x) x[e] = load_img(xin, e, in_bf16);
  cl.sync();
  // r = b - A x, p = r
  apply_sb(P, x, z, i0, i1);
  cl.sync();
  float acc = 0.f;
  for (long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const int u = (int)(e / W), v = (int)(e % W);
    const float ax = fmaf(apply_btst(P, z, u, v), is2, alpha * x[e]);
    const float rv = fmaf(alpha, f[e], b0[e]) - ax;
    r[e] = rv;
    p[e] = rv;
    acc = fmaf(rv, rv, acc);
  }
  acc = block_sum(acc, scratch);
  if (threadIdx.x == 0) part_a = acc;
  cl.sync();
  double rr = cluster_sum(cl, &part_a);

  for (int it = 0; it < P->cg_iters; ++it) {
    if (rr == 0.0) break;
    apply_sb(P, p, z, i0, i1);
    cl.sync();
    acc = 0.f;
    for (long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
      const int u = (int)(e / W), v = (int)(e % W);
      const float apv = fmaf(apply_btst(P, z, u, v), is2, alpha * p[e]);
      ap[e] = apv;
      acc = fmaf(p[e], apv, acc);
    }
    acc = block_sum(acc, scratch);
    if (threadIdx.x == 0) part_b = acc;
    cl.sync();
    const double pap = cluster_sum(cl, &part_b);
    if (pap <= 0.0) break;
    const float a = (float)(rr / pap);
    acc = 0.f;
    for (long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
      x[e] = fmaf(a, p[e], x[e]);
      const float rv = fmaf(-a, ap[e], r[e]);
      r[e] = rv;
      acc = fmaf(rv, rv, acc);
    }
    acc = block_sum(acc, scratch);
    if (threadIdx.x == 0) part_c = acc;
    cl.sync();
    const double rr_new = cluster_sum(cl, &part_c);
    const float beta = (float)(rr_new / rr);
    rr = rr_new;
    for (long e = e0 + threadIdx.x; e < e1; e += blockDim.x) p[e] = fmaf(beta, p[e], r[e]);
    cl.sync();
  }

  // write x_{k+1}, statistics against x_k
  void *dst_ring = static_cast<char *>(P->ring) + (size_t)sa.dst * P->slot_stride * esz;
  float sd = 0.f, sx = 0.f;
  for (long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    float xv = x[e];
    if (sa.dst_ptr) {
      sa.dst_ptr[e] = xv;
    } else {
      store_img(dst_ring, e, xv, P->storage);
      if (P->storage) xv = __bfloat162float(__float2bfloat16_rn(xv));
    }
    const float xo = load_img(xin, e, in_bf16);
    sd = fmaf(xv - xo, xv - xo, sd);
    sx = fmaf(xo, xo, sx);
  }
  sd = block_sum(sd, scratch);
  sx = block_sum(sx, scratch);
  if (threadIdx.x == 0) { part_e = sd; part_d = sx; }
  cl.sync();
  if (sa.update_state && rank == 0 && threadIdx.x == 0) {
    const double tsd = cluster_sum(cl, &part_e), tsx = cluster_sum(cl, &part_d);
    ProbState *st = P->st;
    const double rel = tsx > 0.0 ? sqrt(tsd / tsx) : (tsd > 0.0 ? INFINITY : 0.0);
    st->rel_change = rel;
    st->calls += 1;
    if (rel < st->tol || st->calls >= st->max_calls) {
      st->done = 1;
      st->converged = rel < st->tol ? 1 : 0;
      st->final_slot = sa.dst;
    }
  }
  cl.sync();   // keep every CTA's shared memory alive until rank 0 has read it
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

cudaError_t sr_prepare(int cluster) {
  if (cluster > 8)
    return cudaFuncSetAttribute((const void *)k_sr_step,
                                cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  return cudaSuccess;
}

cudaError_t launch_sr_step(const ProbDev *d_probs, const int *d_sr_probs, int n_sr, int cluster,
                           StepArgs sa, cudaStream_t s) {
  if (n_sr <= 0) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(n_sr * cluster);
  cfg.blockDim = dim3(kSrThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_sr_step, d_probs, d_sr_probs, sa);
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
