// Fourier-domain linear solve of the FP step for a block-circulant blur H (Eq. (7) and
// its footnote): x_{k+1} = IFFT2( C + G . FFT2(f) ),
//   C = conj(K) FFT2(y) / (sigma^2 D) / (H W),  G = alpha / D / (H W),
//   D = |K|^2 / sigma^2 + alpha,  K = FFT2 of the circularly centred PSF.
//
// The 2-D transform is three passes over a half spectrum (H x (W/2 + 1) complex):
//   1. rows, real-to-complex: each row of W reals is packed as W/2 complex values, a
//      W/2-point complex FFT is taken and the W/2 + 1 non-redundant bins are untangled;
//   2. columns: forward FFT of each column, the pointwise solve X = C + G F, inverse FFT
//      (all in shared memory, one read and one write of the spectrum);
//   3. rows, complex-to-real, with the relative-change statistics of the FP step
//      (sum (x_{k+1} - x_k)^2, sum x_k^2) reduced on the fly and, in a batched solve, the
//      termination test of the problem done by the last CTA to finish it.
// Transforms are self-sorting Stockham passes in shared memory with radix 4, 2 and 3
// (sizes 2^a 3^b), twiddles from tables computed on the host in double precision.
// Inverse transforms use IFFT(X) = conj(FFT(conj(X))); the 1/(H W) scale is folded
// into C and G.
#include <cooperative_groups.h>

#include <algorithm>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace red {

namespace {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 mul_mi(float2 a) { return make_float2(a.y, -a.x); }  // * (-i)
__device__ __forceinline__ float2 mul_pi(float2 a) { return make_float2(-a.y, a.x); }  // * (+i)

// Division by a run-time invariant d < 2^16 for numerators t < 2^16: q = hi32(t * m) with
// m = floor(2^32 / d) + 1 (exact in that range; d = 1 handled separately). Replaces the
// integer divisions of the index arithmetic, which otherwise dominate the FFT kernels.
struct FastDiv {
  uint32_t d, m;
  __device__ __forceinline__ explicit FastDiv(int dd) : d((uint32_t)dd), m(dd > 1 ? 0xFFFFFFFFu / (uint32_t)dd + 1u : 0u) {}
  __device__ __forceinline__ int div(int t) const { return d == 1 ? t : (int)__umulhi((uint32_t)t, m); }
  __device__ __forceinline__ void divmod(int t, int &q, int &r) const {
    q = div(t);
    r = t - q * (int)d;
  }
};

// Copies `total` elements with U independent loads in flight per thread (load all, then
// store all), instead of one load-to-use round trip per loop iteration.
template <int U, class Load, class Store>
__device__ __forceinline__ void copy_batched(int total, int tid, int nthr, Load load, Store store) {
  for (int base = tid; base < total; base += U * nthr) {
    float2 v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int idx = base + u * nthr;
      if (idx < total) v[u] = load(idx);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int idx = base + u * nthr;
      if (idx < total) store(idx, v[u]);
    }
  }
}

// Forward Stockham FFT of `nseq` sequences of length n held in shared memory (sequence s
// at x + s * ss). Ping-pongs between x and y; returns the buffer holding the result.
// Pass with radix r after previous passes of product Ns: butterfly j reads elements
// j + q n/r, twiddles them by w_n^{(j mod Ns) q n/(Ns r)}, takes an r-point DFT and writes
// to (j - j mod Ns) r + j mod Ns + q Ns (natural order output).
__device__ float2 *stockham(float2 *x, float2 *y, int n, int nseq, int ss,
                            const float2 *__restrict__ tw, int tid, int nthr) {
  float2 *in = x, *out = y;
  int Ns = 1;
  int rem = n;
  while (rem > 1) {
    const int r = (rem % 4 == 0) ? 4 : ((rem % 2 == 0) ? 2 : 3);
    const int nb = n / r;
    const int tws = n / (Ns * r);
    const int total = nseq * nb;
    const FastDiv dnb(nb), dns(Ns);
    for (int t = tid; t < total; t += nthr) {
      int s, j, g, kk;
      dnb.divmod(t, s, j);
      dns.divmod(j, g, kk);
      const float2 *src = in + s * ss;
      float2 *dst = out + s * ss;
      const int base = g * Ns * r + kk;
      if (r == 4) {
        float2 a0 = src[j], a1 = src[j + nb], a2 = src[j + 2 * nb], a3 = src[j + 3 * nb];
        if (kk) {
          const int ti = kk * tws;
          a1 = cmul(a1, tw[ti]);
          a2 = cmul(a2, tw[2 * ti]);
          a3 = cmul(a3, tw[3 * ti]);
        }
        const float2 t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3);
        const float2 t3 = mul_mi(csub(a1, a3));
        dst[base] = cadd(t0, t2);
        dst[base + Ns] = cadd(t1, t3);
        dst[base + 2 * Ns] = csub(t0, t2);
        dst[base + 3 * Ns] = csub(t1, t3);
      } else if (r == 2) {
        float2 a0 = src[j], a1 = src[j + nb];
        if (kk) a1 = cmul(a1, tw[kk * tws]);
        dst[base] = cadd(a0, a1);
        dst[base + Ns] = csub(a0, a1);
      } else {
        float2 a0 = src[j], a1 = src[j + nb], a2 = src[j + 2 * nb];
        if (kk) {
          const int ti = kk * tws;
          a1 = cmul(a1, tw[ti]);
          a2 = cmul(a2, tw[2 * ti]);
        }
        // w = e^{-2 pi i / 3}: y1 = a0 - s/2 - i (sqrt3/2) d, y2 = a0 - s/2 + i (sqrt3/2) d
        const float2 s12 = cadd(a1, a2), d12 = csub(a1, a2);
        const float2 m = make_float2(a0.x - 0.5f * s12.x, a0.y - 0.5f * s12.y);
        const float h = 0.86602540378443864676f;
        const float2 e = make_float2(h * d12.x, h * d12.y);
        dst[base] = cadd(a0, s12);
        dst[base + Ns] = cadd(m, mul_mi(e));
        dst[base + 2 * Ns] = cadd(m, mul_pi(e));
      }
    }
    __syncthreads();
    float2 *tmp = in;
    in = out;
    out = tmp;
    Ns *= r;
    rem /= r;
  }
  return in;
}

// Pass 1: rows, real to half spectrum. Item (prob, first row).
__global__ void __launch_bounds__(256)
k_fft_r2c(const ProbDev *__restrict__ probs, const Item *__restrict__ items, int tw_cap,
          int buf_cap, const float *src_override, float2 *dst_override, int skip_done) {
  extern __shared__ float2 sm[];
  const Item it = items[blockIdx.x];
  const ProbDev *P = probs + it.prob;
  if (skip_done && P->st->done) return;
  const int M = P->M, W = P->W, H = P->H, Wh = P->Wh;
  const int r0 = it.a;
  const int nr = min(it.b, H - r0);
  float2 *twm = sm;
  float2 *tww = twm + tw_cap;
  float2 *b0 = tww + tw_cap + 1;
  float2 *b1 = b0 + buf_cap;
  const int tid = threadIdx.x, nthr = blockDim.x;
  for (int i = tid; i < M; i += nthr) twm[i] = P->tw_m[i];
  for (int i = tid; i <= M; i += nthr) tww[i] = P->tw_w[i];
  const float *src = src_override ? src_override : P->f;
  const FastDiv fd1(M > 0 ? M : 1);
  for (int idx = tid; idx < nr * M; idx += nthr) {
    int row, n;
    fd1.divmod(idx, row, n);
    b0[row * M + n] = reinterpret_cast<const float2 *>(src + (long)(r0 + row) * W)[n];
  }
  __syncthreads();
  const float2 *Z = stockham(b0, b1, M, nr, M, twm, tid, nthr);
  float2 *dst = dst_override ? dst_override : P->spec;
  const FastDiv fd2(Wh > 0 ? Wh : 1);
  for (int idx = tid; idx < nr * Wh; idx += nthr) {
    int row, kk;
    fd2.divmod(idx, row, kk);
    const float2 zk = Z[row * M + (kk == M ? 0 : kk)];
    const float2 zc = cconj(Z[row * M + (kk == 0 ? 0 : M - kk)]);
    // X_k = ((Z_k + conj Z_{M-k}) - i w^k (Z_k - conj Z_{M-k})) / 2
    const float2 t = cmul(tww[kk], csub(zk, zc));
    const float2 sum = cadd(zk, zc);
    dst[(long)(r0 + row) * Wh + kk] = make_float2(0.5f * (sum.x + t.y), 0.5f * (sum.y - t.x));
  }
}

// Pass 2: columns of the half spectrum. mode 0: forward FFT only (spectra of y and the
// PSF at set-up); mode 1: forward FFT, X = C + G F, inverse FFT (the FP-step solve);
// mode 2: forward FFT, X = K F / (H W), inverse FFT (H x, for the objective).
__global__ void __launch_bounds__(256)
k_fft_cols(const ProbDev *__restrict__ probs, const Item *__restrict__ items, int tw_cap,
           int buf_cap, int mode, float2 *spec_override, int skip_done) {
  extern __shared__ float2 sm[];
  const Item it = items[blockIdx.x];
  const ProbDev *P = probs + it.prob;
  if (skip_done && P->st->done) return;
  const int H = P->H, Wh = P->Wh;
  const int c0 = it.a;
  const int nc = min(it.b, Wh - c0);
  const int hs = H + 1;   // padded column stride in shared memory
  float2 *twh = sm;
  float2 *b0 = twh + tw_cap;
  float2 *b1 = b0 + buf_cap;
  const int tid = threadIdx.x, nthr = blockDim.x;
  for (int i = tid; i < H; i += nthr) twh[i] = P->tw_h[i];
  float2 *spec = spec_override ? spec_override : P->spec;
  const FastDiv fd3(nc > 0 ? nc : 1);
  for (int idx = tid; idx < H * nc; idx += nthr) {
    int r, c;
    fd3.divmod(idx, r, c);
    b0[c * hs + r] = spec[(long)r * Wh + c0 + c];
  }
  __syncthreads();
  float2 *F = stockham(b0, b1, H, nc, hs, twh, tid, nthr);
  if (mode == 0) {
    const FastDiv fd4(nc > 0 ? nc : 1);
    for (int idx = tid; idx < H * nc; idx += nthr) {
      int r, c;
      fd4.divmod(idx, r, c);
      spec[(long)r * Wh + c0 + c] = F[c * hs + r];
    }
    return;
  }
  if (mode == 1) {
    const FastDiv fd5(nc > 0 ? nc : 1);
    for (int idx = tid; idx < H * nc; idx += nthr) {
      int r, c;
      fd5.divmod(idx, r, c);
      const long g = (long)r * Wh + c0 + c;
      const float2 cc = P->Cc[g];
      const float gg = P->Gg[g];
      const float2 f = F[c * hs + r];
      F[c * hs + r] = make_float2(fmaf(gg, f.x, cc.x), -fmaf(gg, f.y, cc.y));  // conj(C + G F)
    }
  } else {
    // mode 2: H x for the objective: conj(K F / (H W))
    const float inv_hw = 1.0f / ((float)H * (float)P->W);
    const FastDiv fd6(nc > 0 ? nc : 1);
    for (int idx = tid; idx < H * nc; idx += nthr) {
      int r, c;
      fd6.divmod(idx, r, c);
      const float2 kk = P->Kh[(long)r * Wh + c0 + c];
      const float2 v = cmul(kk, F[c * hs + r]);
      F[c * hs + r] = make_float2(v.x * inv_hw, -v.y * inv_hw);
    }
  }
  __syncthreads();
  float2 *other = (F == b0) ? b1 : b0;
  const float2 *X = stockham(F, other, H, nc, hs, twh, tid, nthr);
  const FastDiv fd7(nc > 0 ? nc : 1);
  for (int idx = tid; idx < H * nc; idx += nthr) {
    int r, c;
    fd7.divmod(idx, r, c);
    spec[(long)r * Wh + c0 + c] = cconj(X[c * hs + r]);
  }
}

// Pass 3: rows, half spectrum to real, with the FP-step statistics.
__global__ void __launch_bounds__(256)
k_fft_c2r(const ProbDev *__restrict__ probs, const Item *__restrict__ items, int tw_cap,
          int buf_cap, StepArgs sa) {
  extern __shared__ float2 sm[];
  __shared__ int is_last;
  const Item it = items[blockIdx.x];
  const ProbDev *P = probs + it.prob;
  if (sa.update_state && P->st->done) return;
  const int M = P->M, W = P->W, H = P->H, Wh = P->Wh;
  const int r0 = it.a;
  const int nr = min(it.b, H - r0);
  float2 *twm = sm;
  float2 *tww = twm + tw_cap;
  float2 *b0 = tww + tw_cap + 1;
  float2 *b1 = b0 + buf_cap;
  const int tid = threadIdx.x, nthr = blockDim.x;
  for (int i = tid; i < M; i += nthr) twm[i] = P->tw_m[i];
  for (int i = tid; i <= M; i += nthr) tww[i] = P->tw_w[i];
  __syncthreads();
  const float2 *spec = P->spec;
  const FastDiv fd8(M > 0 ? M : 1);
  for (int idx = tid; idx < nr * M; idx += nthr) {
    int row, kk;
    fd8.divmod(idx, row, kk);
    const float2 xk = spec[(long)(r0 + row) * Wh + kk];
    const float2 xc = cconj(spec[(long)(r0 + row) * Wh + (M - kk)]);
    // 2 E_k = X_k + conj X_{M-k};  2 O_k = (X_k - conj X_{M-k}) e^{+2 pi i k / W}
    const float2 e = cadd(xk, xc);
    const float2 o = cmul(csub(xk, xc), cconj(tww[kk]));
    const float2 z = cadd(e, mul_pi(o));          // 2 Z_k = 2 E_k + i 2 O_k
    b0[row * M + kk] = cconj(z);
  }
  __syncthreads();
  const float2 *Y = stockham(b0, b1, M, nr, M, twm, tid, nthr);

  // output row = conj(Y); x[2n] = Re, x[2n+1] = Im; statistics against x_in
  const int esz = P->storage ? 2 : 4;
  float *dst = sa.dst_ptr ? sa.dst_ptr : nullptr;
  void *dst_ring = static_cast<char *>(P->ring) + (size_t)sa.dst * P->slot_stride * esz;
  const void *src_ring = sa.src_ptr ? sa.src_ptr
                                    : static_cast<const char *>(P->ring) +
                                          (size_t)sa.src * P->slot_stride * esz;
  const int src_bf16 = sa.src_ptr ? 0 : P->storage;
  const int warp = tid >> 5, lane = tid & 31, nwarps = nthr >> 5;
  for (int row = warp; row < nr; row += nwarps) {
    const long rowbase = (long)(r0 + row) * W;
    float sd = 0.f, sx = 0.f;
    for (int n = lane; n < M; n += 32) {
      const float2 v = Y[row * M + n];
      const float xe = v.x, xo = -v.y;
      if (dst) {
        reinterpret_cast<float2 *>(dst + rowbase)[n] = make_float2(xe, xo);
      } else {
        store_img(dst_ring, rowbase + 2 * n, xe, P->storage);
        store_img(dst_ring, rowbase + 2 * n + 1, xo, P->storage);
      }
      // statistics use the stored (rounded) values of the new iterate
      const float ye = P->storage ? __bfloat162float(__float2bfloat16_rn(xe)) : xe;
      const float yo = P->storage ? __bfloat162float(__float2bfloat16_rn(xo)) : xo;
      const float pe = load_img(src_ring, rowbase + 2 * n, src_bf16);
      const float po = load_img(src_ring, rowbase + 2 * n + 1, src_bf16);
      sd = fmaf(ye - pe, ye - pe, sd);
      sd = fmaf(yo - po, yo - po, sd);
      sx = fmaf(pe, pe, sx);
      sx = fmaf(po, po, sx);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      sd += __shfl_xor_sync(0xffffffffu, sd, off);
      sx += __shfl_xor_sync(0xffffffffu, sx, off);
    }
    if (lane == 0) P->row_stats[r0 + row] = make_float2(sd, sx);
  }
  if (!sa.update_state) return;

  // last CTA of this problem: fixed-order reduction of the row sums, termination test
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    const unsigned t = atomicAdd(&P->st->counter, 1u);
    is_last = (t == (unsigned)(P->n_row_items - 1));
  }
  __syncthreads();
  if (!is_last || warp != 0) return;
  __threadfence();
  double sd = 0.0, sx = 0.0;
  for (int r = lane; r < H; r += 32) {
    const float2 v = __ldcg(&P->row_stats[r]);
    sd += (double)v.x;
    sx += (double)v.y;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    sd += __shfl_xor_sync(0xffffffffu, sd, off);
    sx += __shfl_xor_sync(0xffffffffu, sx, off);
  }
  if (lane == 0) {
    ProbState *st = P->st;
    const double rel = sx > 0.0 ? sqrt(sd / sx) : (sd > 0.0 ? INFINITY : 0.0);
    st->rel_change = rel;
    st->calls += 1;
    if (rel < st->tol || st->calls >= st->max_calls) {
      st->done = 1;
      st->converged = rel < st->tol ? 1 : 0;
      st->final_slot = sa.dst;
    }
    st->counter = 0;
    __threadfence();
  }
}

// The whole solve of one FP step for one problem in one thread-block cluster, with the
// half spectrum held in the cluster's shared memory (used when it fits):
//   rows R2C of the CTA's row band -> A (rows x (W/2+1), local shared memory)
//   cluster barrier; each CTA gathers its band of spectrum columns from every CTA's A
//   through distributed shared memory, column FFT, X = C + G F, inverse column FFT
//   cluster barrier; each CTA scatters its columns back into the owners' A
//   cluster barrier; rows C2R of the band -> x_{k+1}, statistics, termination test.
// Global traffic per pixel: f (4 B), C and G (~6 B), x_k for the statistics (4 B) and
// x_{k+1} (4 B); the spectrum never leaves the chip.
__device__ __forceinline__ int band_lo(int q, int n, const FastDiv &by_ncta) { return by_ncta.div(q * n); }
__device__ __forceinline__ int band_owner(int h, int ncta, const FastDiv &by_n) {
  return by_n.div((h + 1) * ncta - 1);
}

constexpr int kClusterThreads = 512;

__global__ void __launch_bounds__(kClusterThreads)
k_fft_solve_cluster(const ProbDev *__restrict__ probs, const int *__restrict__ list, StepArgs sa,
                    int tw_cap_m, int tw_cap_h, int a_cap, int buf_cap) {
  extern __shared__ float2 sm[];
  __shared__ float part_d, part_x;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = cl.block_rank();
  const int ncta = cl.num_blocks();
  const ProbDev *P = probs + list[blockIdx.x / ncta];
  if (sa.update_state && P->st->done) return;   // uniform over the cluster
  const int H = P->H, W = P->W, M = P->M, Wh = P->Wh;
  const FastDiv by_ncta(ncta), by_h(H);
  const int r0 = band_lo(rank, H, by_ncta), nr = band_lo(rank + 1, H, by_ncta) - r0;
  const int c0 = band_lo(rank, Wh, by_ncta), nc = band_lo(rank + 1, Wh, by_ncta) - c0;
  const int hs = H + 1;
  float2 *twm = sm;
  float2 *tww = twm + tw_cap_m;
  float2 *twh = tww + tw_cap_m + 1;
  float2 *A = twh + tw_cap_h;
  float2 *X0 = A + a_cap;
  float2 *X1 = X0 + buf_cap;
  const int tid = threadIdx.x, nthr = blockDim.x;
  for (int i = tid; i < M; i += nthr) twm[i] = P->tw_m[i];
  for (int i = tid; i <= M; i += nthr) tww[i] = P->tw_w[i];
  for (int i = tid; i < H; i += nthr) twh[i] = P->tw_h[i];
  // 1. rows of f, real to half spectrum
  const FastDiv fdm(M);
  copy_batched<4>(nr * M, tid, nthr,
      [&](int idx) {
        int row, n;
        fdm.divmod(idx, row, n);
        return reinterpret_cast<const float2 *>(P->f + (long)(r0 + row) * W)[n];
      },
      [&](int idx, float2 v) { X0[idx] = v; });
  __syncthreads();
  const float2 *Z = stockham(X0, X1, M, nr, M, twm, tid, nthr);
  const FastDiv fd10(Wh > 0 ? Wh : 1);
  for (int idx = tid; idx < nr * Wh; idx += nthr) {
    int row, kk;
    fd10.divmod(idx, row, kk);
    const float2 zk = Z[row * M + (kk == M ? 0 : kk)];
    const float2 zc = cconj(Z[row * M + (kk == 0 ? 0 : M - kk)]);
    const float2 t = cmul(tww[kk], csub(zk, zc));
    const float2 s = cadd(zk, zc);
    A[row * Wh + kk] = make_float2(0.5f * (s.x + t.y), 0.5f * (s.y - t.x));
  }
  cl.sync();
  // 2. gather this CTA's spectrum columns from every row band
  const FastDiv fdc(nc > 0 ? nc : 1);
  copy_batched<8>(H * nc, tid, nthr,
      [&](int idx) {
        int h, c;
        fdc.divmod(idx, h, c);
        const int q = band_owner(h, ncta, by_h);
        const float2 *Aq = cl.map_shared_rank(A, q);
        return Aq[(h - band_lo(q, H, by_ncta)) * Wh + c0 + c];
      },
      [&](int idx, float2 v) {
        int h, c;
        fdc.divmod(idx, h, c);
        X0[c * hs + h] = v;
      });
  __syncthreads();
  float2 *F = stockham(X0, X1, H, nc, hs, twh, tid, nthr);
  for (int base = tid; base < H * nc; base += 4 * nthr) {
    float2 cc[4];
    float gg[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int idx = base + u * nthr;
      if (idx < H * nc) {
        int r, c;
        fdc.divmod(idx, r, c);
        const long g = (long)r * Wh + c0 + c;
        cc[u] = P->Cc[g];
        gg[u] = P->Gg[g];
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int idx = base + u * nthr;
      if (idx < H * nc) {
        int r, c;
        fdc.divmod(idx, r, c);
        const float2 fv = F[c * hs + r];
        F[c * hs + r] = make_float2(fmaf(gg[u], fv.x, cc[u].x), -fmaf(gg[u], fv.y, cc[u].y));  // conj(C + G F)
      }
    }
  }
  __syncthreads();
  const float2 *Xs = stockham(F, F == X0 ? X1 : X0, H, nc, hs, twh, tid, nthr);
  cl.sync();   // every CTA has finished reading the A bands
  // 3. scatter the solved columns back to the row bands
  const FastDiv fd13(nc > 0 ? nc : 1);
  for (int idx = tid; idx < H * nc; idx += nthr) {
    int h, c;
    fd13.divmod(idx, h, c);
    const int q = band_owner(h, ncta, by_h);
    float2 *Aq = cl.map_shared_rank(A, q);
    Aq[(h - band_lo(q, H, by_ncta)) * Wh + c0 + c] = cconj(Xs[c * hs + h]);
  }
  cl.sync();
  // 4. rows, half spectrum to real, statistics against x_k
  const FastDiv fd14(M > 0 ? M : 1);
  for (int idx = tid; idx < nr * M; idx += nthr) {
    int row, kk;
    fd14.divmod(idx, row, kk);
    const float2 xk = A[row * Wh + kk];
    const float2 xc = cconj(A[row * Wh + (M - kk)]);
    const float2 e = cadd(xk, xc);
    const float2 o = cmul(csub(xk, xc), cconj(tww[kk]));
    X0[row * M + kk] = cconj(cadd(e, mul_pi(o)));
  }
  __syncthreads();
  const float2 *Y = stockham(X0, X1, M, nr, M, twm, tid, nthr);
  const int esz = P->storage ? 2 : 4;
  void *dst_ring = static_cast<char *>(P->ring) + (size_t)sa.dst * P->slot_stride * esz;
  const void *src_ring = sa.src_ptr ? sa.src_ptr
                                    : static_cast<const char *>(P->ring) + (size_t)sa.src * P->slot_stride * esz;
  const int src_bf16 = sa.src_ptr ? 0 : P->storage;
  float sd = 0.f, sx = 0.f;
  // previous iterate x_k for the statistics: 4 pixel pairs in flight per thread
  for (int b0 = tid; b0 < nr * M; b0 += 4 * nthr) {
    float2 prev[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int idx = b0 + u * nthr;
      if (idx < nr * M) {
        int row, n;
        fdm.divmod(idx, row, n);
        const long base = (long)(r0 + row) * W + 2 * n;
        prev[u] = make_float2(load_img(src_ring, base, src_bf16), load_img(src_ring, base + 1, src_bf16));
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int idx = b0 + u * nthr;
      if (idx >= nr * M) break;
      int row, n;
      fdm.divmod(idx, row, n);
      const long base = (long)(r0 + row) * W + 2 * n;
      const float2 v = Y[row * M + n];
      const float xe = v.x, xo = -v.y;
      float ye = xe, yo = xo;
      if (sa.dst_ptr) {
        reinterpret_cast<float2 *>(sa.dst_ptr + (long)(r0 + row) * W)[n] = make_float2(xe, xo);
      } else {
        store_img(dst_ring, base, xe, P->storage);
        store_img(dst_ring, base + 1, xo, P->storage);
        if (P->storage) {
          ye = __bfloat162float(__float2bfloat16_rn(xe));
          yo = __bfloat162float(__float2bfloat16_rn(xo));
        }
      }
      const float pe = prev[u].x, po = prev[u].y;
      sd = fmaf(ye - pe, ye - pe, sd);
      sd = fmaf(yo - po, yo - po, sd);
      sx = fmaf(pe, pe, sx);
      sx = fmaf(po, po, sx);
    }
  }
  // CTA sums (fixed order), then rank 0 sums the cluster's partials in rank order
  __shared__ float red_d[kClusterThreads / 32], red_x[kClusterThreads / 32];
  const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    sd += __shfl_xor_sync(0xffffffffu, sd, off);
    sx += __shfl_xor_sync(0xffffffffu, sx, off);
  }
  if (lane == 0) { red_d[warp] = sd; red_x[warp] = sx; }
  __syncthreads();
  if (tid == 0) {
    float td = 0.f, tx = 0.f;
    for (int w = 0; w < (nthr >> 5); ++w) { td += red_d[w]; tx += red_x[w]; }
    part_d = td;
    part_x = tx;
  }
  cl.sync();
  if (sa.update_state && rank == 0 && tid == 0) {
    double tsd = 0.0, tsx = 0.0;
    for (int q = 0; q < ncta; ++q) {
      tsd += (double)*cl.map_shared_rank(&part_d, q);
      tsx += (double)*cl.map_shared_rank(&part_x, q);
    }
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
  cl.sync();   // keep shared memory alive until rank 0 has read the partials
}

__global__ void k_spectral_constants(const float2 *__restrict__ khat, const float2 *__restrict__ yhat,
                                     float2 *Cc, float *Gg, int n, double inv_sigma2,
                                     double alpha, double inv_hw) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double kr = khat[i].x, ki = khat[i].y;
  const double yr = yhat[i].x, yi = yhat[i].y;
  const double d = (kr * kr + ki * ki) * inv_sigma2 + alpha;
  // conj(K) Y = (kr yr + ki yi) + i (kr yi - ki yr)
  const double s = inv_sigma2 / d * inv_hw;
  Cc[i] = make_float2((float)((kr * yr + ki * yi) * s), (float)((kr * yi - ki * yr) * s));
  Gg[i] = (float)(alpha / d * inv_hw);
}

}  // namespace

int fft_smem_rows(int tw_cap, int buf_cap) { return (int)((2 * (size_t)tw_cap + 1 + 2 * (size_t)buf_cap) * sizeof(float2)); }
int fft_smem_cols(int tw_cap, int buf_cap) { return (int)(((size_t)tw_cap + 2 * (size_t)buf_cap) * sizeof(float2)); }

// Raises a kernel's dynamic shared-memory limit the first time a launch needs more
// than the 48 KB default (a per-kernel high-water mark; races only repeat the call).
static cudaError_t set_smem(const void *fn, int bytes, int *high_water) {
  if (bytes <= 48 * 1024 || bytes <= *high_water) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) *high_water = bytes;
  return e;
}
static int hw_r2c = 0, hw_cols = 0, hw_c2r = 0;

cudaError_t fft_prepare(int row_tw_cap, int row_buf_cap, int col_tw_cap, int col_buf_cap) {
  const int sr = fft_smem_rows(row_tw_cap, row_buf_cap), sc = fft_smem_cols(col_tw_cap, col_buf_cap);
  cudaError_t e = set_smem((const void *)k_fft_r2c, sr, &hw_r2c);
  if (e == cudaSuccess) e = set_smem((const void *)k_fft_c2r, sr, &hw_c2r);
  if (e == cudaSuccess) e = set_smem((const void *)k_fft_cols, sc, &hw_cols);
  return e;
}

cudaError_t launch_fft_r2c(const ProbDev *d_probs, const Item *d_items, int n_items,
                           int tw_cap, int buf_cap, const float *src_override,
                           float2 *dst_override, int skip_done, cudaStream_t s) {
  if (n_items <= 0) return cudaSuccess;
  const int smem = fft_smem_rows(tw_cap, buf_cap);
  cudaError_t e = set_smem((const void *)k_fft_r2c, smem, &hw_r2c);
  if (e != cudaSuccess) return e;
  k_fft_r2c<<<n_items, 256, smem, s>>>(d_probs, d_items, tw_cap, buf_cap, src_override,
                                       dst_override, skip_done);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_fft_cols(const ProbDev *d_probs, const Item *d_items, int n_items,
                            int tw_cap, int buf_cap, int mode, float2 *spec_override,
                            int skip_done, cudaStream_t s) {
  if (n_items <= 0) return cudaSuccess;
  const int smem = fft_smem_cols(tw_cap, buf_cap);
  cudaError_t e = set_smem((const void *)k_fft_cols, smem, &hw_cols);
  if (e != cudaSuccess) return e;
  k_fft_cols<<<n_items, 256, smem, s>>>(d_probs, d_items, tw_cap, buf_cap, mode, spec_override,
                                        skip_done);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_fft_c2r(const ProbDev *d_probs, const Item *d_items, int n_items,
                           int tw_cap, int buf_cap, StepArgs sa, cudaStream_t s) {
  if (n_items <= 0) return cudaSuccess;
  const int smem = fft_smem_rows(tw_cap, buf_cap);
  cudaError_t e = set_smem((const void *)k_fft_c2r, smem, &hw_c2r);
  if (e != cudaSuccess) return e;
  k_fft_c2r<<<n_items, 256, smem, s>>>(d_probs, d_items, tw_cap, buf_cap, sa);
  count_launches(1);
  return cudaGetLastError();
}

// Shared memory of the cluster solve for one problem (complex elements): twiddles, the
// row band's half spectrum A, two work buffers (row band rows or column band columns).
void fft_cluster_caps(int H, int W, int ncta, int *a_elems, int *buf_elems) {
  const int M = W / 2, Wh = M + 1;
  const int nr = (H + ncta - 1) / ncta, nc = (Wh + ncta - 1) / ncta;
  *a_elems = nr * Wh;
  *buf_elems = std::max(nr * M, nc * (H + 1));
}

int fft_cluster_smem(int tw_cap_m, int tw_cap_h, int a_cap, int buf_cap) {
  return (int)(((size_t)2 * tw_cap_m + 1 + tw_cap_h + a_cap + 2 * (size_t)buf_cap) * sizeof(float2));
}

static int hw_cluster = 0;

cudaError_t fft_cluster_prepare(int smem, int ncta) {
  cudaError_t e = set_smem((const void *)k_fft_solve_cluster, smem, &hw_cluster);
  if (e == cudaSuccess && ncta > 8)
    e = cudaFuncSetAttribute((const void *)k_fft_solve_cluster,
                             cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  return e;
}

cudaError_t launch_fft_solve_cluster(const ProbDev *d_probs, const int *d_list, int n, int ncta,
                                     int tw_cap_m, int tw_cap_h, int a_cap, int buf_cap,
                                     StepArgs sa, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(n * ncta);
  cfg.blockDim = dim3(kClusterThreads);
  cfg.dynamicSmemBytes = fft_cluster_smem(tw_cap_m, tw_cap_h, a_cap, buf_cap);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = ncta;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_fft_solve_cluster, d_probs, d_list, sa, tw_cap_m,
                                     tw_cap_h, a_cap, buf_cap);
  count_launches(1);
  return e;
}

// Largest cluster the device accepts for the cluster solve with this shared memory.
int fft_cluster_max_active(int ncta, int smem) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ncta);
  cfg.blockDim = dim3(kClusterThreads);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = ncta;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, (const void *)k_fft_solve_cluster, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

cudaError_t launch_spectral_constants(const ProbDev *, const float2 *k_hat, const float2 *y_hat,
                                      float2 *Cc, float *Gg, int n, double inv_sigma2,
                                      double alpha, double inv_hw, cudaStream_t s) {
  k_spectral_constants<<<(n + 255) / 256, 256, 0, s>>>(k_hat, y_hat, Cc, Gg, n, inv_sigma2,
                                                       alpha, inv_hw);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace red
