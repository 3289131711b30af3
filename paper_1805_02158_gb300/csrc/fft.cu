// Fourier-domain linear solve of the FP step for a block-circulant blur H (Eq. (7) and
// its footnote): x_{k+1} = IFFT2( C + G . FFT2(f) ),
//   C = conj(K) FFT2(y) / (sigma^2 D) / (H W),  G = alpha / D / (H W),
//   D = |K|^2 / sigma^2 + alpha,  K = FFT2 of the circularly centred PSF.
//
// The 2-D transform works on a half spectrum (H x (W/2 + 1) complex):
//   rows, real-to-complex: each row of W reals is packed as W/2 complex values, a
//     W/2-point complex FFT is taken and the W/2 + 1 non-redundant bins are untangled;
//   columns: forward FFT, the pointwise solve X = C + G F, inverse FFT;
//   rows, complex-to-real, with the relative-change statistics of the FP step.
// Two implementations of the same transforms:
//   * k_fft_solve_cluster: one thread-block cluster per problem, the half spectrum in the
//     cluster's shared memory; each CTA pushes its row band's bins into the column buffers
//     of the CTAs owning the columns (remote stores through distributed shared memory),
//     and after the column solve scatters them back the same way: two cluster barriers
//     per FP step (images up to 384 x 384 with 16 CTAs);
//   * k_fft_r2c / k_fft_cols / k_fft_c2r: three passes through global memory (any size).
// Transforms are self-sorting Stockham passes in shared memory with register-resident
// radix 16, 12, 8, 6, 4, 3 and 2 butterflies (sizes 2^a 3^b): few passes, so few
// barriers. Composite radices are built from radix-2/3/4 kernels with constant roots of
// unity; pass twiddles come from tables computed on the host in double precision.
// Sequences in shared memory are padded (one slot per 16 elements, odd stride) so the
// strided Stockham writes and the column transposes are free of bank conflicts.
// Inverse transforms use IFFT(X) = conj(FFT(conj(X))); the 1/(H W) scale is in C and G.
//
// The same transforms serve the steepest-descent baseline of SD-MPE (Sec. IV): one SD step
// on Eq. (5) for a circulant H is
//   x_{k+1} = x_k - mu grad E(x_k) = IFFT2( C_sd + G_sd . FFT2(x_k) ) + mu alpha f(x_k),
//   C_sd = mu conj(K) FFT2(y) / sigma^2 / (H W),  G_sd = (1 - mu alpha - mu |K|^2 / sigma^2) / (H W),
// so an SD problem's step transforms x_k instead of f and adds mu alpha f at the output.
#include <cooperative_groups.h>

#include <algorithm>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace red {

namespace {

// Asynchronous global -> shared copies (cp.async, 4 or 8 bytes, source aligned to the size):
// each thread issues its copies, commits them as a group, and waits for the group before a
// barrier, so all loads of a phase are in flight together and land in any shared layout.
__device__ __forceinline__ void cp_async8(void *smem_dst, const void *gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async4(void *smem_dst, const void *gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 mul_mi(float2 a) { return make_float2(a.y, -a.x); }  // * (-i)
__device__ __forceinline__ float2 mul_pi(float2 a) { return make_float2(-a.y, a.x); }  // * (+i)

// e^{-2 pi i m / 48}: every root of unity the radix-16/12/8/6 kernels need
__device__ __forceinline__ float2 root48(int m) {
  constexpr float c[48] = {
      1.0f, 0.99144486137381038f, 0.96592582628906831f, 0.92387953251128674f,
      0.8660254037844386f, 0.79335334029123517f, 0.70710678118654757f, 0.60876142900872066f,
      0.5f, 0.38268343236508978f, 0.25881904510252074f, 0.1305261922200516f,
      0.0f, -0.1305261922200516f, -0.25881904510252074f, -0.38268343236508978f,
      -0.5f, -0.60876142900872066f, -0.70710678118654757f, -0.79335334029123517f,
      -0.8660254037844386f, -0.92387953251128674f, -0.96592582628906831f, -0.99144486137381038f,
      -1.0f, -0.99144486137381038f, -0.96592582628906831f, -0.92387953251128674f,
      -0.8660254037844386f, -0.79335334029123517f, -0.70710678118654757f, -0.60876142900872066f,
      -0.5f, -0.38268343236508978f, -0.25881904510252074f, -0.1305261922200516f,
      0.0f, 0.1305261922200516f, 0.25881904510252074f, 0.38268343236508978f,
      0.5f, 0.60876142900872066f, 0.70710678118654757f, 0.79335334029123517f,
      0.8660254037844386f, 0.92387953251128674f, 0.96592582628906831f, 0.99144486137381038f};
  constexpr float s[48] = {
      0.0f, 0.1305261922200516f, 0.25881904510252074f, 0.38268343236508978f,
      0.5f, 0.60876142900872066f, 0.70710678118654757f, 0.79335334029123517f,
      0.8660254037844386f, 0.92387953251128674f, 0.96592582628906831f, 0.99144486137381038f,
      1.0f, 0.99144486137381038f, 0.96592582628906831f, 0.92387953251128674f,
      0.8660254037844386f, 0.79335334029123517f, 0.70710678118654757f, 0.60876142900872066f,
      0.5f, 0.38268343236508978f, 0.25881904510252074f, 0.1305261922200516f,
      0.0f, -0.1305261922200516f, -0.25881904510252074f, -0.38268343236508978f,
      -0.5f, -0.60876142900872066f, -0.70710678118654757f, -0.79335334029123517f,
      -0.8660254037844386f, -0.92387953251128674f, -0.96592582628906831f, -0.99144486137381038f,
      -1.0f, -0.99144486137381038f, -0.96592582628906831f, -0.92387953251128674f,
      -0.8660254037844386f, -0.79335334029123517f, -0.70710678118654757f, -0.60876142900872066f,
      -0.5f, -0.38268343236508978f, -0.25881904510252074f, -0.1305261922200516f};
  return make_float2(c[m % 48], -s[m % 48]);
}

// In-register forward DFTs (natural-order output).
__device__ __forceinline__ void dft_base(float2 (&a)[2]) {
  const float2 t = a[0];
  a[0] = cadd(t, a[1]);
  a[1] = csub(t, a[1]);
}
__device__ __forceinline__ void dft_base(float2 (&a)[3]) {
  // w = e^{-2 pi i / 3}: y1 = a0 - s/2 - i (sqrt3/2) d, y2 = a0 - s/2 + i (sqrt3/2) d
  const float2 s12 = cadd(a[1], a[2]), d12 = csub(a[1], a[2]);
  const float2 m = make_float2(a[0].x - 0.5f * s12.x, a[0].y - 0.5f * s12.y);
  const float h = 0.86602540378443864676f;
  const float2 e = make_float2(h * d12.x, h * d12.y);
  a[0] = cadd(a[0], s12);
  a[1] = cadd(m, mul_mi(e));
  a[2] = cadd(m, mul_pi(e));
}
__device__ __forceinline__ void dft_base(float2 (&a)[4]) {
  const float2 t0 = cadd(a[0], a[2]), t1 = csub(a[0], a[2]), t2 = cadd(a[1], a[3]);
  const float2 t3 = mul_mi(csub(a[1], a[3]));
  a[0] = cadd(t0, t2);
  a[1] = cadd(t1, t3);
  a[2] = csub(t0, t2);
  a[3] = csub(t1, t3);
}

// N = A * B point DFT by one Cooley-Tukey step: B-point DFTs of the A interleaved
// subsequences, twiddles w_N^{n1 k1}, A-point DFTs across them; X[k1 + B k2].
template <int A, int B>
__device__ __forceinline__ void dft_ab(float2 (&x)[A * B]) {
  constexpr int N = A * B;
  float2 y[A][B];
#pragma unroll
  for (int n1 = 0; n1 < A; ++n1) {
    float2 t[B];
#pragma unroll
    for (int n2 = 0; n2 < B; ++n2) t[n2] = x[n1 + A * n2];
    dft_base(t);
#pragma unroll
    for (int k1 = 0; k1 < B; ++k1) {
      const int m = (n1 * k1) % N;
      if (m == 0)
        y[n1][k1] = t[k1];
      else if (4 * m == N)
        y[n1][k1] = mul_mi(t[k1]);
      else if (2 * m == N)
        y[n1][k1] = make_float2(-t[k1].x, -t[k1].y);
      else
        y[n1][k1] = cmul(t[k1], root48(m * (48 / N)));
    }
  }
#pragma unroll
  for (int k1 = 0; k1 < B; ++k1) {
    float2 t[A];
#pragma unroll
    for (int n1 = 0; n1 < A; ++n1) t[n1] = y[n1][k1];
    dft_base(t);
#pragma unroll
    for (int k2 = 0; k2 < A; ++k2) x[k1 + B * k2] = t[k2];
  }
}

template <int R> __device__ __forceinline__ void dft(float2 (&a)[R]);
template <> __device__ __forceinline__ void dft<2>(float2 (&a)[2]) { dft_base(a); }
template <> __device__ __forceinline__ void dft<3>(float2 (&a)[3]) { dft_base(a); }
template <> __device__ __forceinline__ void dft<4>(float2 (&a)[4]) { dft_base(a); }
template <> __device__ __forceinline__ void dft<6>(float2 (&a)[6]) { dft_ab<2, 3>(a); }
template <> __device__ __forceinline__ void dft<8>(float2 (&a)[8]) { dft_ab<2, 4>(a); }
template <> __device__ __forceinline__ void dft<12>(float2 (&a)[12]) { dft_ab<4, 3>(a); }
template <> __device__ __forceinline__ void dft<16>(float2 (&a)[16]) { dft_ab<4, 4>(a); }

// padded position of element e of a shared-memory sequence (one pad slot per 16)
__device__ __forceinline__ int pidx(int e) { return e + (e >> 4); }

// One Stockham pass of radix R over nseq sequences (stride ss) of length n, after passes
// of product Ns: butterfly j reads elements j + q n/R, twiddles them by
// w_n^{(j mod Ns) q n/(Ns R)}, takes an R-point DFT and writes positions
// (j - j mod Ns) R + j mod Ns + q Ns (natural-order output overall).
template <int R>
__device__ __forceinline__ void stockham_pass(const float2 *in, float2 *out, int n, int nseq, int ss,
                                              int Ns, const float2 *__restrict__ tw, int tid,
                                              int nthr) {
  const int nb = n / R;
  const int tws = n / (Ns * R);
  const FastDiv dnb(nb), dns(Ns);
  for (int t = tid; t < nseq * nb; t += nthr) {
    int s, j, g, kk;
    dnb.divmod(t, s, j);
    dns.divmod(j, g, kk);
    const float2 *src = in + s * ss;
    float2 *dst = out + s * ss;
    float2 a[R];
#pragma unroll
    for (int q = 0; q < R; ++q) a[q] = src[pidx(j + q * nb)];
    if (kk) {
#pragma unroll
      for (int q = 1; q < R; ++q) a[q] = cmul(a[q], tw[kk * q * tws]);
    }
    dft<R>(a);
    const int base = g * Ns * R + kk;
#pragma unroll
    for (int q = 0; q < R; ++q) dst[pidx(base + q * Ns)] = a[q];
  }
}

__device__ __forceinline__ int pick_radix(int rem) {
  if (rem % 16 == 0) return 16;
  if (rem % 12 == 0) return 12;
  if (rem % 8 == 0) return 8;
  if (rem % 6 == 0) return 6;
  if (rem % 4 == 0) return 4;
  if (rem % 3 == 0) return 3;
  return 2;
}

// Forward FFT of nseq padded sequences of length n (2^a 3^b) held at x + s * ss; ping-pongs
// between x and y and returns the buffer holding the result. Ends with a barrier. Not
// inlined: one copy of the unrolled radix passes serves every call site (instruction
// cache). Powers of two take a copy with the radix-16/8/4/2 passes only, whose smaller
// code stays resident in the instruction cache across the transform phases.
template <bool POW2>
__device__ __forceinline__ float2 *fft_smem_impl(float2 *x, float2 *y, int n, int nseq, int ss,
                                                 const float2 *__restrict__ tw, int tid, int nthr) {
  float2 *in = x, *out = y;
  int Ns = 1, rem = n;
  while (rem > 1) {
    const int r = pick_radix(rem);
    if (POW2) {
      switch (r) {
        case 16: stockham_pass<16>(in, out, n, nseq, ss, Ns, tw, tid, nthr); break;
        case 8: stockham_pass<8>(in, out, n, nseq, ss, Ns, tw, tid, nthr); break;
        case 4: stockham_pass<4>(in, out, n, nseq, ss, Ns, tw, tid, nthr); break;
        default: stockham_pass<2>(in, out, n, nseq, ss, Ns, tw, tid, nthr); break;
      }
    } else {
      switch (r) {
        case 16: stockham_pass<16>(in, out, n, nseq, ss, Ns, tw, tid, nthr); break;
        case 12: stockham_pass<12>(in, out, n, nseq, ss, Ns, tw, tid, nthr); break;
        case 8: stockham_pass<8>(in, out, n, nseq, ss, Ns, tw, tid, nthr); break;
        case 6: stockham_pass<6>(in, out, n, nseq, ss, Ns, tw, tid, nthr); break;
        case 4: stockham_pass<4>(in, out, n, nseq, ss, Ns, tw, tid, nthr); break;
        case 3: stockham_pass<3>(in, out, n, nseq, ss, Ns, tw, tid, nthr); break;
        default: stockham_pass<2>(in, out, n, nseq, ss, Ns, tw, tid, nthr); break;
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

__device__ __noinline__ float2 *fft_smem_pow2(float2 *x, float2 *y, int n, int nseq, int ss,
                                              const float2 *__restrict__ tw, int tid, int nthr) {
  return fft_smem_impl<true>(x, y, n, nseq, ss, tw, tid, nthr);
}

__device__ __noinline__ float2 *fft_smem_mixed(float2 *x, float2 *y, int n, int nseq, int ss,
                                               const float2 *__restrict__ tw, int tid, int nthr) {
  return fft_smem_impl<false>(x, y, n, nseq, ss, tw, tid, nthr);
}

__device__ __forceinline__ float2 *fft_smem(float2 *x, float2 *y, int n, int nseq, int ss,
                                            const float2 *__restrict__ tw, int tid, int nthr) {
  return (n & (n - 1)) == 0 ? fft_smem_pow2(x, y, n, nseq, ss, tw, tid, nthr)
                            : fft_smem_mixed(x, y, n, nseq, ss, tw, tid, nthr);
}

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

// Bin k of the half spectrum from the packed M-point transform Z of one row (padded):
// X_k = ((Z_k + conj Z_{M-k}) - i w^k (Z_k - conj Z_{M-k})) / 2, w = e^{-2 pi i / W}.
__device__ __forceinline__ float2 r2c_bin(const float2 *Z, int M, int kk, const float2 *tww) {
  const float2 zk = Z[pidx(kk == M ? 0 : kk)];
  const float2 zc = cconj(Z[pidx(kk == 0 ? 0 : M - kk)]);
  const float2 t = cmul(tww[kk], csub(zk, zc));
  const float2 s = cadd(zk, zc);
  return make_float2(0.5f * (s.x + t.y), 0.5f * (s.y - t.x));
}

// conj(2 Z_k) with 2 Z_k = (X_k + conj X_{M-k}) + i (X_k - conj X_{M-k}) e^{+2 pi i k / W}:
// the forward transform of it, conjugated, is W times the row's real samples (packed).
__device__ __forceinline__ float2 c2r_pre(float2 xk, float2 xmk, float2 twk) {
  const float2 xc = cconj(xmk);
  const float2 e = cadd(xk, xc);
  const float2 o = cmul(csub(xk, xc), cconj(twk));
  return cconj(cadd(e, mul_pi(o)));
}

// Writes of x_{k+1} and the relative-change statistics against x_k.
struct StepOut {
  const ProbDev *P;
  StepArgs sa;
  void *dst_ring;
  const void *src_ring;
  int src_type;
  __device__ __forceinline__ void init(const ProbDev *p, const StepArgs &s) {
    P = p;
    sa = s;
    const int esz = store_bytes(P->storage);
    dst_ring = static_cast<char *>(P->ring) + (size_t)sa.dst * P->slot_stride * esz;
    src_ring = sa.src_ptr ? sa.src_ptr
                          : static_cast<const char *>(P->ring) + (size_t)sa.src * P->slot_stride * esz;
    src_type = sa.src_ptr ? kStoreF32 : P->storage;
  }
  __device__ __forceinline__ float2 prev(long base) const {
    return make_float2(load_img(src_ring, base, src_type), load_img(src_ring, base + 1, src_type));
  }
  // mu alpha f at (base, base + 1) for an SD problem's step output, 0 for an FP step
  __device__ __forceinline__ float2 sd_term(long base) const {
    if (P->baseline != kBaseSD) return make_float2(0.f, 0.f);
    const float ma = P->sd->mu_alpha_f;
    const float2 fv = *reinterpret_cast<const float2 *>(P->f + base);
    return make_float2(ma * fv.x, ma * fv.y);
  }
  // writes x_{k+1}[base], [base+1] = (xe, xo); accumulates the statistics against pv
  __device__ __forceinline__ void put(long base, float xe, float xo, float2 pv, float &sd,
                                      float &sx) const {
    float ye = xe, yo = xo;
    if (sa.dst_ptr) {
      *reinterpret_cast<float2 *>(sa.dst_ptr + base) = make_float2(xe, xo);
    } else {
      store_img(dst_ring, base, xe, P->storage);
      store_img(dst_ring, base + 1, xo, P->storage);
      ye = round_to_storage(xe, P->storage);
      yo = round_to_storage(xo, P->storage);
    }
    sd = fmaf(ye - pv.x, ye - pv.x, sd);
    sd = fmaf(yo - pv.y, yo - pv.y, sd);
    sx = fmaf(pv.x, pv.x, sx);
    sx = fmaf(pv.y, pv.y, sx);
  }
};

// Termination test of Algorithm 3 after an FP step (one thread).
__device__ __forceinline__ void finish_step(ProbState *st, double sd, double sx, int dst_slot) {
  const double rel = sx > 0.0 ? sqrt(sd / sx) : (sd > 0.0 ? INFINITY : 0.0);
  st->rel_change = rel;
  st->calls += 1;
  if (rel < st->ve_stop_tol) st->ve_off = 1;   // extrapolation ends, baseline steps follow
  if (rel < st->tol || st->calls >= st->max_calls) {
    st->done = 1;
    st->converged = rel < st->tol ? 1 : 0;
    st->final_slot = dst_slot;
  }
}

// ---------------------------------------------------------------------------------------
// three-pass path
// ---------------------------------------------------------------------------------------

// Pass 1: rows, real to half spectrum. Item (prob, first row, rows).
__global__ void __launch_bounds__(256)
k_fft_r2c(const ProbDev *__restrict__ probs, const Item *__restrict__ items, int tw_cap,
          int buf_cap, const float *src_override, float2 *dst_override, int skip_done,
          StepArgs sa, int is_step) {
  extern __shared__ float2 sm[];
  const Item it = items[blockIdx.x];
  const ProbDev *P = probs + it.prob;
  if ((skip_done & 1) && P->st->done) return;     // bit 0: finished problems
  if ((skip_done & 2) && P->st->frozen) return;   // bit 1: frozen problems (full-cycle step)
  const int M = P->M, W = P->W, H = P->H, Wh = P->Wh;
  const int ss = fft_seq_stride(M);
  const int r0 = it.a;
  const int nr = min(it.b, H - r0);
  float2 *twm = sm;
  float2 *tww = twm + tw_cap;
  float2 *b0 = tww + tw_cap + 1;
  float2 *b1 = b0 + buf_cap;
  const int tid = threadIdx.x, nthr = blockDim.x;
  for (int i = tid; i < M; i += nthr) twm[i] = P->tw_m[i];
  for (int i = tid; i <= M; i += nthr) tww[i] = P->tw_w[i];
  const float *src = src_override ? src_override : ((skip_done & kFftSrcY) ? P->y : P->f);
  // an SD problem's step transforms x_k (its ring slot, any storage type)
  const bool sd_step = is_step && P->baseline == kBaseSD;
  StepOut xin;
  if (sd_step) xin.init(P, sa);
  const FastDiv dm(M), dwh(Wh);
  copy_batched<4>(nr * M, tid, nthr,
      [&](int idx) {
        int row, n;
        dm.divmod(idx, row, n);
        if (sd_step) return xin.prev((long)(r0 + row) * W + 2 * n);
        return reinterpret_cast<const float2 *>(src + (long)(r0 + row) * W)[n];
      },
      [&](int idx, float2 v) {
        int row, n;
        dm.divmod(idx, row, n);
        b0[row * ss + pidx(n)] = v;
      });
  __syncthreads();
  const float2 *Z = fft_smem(b0, b1, M, nr, ss, twm, tid, nthr);
  float2 *dst = dst_override ? dst_override : P->spec;
  for (int idx = tid; idx < nr * Wh; idx += nthr) {
    int row, kk;
    dwh.divmod(idx, row, kk);
    dst[(long)(r0 + row) * Wh + kk] = r2c_bin(Z + row * ss, M, kk, tww);
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
  if ((skip_done & 1) && P->st->done) return;     // bit 0: finished problems
  if ((skip_done & 2) && P->st->frozen) return;   // bit 1: frozen problems (full-cycle step)
  const int H = P->H, Wh = P->Wh;
  const int c0 = it.a;
  const int nc = min(it.b, Wh - c0);
  const int hs = fft_seq_stride(H);
  float2 *twh = sm;
  float2 *b0 = twh + tw_cap;
  float2 *b1 = b0 + buf_cap;
  const int tid = threadIdx.x, nthr = blockDim.x;
  for (int i = tid; i < H; i += nthr) twh[i] = P->tw_h[i];
  float2 *spec = spec_override ? spec_override : P->spec;
  const FastDiv dnc(nc > 0 ? nc : 1);
  copy_batched<8>(H * nc, tid, nthr,
      [&](int idx) {
        int r, c;
        dnc.divmod(idx, r, c);
        return spec[(long)r * Wh + c0 + c];
      },
      [&](int idx, float2 v) {
        int r, c;
        dnc.divmod(idx, r, c);
        b0[c * hs + pidx(r)] = v;
      });
  __syncthreads();
  float2 *F = fft_smem(b0, b1, H, nc, hs, twh, tid, nthr);
  if (mode == 0) {
    for (int idx = tid; idx < H * nc; idx += nthr) {
      int r, c;
      dnc.divmod(idx, r, c);
      spec[(long)r * Wh + c0 + c] = F[c * hs + pidx(r)];
    }
    return;
  }
  const float inv_hw = 1.0f / ((float)H * (float)P->W);
  // kU constants (C and G, or K) in flight per thread before any is used: one memory
  // latency per kU elements instead of one per element
  constexpr int kU = 8;
  for (int base = tid; base < H * nc; base += kU * nthr) {
    float2 cv[kU];
    float gv[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int idx = base + u * nthr;
      gv[u] = 0.f;
      if (idx < H * nc) {
        int r, c;
        dnc.divmod(idx, r, c);
        const long g = (long)r * Wh + c0 + c;
        if (mode == 1) {
          cv[u] = P->Cc[g];
          gv[u] = P->Gg[g];
        } else {
          cv[u] = P->Kh[g];
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int idx = base + u * nthr;
      if (idx < H * nc) {
        int r, c;
        dnc.divmod(idx, r, c);
        const float2 fv = F[c * hs + pidx(r)];
        float2 xv;
        if (mode == 1) {
          xv = make_float2(fmaf(gv[u], fv.x, cv[u].x), fmaf(gv[u], fv.y, cv[u].y));
        } else {
          const float2 kv = cmul(cv[u], fv);
          xv = make_float2(kv.x * inv_hw, kv.y * inv_hw);
        }
        F[c * hs + pidx(r)] = cconj(xv);
      }
    }
  }
  __syncthreads();
  const float2 *X = fft_smem(F, F == b0 ? b1 : b0, H, nc, hs, twh, tid, nthr);
  for (int idx = tid; idx < H * nc; idx += nthr) {
    int r, c;
    dnc.divmod(idx, r, c);
    spec[(long)r * Wh + c0 + c] = cconj(X[c * hs + pidx(r)]);
  }
}

// Pass 3: rows, half spectrum to real, with the FP-step statistics and (batched solves)
// the termination test by the last CTA of the problem.
__global__ void __launch_bounds__(256)
k_fft_c2r(const ProbDev *__restrict__ probs, const Item *__restrict__ items, int tw_cap,
          int buf_cap, StepArgs sa) {
  extern __shared__ float2 sm[];
  __shared__ int is_last;
  const Item it = items[blockIdx.x];
  const ProbDev *P = probs + it.prob;
  if (sa.update_state && P->st->done) return;
  if (sa.skip_frozen && P->st->frozen) return;
  const int M = P->M, W = P->W, H = P->H, Wh = P->Wh;
  const int ss = fft_seq_stride(M);
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
  const FastDiv dm(M);
  for (int base = tid; base < nr * M; base += 4 * nthr) {   // 8 spectrum loads in flight
    float2 xa[4], xb[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int idx = base + u * nthr;
      if (idx < nr * M) {
        int row, kk;
        dm.divmod(idx, row, kk);
        const float2 *xr = spec + (long)(r0 + row) * Wh;
        xa[u] = xr[kk];
        xb[u] = xr[M - kk];
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int idx = base + u * nthr;
      if (idx < nr * M) {
        int row, kk;
        dm.divmod(idx, row, kk);
        b0[row * ss + pidx(kk)] = c2r_pre(xa[u], xb[u], tww[kk]);
      }
    }
  }
  __syncthreads();
  const float2 *Y = fft_smem(b0, b1, M, nr, ss, twm, tid, nthr);

  StepOut out;
  out.init(P, sa);
  const int warp = tid >> 5, lane = tid & 31, nwarps = nthr >> 5;
  for (int row = warp; row < nr; row += nwarps) {
    const long rowbase = (long)(r0 + row) * W;
    float sd = 0.f, sx = 0.f;
    for (int n0 = lane; n0 < M; n0 += 4 * 32) {   // x_k (and the SD term) loaded 4 at a time
      float2 pv[4], tv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int n = n0 + 32 * u;
        if (n < M) {
          pv[u] = out.prev(rowbase + 2 * n);
          tv[u] = out.sd_term(rowbase + 2 * n);
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int n = n0 + 32 * u;
        if (n < M) {
          const float2 v = Y[row * ss + pidx(n)];
          out.put(rowbase + 2 * n, v.x + tv[u].x, -v.y + tv[u].y, pv[u], sd, sx);
        }
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      sd += __shfl_xor_sync(0xffffffffu, sd, off);
      sx += __shfl_xor_sync(0xffffffffu, sx, off);
    }
    if (lane == 0) P->row_stats[r0 + row] = make_float2(sd, sx);
  }
  if (!sa.update_state) return;

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
    finish_step(P->st, sd, sx, sa.dst);
    P->st->counter = 0;
    __threadfence();
  }
}

// ---------------------------------------------------------------------------------------
// cluster path
// ---------------------------------------------------------------------------------------

// The whole solve of one FP step for one problem in one thread-block cluster, with the
// half spectrum held in the cluster's shared memory:
//   rows R2C of the CTA's row band; every bin is stored straight into the column buffer
//   Rb of the CTA owning its column (distributed shared memory)
//   cluster barrier; column FFT, X = C + G F, inverse column FFT; each CTA stores its
//   columns back into the row-band buffer A of the rows' owners (A is touched by nobody
//   before, so no barrier is needed first)
//   cluster barrier; rows C2R of the band -> x_{k+1}, statistics; every CTA stores its
//   partial statistics into rank 0's shared memory, and after a third cluster barrier rank
//   0 sums them and runs the termination test.
// Global traffic per pixel: f (4 B), C and G (~6 B), x_k for the statistics (4 B) and
// x_{k+1} (4 B); the spectrum never leaves the chip.
constexpr int kClusterThreads = 256;   // two CTAs per SM fit, so 16-CTA clusters co-reside

__device__ __forceinline__ int band_lo(int q, int n, const FastDiv &by_ncta) { return by_ncta.div(q * n); }
__device__ __forceinline__ int band_owner(int h, int ncta, const FastDiv &by_n) {
  return by_n.div((h + 1) * ncta - 1);
}

__global__ void __launch_bounds__(kClusterThreads, 2)
k_fft_solve_cluster(const ProbDev *__restrict__ probs, const int *__restrict__ list, StepArgs sa,
                    int tw_cap_m, int tw_cap_h, int a_cap, int buf_cap, int cg_cap) {
  extern __shared__ float2 sm[];
  __shared__ float red_d[kClusterThreads / 32], red_x[kClusterThreads / 32];
  __shared__ float2 cl_stats[16];   // on rank 0: every CTA's (sum d^2, sum x^2), by rank
  cg::cluster_group cl = cg::this_cluster();
  const int rank = cl.block_rank();
  const int ncta = cl.num_blocks();
  const ProbDev *P = probs + list[blockIdx.x / ncta];
  // both tests are uniform over the cluster (one problem per cluster)
  if (sa.update_state && P->st->done) return;
  if (sa.skip_frozen && P->st->frozen) return;
  const int H = P->H, W = P->W, M = P->M, Wh = P->Wh;
  const int ssm = fft_seq_stride(M), ssh = fft_seq_stride(H);
  const FastDiv by_ncta(ncta), by_h(H);
  const int r0 = band_lo(rank, H, by_ncta), nr = band_lo(rank + 1, H, by_ncta) - r0;
  const int c0 = band_lo(rank, Wh, by_ncta), nc = band_lo(rank + 1, Wh, by_ncta) - c0;
  float2 *twm = sm;
  float2 *tww = twm + tw_cap_m;
  float2 *twh = tww + tw_cap_m + 1;
  float2 *A = twh + tw_cap_h;       // row band of the solved half spectrum (phase 3 -> 4)
  float2 *X0 = A + a_cap;
  float2 *X1 = X0 + buf_cap;
  float2 *Rb = X1 + buf_cap;        // this CTA's spectrum columns, pushed by every band
  const int tid = threadIdx.x, nthr = blockDim.x;
  const FastDiv fdm(M), fdwh(Wh), fdc(nc > 0 ? nc : 1);
  StepOut out;
  out.init(P, sa);
  // 1. group 0: twiddle tables and the band's rows (f, or x_k for an SD step) straight into
  //    the padded row buffer; group 1 (when cg_cap > 0): C and G of the CTA's columns, needed
  //    only after the column transform, so their latency hides behind it
  const bool sd_step = P->baseline == kBaseSD;
  for (int i = tid; i < M; i += nthr) cp_async8(twm + i, P->tw_m + i);
  for (int i = tid; i <= M; i += nthr) cp_async8(tww + i, P->tw_w + i);
  for (int i = tid; i < H; i += nthr) cp_async8(twh + i, P->tw_h + i);
  if (!sd_step || out.src_type == kStoreF32) {
    const float *rows = sd_step ? static_cast<const float *>(out.src_ring) : P->f;
    for (int idx = tid; idx < nr * M; idx += nthr) {
      int row, n;
      fdm.divmod(idx, row, n);
      cp_async8(X0 + row * ssm + pidx(n), rows + (long)(r0 + row) * W + 2 * n);
    }
  } else {   // SD step from a 16-bit ring: converted on the way in
    for (int idx = tid; idx < nr * M; idx += nthr) {
      int row, n;
      fdm.divmod(idx, row, n);
      X0[row * ssm + pidx(n)] = out.prev((long)(r0 + row) * W + 2 * n);
    }
  }
  cp_async_commit();
  float2 *Cs = Rb + buf_cap;                              // cg_cap complex C values
  float *Gs = reinterpret_cast<float *>(Cs + cg_cap);     // cg_cap real G values
  const bool cg_staged = cg_cap >= H * nc;
  if (cg_staged) {
    for (int idx = tid; idx < H * nc; idx += nthr) {
      int r, c;
      fdc.divmod(idx, r, c);
      const long g = (long)r * Wh + c0 + c;
      cp_async8(Cs + idx, P->Cc + g);
      cp_async4(Gs + idx, P->Gg + g);
    }
  }
  cp_async_commit();
  cp_async_wait<1>();   // group 0 landed (group 1 may still be in flight)
  __syncthreads();
  const float2 *Z = fft_smem(X0, X1, M, nr, ssm, twm, tid, nthr);
  // 2. push: every half-spectrum bin of the band's rows goes straight into the column
  //    buffer of the CTA that owns its column (remote stores, no round trip), then one
  //    cluster barrier makes the columns complete
  const FastDiv by_wh(Wh);
  for (int idx = tid; idx < nr * Wh; idx += nthr) {
    int row, kk;
    fdwh.divmod(idx, row, kk);
    const float2 v = r2c_bin(Z + row * ssm, M, kk, tww);
    const int q = band_owner(kk, ncta, by_wh);
    float2 *Rq = cl.map_shared_rank(Rb, q);
    Rq[(kk - band_lo(q, Wh, by_ncta)) * ssh + pidx(r0 + row)] = v;
  }
  cl.sync();
  float2 *F = fft_smem(Rb, X0, H, nc, ssh, twh, tid, nthr);
  if (cg_staged) {
    cp_async_wait<0>();
    __syncthreads();
  }
  for (int base = tid; base < H * nc; base += 4 * nthr) {
    float2 cc[4];
    float gg[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int idx = base + u * nthr;
      if (idx < H * nc) {
        if (cg_staged) {
          cc[u] = Cs[idx];
          gg[u] = Gs[idx];
        } else {
          int r, c;
          fdc.divmod(idx, r, c);
          const long g = (long)r * Wh + c0 + c;
          cc[u] = P->Cc[g];
          gg[u] = P->Gg[g];
        }
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int idx = base + u * nthr;
      if (idx < H * nc) {
        int r, c;
        fdc.divmod(idx, r, c);
        const float2 fv = F[c * ssh + pidx(r)];
        F[c * ssh + pidx(r)] = make_float2(fmaf(gg[u], fv.x, cc[u].x), -fmaf(gg[u], fv.y, cc[u].y));
      }
    }
  }
  __syncthreads();
  const float2 *Xs = fft_smem(F, F == Rb ? X0 : Rb, H, nc, ssh, twh, tid, nthr);
  // 3. scatter the solved columns back to the row bands (A is read only by its own CTA,
  //    after the next barrier, so no barrier is needed before the remote stores)
  for (int idx = tid; idx < H * nc; idx += nthr) {
    int h, c;
    fdc.divmod(idx, h, c);
    const int q = band_owner(h, ncta, by_h);
    float2 *Aq = cl.map_shared_rank(A, q);
    Aq[(h - band_lo(q, H, by_ncta)) * Wh + c0 + c] = cconj(Xs[c * ssh + pidx(h)]);
  }
  cl.sync();
  // 4. x_k of the band for the statistics into Rb (free since the barrier: every CTA has
  //    finished reading its columns), in flight during the inverse row transform; then rows,
  //    half spectrum to real, statistics against x_k
  const int esz = store_bytes(out.src_type);
  char *prev_s = reinterpret_cast<char *>(Rb);
  {
    const char *src = static_cast<const char *>(out.src_ring) + (size_t)r0 * W * esz;
    for (int idx = tid; idx < nr * M; idx += nthr) {
      if (esz == 4)
        cp_async8(prev_s + 8 * idx, src + 8 * (size_t)idx);
      else
        cp_async4(prev_s + 4 * idx, src + 4 * (size_t)idx);
    }
    cp_async_commit();
  }
  for (int idx = tid; idx < nr * M; idx += nthr) {
    int row, kk;
    fdm.divmod(idx, row, kk);
    X0[row * ssm + pidx(kk)] = c2r_pre(A[row * Wh + kk], A[row * Wh + (M - kk)], tww[kk]);
  }
  __syncthreads();
  const float2 *Y = fft_smem(X0, X1, M, nr, ssm, twm, tid, nthr);
  cp_async_wait<0>();
  __syncthreads();
  float sd = 0.f, sx = 0.f;
  for (int idx = tid; idx < nr * M; idx += nthr) {
    int row, n;
    fdm.divmod(idx, row, n);
    const float2 v = Y[row * ssm + pidx(n)];
    const long e = (long)(r0 + row) * W + 2 * n;
    const float2 pv = make_float2(load_img(prev_s, 2 * (long)idx, out.src_type),
                                  load_img(prev_s, 2 * (long)idx + 1, out.src_type));
    const float2 t = out.sd_term(e);
    out.put(e, v.x + t.x, -v.y + t.y, pv, sd, sx);
  }
  // CTA sums (fixed order); the per-CTA partials are summed below by rank 0
  const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    sd += __shfl_xor_sync(0xffffffffu, sd, off);
    sx += __shfl_xor_sync(0xffffffffu, sx, off);
  }
  if (lane == 0) {
    red_d[warp] = sd;
    red_x[warp] = sx;
  }
  __syncthreads();
  if (!sa.update_state) return;   // uniform over the cluster (a launch argument)
  // per-CTA partials into rank 0's shared memory, one cluster barrier (release / acquire at
  // cluster scope), then rank 0 sums them in rank order: no GPU-scope fence, no atomic
  if (tid == 0) {
    float td = 0.f, tx = 0.f;
    for (int w = 0; w < (nthr >> 5); ++w) {
      td += red_d[w];
      tx += red_x[w];
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
    finish_step(P->st, tsd, tsx, sa.dst);
  }
}

// FP solve (sd == null): C = conj(K) Y / (sigma^2 D) / (H W), G = alpha / D / (H W) with
// D = |K|^2 / sigma^2 + alpha. SD step: C_sd = mu conj(K) Y / sigma^2 / (H W),
// G_sd = (1 - mu alpha - mu |K|^2 / sigma^2) / (H W).
__device__ __forceinline__ void spectral_constant_at(const float2 *__restrict__ khat,
                                                     const float2 *__restrict__ yhat, float2 *Cc,
                                                     float *Gg, int i, double inv_sigma2,
                                                     double alpha, double inv_hw,
                                                     const SdParams *sd) {
  const double kr = khat[i].x, ki = khat[i].y;
  const double yr = yhat[i].x, yi = yhat[i].y;
  const double k2 = kr * kr + ki * ki;
  // conj(K) Y = (kr yr + ki yi) + i (kr yi - ki yr)
  double s, g;
  if (sd) {
    const double mu = sd->mu;
    s = mu * inv_sigma2 * inv_hw;
    g = (1.0 - mu * alpha - mu * k2 * inv_sigma2) * inv_hw;
  } else {
    const double d = k2 * inv_sigma2 + alpha;
    s = inv_sigma2 / d * inv_hw;
    g = alpha / d * inv_hw;
  }
  Cc[i] = make_float2((float)((kr * yr + ki * yi) * s), (float)((kr * yi - ki * yr) * s));
  Gg[i] = (float)g;
}

__global__ void k_spectral_constants(const float2 *__restrict__ khat, const float2 *__restrict__ yhat,
                                     float2 *Cc, float *Gg, int n, double inv_sigma2,
                                     double alpha, double inv_hw, const SdParams *sd) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  spectral_constant_at(khat, yhat, Cc, Gg, i, inv_sigma2, alpha, inv_hw, sd);
}

// The same for several problems in one launch: item {prob, first frequency}, 256 each.
__global__ void __launch_bounds__(256)
k_spectral_constants_items(const ProbDev *__restrict__ probs, const Item *__restrict__ items) {
  const Item it = items[blockIdx.x];
  const ProbDev *P = probs + it.prob;
  const int i = it.a + threadIdx.x;
  if (i >= P->H * P->Wh) return;
  spectral_constant_at(P->Kh, P->spec, const_cast<float2 *>(P->Cc), const_cast<float *>(P->Gg), i,
                       P->inv_sigma2_d, P->alpha_d, 1.0 / ((double)P->H * P->W),
                       P->baseline == kBaseSD ? P->sd : nullptr);
}

// max |K(w)|^2 over the half spectrum (rows u < H, columns v <= W/2), K the DFT of the
// PSF taps, evaluated directly: K(u, v) = sum_{a, b} psf[a][b] e^{-2 pi i (u a / H + v b / W)}
// (|K| does not depend on where the PSF is centred). The phase is reduced exactly in
// integers (t = (u a mod H) W + (v b mod W) H over H W, below 2^23), so FP32 keeps it to
// rounding. Each thread takes frequencies by a grid stride and folds its maximum into the
// bits of sd->kmax_bits.
__global__ void __launch_bounds__(256)
k_psf_spectrum_max(const float *__restrict__ psf, int kh, int kw, int H, int W, SdParams *sd) {
  const int Wh = W / 2 + 1;
  const long nf = (long)H * Wh;
  const float inv_hw2 = 2.0f / ((float)H * (float)W);
  float best = 0.f;
  for (long f = blockIdx.x * (long)blockDim.x + threadIdx.x; f < nf; f += (long)gridDim.x * blockDim.x) {
    const int u = (int)(f / Wh), v = (int)(f - (long)u * Wh);
    float re = 0.f, im = 0.f;
    for (int a = 0; a < kh; ++a) {
      const int pu = (int)(((long)u * a) % H) * W;
      for (int b = 0; b < kw; ++b) {
        const int t = pu + (int)(((long)v * b) % W) * H;   // < 2 H W
        float sn, cs;
        sincospif((float)t * inv_hw2, &sn, &cs);
        const float w = psf[a * kw + b];
        re = fmaf(w, cs, re);
        im = fmaf(-w, sn, im);
      }
    }
    best = fmaxf(best, fmaf(re, re, im * im));
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) best = fmaxf(best, __shfl_xor_sync(0xffffffffu, best, off));
  if ((threadIdx.x & 31) == 0) atomicMax(&sd->kmax_bits, __float_as_uint(best));
}

// mu = 1 / (max |K|^2 / sigma^2 + alpha), or the configured step size.
__global__ void k_sd_finish(SdParams *sd, double inv_sigma2, double alpha, double mu_given) {
  const double kmax = (double)__uint_as_float(sd->kmax_bits);
  const double mu = mu_given > 0.0 ? mu_given : 1.0 / (kmax * inv_sigma2 + alpha);
  sd->mu = mu;
  sd->mu_f = (float)mu;
  sd->mu_alpha_f = (float)(mu * alpha);
}

}  // namespace

// ---------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------

int fft_smem_rows(int tw_cap, int buf_cap) {
  return (int)((2 * (size_t)tw_cap + 1 + 2 * (size_t)buf_cap) * sizeof(float2));
}
int fft_smem_cols(int tw_cap, int buf_cap) {
  return (int)(((size_t)tw_cap + 2 * (size_t)buf_cap) * sizeof(float2));
}

// Raises a kernel's dynamic shared-memory limit the first time a launch needs more
// than the 48 KB default (a per-kernel high-water mark; races only repeat the call).
static cudaError_t set_smem(const void *fn, int bytes, int *high_water) {
  if (bytes <= 48 * 1024 || bytes <= *high_water) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) *high_water = bytes;
  return e;
}
static int hw_r2c = 0, hw_cols = 0, hw_c2r = 0, hw_cluster = 0;

cudaError_t fft_prepare(int row_tw_cap, int row_buf_cap, int col_tw_cap, int col_buf_cap) {
  const int sr = fft_smem_rows(row_tw_cap, row_buf_cap), sc = fft_smem_cols(col_tw_cap, col_buf_cap);
  cudaError_t e = set_smem((const void *)k_fft_r2c, sr, &hw_r2c);
  if (e == cudaSuccess) e = set_smem((const void *)k_fft_c2r, sr, &hw_c2r);
  if (e == cudaSuccess) e = set_smem((const void *)k_fft_cols, sc, &hw_cols);
  return e;
}

cudaError_t launch_fft_r2c(const ProbDev *d_probs, const Item *d_items, int n_items,
                           int tw_cap, int buf_cap, const float *src_override,
                           float2 *dst_override, int skip_done, cudaStream_t s,
                           const StepArgs *step) {
  if (n_items <= 0) return cudaSuccess;
  const int smem = fft_smem_rows(tw_cap, buf_cap);
  cudaError_t e = set_smem((const void *)k_fft_r2c, smem, &hw_r2c);
  if (e != cudaSuccess) return e;
  const StepArgs sa = step ? *step : StepArgs{};
  k_fft_r2c<<<n_items, 256, smem, s>>>(d_probs, d_items, tw_cap, buf_cap, src_override,
                                       dst_override, skip_done, sa, step ? 1 : 0);
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

// Shared memory of the cluster solve for one problem (complex elements): the row band's
// half spectrum A, two work buffers (the band's padded rows or columns), the column buffer
// (also the band's x_k at the end), and cg_elems C and G values of the CTA's columns.
void fft_cluster_caps(int H, int W, int ncta, int *a_elems, int *buf_elems, int *cg_elems) {
  const int M = W / 2, Wh = M + 1;
  const int nr = (H + ncta - 1) / ncta, nc = (Wh + ncta - 1) / ncta;
  *a_elems = nr * Wh;
  *buf_elems = std::max(nr * fft_seq_stride(M), nc * fft_seq_stride(H));
  *cg_elems = nc * H;
}

// cg_cap = 0: C and G are read from global memory in the solve phase.
int fft_cluster_smem(int tw_cap_m, int tw_cap_h, int a_cap, int buf_cap, int cg_cap) {
  return (int)(((size_t)2 * tw_cap_m + 1 + tw_cap_h + a_cap + 3 * (size_t)buf_cap) * sizeof(float2) +
               (size_t)cg_cap * (sizeof(float2) + sizeof(float)));
}

cudaError_t fft_cluster_prepare(int smem, int ncta) {
  cudaError_t e = set_smem((const void *)k_fft_solve_cluster, smem, &hw_cluster);
  if (e == cudaSuccess && ncta > 8)
    e = cudaFuncSetAttribute((const void *)k_fft_solve_cluster,
                             cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  return e;
}

cudaError_t launch_fft_solve_cluster(const ProbDev *d_probs, const int *d_list, int n, int ncta,
                                     int tw_cap_m, int tw_cap_h, int a_cap, int buf_cap,
                                     int cg_cap, StepArgs sa, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(n * ncta);
  cfg.blockDim = dim3(kClusterThreads);
  cfg.dynamicSmemBytes = fft_cluster_smem(tw_cap_m, tw_cap_h, a_cap, buf_cap, cg_cap);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = ncta;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_fft_solve_cluster, d_probs, d_list, sa, tw_cap_m,
                                     tw_cap_h, a_cap, buf_cap, cg_cap);
  count_launches(1);
  return e;
}

// Number of clusters of `ncta` CTAs of the cluster solve the device can hold at once.
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
                                      double alpha, double inv_hw, cudaStream_t s,
                                      const SdParams *sd) {
  k_spectral_constants<<<(n + 255) / 256, 256, 0, s>>>(k_hat, y_hat, Cc, Gg, n, inv_sigma2,
                                                       alpha, inv_hw, sd);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_spectral_constants_items(const ProbDev *d_probs, const Item *d_items,
                                            int n_items, cudaStream_t s) {
  if (n_items <= 0) return cudaSuccess;
  k_spectral_constants_items<<<n_items, 256, 0, s>>>(d_probs, d_items);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_sd_step_size(const ProbDev *, const float *psf, int kh, int kw, int H, int W,
                                double inv_sigma2, double alpha, double mu_given, SdParams *sd,
                                cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(sd, 0, sizeof(SdParams), s);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const long nf = (long)H * (W / 2 + 1);
  const int ctas = (int)std::min<long>((nf + 255) / 256, 4L * sms);
  k_psf_spectrum_max<<<ctas, 256, 0, s>>>(psf, kh, kw, H, W, sd);
  k_sd_finish<<<1, 1, 0, s>>>(sd, inv_sigma2, alpha, mu_given);
  count_launches(2);
  return cudaGetLastError();
}

}  // namespace red
