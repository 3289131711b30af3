// Vector extrapolation on the device (Sec. III-B): MPE (Algorithm 1) and RRE (Eq. (19)).
//
// From the stored iterates x_m .. x_{m+kappa+1} (K = kappa + 1 differences):
//   1. k_gram:     G = U^T U, U = [x_{m+1} - x_m, ..., x_{m+K} - x_{m+K-1}], formed on the fly.
//                  HBM-bound tall-skinny reduction: each work unit (problem, chunk of
//                  2048 pixels) reads the K + 1 vectors once with 16-byte loads. The
//                  differences are split exactly (TwoSum: u = s + e), the products are
//                  exact (TwoProduct with FMA) and accumulated in double-float (hi + lo)
//                  per thread, then reduced across the warp and the CTA in double-float
//                  (TwoSum on FP32 units) and published as one (hi, lo) pair per entry.
//                  The result has FP64-level accuracy without FP64 arithmetic in the pixel
//                  loop or the reductions (FP64 throughput on this part is a small fraction
//                  of FP32).
//   2. gamma solve: per problem, one warp of the last Gram CTA of that problem to finish
//                  (no launch of its own): sums the chunk partials in a fixed order (in
//                  double-float), then, for MPE and RRE in double-float arithmetic on FP32
//                  units, G = U^T D U (the Cholesky factor of G, R = D^{1/2} U, without its
//                  square roots; R is the R of Algorithm 2's QR up to signs) and MPE:
//                  R_{kappa-1} c' = -r_{kappa+1}, c_kappa = 1 (Algorithm 1 step 2, solved as
//                  G_{kappa-1} c' = -g) or RRE: G d = 1, gamma = c / sum c (d / sum d); or
//                  SVD-MPE in FP64: Cholesky R, gamma = v / sum v with v the right singular
//                  vector of R for its smallest singular value (one-sided Jacobi on R,
//                  lane-parallel); with the rank-loss and existence rules of the oracle.
//   3. k_combine:  Algorithm 1 steps 3-4 evaluated without Q as
//                  x_(m,kappa) = x_m + U_{kappa-1} xi (= x_m + Q_{kappa-1} R_{kappa-1} xi),
//                  xi_j = 1 - sum_{i<=j} gamma_i; reads K vectors, writes one.
// Chunks are fixed per problem, so the reduction order (and the result) does not depend
// on the launch shape or on other problems in the batch.
//
// Cycling with frozen gamma (a remark of Sec. III-C): with ProbDev::ve_freeze = n > 0, the
// n-th successful gamma solve sets the problem's `frozen` flag; from then on the Gram (and
// with it the solve) skips the problem (VeArgs::skip_frozen), its xi stays in ve_coef, and every
// cycle's combine applies it to x_m .. x_{m+kappa} (the combine never reads x_{m+kappa+1}
// unless the extrapolation broke down, which a frozen gamma cannot).
//
// Extrapolation ended by its own criterion (the additional-iterations remark of Sec.
// III-C): with ProbState::ve_stop_tol > 0, the first FP step whose relative change is
// below it sets `ve_off` (in the Fourier solve's or the SR kernel's statistics epilogue);
// from then on the Gram skips the problem and the combine passes the last FP iterate on
// unchanged, as after a breakdown, so every later step is a plain baseline step.
#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "runtime.h"

namespace red {

namespace {

// Threads per Gram and per combine work unit (one chunk of kGramChunk pixels). The Gram:
// 8 pixels per thread, one round of 16-byte loads per vector in flight. The combine: 4
// rounds of one float4 per vector per thread (measured faster than one round with 512
// threads: 7.8 vs 9.7 us on ten 256^2 problems, k = 5).
constexpr int kGramThreads = 256;
constexpr int kCombineThreads = 128;

__device__ __forceinline__ void two_diff(float a, float b, float &s, float &e) {
  s = __fsub_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(-b, bb));
}

__device__ __forceinline__ const float *vec_ptr(const ProbDev *P, const VeArgs &va, int i) {
  if (va.ptrs[i]) return va.ptrs[i];
  return static_cast<const float *>(P->ring) + (size_t)va.slots[i] * P->slot_stride;
}

// A 16-bit ring slot (BF16 or FP16 storage).
__device__ __forceinline__ const void *vec_ptr_16(const ProbDev *P, const VeArgs &va, int i) {
  return static_cast<const char *>(P->ring) + (size_t)va.slots[i] * P->slot_stride * 2;
}

// s + e = a + b exactly (TwoSum, round to nearest): the double-float adds below.
__device__ __forceinline__ void df_add(float &h, float &l, float h2, float l2) {
  const float s = __fadd_rn(h, h2);
  const float z = __fsub_rn(s, h);
  const float e = __fadd_rn(__fsub_rn(h, __fsub_rn(s, z)), __fsub_rn(h2, z));
  h = s;
  l = __fadd_rn(__fadd_rn(l, l2), e);
}

// Double-word ("double-float") arithmetic on FP32 units for the MPE / RRE solve: a value is
// h + l with |l| <= ulp(h) / 2, unit roundoff u = 2^-24. The algorithms are those of Joldes,
// Muller and Popescu, "Tight and rigorous error bounds for basic building blocks of
// double-word arithmetic" (ACM TOMS 44(2), 2017), with their relative error bounds:
// AccurateDWPlusDW (3u^2 + 13u^3), DWTimesDW3 (4u^2), DWTimesFP3 (2u^2), DWDivDW2
// (15u^2 + 56u^3); TwoSum is Knuth's, Fast2Sum Dekker's (|a| >= |b| or a = 0). Every
// operation is an explicitly rounded intrinsic, so no contraction changes them.
struct Dw {
  float h, l;
};
__device__ __forceinline__ Dw dw_of(float h, float l = 0.f) { return Dw{h, l}; }
__device__ __forceinline__ Dw two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float z = __fsub_rn(s, a);
  return Dw{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z))};
}
__device__ __forceinline__ Dw fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return Dw{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ Dw dw_add(Dw x, Dw y) {
  const Dw s = two_sum(x.h, y.h);
  const Dw t = two_sum(x.l, y.l);
  const Dw v = fast_two_sum(s.h, __fadd_rn(s.l, t.h));
  return fast_two_sum(v.h, __fadd_rn(t.l, v.l));
}
__device__ __forceinline__ Dw dw_neg(Dw x) { return Dw{-x.h, -x.l}; }
__device__ __forceinline__ Dw dw_sub(Dw x, Dw y) { return dw_add(x, dw_neg(y)); }
__device__ __forceinline__ Dw dw_abs(Dw x) { return x.h < 0.f ? dw_neg(x) : x; }
__device__ __forceinline__ Dw dw_mul(Dw x, Dw y) {
  const float ch = __fmul_rn(x.h, y.h);
  const float cl1 = __fmaf_rn(x.h, y.h, -ch);
  const float tl1 = __fmaf_rn(x.h, y.l, __fmul_rn(x.l, y.l));
  const float cl2 = __fmaf_rn(x.l, y.h, tl1);
  return fast_two_sum(ch, __fadd_rn(cl1, cl2));
}
__device__ __forceinline__ Dw dw_mul_f(Dw x, float y) {
  const float ch = __fmul_rn(x.h, y);
  const float cl1 = __fmaf_rn(x.h, y, -ch);
  return fast_two_sum(ch, __fmaf_rn(x.l, y, cl1));
}
__device__ __forceinline__ Dw dw_div(Dw x, Dw y) {
  const float th = __fdiv_rn(x.h, y.h);
  const Dw r = dw_mul_f(y, th);
  const float d = __fadd_rn(__fsub_rn(x.h, r.h), __fsub_rn(x.l, r.l));
  return fast_two_sum(th, __fdiv_rn(d, y.h));
}
// x - a * b
__device__ __forceinline__ Dw dw_fnma(Dw a, Dw b, Dw x) { return dw_sub(x, dw_mul(a, b)); }

template <int K>
struct GramAcc {
  float hi[K * (K + 1) / 2];
  float lo[K * (K + 1) / 2];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int i = 0; i < K * (K + 1) / 2; ++i) hi[i] = lo[i] = 0.f;
  }
  // one pixel: x[0..K]
  __device__ __forceinline__ void add(const float (&x)[K + 1]) {
    float s[K], e[K];
#pragma unroll
    for (int i = 0; i < K; ++i) two_diff(x[i + 1], x[i], s[i], e[i]);
    int idx = 0;
#pragma unroll
    for (int i = 0; i < K; ++i) {
#pragma unroll
      for (int j = i; j < K; ++j) {
        const float p = __fmul_rn(s[i], s[j]);
        const float pe = __fmaf_rn(s[i], s[j], -p);
        const float cross = __fmaf_rn(s[i], e[j], __fmul_rn(e[i], s[j]));
        // TwoSum(hi, p)
        const float h = hi[idx];
        const float t = __fadd_rn(h, p);
        const float z = __fsub_rn(t, h);
        const float err = __fadd_rn(__fsub_rn(h, __fsub_rn(t, z)), __fsub_rn(p, z));
        hi[idx] = t;
        lo[idx] = __fadd_rn(lo[idx], __fadd_rn(err, __fadd_rn(pe, cross)));
        ++idx;
      }
    }
  }
};

template <int K>
__device__ void ve_solve_k(const ProbDev *P, int update_state);

// The last CTA of a problem to finish its Gram partial sums runs the gamma solve (one warp),
// so the solve needs no launch of its own: every CTA publishes its partials, fences, and
// counts itself in st->counter2; the one that completes the count reads all partials.
__device__ __forceinline__ bool last_gram_cta(const ProbDev *P) {
  __shared__ int is_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    is_last = atomicAdd(&P->st->counter2, 1u) == (unsigned)(P->n_chunks - 1);
  }
  __syncthreads();
  return is_last != 0;
}

template <int K>
__global__ void __launch_bounds__(kGramThreads)
k_gram(const ProbDev *__restrict__ probs, const Item *__restrict__ items, VeArgs va) {
  constexpr int NP = K * (K + 1) / 2;
  __shared__ float2 red[kGramThreads / 32][NP];
  const Item it = items[blockIdx.x];
  const ProbDev *P = probs + it.prob;
  if (va.update_state && P->st->done) return;
  if (va.skip_frozen && P->st->frozen) return;
  if (va.update_state && P->st->ve_off) return;   // extrapolation has ended for this problem
  const int N = P->N;
  const int begin = it.a * kGramChunk;
  const int end = min(N, begin + kGramChunk);
  GramAcc<K> acc;
  acc.zero();
  const int tid = threadIdx.x;
  const int stype = (va.ptrs[0] == nullptr) ? P->storage : kStoreF32;
  if (stype == kStoreF32) {
    const float *xp[K + 1];
#pragma unroll
    for (int i = 0; i <= K; ++i) xp[i] = vec_ptr(P, va, i);
    bool aligned = ((begin & 3) == 0);
#pragma unroll
    for (int i = 0; i <= K; ++i) aligned = aligned && ((reinterpret_cast<uintptr_t>(xp[i]) & 15) == 0);
    int p0 = begin;
    if (aligned) {
      const int nv = (end - begin) >> 2;
      const int step = blockDim.x;
      constexpr bool kDual = K <= 6;   // two loads per vector in flight where registers allow
      for (int v = tid; v < nv; v += (kDual ? 2 : 1) * step) {
        float4 q0[K + 1], q1[K + 1];
        const bool has1 = kDual && v + step < nv;
#pragma unroll
        for (int i = 0; i <= K; ++i) {
          const float4 *src = reinterpret_cast<const float4 *>(xp[i] + begin);
          q0[i] = __ldcs(src + v);
          if (has1) q1[i] = __ldcs(src + v + step);
        }
        float x[K + 1];
#pragma unroll
        for (int i = 0; i <= K; ++i) x[i] = q0[i].x;
        acc.add(x);
#pragma unroll
        for (int i = 0; i <= K; ++i) x[i] = q0[i].y;
        acc.add(x);
#pragma unroll
        for (int i = 0; i <= K; ++i) x[i] = q0[i].z;
        acc.add(x);
#pragma unroll
        for (int i = 0; i <= K; ++i) x[i] = q0[i].w;
        acc.add(x);
        if (has1) {
#pragma unroll
          for (int i = 0; i <= K; ++i) x[i] = q1[i].x;
          acc.add(x);
#pragma unroll
          for (int i = 0; i <= K; ++i) x[i] = q1[i].y;
          acc.add(x);
#pragma unroll
          for (int i = 0; i <= K; ++i) x[i] = q1[i].z;
          acc.add(x);
#pragma unroll
          for (int i = 0; i <= K; ++i) x[i] = q1[i].w;
          acc.add(x);
        }
      }
      p0 = begin + (nv << 2);
    }
    for (int p = p0 + tid; p < end; p += blockDim.x) {
      float x[K + 1];
#pragma unroll
      for (int i = 0; i <= K; ++i) x[i] = xp[i][p];
      acc.add(x);
    }
  } else {
    const void *xp[K + 1];
#pragma unroll
    for (int i = 0; i <= K; ++i) xp[i] = vec_ptr_16(P, va, i);
    for (int p = begin + tid; p < end; p += blockDim.x) {
      float x[K + 1];
#pragma unroll
      for (int i = 0; i <= K; ++i) x[i] = load_img(xp[i], p, stype);
      acc.add(x);
    }
  }
  // warp and CTA reductions in double-float (FP32 units, TwoSum), fixed order
  const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    float h = acc.hi[q], l = acc.lo[q];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
      df_add(h, l, __shfl_xor_sync(0xffffffffu, h, off), __shfl_xor_sync(0xffffffffu, l, off));
    if (lane == 0) red[warp][q] = make_float2(h, l);
  }
  __syncthreads();
  if (tid < NP) {   // partials stay double-float (hi, lo): the solve sums them in FP32 units
    float h = 0.f, l = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) df_add(h, l, red[w][tid].x, red[w][tid].y);
    P->gram_part[(size_t)it.a * kMaxPairs + tid] = make_float2(h, l);
  }
  if (!last_gram_cta(P)) return;
  __threadfence();
  if (warp == 0) ve_solve_k<K>(P, va.update_state);
  if (tid == 0) P->st->counter2 = 0;
}

// Generic FP64 path for K > 10 (rarely used; correct but not tuned).
__global__ void __launch_bounds__(256)
k_gram_generic(const ProbDev *__restrict__ probs, const Item *__restrict__ items, VeArgs va) {
  __shared__ double red[kMaxPairs];
  const Item it = items[blockIdx.x];
  const ProbDev *P = probs + it.prob;
  if (va.update_state && P->st->done) return;
  if (va.skip_frozen && P->st->frozen) return;
  if (va.update_state && P->st->ve_off) return;   // extrapolation has ended for this problem
  const int K = va.nvec - 1;
  const int NP = K * (K + 1) / 2;
  const int begin = it.a * kGramChunk;
  const int end = min(P->N, begin + kGramChunk);
  for (int q = threadIdx.x; q < NP; q += blockDim.x) red[q] = 0.0;
  __syncthreads();
  // thread t accumulates pair q = t mod NP over a strided subset of pixels, then atomics
  // are avoided by a fixed two-level order: each thread owns one pair.
  for (int q = threadIdx.x; q < NP; q += blockDim.x) {
    int i = 0, rem = q;
    while (rem >= K - i) { rem -= K - i; ++i; }
    const int j = i + rem;
    double s = 0.0;
    for (int p = begin; p < end; ++p) {
      const float *xi0 = vec_ptr(P, va, i), *xi1 = vec_ptr(P, va, i + 1);
      const float *xj0 = vec_ptr(P, va, j), *xj1 = vec_ptr(P, va, j + 1);
      const double ui = (double)xi1[p] - (double)xi0[p];
      const double uj = (double)xj1[p] - (double)xj0[p];
      s += ui * uj;
    }
    red[q] = s;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < NP; q += blockDim.x) {
    const float hi = __double2float_rn(red[q]);
    P->gram_part[(size_t)it.a * kMaxPairs + q] = make_float2(hi, __double2float_rn(red[q] - (double)hi));
  }
  if (!last_gram_cta(P)) return;
  __threadfence();
  if (threadIdx.x < 32) {
    if (K == 11) ve_solve_k<11>(P, va.update_state);
    else ve_solve_k<12>(P, va.update_state);
  }
  if (threadIdx.x == 0) P->st->counter2 = 0;
}

// SVD-MPE weights: the right singular vector of the K x K factor R for its smallest
// singular value, by one-sided (Hestenes) Jacobi: plane rotations of column pairs of R
// until every pair is orthogonal to 1e-15, accumulated in V. Lane i < K holds row i of R
// and of V; the three column inner products of a rotation are warp sums (fixed xor tree),
// so every lane takes the same rotation. Returns false when sum v vanishes.
template <int K>
__device__ bool svd_mpe_gamma(const double (&R)[K][K], double (&gamma)[K]) {
  const int lane = threadIdx.x & 31;
  double a[K], v[K];
#pragma unroll
  for (int j = 0; j < K; ++j) {
    a[j] = 0.0;
#pragma unroll
    for (int i = 0; i < K; ++i)
      if (lane == i) a[j] = R[i][j];
    v[j] = (lane == j) ? 1.0 : 0.0;
  }
  auto wsum = [](double x) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
    return x;
  };
  // (the pair loops are rolled: SVD-MPE is not on the timed path, and unrolling them for
  // every K would dominate the library's build time)
  for (int sweep = 0; sweep < 40; ++sweep) {
    bool rotated = false;
#pragma unroll 1
    for (int p = 0; p < K - 1; ++p) {
#pragma unroll 1
      for (int q = p + 1; q < K; ++q) {
        const double al = wsum(a[p] * a[p]), be = wsum(a[q] * a[q]), ga = wsum(a[p] * a[q]);
        if (ga == 0.0 || fabs(ga) <= 1e-15 * sqrt(al * be)) continue;
        rotated = true;
        const double zeta = (be - al) / (2.0 * ga);
        const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
        const double ap = a[p], aq = a[q], vp = v[p], vq = v[q];
        a[p] = c * ap - s * aq;
        a[q] = s * ap + c * aq;
        v[p] = c * vp - s * vq;
        v[q] = s * vp + c * vq;
      }
    }
    if (!rotated) break;
  }
  // smallest column norm of the rotated R = smallest singular value
  int jmin = 0;
  double nmin = wsum(a[0] * a[0]);
#pragma unroll
  for (int j = 1; j < K; ++j) {
    const double nj = wsum(a[j] * a[j]);
    if (nj < nmin) {
      nmin = nj;
      jmin = j;
    }
  }
  double vj = 0.0;
#pragma unroll
  for (int j = 0; j < K; ++j)
    if (j == jmin) vj = v[j];
  double sv = 0.0, sa = 0.0;
#pragma unroll
  for (int i = 0; i < K; ++i) {
    gamma[i] = __shfl_sync(0xffffffffu, vj, i);
    sv += gamma[i];
    sa += fabs(gamma[i]);
  }
  if (fabs(sv) <= kSumTol * sa) return false;
#pragma unroll
  for (int i = 0; i < K; ++i) gamma[i] /= sv;
  return true;
}

__device__ __forceinline__ Dw shfl_xor_dw(Dw x, int off) {
  return Dw{__shfl_xor_sync(0xffffffffu, x.h, off), __shfl_xor_sync(0xffffffffu, x.l, off)};
}
__device__ __forceinline__ Dw shfl_up_dw(Dw x, int off) {
  return Dw{__shfl_up_sync(0xffffffffu, x.h, off), __shfl_up_sync(0xffffffffu, x.l, off)};
}
// Sum over the warp by a fixed xor tree; every lane ends with the same value (each step
// adds the same two operands on both lanes of a pair, and the double-word sum is
// commutative: its TwoSum error terms are exact).
__device__ __forceinline__ Dw warp_sum_dw(Dw x) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) x = dw_add(x, shfl_xor_dw(x, off));
  return x;
}

// The tiny solve for gamma, one warp per problem, written as short loops over shared
// memory: it runs once per cycle on whichever SM finishes the Gram last, with a cold
// instruction cache, so its cost is set by the instructions it fetches at least as much as
// by its arithmetic.
//   1. G: the chunk partials pass through shared memory 32 chunks at a time (lane r loads
//      chunk r's partials), and lane q sums entry q over the chunks in increasing order
//      (double-float TwoSum).
//   2. MPE and RRE, in double-word arithmetic on FP32 units: G = U^T D U by right-looking
//      LDL^T (column j: pivot d_j, U_jb = A_jb / d_j on lanes b, trailing update
//      A_ab -= A_ja U_jb on lanes over the pairs a <= b); the pivots d_j are the r_jj^2 of
//      Algorithm 2's R = D^{1/2} U, so the rank test is the oracle's. Then U^T z = rhs and
//      U c = z / D by columns over the lanes (MPE: rhs = -g, the first kappa entries of G's
//      last column, and c_kappa = 1; RRE: rhs = 1), sum c and sum |c| by xor trees, gamma_j =
//      c_j / sum c on lane j, xi_j = 1 - sum_{i<=j} gamma_i by a lane scan.
//   3. SVD-MPE: every lane reads G, factors G = R^T R in FP64 and runs the lane-parallel
//      rotations of svd_mpe_gamma; lane 0 writes the results.
template <int K>
__device__ void ve_solve_k(const ProbDev *P, int update_state) {
  constexpr int NP = K * (K + 1) / 2;
  constexpr int kap = K - 1;
  constexpr int QL = (NP + 31) / 32;   // Gram entries per lane
  __shared__ float2 tile[32][NP];      // 32 chunks' partials
  __shared__ Dw A[K][K];               // G's upper triangle, then the trailing updates
  __shared__ Dw Us[K][K];              // strict upper part of U
  __shared__ Dw dg[K], z[K];
  const int lane = threadIdx.x & 31;
  ProbState *st = P->st;

  // 1. G
  Dw acc[QL];
#pragma unroll
  for (int i = 0; i < QL; ++i) acc[i] = dw_of(0.f);
  const int nc = P->n_chunks;
#pragma unroll 1
  for (int c0 = 0; c0 < nc; c0 += 32) {
    const int c = c0 + lane;
    const float2 *src = P->gram_part + (size_t)min(c, nc - 1) * kMaxPairs;
#pragma unroll
    for (int q = 0; q < NP; ++q) tile[lane][q] = c < nc ? __ldcg(src + q) : make_float2(0.f, 0.f);
    __syncwarp();
    const int rows = min(32, nc - c0);
#pragma unroll
    for (int i = 0; i < QL; ++i) {
      const int q = lane + 32 * i;
      if (q < NP) {
#pragma unroll 4
        for (int r = 0; r < rows; ++r) {
          const float2 v = tile[r][q];
          df_add(acc[i].h, acc[i].l, v.x, v.y);
        }
      }
    }
    __syncwarp();
  }
#pragma unroll
  for (int i = 0; i < QL; ++i) {
    const int q = lane + 32 * i;
    if (q < NP) {
      int r = 0, rem = q;   // q -> (r, r + rem) in the row-major upper triangle
      while (rem >= K - r) {
        rem -= K - r;
        ++r;
      }
      A[r][r + rem] = acc[i];
    }
  }
  __syncwarp();

  if (P->ve_method == kVeSvdMpe) {
    double G[K][K];
#pragma unroll
    for (int i = 0; i < K; ++i)
#pragma unroll
      for (int j = i; j < K; ++j) G[i][j] = (double)A[i][j].h + (double)A[i][j].l;
    double R[K][K], inv[K], gamma[K];
    bool bad = false, last_bad = false;   // rank loss in one of the first kappa columns / the last
#pragma unroll
    for (int a = 0; a < K; ++a)
#pragma unroll
      for (int b = 0; b < K; ++b) R[a][b] = 0.0;
#pragma unroll
    for (int jj = 0; jj < K; ++jj) {
      if (bad || last_bad) continue;
      double sj = G[jj][jj];
#pragma unroll
      for (int a = 0; a < jj; ++a) sj -= R[a][jj] * R[a][jj];
      if (G[jj][jj] == 0.0 || sj <= kRankTol * G[jj][jj]) {
        if (jj < K - 1) bad = true;
        else last_bad = true;
        continue;
      }
      R[jj][jj] = sqrt(sj);
      inv[jj] = 1.0 / R[jj][jj];
#pragma unroll
      for (int b = jj + 1; b < K; ++b) {
        double t = G[jj][b];
#pragma unroll
        for (int a = 0; a < jj; ++a) t -= R[a][jj] * R[a][b];
        R[jj][b] = t * inv[jj];
      }
    }
    const bool ok = !bad && svd_mpe_gamma<K>(R, gamma);
    if (lane != 0) return;
    if (update_state) {
      st->ve_steps += 1;
      st->solved = 1;   // this cycle's combine uses a fresh gamma
    }
    if (!ok) {
      st->ve_status = 1;
      if (update_state) st->ve_breakdowns += 1;
      return;
    }
    st->ve_status = 0;
    if (update_state) {
      st->ve_ok += 1;
      if (P->ve_freeze > 0 && st->ve_ok >= P->ve_freeze) st->frozen = 1;
    }
    double run = 0.0, sabs = 0.0;
#pragma unroll
    for (int j = 0; j < K; ++j) {
      P->gamma[j] = gamma[j];
      sabs += fabs(gamma[j]);
      if (j < kap) {
        run += gamma[j];
        P->ve_coef[j] = 1.0 - run;   // xi_j
      }
    }
    st->sum_abs_gamma = sabs;
    return;
  }

  // 2. MPE / RRE
  const float rank_tol = (float)kRankTol, sum_tol = (float)kSumTol;
  // lane j keeps G_jj (the rank test's reference) and -G_{j,kappa} (MPE's right-hand side)
  const float gdiag = lane < K ? A[lane][lane].h : 0.f;
  const Dw rhs_mpe = lane < kap ? dw_neg(A[lane][kap]) : dw_of(0.f);
  int fail = -1;   // first column with rank loss
#pragma unroll 1
  for (int j = 0; j < K; ++j) {
    const Dw dj = A[j][j];
    const float gjj = __shfl_sync(0xffffffffu, gdiag, j);
    if (gjj == 0.f || dj.h <= rank_tol * gjj) {
      fail = j;
      break;
    }
    if (lane == 0) dg[j] = dj;
    if (j + 1 + lane < K) Us[j][j + 1 + lane] = dw_div(A[j][j + 1 + lane], dj);
    __syncwarp();
    const int m = K - 1 - j;   // trailing order
#pragma unroll 1
    for (int p = lane; p < m * (m + 1) / 2; p += 32) {
      int r = 0, rem = p;
      while (rem >= m - r) {
        rem -= m - r;
        ++r;
      }
      const int a = j + 1 + r, b = a + rem;
      A[a][b] = dw_fnma(A[j][a], Us[j][b], A[a][b]);
    }
    __syncwarp();
  }
  const bool last_bad = fail == K - 1;
  bool ok = fail < 0 || last_bad;
  const bool use_mpe = (P->ve_method == kVeMpe) || (P->ve_method == kVeRre && last_bad);
  Dw c = dw_of(0.f);
  if (ok) {
    const int n = use_mpe ? kap : K;
    if (lane < n) z[lane] = use_mpe ? rhs_mpe : dw_of(1.f);
    __syncwarp();
#pragma unroll 1
    for (int a = 0; a < n; ++a) {   // U^T z = rhs (unit lower), by columns
      const Dw za = z[a];
      if (lane > a && lane < n) z[lane] = dw_fnma(Us[a][lane], za, z[lane]);
      __syncwarp();
    }
    if (lane < n) z[lane] = dw_div(z[lane], dg[lane]);
    __syncwarp();
#pragma unroll 1
    for (int a = n - 1; a > 0; --a) {   // U c = z / D (unit upper), by columns
      const Dw ca = z[a];
      if (lane < a) z[lane] = dw_fnma(Us[lane][a], ca, z[lane]);
      __syncwarp();
    }
    c = lane < n ? z[lane] : ((use_mpe && lane == kap) ? dw_of(1.f) : dw_of(0.f));
    const Dw ssum = warp_sum_dw(c);
    const Dw sa = warp_sum_dw(dw_abs(c));
    // MPE's existence rule (sum c = 0); RRE's sum d = 1^T G^-1 1 > 0 always
    if (use_mpe && fabsf(ssum.h) <= sum_tol * sa.h) ok = false;
    c = dw_div(c, ssum);   // gamma_j on lane j (zero on lanes >= K)
  }
  if (lane == 0) {
    if (update_state) {
      st->ve_steps += 1;
      st->solved = 1;   // this cycle's combine uses a fresh gamma
    }
    st->ve_status = ok ? 0 : 1;
    if (update_state) {
      if (!ok) st->ve_breakdowns += 1;
      else {
        st->ve_ok += 1;
        if (P->ve_freeze > 0 && st->ve_ok >= P->ve_freeze) st->frozen = 1;
      }
    }
  }
  if (!ok) return;
  // xi_j = 1 - sum_{i<=j} gamma_i (inclusive scan over the lanes), sum |gamma|
  Dw pre = c;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const Dw t = shfl_up_dw(pre, off);
    if (lane >= off) pre = dw_add(t, pre);
  }
  const Dw sabs = warp_sum_dw(dw_abs(c));
  const Dw xi = dw_sub(dw_of(1.f), pre);
  if (lane < K) P->gamma[lane] = (double)c.h + (double)c.l;
  if (lane < kap) P->ve_coef[lane] = (double)xi.h + (double)xi.l;
  if (lane == 0) st->sum_abs_gamma = (double)sabs.h + (double)sabs.l;
}

// Algorithm 1 steps 3-4 without Q: x_(m,kappa) = x_m + sum_{j<kappa} xi_j (x_{m+j+1} - x_{m+j}).
// On breakdown the output is the last iterate x_{m+kappa+1}.
template <int K>
__global__ void __launch_bounds__(kCombineThreads)
k_combine(const ProbDev *__restrict__ probs, const Item *__restrict__ items, VeArgs va) {
  constexpr int kap = K - 1;
  const Item it = items[blockIdx.x];
  const ProbDev *P = probs + it.prob;
  if (va.update_state && P->st->done) return;
  const int begin = it.a * kGramChunk;
  const int end = min(P->N, begin + kGramChunk);
  // the last iterate passes on unchanged after a breakdown, and once extrapolation has
  // ended (ve_stop_tol): the next cycle's steps are then plain baseline steps
  const bool ve_off = va.update_state && P->st->ve_off;
  const int brk = P->st->ve_status || ve_off;
  if (va.update_state && it.a == 0 && threadIdx.x == 0) {
    // one thread per problem: a combine without a fresh solve reuses the frozen xi
    ProbState *st = P->st;
    if (!st->solved && !ve_off) {
      st->ve_steps += 1;
      st->frozen_steps += 1;
    }
    st->solved = 0;
  }
  float xi[kap > 0 ? kap : 1];
#pragma unroll
  for (int j = 0; j < kap; ++j) xi[j] = (float)P->ve_coef[j];
  const bool explicit_io = va.ptrs[0] != nullptr;
  const int stype = explicit_io ? kStoreF32 : P->storage;
  const int esz = store_bytes(stype);
  void *out = va.out_ptr ? (void *)va.out_ptr
                         : static_cast<char *>(P->ring) + (size_t)va.out_slot * P->slot_stride * esz;
  const void *xs[K + 1];
#pragma unroll
  for (int i = 0; i <= K; ++i)
    xs[i] = va.ptrs[i] ? (const void *)va.ptrs[i]
                       : static_cast<const char *>(P->ring) + (size_t)va.slots[i] * P->slot_stride * esz;
  bool vec = stype == kStoreF32 && ((begin & 3) == 0) && ((reinterpret_cast<uintptr_t>(out) & 15) == 0);
#pragma unroll
  for (int i = 0; i <= K; ++i) vec = vec && ((reinterpret_cast<uintptr_t>(xs[i]) & 15) == 0);
  int p0 = begin;
  if (vec) {
    const int nv = (end - begin) >> 2;
    for (int v = threadIdx.x; v < nv; v += blockDim.x) {
      float4 r;
      if (brk) {
        r = reinterpret_cast<const float4 *>(static_cast<const float *>(xs[K]) + begin)[v];
      } else {
        float4 x[K];
#pragma unroll
        for (int i = 0; i < K; ++i)
          x[i] = __ldcs(reinterpret_cast<const float4 *>(static_cast<const float *>(xs[i]) + begin) + v);
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int j = 0; j < kap; ++j) {
          acc.x = fmaf(xi[j], x[j + 1].x - x[j].x, acc.x);
          acc.y = fmaf(xi[j], x[j + 1].y - x[j].y, acc.y);
          acc.z = fmaf(xi[j], x[j + 1].z - x[j].z, acc.z);
          acc.w = fmaf(xi[j], x[j + 1].w - x[j].w, acc.w);
        }
        r = make_float4(x[0].x + acc.x, x[0].y + acc.y, x[0].z + acc.z, x[0].w + acc.w);
      }
      reinterpret_cast<float4 *>(static_cast<float *>(out) + begin)[v] = r;
    }
    p0 = begin + (nv << 2);
  }
  for (int p = p0 + threadIdx.x; p < end; p += blockDim.x) {
    float val;
    if (brk) {
      val = load_img(xs[K], p, stype);
    } else {
      float prev = load_img(xs[0], p, stype);
      const float x0 = prev;
      float acc = 0.f;
#pragma unroll
      for (int j = 0; j < kap; ++j) {
        const float nx = load_img(xs[j + 1], p, stype);
        acc = fmaf(xi[j], nx - prev, acc);
        prev = nx;
      }
      val = x0 + acc;
    }
    store_img(out, p, val, stype);
  }
}

// mode 0: ring slot `slot` <- ptrs[prob] (f32);  mode 1: ptrs[prob] <- final slot (f32)
__global__ void __launch_bounds__(256)
k_copy_slots(const ProbDev *__restrict__ probs, const Item *__restrict__ items, int mode, int slot,
             float *const *ptrs) {
  const Item it = items[blockIdx.x];
  const ProbDev *P = probs + it.prob;
  const int begin = it.a * kGramChunk;
  const int end = min(P->N, begin + kGramChunk);
  const int esz = store_bytes(P->storage);
  float *user = ptrs[it.prob];
  if (mode == 0) {
    void *dst = static_cast<char *>(P->ring) + (size_t)slot * P->slot_stride * esz;
    for (int p = begin + threadIdx.x; p < end; p += blockDim.x) store_img(dst, p, user[p], P->storage);
  } else {
    const void *src = static_cast<const char *>(P->ring) + (size_t)P->st->final_slot * P->slot_stride * esz;
    for (int p = begin + threadIdx.x; p < end; p += blockDim.x) user[p] = load_img(src, p, P->storage);
  }
}

// One problem's ring slot <-> a float32 image (storage conversion included).
__global__ void k_slot_io(const ProbDev *__restrict__ P, int slot, float *img, int to_slot) {
  const int esz = store_bytes(P->storage);
  char *ring = static_cast<char *>(P->ring) + (size_t)slot * P->slot_stride * esz;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < P->N; e += (long)gridDim.x * blockDim.x) {
    if (to_slot)
      store_img(ring, e, img[e], P->storage);
    else
      img[e] = load_img(ring, e, P->storage);
  }
}

}  // namespace

// SMs of the current device (grid size of the grid-stride slot copies).
static int current_device_sms() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) {
    cudaGetLastError();
    return 1;
  }
  return n;
}

cudaError_t launch_convert_to_slot(const ProbDev *d_prob, const float *src, int slot, cudaStream_t s) {
  k_slot_io<<<current_device_sms(), 256, 0, s>>>(d_prob, slot, const_cast<float *>(src), 1);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_fetch_slot(const ProbDev *d_prob, int slot, float *dst, cudaStream_t s) {
  k_slot_io<<<current_device_sms(), 256, 0, s>>>(d_prob, slot, dst, 0);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_gram(const ProbDev *d_probs, const Item *d_items, int n_items,
                        const VeArgs &va, cudaStream_t s) {
  if (n_items <= 0) return cudaSuccess;
  const int K = va.nvec - 1;
  switch (K) {
#define RED_GRAM_CASE(k) \
  case k: k_gram<k><<<n_items, kGramThreads, 0, s>>>(d_probs, d_items, va); break;
    RED_GRAM_CASE(1) RED_GRAM_CASE(2) RED_GRAM_CASE(3) RED_GRAM_CASE(4) RED_GRAM_CASE(5)
    RED_GRAM_CASE(6) RED_GRAM_CASE(7) RED_GRAM_CASE(8) RED_GRAM_CASE(9) RED_GRAM_CASE(10)
#undef RED_GRAM_CASE
    default:
      k_gram_generic<<<n_items, 256, 0, s>>>(d_probs, d_items, va);
  }
  count_launches(1);
  return cudaGetLastError();
}

#define RED_K_CASES(M) \
  M(1) M(2) M(3) M(4) M(5) M(6) M(7) M(8) M(9) M(10) M(11) M(12)

cudaError_t launch_combine(const ProbDev *d_probs, const Item *d_items, int n_items,
                           const VeArgs &va, cudaStream_t s) {
  if (n_items <= 0) return cudaSuccess;
  switch (va.nvec - 1) {
#define RED_COMBINE_CASE(k) \
  case k: k_combine<k><<<n_items, kCombineThreads, 0, s>>>(d_probs, d_items, va); break;
    RED_K_CASES(RED_COMBINE_CASE)
#undef RED_COMBINE_CASE
    default: return cudaErrorInvalidValue;
  }
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_copy_slots(const ProbDev *d_probs, const Item *d_items, int n_items, int mode,
                              int slot, float *const *d_ptrs, cudaStream_t s) {
  if (n_items <= 0) return cudaSuccess;
  k_copy_slots<<<n_items, 256, 0, s>>>(d_probs, d_items, mode, slot, d_ptrs);
  count_launches(1);
  return cudaGetLastError();
}

// ---- allocation-free extrapolation ------------------------------------------------------
// The same three steps over plain device vectors, with every scratch word (Gram partial
// sums, xi, gamma, status) in one file-scope device array instead of a problem's buffers.
namespace {

constexpr int kStaticGramCtas = 1024;                      // Gram partial rows (max)
constexpr int kStaticPartials = kStaticGramCtas * kMaxPairs;
constexpr int kStaticStateDoubles = 16;
constexpr int kStaticDoubles = kStaticPartials + 2 * kMaxK + kStaticStateDoubles;
static_assert(sizeof(ProbState) <= kStaticStateDoubles * sizeof(double), "state block");

// 638,976 + 320 bytes: per-CTA Gram partials | xi | gamma | ProbState
static __device__ __align__(256) double g_ve_scratch[kStaticDoubles];

struct StaticVe {
  const float *x[kMaxK + 1];
  float *out;
  long n;
  int n_chunks;       // kGramChunk-pixel chunks of the vectors
  float2 *part;       // gridDim.x (Gram launch) rows of kMaxPairs (hi, lo) partial sums
  int n_part;
  int method;
  double *coef, *gamma;
  ProbState *st;
};

// Gram partials: CTA b accumulates chunks b, b + gridDim.x, ... (double-float, exact
// products as in k_gram) and writes one row of partial sums.
template <int K>
__global__ void __launch_bounds__(128) k_gram_static(StaticVe a) {
  constexpr int NP = K * (K + 1) / 2;
  __shared__ float2 red[4][NP];
  GramAcc<K> acc;
  acc.zero();
  const int tid = threadIdx.x;
  bool aligned = true;
#pragma unroll
  for (int i = 0; i <= K; ++i) aligned = aligned && ((reinterpret_cast<uintptr_t>(a.x[i]) & 15) == 0);
  for (long c = blockIdx.x; c < a.n_chunks; c += gridDim.x) {
    const long begin = c * kGramChunk;
    const long end = min(a.n, begin + kGramChunk);
    long p0 = begin;
    if (aligned) {   // begin is a multiple of 4
      const int nv = (int)((end - begin) >> 2);
      for (int v = tid; v < nv; v += blockDim.x) {
        float4 q[K + 1];
#pragma unroll
        for (int i = 0; i <= K; ++i) q[i] = __ldcs(reinterpret_cast<const float4 *>(a.x[i] + begin) + v);
        float x[K + 1];
#pragma unroll
        for (int i = 0; i <= K; ++i) x[i] = q[i].x;
        acc.add(x);
#pragma unroll
        for (int i = 0; i <= K; ++i) x[i] = q[i].y;
        acc.add(x);
#pragma unroll
        for (int i = 0; i <= K; ++i) x[i] = q[i].z;
        acc.add(x);
#pragma unroll
        for (int i = 0; i <= K; ++i) x[i] = q[i].w;
        acc.add(x);
      }
      p0 = begin + ((long)nv << 2);
    }
    for (long p = p0 + tid; p < end; p += blockDim.x) {
      float x[K + 1];
#pragma unroll
      for (int i = 0; i <= K; ++i) x[i] = a.x[i][p];
      acc.add(x);
    }
  }
  const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    float h = acc.hi[q], l = acc.lo[q];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
      df_add(h, l, __shfl_xor_sync(0xffffffffu, h, off), __shfl_xor_sync(0xffffffffu, l, off));
    if (lane == 0) red[warp][q] = make_float2(h, l);
  }
  __syncthreads();
  if (tid < NP) {
    float h = 0.f, l = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) df_add(h, l, red[w][tid].x, red[w][tid].y);
    a.part[(size_t)blockIdx.x * kMaxPairs + tid] = make_float2(h, l);
  }
}

// The gamma solve of ve_solve_k on a descriptor that points into the static scratch.
template <int K>
__global__ void __launch_bounds__(32) k_ve_solve_static(StaticVe a) {
  ProbDev P{};
  P.n_chunks = a.n_part;
  P.gram_part = a.part;
  P.ve_method = a.method;
  P.ve_coef = a.coef;
  P.gamma = a.gamma;
  P.st = a.st;
  ve_solve_k<K>(&P, 0);
}

// x_(m,kappa) = x_m + sum_j xi_j (x_{m+j+1} - x_{m+j}); the last iterate on breakdown.
template <int K>
__global__ void __launch_bounds__(256) k_combine_static(StaticVe a) {
  constexpr int kap = K - 1;
  const int brk = a.st->ve_status;
  float xi[kap > 0 ? kap : 1];
#pragma unroll
  for (int j = 0; j < kap; ++j) xi[j] = (float)a.coef[j];
  bool vec = (reinterpret_cast<uintptr_t>(a.out) & 15) == 0;
#pragma unroll
  for (int i = 0; i <= K; ++i) vec = vec && ((reinterpret_cast<uintptr_t>(a.x[i]) & 15) == 0);
  const long stride = (long)gridDim.x * blockDim.x;
  long p0 = 0;
  if (vec) {
    const long nv = a.n >> 2;
    for (long v = blockIdx.x * (long)blockDim.x + threadIdx.x; v < nv; v += stride) {
      float4 r;
      if (brk) {
        r = reinterpret_cast<const float4 *>(a.x[K])[v];
      } else {
        float4 x[K];
#pragma unroll
        for (int i = 0; i < K; ++i) x[i] = __ldcs(reinterpret_cast<const float4 *>(a.x[i]) + v);
        float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int j = 0; j < kap; ++j) {
          s.x = fmaf(xi[j], x[j + 1].x - x[j].x, s.x);
          s.y = fmaf(xi[j], x[j + 1].y - x[j].y, s.y);
          s.z = fmaf(xi[j], x[j + 1].z - x[j].z, s.z);
          s.w = fmaf(xi[j], x[j + 1].w - x[j].w, s.w);
        }
        r = make_float4(x[0].x + s.x, x[0].y + s.y, x[0].z + s.z, x[0].w + s.w);
      }
      reinterpret_cast<float4 *>(a.out)[v] = r;
    }
    p0 = nv << 2;
  }
  for (long p = p0 + blockIdx.x * (long)blockDim.x + threadIdx.x; p < a.n; p += stride) {
    float val;
    if (brk) {
      val = a.x[K][p];
    } else {
      float prev = a.x[0][p];
      const float x0 = prev;
      float s = 0.f;
#pragma unroll
      for (int j = 0; j < kap; ++j) {
        const float nx = a.x[j + 1][p];
        s = fmaf(xi[j], nx - prev, s);
        prev = nx;
      }
      val = x0 + s;
    }
    a.out[p] = val;
  }
}

// Device address of g_ve_scratch and the device's SM count, looked up once per device
// with that device current.
std::mutex g_static_mu;
std::vector<double *> g_static_addr;
std::vector<int> g_static_sms;

double *static_scratch(int dev, int *sms) {
  std::lock_guard<std::mutex> lk(g_static_mu);
  if ((int)g_static_addr.size() <= dev) {
    g_static_addr.resize(dev + 1, nullptr);
    g_static_sms.resize(dev + 1, 0);
  }
  if (!g_static_addr[dev]) {
    void *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_ve_scratch);
    if (e != cudaSuccess)
      throw Fail{RED_ECUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e)};
    int n = 0;
    e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess || n < 1)
      throw Fail{RED_ECUDA, std::string("cudaDeviceGetAttribute(SM count): ") + cudaGetErrorString(e)};
    g_static_sms[dev] = n;
    g_static_addr[dev] = static_cast<double *>(ptr);
  }
  *sms = g_static_sms[dev];
  return g_static_addr[dev];
}

}  // namespace
}  // namespace red

using namespace red;

extern "C" red_status red_ve_extrapolate_static(const void *const *xs_dev, int n_vec, int64_t n,
                                                int method, void *x_out_dev, double *gamma_host,
                                                void *stream) {
  return guarded([&] {
    CHECK_ARG(xs_dev && x_out_dev, "null argument");
    CHECK_ARG(n_vec >= 3 && n_vec <= kMaxK + 1, "n_vec must be in [3, 13]");
    CHECK_ARG(method == RED_VE_MPE || method == RED_VE_RRE || method == RED_VE_SVDMPE,
              "method must be RED_VE_MPE, RED_VE_RRE or RED_VE_SVDMPE");
    CHECK_ARG(n >= 1, "n must be positive");
    const int64_t max_n = 2147483647;   // chunk counts and launch sizes are 32-bit
    if (n > max_n)
      throw Fail{RED_EINVAL, "n = " + std::to_string(n) + " exceeds the limit of " +
                                 std::to_string(max_n) + " elements per vector"};
    int dev = 0;
    CUDA_OK(cudaGetDevice(&dev));
    int sms = 0;
    double *scratch = static_scratch(dev, &sms);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    StaticVe a{};
    for (int i = 0; i < n_vec; ++i) {
      CHECK_ARG(xs_dev[i] != nullptr, "null vector");
      a.x[i] = static_cast<const float *>(xs_dev[i]);
    }
    a.out = static_cast<float *>(x_out_dev);
    a.n = n;
    a.n_chunks = (int)((n + kGramChunk - 1) / kGramChunk);
    a.n_part = std::min(a.n_chunks, kStaticGramCtas);
    a.part = reinterpret_cast<float2 *>(scratch);
    a.method = method;
    a.coef = scratch + kStaticPartials;
    a.gamma = a.coef + kMaxK;
    a.st = reinterpret_cast<ProbState *>(a.gamma + kMaxK);
    // the state block starts at zero; every partial, xi and gamma read is written first
    CUDA_OK(cudaMemsetAsync(a.st, 0, sizeof(ProbState), s));
    const int K = n_vec - 1;
    // grid-stride combine: at most 4 resident 256-thread CTAs per SM of this device
    const int comb_ctas = (int)std::min<int64_t>((n / 4 + 255) / 256 + 1, 4 * (int64_t)sms);
    switch (K) {
#define RED_STATIC_CASE(k)                                      \
  case k:                                                       \
    k_gram_static<k><<<a.n_part, 128, 0, s>>>(a);               \
    k_ve_solve_static<k><<<1, 32, 0, s>>>(a);                   \
    k_combine_static<k><<<comb_ctas, 256, 0, s>>>(a);           \
    break;
      RED_K_CASES(RED_STATIC_CASE)
#undef RED_STATIC_CASE
      default: throw Fail{RED_EINVAL, "n_vec must be in [3, 13]"};
    }
    count_launches(3);
    CUDA_OK(cudaGetLastError());
    double hg[kMaxK];
    ProbState hs;
    CUDA_OK(cudaMemcpyAsync(hg, a.gamma, kMaxK * sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_OK(cudaMemcpyAsync(&hs, a.st, sizeof(ProbState), cudaMemcpyDeviceToHost, s));
    CUDA_OK(cudaStreamSynchronize(s));
    if (hs.ve_status) return RED_EVE_BREAKDOWN;
    if (gamma_host)
      for (int i = 0; i < K; ++i) gamma_host[i] = hg[i];
    return RED_OK;
  });
}
