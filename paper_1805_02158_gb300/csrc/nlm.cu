// Non-local-means denoiser f(x): the denoising engine called once per FP step (Eq. (7)),
// the dominant cost of RED (Sec. II-B: "hundreds of denoising activations").
//
// Definition (same as the FP64 oracle): for every pixel p,
//   f(p) = sum_d w(p,d) xp(p+d) / sum_d w(p,d),  d in [-5,5]^2 (11x11 search window),
//   w(p,d) = exp(-(1/(25 h^2)) sum_{t in [-2,2]^2} (xp(p+t) - xp(p+d+t))^2),
// xp = x extended by half-sample symmetric reflection.
//
// GB300 mapping. One warp = a tile of 60 output columns x kNlmR = 6 output rows (warp-sized work
// units balance evenly over the SMs; a CTA is 1-4 independent warps); the tile plus a
// 7-pixel halo (search radius 5 + patch radius 2) is staged once in shared memory, prescaled by k = sqrt(log2(e) / (25 h^2)) so that a weight is a single
// ex2.approx of a negated patch distance. Each lane owns 2 adjacent columns and kNlmR rows:
//   * the lane's own patch rows a(rr) (12 x 2 values) stay in registers for all 121 offsets;
//   * for each dx the lane loads the kNlmR + 14 candidate rows it needs for all 11 dy once, so
//     the dy loop (fully unrolled) only renames registers;
//   * vertical 5-row sums of squared differences slide down the column with 2 FMAs/row;
//   * horizontal 5-column sums use 4 warp shuffles per row (the warp covers 64 columns
//     and outputs the inner 60).
// Per output pixel and offset: ~8.7 FP32 ops, 1 MUFU.EX2, 2 SHFL; no shared-memory
// traffic in the inner loop beyond one candidate row per dy. Two alternatives measured on
// GB300 and not kept: the same arithmetic in packed f32x2 instructions (no faster:
// fma.rn.f32x2 has the lane throughput of scalar FMA, 38.2 vs 37.1 T lane-op/s), and the
// ragged right strip of 256-wide images (16 columns) packed three narrow lane segments to
// a warp (10.6 % fewer instructions, but a slower busiest SM: 58-61 vs 53 us).
//
// Work decomposition is fixed to a (kNlmR-row, 2-column) grid in image coordinates, so a
// pixel's arithmetic (and result, bit for bit) does not depend on the CTA shape chosen
// by the autotuner or on which other problems share the launch.
#include <cstdlib>
#include <vector>

#include "common.cuh"

namespace red {

namespace {

constexpr int kCols = kNlmTW + 14;   // staged columns: [tc0 - 7, tc0 + 67)
constexpr int kStride = 76;          // shared-memory row stride (floats)
constexpr unsigned kFull = 0xffffffffu;
constexpr int kStageU = 48;          // tile loads in flight per lane (the whole tile at once)

// Half-sample symmetric reflection for indices within one side length of the image,
// then clamped into it.
__device__ __forceinline__ int reflect_clamp(int i, int n) {
  i = i < 0 ? -1 - i : (i >= n ? 2 * n - 1 - i : i);
  return min(max(i, 0), n - 1);
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

template <int R, int MINB>
__global__ void __launch_bounds__(128, MINB)
k_nlm(const ProbDev *__restrict__ probs, const Item *__restrict__ items, int n_items, StepArgs sa,
      int src_type_override, float *f_override) {
  extern __shared__ float smem_tiles[];
  // one independent tile of 60 x R outputs per warp (work units are warp-sized so they
  // spread evenly over the SMs); the warp stages its own tile + 7-pixel halo
  const int item = blockIdx.x * blockDim.y + threadIdx.y;
  if (item >= n_items) return;
  const Item it = items[item];
  const ProbDev *P = probs + it.prob;
  if (sa.update_state && P->st->done) return;
  if (sa.skip_frozen && P->st->frozen) return;
  float *tile = smem_tiles + threadIdx.y * ((R + 14) * kStride);

  const int H = P->H, W = P->W;
  const int tr0 = it.a, tc0 = it.b;
  const int rows = R + 14;
  const float k = P->nlm_k;

  const void *src;
  int stype;
  if (sa.src_ptr) {
    src = sa.src_ptr;
    stype = src_type_override;
  } else {
    stype = P->storage;
    src = static_cast<const char *>(P->ring) + (size_t)sa.src * P->slot_stride * store_bytes(stype);
  }

  // Stage the tile: kStageU loads in flight per lane. One reflection is exact for every
  // pixel an output inside the image needs (halo 7 <= side); the clamp only keeps
  // rows/columns of partial tiles, whose outputs are not stored, inside the image.
  const int tid = threadIdx.x;
  const int total = rows * kCols;
  for (int base = tid; base < total; base += kStageU * 32) {
    float v[kStageU];
#pragma unroll
    for (int u = 0; u < kStageU; ++u) {
      const int idx = base + u * 32;
      if (idx < total) {
        const int rr = idx / kCols;
        const int cc = idx - rr * kCols;
        const int gr = reflect_clamp(tr0 - 7 + rr, H);
        const int gc = reflect_clamp(tc0 - 7 + cc, W);
        v[u] = load_img(src, (long)gr * W + gc, stype);
      }
    }
#pragma unroll
    for (int u = 0; u < kStageU; ++u) {
      const int idx = base + u * 32;
      if (idx < total) {
        const int rr = idx / kCols;
        tile[rr * kStride + (idx - rr * kCols)] = k * v[u];
      }
    }
  }
  __syncwarp();

  const int lane = threadIdx.x;
  const int r0 = 0;                   // the warp's first output row, tile-local
  const int sc0 = 2 * lane + 5;       // staged column of the lane's first column

  // own patch rows: staged rows r0 + 5 .. r0 + R + 8 (output rows r0-2 .. r0+R+1)
  float a0[R + 4], a1[R + 4];
#pragma unroll
  for (int rr = 0; rr < R + 4; ++rr) {
    a0[rr] = tile[(r0 + 5 + rr) * kStride + sc0];
    a1[rr] = tile[(r0 + 5 + rr) * kStride + sc0 + 1];
  }
  float num0[R], num1[R], den0[R], den1[R];
#pragma unroll
  for (int r = 0; r < R; ++r) num0[r] = num1[r] = den0[r] = den1[r] = 0.f;

#pragma unroll 1
  for (int dx = -5; dx <= 5; ++dx) {
    // candidate rows for dy = -5..5: staged rows r0 .. r0 + R + 13
    const float *bcol = tile + sc0 + dx;
    float b0[R + 14], b1[R + 14];
#pragma unroll
    for (int t = 0; t < R + 14; ++t) {
      b0[t] = bcol[(r0 + t) * kStride];
      b1[t] = bcol[(r0 + t) * kStride + 1];
    }
#pragma unroll
    for (int dyi = 0; dyi < 11; ++dyi) {
      float d0[R + 4], d1[R + 4];
#pragma unroll
      for (int rr = 0; rr < R + 4; ++rr) {
        d0[rr] = a0[rr] - b0[rr + dyi];
        d1[rr] = a1[rr] - b1[rr + dyi];
      }
      // negated 5-row sums of squared differences (so a weight is ex2 of the sum)
      float v0 = (-d0[0]) * d0[0];
      float v1 = (-d1[0]) * d1[0];
#pragma unroll
      for (int t = 1; t < 5; ++t) {
        v0 = fmaf(-d0[t], d0[t], v0);
        v1 = fmaf(-d1[t], d1[t], v1);
      }
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (r > 0) {
          v0 = fmaf(-d0[r + 4], d0[r + 4], fmaf(d0[r - 1], d0[r - 1], v0));
          v1 = fmaf(-d1[r + 4], d1[r + 4], fmaf(d1[r - 1], d1[r - 1], v1));
        }
        const float p = v0 + v1;
        const float pl = __shfl_up_sync(kFull, p, 1);
        const float pr = __shfl_down_sync(kFull, p, 1);
        const float v1l = __shfl_up_sync(kFull, v1, 1);
        const float v0r = __shfl_down_sync(kFull, v0, 1);
        const float D0 = (pl + p) + v0r;
        const float D1 = (v1l + p) + pr;
        const float w0 = ex2_approx(D0);
        const float w1 = ex2_approx(D1);
        num0[r] = fmaf(w0, b0[r + 2 + dyi], num0[r]);
        num1[r] = fmaf(w1, b1[r + 2 + dyi], num1[r]);
        den0[r] += w0;
        den1[r] += w1;
      }
    }
  }

  if (lane == 0 || lane == 31) return;  // halo lanes
  float *dst = f_override ? f_override : P->f;
  const float inv_k = 1.0f / k;
  const int c = tc0 - 2 + 2 * lane;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int gr = tr0 + r0 + r;
    if (gr >= H) break;
    if (c < W) dst[(long)gr * W + c] = (num0[r] / den0[r]) * inv_k;
    if (c + 1 < W) dst[(long)gr * W + c + 1] = (num1[r] / den1[r]) * inv_k;
  }
}

}  // namespace

// Work items of one image: a warp tile per band of kNlmR rows and 60 columns.
void nlm_items(int prob, int H, int W, std::vector<Item> &out) {
  for (int r0 = 0; r0 < H; r0 += kNlmR)
    for (int c0 = 0; c0 < W; c0 += kNlmTW) out.push_back({prob, r0, c0, 0});
}

cudaError_t nlm_prepare(int wy) {
  (void)wy;   // at most 4 warps per CTA x 8.5 KB of staged tile: under the 48 KB default
  return cudaSuccess;
}

// occ: 3 or 4 resident CTAs per SM (the register budget: 161 or 128 per thread); the
// arithmetic, and so the result, is the same for both.
cudaError_t launch_nlm(const ProbDev *d_probs, const Item *d_items, int n_items, int wy,
                       StepArgs sa, int src_type, cudaStream_t s, float *f_override, int occ) {
  if (n_items <= 0) return cudaSuccess;
  if (wy < 1 || wy > 4) return cudaErrorInvalidValue;   // kernel is bounded at 128 threads
  const size_t smem = (size_t)wy * (kNlmR + 14) * kStride * sizeof(float);
  dim3 block(32, wy);
  const int ctas = (n_items + wy - 1) / wy;
  if (occ >= 4)
    k_nlm<kNlmR, 4><<<ctas, block, smem, s>>>(d_probs, d_items, n_items, sa, src_type, f_override);
  else
    k_nlm<kNlmR, 3><<<ctas, block, smem, s>>>(d_probs, d_items, n_items, sa, src_type, f_override);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace red
