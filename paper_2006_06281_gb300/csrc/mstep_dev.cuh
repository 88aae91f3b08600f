// Device code of the M-step of fast CPD on sm_103a (shared by the per-pair
// kernels in mstep.cu and the batched persistent kernel in batch.cu) (Eq. 17 full basis, Eq. 20 top-K basis) and
// the variance update (Eq. 18), fused into the last kernel.
//
// Both dense products of the M-step are skinny (3 right-hand sides) and
// HBM-bound, so both run through one streaming kernel, `colsum`:
//     out[c][d] = sum_r A[r][c] * V[r][d]     (A row-major, d = 0..2)
// Each thread owns W consecutive columns (two 16-byte vectors = 32 bytes per
// row; 32-byte segments measured steadier across physical placements than
// 16-byte ones), walks a chunk of rows with loads in flight, and takes V[r]
// from shared memory;
// the row chunks are split over blocks and summed in a fixed order.
//   projection  A = U  (M x K), V = R = Ytil - X  ->  a_k = (U^T R)_k
//   expansion   A = U^T (K x M, stored once at setup), V = B  ->  (U B)_m
// with the diagonal update in between: s_k = l_k / (l_k + lambda sigma2),
// B_k = s_k a_k ("only a diagonal changes per iteration", Sec. III) and
// C_k = a_k / (l_k + lambda sigma2) for W.
// The expansion's reduction kernel writes T = X + U B and evaluates, per row
// in FP64, the Eq. 18 term with the new T, shifted to the old T (no
// cancellation of O(1) terms):
//   sum_n p^_mn |y_n - t_new|^2
//     = V_m/P1_m + 2 (t_old - t_new).(Ytil_m - t_old) + |t_old - t_new|^2;
// its last block sums the block partials in a fixed order and advances the
// device state (sigma2, history, stop test).
#pragma once

#include "common.cuh"

#include <cuda_fp16.h>
#include <math.h>

namespace fcpd {
namespace dev {

template <typename F> struct L16;
template <> struct L16<float> {
  using t = float4;
  static constexpr int W = 4;
};
template <> struct L16<double> {
  using t = double2;
  static constexpr int W = 2;
};
template <> struct L16<__half> {     // FP16 basis of the mixed-precision mode
  using t = uint4;
  static constexpr int W = 8;
};

__device__ __forceinline__ float lane_of(const float4& v, int i) {
  return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w;
}
__device__ __forceinline__ double lane_of(const double2& v, int i) { return i == 0 ? v.x : v.y; }
// FP16 lane i of a 16-byte vector.  By default the half's exponent and
// mantissa bits are moved to bit 13 of an FP32 word with integer operations:
// that word holds the FP16 value times 2^-112 exactly (normal and subnormal
// alike), and colsum_body pre-scales the other factor by 2^112, so every
// product is the same as with a conversion instruction while the work goes
// to the integer pipe.  FCPD_H2F_CVT selects the conversion instruction.
__device__ __forceinline__ float lane_of(const uint4& v, int i) {
  const unsigned int w = i < 2 ? v.x : i < 4 ? v.y : i < 6 ? v.z : v.w;
#ifdef FCPD_H2F_CVT
  const __half2 h = *reinterpret_cast<const __half2*>(&w);
  return (i & 1) ? __high2float(h) : __low2float(h);
#else
  const unsigned int b = (i & 1) ? (((w >> 3) & 0x0FFFE000u) | (w & 0x80000000u))
                                 : (((w << 13) & 0x0FFFE000u) | ((w << 16) & 0x80000000u));
  return __uint_as_float(b);
#endif
}
// Factor that undoes lane_of's 2^-112 inside each product (1 where lane_of
// is exact).  The products u * (v * 2^112) then equal u * v exactly; this
// relies on FP32 subnormals not being flushed (no -ftz / fast-math).
template <typename S> __device__ __forceinline__ float lane_scale() { return 1.0f; }
#ifndef FCPD_H2F_CVT
template <> __device__ __forceinline__ float lane_scale<__half>() { return 0x1p112f; }
#endif

constexpr int kThreadsP = 128;   // streaming kernel block
constexpr int kRTile = 256;      // rows of V staged per shared-memory tile
constexpr int kThreadsD = 256;   // reduction kernels
#ifndef FCPD_MRED_COLS
#define FCPD_MRED_COLS 64
#endif
constexpr int kMRedCols = FCPD_MRED_COLS;   // columns per reduction block
constexpr int kMRedSub = kThreadsD / kMRedCols;
static_assert(kMRedCols * kMRedSub == kThreadsD, "columns per block must divide the block");

// ---------------------------------------------------------------- colsum
// 16-byte vectors of A per thread and row (the plan pads rows to this):
// two (32 bytes) for FP32/FP64; one (8 columns) for an FP16 basis, whose
// threads do twice the arithmetic per byte -- measured at M = N = 20000:
// 5.0 TB/s with one vector, 3.6 TB/s with two.
#ifndef FCPD_COLSUM_VEC_H
#define FCPD_COLSUM_VEC_H 1
#endif
template <typename S> __host__ __device__ constexpr int colsum_vectors() {
  return sizeof(S) == 2 ? FCPD_COLSUM_VEC_H : 2;
}

// S is the storage type of A (F itself, or FP16 for a basis stored in half
// precision); products and sums are in F.
template <typename F, typename S, int THREADS>
__device__ __forceinline__ void colsum_body(const S* FCPD_RESTRICT A, int64_t ldA, int rows, int cols, const typename Vec<F>::t4* FCPD_RESTRICT V,
       int rows_per_chunk, F* FCPD_RESTRICT part, int64_t ldP, DevState* FCPD_RESTRICT st, int gate,
       int clear_row_flags, int bx, int by, int gx, int gy) {
  if (gate && iteration_gated(st)) return;
  // the E-step's row list was consumed by fixB before this kernel
  if (clear_row_flags && bx == 0 && by == 0 && threadIdx.x == 0) st->n_flag_rows = 0;
  using V4 = typename Vec<F>::t4;
  using LT = typename L16<S>::t;
  constexpr int L = L16<S>::W;           // elements per 16-byte vector
  constexpr int NV = colsum_vectors<S>();
  constexpr int W = NV * L;              // columns per thread (NV x 16 bytes of A per row)
  __shared__ V4 sV[kRTile];
  const int c0 = (bx * THREADS + threadIdx.x) * W;
  const int r0 = by * rows_per_chunk;
  const int r1 = min(rows, r0 + rows_per_chunk);
  F acc[W][3];
#pragma unroll
  for (int w = 0; w < W; ++w) acc[w][0] = acc[w][1] = acc[w][2] = (F)0;
  for (int base = r0; base < r1; base += kRTile) {
    const int cnt = min(kRTile, r1 - base);
    __syncthreads();
    for (int i = threadIdx.x; i < cnt; i += THREADS) {
      V4 v = V[base + i];
      if constexpr (sizeof(S) == 2) {          // exact power-of-two pre-scale (see lane_of)
        const F k = (F)lane_scale<S>();
        v.x *= k; v.y *= k; v.z *= k;
      }
      sV[i] = v;
    }
    __syncthreads();
    if (c0 < cols) {
      const S* ap = A + (size_t)base * ldA + c0;
#pragma unroll 4
      for (int i = 0; i < cnt; ++i) {
        const LT* row = reinterpret_cast<const LT*>(ap + (size_t)i * ldA);
        const LT u0 = __ldg(row), u1 = NV > 1 ? __ldg(row + 1) : u0;
        const V4 r = sV[i];
#pragma unroll
        for (int w = 0; w < W; ++w) {
          const F uw = (F)(w < L ? lane_of(u0, w) : lane_of(u1, w - L));
          acc[w][0] = fma(uw, r.x, acc[w][0]);
          acc[w][1] = fma(uw, r.y, acc[w][1]);
          acc[w][2] = fma(uw, r.z, acc[w][2]);
        }
      }
    }
  }
  if (c0 < cols) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      F* out = part + ((size_t)by * 3 + d) * ldP + c0;
      if constexpr (sizeof(F) == 4) {
#pragma unroll
        for (int v = 0; v < W / 4; ++v)
          reinterpret_cast<float4*>(out)[v] =
              make_float4(acc[4 * v][d], acc[4 * v + 1][d], acc[4 * v + 2][d], acc[4 * v + 3][d]);
      } else {
#pragma unroll
        for (int v = 0; v < W / 2; ++v)
          reinterpret_cast<double2*>(out)[v] = make_double2(acc[2 * v][d], acc[2 * v + 1][d]);
      }
    }
  }
}

// Sum of the chunk partials of column `col` (accumulated in F: FP32 partials
// are summed in FP32 -- GB300's FP64 rate is a small fraction of FP32 -- in a
// fixed order; the FP64 path sums in FP64).  A block serves COLS columns;
// kThreadsD / COLS threads per column each take a strided subset; the subsets
// are added in order through `part`.  Fewer columns per block shorten each
// thread's chain of dependent loads when there are many chunks.
template <typename F, int COLS = kMRedCols>
__device__ __forceinline__ void chunk_sums(const F* FCPD_RESTRICT partials, int chunks, int64_t ldP, int col,
                                           int ncols, F (&a)[3], F (*part)[3][COLS]) {
  constexpr int SUB = kThreadsD / COLS;
  const int c = threadIdx.x % COLS, sub = threadIdx.x / COLS;
  F s[3] = {(F)0, (F)0, (F)0};
  if (col < ncols) {
#pragma unroll 4
    for (int k = sub; k < chunks; k += SUB)
#pragma unroll
      for (int d = 0; d < 3; ++d) s[d] += __ldcg(partials + ((size_t)k * 3 + d) * ldP + col);
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) part[sub][d][c] = s[d];
  __syncthreads();
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    F t = (F)0;
#pragma unroll
    for (int j = 0; j < SUB; ++j) t += part[j][d][c];
    a[d] = t;
  }
}

// Diagonal update (once per column k) with the sigma2 of this iteration's
// E-step: B_k = s_k a_k, C_k = a_k / (l_k + lambda sigma2).  COLS columns per
// block (as chunk_sums).
template <typename F, int COLS = kMRedCols>
__device__ __forceinline__ void diag_update_body(const F* FCPD_RESTRICT partP, int chunks, int64_t ldU, int K, const double* FCPD_RESTRICT lam,
            typename Vec<F>::t4* FCPD_RESTRICT B4, typename Vec<F>::t4* FCPD_RESTRICT C4,
            const DevState* FCPD_RESTRICT st, int gate, int bx, int by, int gx, int gy) {
  static_assert(COLS <= kThreadsD && kThreadsD % COLS == 0, "columns per block must divide the block");
  if (gate && iteration_gated(st)) return;
  __shared__ F part[kThreadsD / COLS][3][COLS];
  __shared__ double lamsig;
  if (threadIdx.x == 0) lamsig = st->lambda * st->sigma2;
  const int k = bx * COLS + threadIdx.x % COLS;
  F a[3];
  chunk_sums<F, COLS>(partP, chunks, ldU, k, K, a, part);
  if (threadIdx.x >= COLS || k >= K) return;
  const double inv = 1.0 / (lam[k] + lamsig);          // one FP64 division per column
  const double s = lam[k] * inv;
  using V4 = typename Vec<F>::t4;
  V4 b, cw;
  b.x = (F)(s * a[0]); b.y = (F)(s * a[1]); b.z = (F)(s * a[2]); b.w = (F)0;
  cw.x = (F)(a[0] * inv); cw.y = (F)(a[1] * inv); cw.z = (F)(a[2] * inv); cw.w = (F)0;
  B4[k] = b;
  C4[k] = cw;
}

// T = X + U B (X may be null: W = U C) from the expansion partials; with EPI
// the Eq. 18 epilogue and the device-state update of the iteration.
// Eq. 18 terms of model point m after its update from `to` to `tn` (yt:
// Ytil_m with sum_n p^_mn |y_n - t_m|^2 in w): the shifted-form contribution,
// the squared change of t_m, and the squared ground-truth error.
template <typename V4>
__device__ __forceinline__ void point_terms(const V4& to, const V4& tn, const V4& yt,
                                            const V4* FCPD_RESTRICT Yhat4, int m, double& contrib, double& dT2,
                                            double& gt2) {
  const double dx = (double)to.x - tn.x, dy = (double)to.y - tn.y, dz = (double)to.z - tn.z;
  const double gx = (double)yt.x - to.x, gy = (double)yt.y - to.y, gz = (double)yt.z - to.z;
  dT2 = dx * dx + dy * dy + dz * dz;
  contrib = (double)yt.w + 2.0 * (dx * gx + dy * gy + dz * gz) + dT2;
  gt2 = 0.0;
  if (Yhat4) {
    const V4 h = Yhat4[m];
    const double ex = (double)tn.x - h.x, ey = (double)tn.y - h.y, ez = (double)tn.z - h.z;
    gt2 = ex * ex + ey * ey + ez * ez;
  }
}

// End of an iteration from the totals over all model points (t0: Eq. 18
// numerator, t1: sum |dT|^2, t2: sum of squared ground-truth errors):
// sigma2, the history entry, the iteration count and the stop tests.  One
// thread.
__device__ __forceinline__ void finish_iteration(DevState* FCPD_RESTRICT st, double t0, double t1, double t2, int M) {
  const int it = st->iter;
  const double s2new = t0 / (3.0 * (double)M);
  const double rm = st->has_gt ? sqrt(t2 / (double)M) : nan("");
  // passes A and B evaluate 2 M N pairs when dense; the pruned ones count theirs
  const double frac = prune_active(st) ? (double)st->pairs_eval / (2.0 * (double)M * (double)st->N) : 1.0;
  st->pairs_eval = 0;
  st->last_eval_frac = frac;
  if (st->hist && it < kHistCap) {
    st->hist[it] = s2new;
    st->hist[kHistCap + it] = st->loglik;
    st->hist[2 * kHistCap + it] = rm;
    st->hist[3 * kHistCap + it] = frac;
  }
  st->last_dT2 = t1;
  st->last_rmse = rm;
  if (!(s2new > 0.0) || !isfinite(s2new)) st->status = (int)CPD_ENUMERIC;
  else st->sigma2 = s2new;
  st->iter = it + 1;
  if (st->tol > 0.0 && sqrt(t1 / (double)M) <= st->tol) st->done = 1;
  if (st->gt_tol > 0.0 && st->has_gt && rm <= st->gt_tol) st->done = 1;
}

// With EPI, returns true in the block that completed the iteration (wrote
// sigma2 and the history); false otherwise.
template <typename F, bool EPI>
__device__ __forceinline__ bool expand_finish_body(const F* FCPD_RESTRICT partE, int chunks, int64_t ldM, int M,
              const typename Vec<F>::t4* FCPD_RESTRICT X4, const typename Vec<F>::t4* FCPD_RESTRICT Yt4,
              typename Vec<F>::t4* FCPD_RESTRICT Tout, const typename Vec<F>::t4* FCPD_RESTRICT Yhat4,
              double* FCPD_RESTRICT sums, DevState* FCPD_RESTRICT st, int gate, int bx, int by, int gx, int gy) {
  if (gate && iteration_gated(st)) return false;
  using V4 = typename Vec<F>::t4;
  __shared__ F part[kMRedSub][3][kMRedCols];
  __shared__ double sh3[32][3];
  __shared__ bool last;
  const int m = bx * kMRedCols + threadIdx.x % kMRedCols;
  // the row's own inputs are loaded first, in flight during the chunk sums
  const bool row = threadIdx.x < kMRedCols && m < M;
  V4 x{}, to{}, yt{}, yh{};
  if (row) {
    if (X4) x = X4[m];
    if constexpr (EPI) {
      to = Tout[m];
      yt = Yt4[m];
      if (Yhat4) yh = Yhat4[m];
    }
  }
  F a[3];
  chunk_sums<F>(partE, chunks, ldM, m, M, a, part);
  double contrib = 0.0, dT2 = 0.0, gt2 = 0.0;
  if (row) {
    V4 tn;
    tn.x = (F)((double)x.x + (double)a[0]); tn.y = (F)((double)x.y + (double)a[1]);
    tn.z = (F)((double)x.z + (double)a[2]); tn.w = (F)0;
    if constexpr (EPI) point_terms<V4>(to, tn, yt, Yhat4 ? &yh : nullptr, 0, contrib, dT2, gt2);
    Tout[m] = tn;
  }
  if constexpr (EPI) {
    // only the first kMRedCols threads hold a row's terms
    block_sum3(contrib, dT2, gt2, sh3, (kMRedCols + 31) / 32);
    if (threadIdx.x == 0) {
      sums[(size_t)bx * 3] = contrib;
      sums[(size_t)bx * 3 + 1] = dT2;
      sums[(size_t)bx * 3 + 2] = gt2;
      __threadfence();
      last = atomicAdd(&st->ticket_e, 1u) == gx - 1;
    }
    __syncthreads();
    if (last) {
      __threadfence();
      double a0 = 0, a1 = 0, a2 = 0;
      for (int i = threadIdx.x; i < (int)gx; i += blockDim.x) {
        a0 += __ldcg(sums + (size_t)i * 3);
        a1 += __ldcg(sums + (size_t)i * 3 + 1);
        a2 += __ldcg(sums + (size_t)i * 3 + 2);
      }
      block_sum3(a0, a1, a2, sh3, (int)(blockDim.x >> 5));
      if (threadIdx.x == 0) {
        finish_iteration(st, a0, a1, a2, M);
        st->ticket_e = 0;
      }
    }
    return last;
  }
  return false;
}

}  // namespace dev
}  // namespace fcpd
