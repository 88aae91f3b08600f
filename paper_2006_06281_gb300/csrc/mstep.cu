// M-step of fast CPD on sm_103a (Eq. 17 full basis, Eq. 20 top-K basis) and
// the variance update (Eq. 18), fused.
//
//   project  A = U^T R with R = Ytil - X (K x 3).  U is M x ldU row-major;
//            each thread streams 16-byte vectors of W consecutive columns down
//            a chunk of rows (coalesced HBM reads), rows of R are broadcast
//            from shared memory; the row chunks are split over blocks and
//            summed by `project_reduce` in a fixed order.
//   diag     s_k = l_k / (l_k + lambda sigma2) -- "only a diagonal is
//            updated" per iteration; B_k = s_k A_k, C_k = A_k/(l_k + lambda sigma2).
//   expand   T = X + U B.  Each warp owns kRows rows and sweeps them with
//            16-byte loads while B tiles are shared through shared memory.
//            Epilogue (per row, FP64): the Eq. 18 term with the new T,
//              sum_n p^_mn |y_n - t_new|^2
//                = V_m/P1_m + 2 (t_old - t_new).(Ytil_m - t_old) + |t_old - t_new|^2,
//            which is Eq. 18's trace form shifted to t_old (no cancellation of
//            O(1) terms); the last block sums the block partials in a fixed
//            order and advances the device state (sigma2, history, stop test).
#include "common.cuh"

#include <math.h>

#include <algorithm>

namespace fcpd {

namespace {

template <typename F> struct L16;
template <> struct L16<float> {
  using t = float4;
  static constexpr int W = 4;
};
template <> struct L16<double> {
  using t = double2;
  static constexpr int W = 2;
};

__device__ __forceinline__ float lane_of(const float4& v, int i) {
  return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w;
}
__device__ __forceinline__ double lane_of(const double2& v, int i) { return i == 0 ? v.x : v.y; }

constexpr int kThreadsP = 128;   // projection block
constexpr int kRTile = 256;      // rows of R staged per shared-memory tile
constexpr int kThreadsE = 256;   // expansion block (8 warps)
constexpr int kRows = 4;         // rows per warp in the expansion
constexpr int kThreadsD = 256;   // diagonal-update block

template <typename F> __host__ __device__ constexpr int ktile_e() { return sizeof(F) == 4 ? 2048 : 1024; }

// ---------------------------------------------------------------- project
template <typename F>
__global__ void __launch_bounds__(kThreadsP)
project(const F* __restrict__ U, int64_t ldU, int M, int K, const typename Vec<F>::t4* __restrict__ R4,
        int rows_per_chunk, F* __restrict__ partP, const DevState* __restrict__ st, int gate) {
  if (gate && iteration_gated(st)) return;
  using V4 = typename Vec<F>::t4;
  using LT = typename L16<F>::t;
  constexpr int W = L16<F>::W;
  __shared__ V4 sR[kRTile];
  const int k0 = (blockIdx.x * kThreadsP + threadIdx.x) * W;
  const int r0 = blockIdx.y * rows_per_chunk;
  const int r1 = min(M, r0 + rows_per_chunk);
  F acc[W][3];
#pragma unroll
  for (int w = 0; w < W; ++w) acc[w][0] = acc[w][1] = acc[w][2] = (F)0;
  for (int base = r0; base < r1; base += kRTile) {
    const int cnt = min(kRTile, r1 - base);
    __syncthreads();
    for (int i = threadIdx.x; i < cnt; i += kThreadsP) sR[i] = R4[base + i];
    __syncthreads();
    if (k0 < K) {
      const F* up = U + (size_t)base * ldU + k0;
#pragma unroll 8
      for (int i = 0; i < cnt; ++i) {
        const LT u = __ldg(reinterpret_cast<const LT*>(up + (size_t)i * ldU));
        const V4 r = sR[i];
#pragma unroll
        for (int w = 0; w < W; ++w) {
          const F uw = lane_of(u, w);
          acc[w][0] = fma(uw, r.x, acc[w][0]);
          acc[w][1] = fma(uw, r.y, acc[w][1]);
          acc[w][2] = fma(uw, r.z, acc[w][2]);
        }
      }
    }
  }
  if (k0 < K) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      F* out = partP + ((size_t)blockIdx.y * 3 + d) * ldU + k0;
      if constexpr (W == 4) {
        *reinterpret_cast<float4*>(out) = make_float4(acc[0][d], acc[1][d], acc[2][d], acc[3][d]);
      } else {
        *reinterpret_cast<double2*>(out) = make_double2(acc[0][d], acc[1][d]);
      }
    }
  }
}

// Sums the projection partials (FP64, fixed order) and applies the diagonal
// update with the sigma2 of this iteration's E-step.
template <typename F>
__global__ void __launch_bounds__(kThreadsD)
project_reduce(const F* __restrict__ partP, int chunks, int64_t ldU, int K, const double* __restrict__ lam,
               typename Vec<F>::t4* __restrict__ B4, typename Vec<F>::t4* __restrict__ C4,
               const DevState* __restrict__ st, int gate) {
  if (gate && iteration_gated(st)) return;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  double a[3] = {0.0, 0.0, 0.0};
  for (int c = 0; c < chunks; ++c)
#pragma unroll
    for (int d = 0; d < 3; ++d) a[d] += (double)partP[((size_t)c * 3 + d) * ldU + k];
  const double den = lam[k] + st->lambda * st->sigma2;
  const double s = lam[k] / den;
  using V4 = typename Vec<F>::t4;
  V4 b, cw;
  b.x = (F)(s * a[0]); b.y = (F)(s * a[1]); b.z = (F)(s * a[2]); b.w = (F)0;
  cw.x = (F)(a[0] / den); cw.y = (F)(a[1] / den); cw.z = (F)(a[2] / den); cw.w = (F)0;
  B4[k] = b;
  C4[k] = cw;
}

// ----------------------------------------------------------------- expand
template <typename F, bool EPI>
__global__ void __launch_bounds__(kThreadsE)
expand(const F* __restrict__ U, int64_t ldU, int M, int K, const typename Vec<F>::t4* __restrict__ B4,
       const typename Vec<F>::t4* __restrict__ X4, const typename Vec<F>::t4* __restrict__ Yt4,
       typename Vec<F>::t4* __restrict__ Tout, const typename Vec<F>::t4* __restrict__ Yhat4,
       double* __restrict__ sums, DevState* __restrict__ st, int gate) {
  if (gate && iteration_gated(st)) return;
  using V4 = typename Vec<F>::t4;
  using LT = typename L16<F>::t;
  constexpr int W = L16<F>::W;
  constexpr int KT = ktile_e<F>();
  extern __shared__ __align__(32) unsigned char smem_raw[];
  V4* sB = reinterpret_cast<V4*>(smem_raw);
  __shared__ double sh[32];
  __shared__ bool last;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row0 = (blockIdx.x * (kThreadsE / 32) + warp) * kRows;
  F acc[kRows][3];
#pragma unroll
  for (int r = 0; r < kRows; ++r) acc[r][0] = acc[r][1] = acc[r][2] = (F)0;
  for (int kb = 0; kb < K; kb += KT) {
    __syncthreads();
    for (int i = threadIdx.x; i < KT; i += kThreadsE) {
      const int k = kb + i;
      V4 z;
      z.x = z.y = z.z = z.w = (F)0;
      sB[i] = k < K ? B4[k] : z;
    }
    __syncthreads();
    const int kcnt = min(KT, K - kb);
    for (int kk = lane * W; kk < kcnt; kk += 32 * W) {
      V4 b[W];
#pragma unroll
      for (int w = 0; w < W; ++w) b[w] = sB[kk + w];
#pragma unroll
      for (int r = 0; r < kRows; ++r) {
        const int m = row0 + r;
        if (m < M) {
          const LT u = __ldg(reinterpret_cast<const LT*>(U + (size_t)m * ldU + kb + kk));
#pragma unroll
          for (int w = 0; w < W; ++w) {
            const F uw = lane_of(u, w);
            acc[r][0] = fma(uw, b[w].x, acc[r][0]);
            acc[r][1] = fma(uw, b[w].y, acc[r][1]);
            acc[r][2] = fma(uw, b[w].z, acc[r][2]);
          }
        }
      }
    }
  }
#pragma unroll
  for (int r = 0; r < kRows; ++r)
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      F v = acc[r][d];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      acc[r][d] = v;
    }
  double contrib = 0.0, dT2 = 0.0, gt2 = 0.0;
  if (lane < kRows) {
    F s0 = 0, s1 = 0, s2 = 0;
#pragma unroll
    for (int r = 0; r < kRows; ++r)
      if (lane == r) { s0 = acc[r][0]; s1 = acc[r][1]; s2 = acc[r][2]; }
    const int m = row0 + lane;
    if (m < M) {
      double x0 = 0, x1 = 0, x2 = 0;
      if (X4) { const V4 x = X4[m]; x0 = x.x; x1 = x.y; x2 = x.z; }
      V4 tn;
      tn.x = (F)(x0 + (double)s0); tn.y = (F)(x1 + (double)s1); tn.z = (F)(x2 + (double)s2); tn.w = (F)0;
      if constexpr (EPI) {
        const V4 to = Tout[m];
        const V4 yt = Yt4[m];
        const double dx = (double)to.x - tn.x, dy = (double)to.y - tn.y, dz = (double)to.z - tn.z;
        const double gx = (double)yt.x - to.x, gy = (double)yt.y - to.y, gz = (double)yt.z - to.z;
        dT2 = dx * dx + dy * dy + dz * dz;
        contrib = (double)yt.w + 2.0 * (dx * gx + dy * gy + dz * gz) + dT2;
        if (Yhat4) {
          const V4 h = Yhat4[m];
          const double ex = (double)tn.x - h.x, ey = (double)tn.y - h.y, ez = (double)tn.z - h.z;
          gt2 = ex * ex + ey * ey + ez * ez;
        }
      }
      Tout[m] = tn;
    }
  }
  if constexpr (EPI) {
    const double b0 = block_sum(contrib, sh);
    const double b1 = block_sum(dT2, sh);
    const double b2 = block_sum(gt2, sh);
    if (threadIdx.x == 0) {
      sums[(size_t)blockIdx.x * 3] = b0;
      sums[(size_t)blockIdx.x * 3 + 1] = b1;
      sums[(size_t)blockIdx.x * 3 + 2] = b2;
      __threadfence();
      last = atomicAdd(&st->ticket_e, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last) {
      __threadfence();
      const volatile double* vs = sums;
      double a0 = 0, a1 = 0, a2 = 0;
      for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
        a0 += vs[(size_t)i * 3];
        a1 += vs[(size_t)i * 3 + 1];
        a2 += vs[(size_t)i * 3 + 2];
      }
      const double t0 = block_sum(a0, sh);
      const double t1 = block_sum(a1, sh);
      const double t2 = block_sum(a2, sh);
      if (threadIdx.x == 0) {
        const int it = st->iter;
        const double s2new = t0 / (3.0 * (double)M);
        const double rm = st->has_gt ? sqrt(t2 / (double)M) : nan("");
        if (st->hist && it < kHistCap) {
          st->hist[it] = s2new;
          st->hist[kHistCap + it] = st->loglik;
          st->hist[2 * kHistCap + it] = rm;
        }
        st->last_dT2 = t1;
        st->last_rmse = rm;
        if (!(s2new > 0.0) || !isfinite(s2new)) st->status = (int)CPD_ENUMERIC;
        else st->sigma2 = s2new;
        st->iter = it + 1;
        if (st->tol > 0.0 && sqrt(t1 / (double)M) <= st->tol) st->done = 1;
        if (st->gt_tol > 0.0 && st->has_gt && rm <= st->gt_tol) st->done = 1;
        st->ticket_e = 0;
      }
    }
  }
}

int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

template <typename F>
size_t expand_smem() { return sizeof(typename Vec<F>::t4) * ktile_e<F>(); }

}  // namespace

// The expansion uses 32 KB of dynamic shared memory, within the default
// 48 KB limit; the attribute is set explicitly so a larger tile stays legal.
void mstep_prepare() {
  cudaFuncSetAttribute(expand<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)expand_smem<float>());
  cudaFuncSetAttribute(expand<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)expand_smem<float>());
  cudaFuncSetAttribute(expand<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)expand_smem<double>());
  cudaFuncSetAttribute(expand<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)expand_smem<double>());
}

MstepPlan plan_mstep(int64_t M, int64_t K, bool fp64, int sms) {
  MstepPlan p{};
  const int W = fp64 ? 2 : 4;
  const int64_t ldU = cdiv(K, W) * W;
  p.p_col_tiles = (int)cdiv(ldU, (int64_t)kThreadsP * W);
  const int64_t target = (int64_t)sms * 8;
  int64_t chunks = std::max<int64_t>(1, cdiv(target, p.p_col_tiles));
  int64_t rpc = std::max<int64_t>(16, cdiv(M, chunks));
  p.p_rows_per_chunk = (int)rpc;
  p.p_row_chunks = (int)cdiv(M, rpc);
  p.partP_elems = (int64_t)p.p_row_chunks * 3 * ldU;
  p.e_blocks = (int)cdiv(M, (kThreadsE / 32) * kRows);
  p.sums_elems = (int64_t)p.e_blocks * 3;
  return p;
}

template <typename F>
void launch_mstep(const MstepPlan& pl, const F* U, int64_t ldU, const double* lam, int64_t M, int64_t K,
                  const typename Vec<F>::t4* X4, const typename Vec<F>::t4* R4,
                  const typename Vec<F>::t4* Yt4, typename Vec<F>::t4* T4,
                  const typename Vec<F>::t4* Yhat4, F* partP, double* sums, typename Vec<F>::t4* B4,
                  typename Vec<F>::t4* C4, DevState* st, bool iteration, cudaStream_t s, cudaEvent_t* ev) {
  const int g = iteration ? 1 : 0;
  project<F><<<dim3(pl.p_col_tiles, pl.p_row_chunks), kThreadsP, 0, s>>>(U, ldU, (int)M, (int)K, R4,
                                                                       pl.p_rows_per_chunk, partP, st, g);
  record_after(ev, 0, s);
  project_reduce<F><<<(unsigned)cdiv(K, kThreadsD), kThreadsD, 0, s>>>(partP, pl.p_row_chunks, ldU, (int)K,
                                                                       lam, B4, C4, st, g);
  record_after(ev, 1, s);
  if (iteration) {
    expand<F, true><<<pl.e_blocks, kThreadsE, expand_smem<F>(), s>>>(U, ldU, (int)M, (int)K, B4, X4, Yt4,
                                                                      T4, Yhat4, sums, st, g);
  } else {
    expand<F, false><<<pl.e_blocks, kThreadsE, expand_smem<F>(), s>>>(U, ldU, (int)M, (int)K, B4, X4, Yt4,
                                                                       T4, nullptr, sums, st, 0);
  }
  record_after(ev, 2, s);
}

template <typename F>
void launch_w(const MstepPlan& pl, const F* U, int64_t ldU, int64_t M, int64_t K,
              const typename Vec<F>::t4* C4, typename Vec<F>::t4* W4, cudaStream_t s) {
  expand<F, false><<<pl.e_blocks, kThreadsE, expand_smem<F>(), s>>>(U, ldU, (int)M, (int)K, C4, nullptr,
                                                                     nullptr, W4, nullptr, nullptr, nullptr, 0);
}

template void launch_mstep<float>(const MstepPlan&, const float*, int64_t, const double*, int64_t, int64_t,
                                  const float4*, const float4*, const float4*, float4*, const float4*,
                                  float*, double*, float4*, float4*, DevState*, bool, cudaStream_t, cudaEvent_t*);
template void launch_mstep<double>(const MstepPlan&, const double*, int64_t, const double*, int64_t, int64_t,
                                   const dvec4*, const dvec4*, const dvec4*, dvec4*, const dvec4*, double*,
                                   double*, dvec4*, dvec4*, DevState*, bool, cudaStream_t, cudaEvent_t*);
template void launch_w<float>(const MstepPlan&, const float*, int64_t, int64_t, int64_t, const float4*,
                              float4*, cudaStream_t);
template void launch_w<double>(const MstepPlan&, const double*, int64_t, int64_t, int64_t, const dvec4*,
                               dvec4*, cudaStream_t);

}  // namespace fcpd
