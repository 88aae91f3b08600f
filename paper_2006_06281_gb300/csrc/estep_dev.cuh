// Device code of the E-step of fast CPD on sm_103a (shared by the per-pair
// kernels in estep.cu and the batched persistent kernel in batch.cu): Eq. 4 (posterior with the uniform-outlier
// constant c) followed by Eq. 5 (the corresponding constraint: every row of P
// rescaled to sum to 1), reduced to Ytil = P^ Y without storing P.
//
// The M x N posterior is evaluated twice, n-body style, instead of being
// materialised:
//   pass A  each thread owns scene points y_n (columns) in registers and
//           streams model-point tiles t_m through shared memory, accumulating
//           den_n = sum_m e_mn (+ c in the reduction);
//   pass B  each thread owns model points t_m (rows) and streams scene tiles
//           {y_n, den_n} through shared memory, accumulating
//           P1_m = sum_n e_mn/den_n, sum_n (e_mn/den_n) y_n and
//           V_m = sum_n (e_mn/den_n) |y_n - t_m|^2.
// Both passes split their long dimension over blocks; a reduction kernel
// sums the split partials in a fixed order (deterministic), applies Eq. 5
// (Ytil_m = PY_m / P1_m) and checks the row mass.
//
// FP32 form: coordinates are pre-scaled by q = sqrt(log2(e) / (2 sigma2)), so
// e_mn = 2^(-|q y_n - q t_m|^2) is one MUFU ex2 per pair, and pass B folds
// 1/den_n into the exponent: e_mn / den_n = 2^(-log2 den_n - |q y - q t|^2).
// FP32 flushes Gaussians below 2^-126 (about 13 sigma away).  A column whose
// denominator or a row whose mass falls below 2^-88 / 2^-90 (where flushed
// terms could matter) is listed and recomputed exactly by one warp in the log
// domain (max exponent first, then the shifted sum), so FP32 results stay
// valid wherever the FP64 definition is; the status becomes CPD_ENUMERIC only
// if the mass is 0 even in double precision.
// FP64 form: exp(-|y - t|^2 / (2 sigma2)) in double, times 1/den_n.
#pragma once

#include "common.cuh"

#include <math.h>

namespace fcpd {
namespace dev {

// Launch shapes of the FP32 passes (compile-time, overridable with -D for
// tuning sweeps; the defaults were the fastest of nine shapes measured on
// GB300 at M = N = 20000: pass A 0.098 ms vs 0.112 ms for 128 threads x 8
// columns, pass B 0.176 ms vs 0.186 ms for 128 threads x 4 rows).
#ifndef FCPD_EA_THREADS
#define FCPD_EA_THREADS 256
#endif
#ifndef FCPD_EA_COLS
#define FCPD_EA_COLS 16
#endif
#ifndef FCPD_EA_UNROLL
#define FCPD_EA_UNROLL 1
#endif
#ifndef FCPD_EB_THREADS
#define FCPD_EB_THREADS 256
#endif
#ifndef FCPD_EB_ROWS
#define FCPD_EB_ROWS 8
#endif
#ifndef FCPD_EB_UNROLL
#define FCPD_EB_UNROLL 1
#endif
constexpr int kThreadsA = FCPD_EA_THREADS;   // pass A block
constexpr int kColsA32 = FCPD_EA_COLS;       // scene points per thread, FP32
constexpr int kUnrollA = FCPD_EA_UNROLL;     // model points in flight per thread
constexpr int kColsA64 = 4;                  // scene points per thread, FP64
constexpr int kTileA = 128;                  // model points per shared-memory tile
constexpr int kThreadsB = FCPD_EB_THREADS;   // pass B block
constexpr int kRowsB32 = FCPD_EB_ROWS;       // model points per thread, FP32
constexpr int kUnrollB = FCPD_EB_UNROLL;     // scene points in flight per thread
constexpr int kRowsB64 = 2;                  // model points per thread, FP64
constexpr int kTileB = 128;                  // scene points per shared-memory tile
constexpr int kThreadsR = 256;   // reduction kernels
constexpr int kThreadsF = 256;   // log-domain fix-up kernels (one warp per item)
constexpr float kFar = 1e18f;    // padding coordinate: its Gaussian weight is exactly 0
constexpr double kColFloor = 0x1p-88;   // FP32 column sums below this take the exact path
constexpr double kRowFloor = 0x1p-90;   // FP32 row masses below this take the exact path

// q = sqrt(log2(e) / (2 sigma2)) in FP32 (GB300's FP64 rate is a small
// fraction of FP32; every kernel derives q with this same function, so the
// scaled coordinates agree bitwise between passes).
__device__ __forceinline__ float scale_q(double sigma2) {
  return sqrtf(1.44269504f / (2.0f * (float)sigma2));
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Packed FP32 pairs (two lanes of one 64-bit register) for the f32x2
// arithmetic of sm_100-class GPUs: one instruction issues two FP32 ops,
// leaving issue slots for the MUFU ex2 and shared-memory loads.
typedef unsigned long long f2_t;
__device__ __forceinline__ f2_t f2_pack(float a, float b) {
  f2_t r;
  asm("mov.b64 %0, {%1,%2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void f2_unpack(f2_t r, float& a, float& b) {
  asm("mov.b64 {%0,%1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ f2_t f2_sub(f2_t a, f2_t b) {
  f2_t d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2_t f2_add(f2_t a, f2_t b) {
  f2_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2_t f2_mul(f2_t a, f2_t b) {
  f2_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2_t f2_fma(f2_t a, f2_t b, f2_t c) {
  f2_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// Shared-memory tile of the FP32 passes (kTileA = kTileB records of two
// 16-byte halves).  Declared once at namespace scope so that every kernel
// -- and every instantiation of the pass bodies inside one kernel -- holds a
// single copy.
static_assert(kTileA == kTileB, "passes A and B share one tile buffer");
__shared__ ulonglong2 s_pass_tile[kTileA][2];

// ------------------------------------------------------------------ pass A
// FP32 pass A: each thread owns kColsA32 scene points as kColsA32/2 packed
// pairs; a model point is broadcast from shared memory as duplicated pairs
// {(x,x),(y,y)},{(z,z),-}.  Per pair of Gaussians: 3 sub + 1 mul + 2 fma on
// f32x2, two MUFU ex2 and two scalar adds.
// COLS < kColsA32 serves a partial last tile: the tile still starts at
// bx * kThreadsA * kColsA32 but each thread covers only COLS scene points.
template <int COLS = kColsA32>
__device__ __forceinline__ void passA_f32_body(const float4* FCPD_RESTRICT T4, int M, int rows_per_chunk, const float4* FCPD_RESTRICT Y4,
          int N, float* FCPD_RESTRICT partA, DevState* FCPD_RESTRICT st, int gate, int bx, int by, int gx, int gy) {
  if (gate && iteration_gated(st)) return;
  static_assert(COLS % 2 == 0 && COLS <= kColsA32, "scene points per thread: even, at most kColsA32");
  constexpr int P = COLS / 2;
  ulonglong2 (*sT)[2] = s_pass_tile;
  const float q = scale_q(st->sigma2);
  const int nbase = bx * (kThreadsA * kColsA32) + threadIdx.x;
  f2_t yx[P], yy[P], yz[P];
  float acc[2 * P];
#pragma unroll
  for (int p = 0; p < P; ++p) {
    const int n0 = nbase + (2 * p) * kThreadsA, n1 = n0 + kThreadsA;
    const float4 far4 = make_float4(-kFar / q, -kFar / q, -kFar / q, 0.f);
    const float4 y0 = n0 < N ? Y4[n0] : far4;
    const float4 y1 = n1 < N ? Y4[n1] : far4;
    yx[p] = f2_pack(q * y0.x, q * y1.x);
    yy[p] = f2_pack(q * y0.y, q * y1.y);
    yz[p] = f2_pack(q * y0.z, q * y1.z);
    acc[2 * p] = acc[2 * p + 1] = 0.f;
  }
  const int r0 = by * rows_per_chunk;
  const int r1 = min(M, r0 + rows_per_chunk);
  for (int base = r0; base < r1; base += kTileA) {
    __syncthreads();
    for (int i = threadIdx.x; i < kTileA; i += kThreadsA) {
      const int m = base + i;
      float tx = kFar, ty = kFar, tz = kFar;
      if (m < r1) {
        const float4 t = T4[m];
        tx = q * t.x; ty = q * t.y; tz = q * t.z;
      }
      sT[i][0] = make_ulonglong2(f2_pack(tx, tx), f2_pack(ty, ty));
      sT[i][1] = make_ulonglong2(f2_pack(tz, tz), 0ull);
    }
    __syncthreads();
    const int cnt = min(kTileA, r1 - base);
#pragma unroll kUnrollA
    for (int i = 0; i < cnt; ++i) {
      const ulonglong2 a = sT[i][0];
      const f2_t tz2 = sT[i][1].x;
#pragma unroll
      for (int p = 0; p < P; ++p) {
        const f2_t dx = f2_sub(yx[p], a.x), dy = f2_sub(yy[p], a.y), dz = f2_sub(yz[p], tz2);
        f2_t d2 = f2_mul(dx, dx);
        d2 = f2_fma(dy, dy, d2);
        d2 = f2_fma(dz, dz, d2);
        float d0, d1;
        f2_unpack(d2, d0, d1);                  // register halves: no move
        acc[2 * p] += ex2_approx(-d0);          // scalar adds: no repacking of
        acc[2 * p + 1] += ex2_approx(-d1);      // the MUFU results
      }
    }
  }
#pragma unroll
  for (int p = 0; p < P; ++p) {
    const float a0 = acc[2 * p], a1 = acc[2 * p + 1];
    const int n0 = nbase + (2 * p) * kThreadsA, n1 = n0 + kThreadsA;
    if (n0 < N) partA[(size_t)by * N + n0] = a0;
    if (n1 < N) partA[(size_t)by * N + n1] = a1;
  }
}

__device__ __forceinline__ void passA_f64_body(const dvec4* FCPD_RESTRICT T4, int M, int rows_per_chunk, const dvec4* FCPD_RESTRICT Y4,
          int N, double* FCPD_RESTRICT partA, const DevState* FCPD_RESTRICT st, int gate, int bx, int by, int gx, int gy) {
  if (gate && iteration_gated(st)) return;
  __shared__ dvec4 sT[kTileA];
  const double inv2s2 = 1.0 / (2.0 * st->sigma2);
  const int nbase = bx * (kThreadsA * kColsA64) + threadIdx.x;
  double yx[kColsA64], yy[kColsA64], yz[kColsA64], acc[kColsA64];
#pragma unroll
  for (int j = 0; j < kColsA64; ++j) {
    const int n = nbase + j * kThreadsA;
    const dvec4 y = n < N ? Y4[n] : dvec4{0, 0, 0, 0};
    yx[j] = y.x; yy[j] = y.y; yz[j] = y.z;
    acc[j] = 0.0;
  }
  const int r0 = by * rows_per_chunk;
  const int r1 = min(M, r0 + rows_per_chunk);
  for (int base = r0; base < r1; base += kTileA) {
    __syncthreads();
    for (int i = threadIdx.x; i < kTileA; i += kThreadsA) {
      const int m = base + i;
      sT[i] = m < r1 ? T4[m] : dvec4{0, 0, 0, 0};
    }
    __syncthreads();
    const int cnt = min(kTileA, r1 - base);
    for (int i = 0; i < cnt; ++i) {
      const dvec4 t = sT[i];
#pragma unroll
      for (int j = 0; j < kColsA64; ++j) {
        const double dx = yx[j] - t.x, dy = yy[j] - t.y, dz = yz[j] - t.z;
        acc[j] += exp(-(dx * dx + dy * dy + dz * dz) * inv2s2);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < kColsA64; ++j) {
    const int n = nbase + j * kThreadsA;
    if (n < N) partA[(size_t)by * N + n] = acc[j];
  }
}

__device__ __forceinline__ double outlier_c(const DevState* st, int M, int N) {
  const double w = st->w;
  const double t = 2.0 * kPi * st->sigma2;         // (2 pi sigma2)^(D/2), D = 3
  return t * sqrt(t) * (w / (1.0 - w)) * ((double)M / (double)N);
}
// The same constant in FP32 arithmetic (relative error a few 2^-24, below
// that of the FP32 Gaussian sums it is added to): GB300's FP64 square root
// and divisions would stand on the critical path of every reduction block.
__device__ __forceinline__ double outlier_c_f32(const DevState* st, int M, int N) {
  const float w = (float)st->w;
  const float t = (float)(2.0 * kPi * st->sigma2);
  return (double)(t * sqrtf(t) * (w / (1.f - w)) * ((float)M / (float)N));
}

// ------------------------------------------------- pass A reduction (+ c)
// den_n = sum of the split partials + c (Eq. 4).  Prepares pass B's scene
// records and reduces the Eq. 3 log-likelihood sum_n ln den_n (+ constants).
// A block owns kRedCols columns; kRedSub threads per column each sum a strided
// subset of the chunks (coalesced across columns), then the subsets are added
// in a fixed order -- deterministic.
#ifndef FCPD_RED_COLS
#define FCPD_RED_COLS 64
#endif
constexpr int kRedCols = FCPD_RED_COLS;
constexpr int kRedSub = kThreadsR / kRedCols;
static_assert(kRedCols * kRedSub == kThreadsR, "columns per block must divide the block");

template <typename F>
// Returns true in the block that completed the reduction over all gx blocks
// (the one that wrote the log-likelihood).  defer: the log-likelihood is
// zeroed (for fixA's terms) and left to loglik_finish, off the critical
// path, which sums the FP32 exponent offsets -log2 den_n in Yb (FP32) or
// the block sums written here (FP64).
__device__ __forceinline__ bool reduceA_body(const F* FCPD_RESTRICT partA, int chunks, int M, const typename Vec<F>::t4* FCPD_RESTRICT Y4,
        int N, typename Vec<F>::t4* FCPD_RESTRICT Yb, double* FCPD_RESTRICT den_out,
        double* FCPD_RESTRICT sums, int* FCPD_RESTRICT flag_cols, DevState* FCPD_RESTRICT st, int gate, int bx, int by, int gx, int gy,
        int defer = 0) {
  if (gate && iteration_gated(st)) return false;
  __shared__ double sh[32];
  __shared__ F part[kRedSub][kRedCols];
  __shared__ bool last;
  __shared__ double c_sh;
  const double s2 = st->sigma2;
  const double w = st->w;
  if (threadIdx.x == 0) c_sh = sizeof(F) == 4 ? outlier_c_f32(st, M, N) : outlier_c(st, M, N);   // once per block
  const int col = threadIdx.x % kRedCols, sub = threadIdx.x / kRedCols;
  const int n = bx * kRedCols + col;
  typename Vec<F>::t4 y{};                    // y_n, in flight with the partial loads
  if (sub == 0 && n < N) y = Y4[n];
  F s = (F)0;   // FP32 partials summed in FP32 (fixed order), FP64 in FP64
  if (n < N) {
#pragma unroll 8
    for (int k = sub; k < chunks; k += kRedSub) s += __ldcg(partA + (size_t)k * N + n);
  }
  part[sub][col] = s;
  __syncthreads();
  const double c = c_sh;
  double lnden = 0.0;
  int bad = 0;
  if (sub == 0 && n < N) {
    F tot = (F)0;
#pragma unroll
    for (int j = 0; j < kRedSub; ++j) tot += part[j][col];
    const double den = (double)tot + c;
    if constexpr (sizeof(F) == 4) {
      const float q = scale_q(s2);
      if (!(den >= kColFloor) || !isfinite(den)) {
        // Gaussians flushed by FP32 may dominate: exact log-domain path
        flag_cols[atomicAdd(&st->n_flag_cols, 1)] = n;
        Yb[n] = make_float4(q * y.x, q * y.y, q * y.z, 0.f);
      } else {
        const float lid = -log2f((float)den);          // exponent offset of pass B
        Yb[n] = make_float4(q * y.x, q * y.y, q * y.z, lid);
        if (den_out) den_out[n] = den;
        lnden = -0.69314718055994531 * (double)lid;    // ln den from the same log2
      }
    } else {
      // the column of Eq. 4 is 0/0 in double precision: the definition fails
      bad = !(den > 0.0) || !isfinite(den);
      Yb[n] = dvec4{y.x, y.y, y.z, bad ? 0.0 : 1.0 / den};
      if (den_out) den_out[n] = den;
      lnden = bad ? 0.0 : log(den);
    }
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicExch(&st->status, (int)CPD_ENUMERIC);
  if (sizeof(F) == 4 && defer) {
    if (bx == 0 && threadIdx.x == 0) st->loglik = 0.0;
    return false;
  }
  const double bs = block_sum(lnden, sh);
  if (defer) {
    if (threadIdx.x == 0) {
      sums[bx] = bs;
      if (bx == 0) st->loglik = 0.0;
    }
    return false;
  }
  if (threadIdx.x == 0) {
    sums[bx] = bs;
    __threadfence();
    last = atomicAdd(&st->ticket_a, 1u) == gx - 1;
  }
  __syncthreads();
  if (last) {
    __threadfence();
    double v = 0.0;
    for (int i = threadIdx.x; i < (int)gx; i += blockDim.x) v += __ldcg(sums + i);
    const double tot = block_sum(v, sh);
    if (threadIdx.x == 0) {
      st->loglik = tot + (double)N * log((1.0 - w) / (double)M) - 1.5 * (double)N * log(2.0 * kPi * s2);
      st->ticket_a = 0;
    }
  }
  return last;
}

// Exact FP32 column denominators in the log domain for the listed columns:
// den_n = 2^a (sum_m 2^(-d'^2_mn - a)) + c with a = max_m (-d'^2_mn).
// defer_loglik: the column's Eq. 3 term is taken from Yb by loglik_finish.
__device__ __forceinline__ void fixA_f32_body(const float4* FCPD_RESTRICT T4, int M, const float4* FCPD_RESTRICT Y4, int N,
         float4* FCPD_RESTRICT Yb, double* FCPD_RESTRICT den_out, const int* FCPD_RESTRICT flag_cols,
         DevState* FCPD_RESTRICT st, int gate, int bx, int by, int gx, int gy, int defer_loglik = 0) {
  if (gate && iteration_gated(st)) return;
  const int count = st->n_flag_cols;
  if (count == 0) return;
  const float q = scale_q(st->sigma2);
  const double c = outlier_c(st, M, N);
  const int lane = threadIdx.x & 31;
  const int nwarps = gx * (kThreadsF / 32);
  for (int j = bx * (kThreadsF / 32) + (threadIdx.x >> 5); j < count; j += nwarps) {
    const int n = flag_cols[j];
    const float4 y = Y4[n];
    const float yx = q * y.x, yy = q * y.y, yz = q * y.z;
    float amax = -INFINITY;
    for (int m = lane; m < M; m += 32) {
      const float4 t = T4[m];
      const float dx = yx - q * t.x, dy = yy - q * t.y, dz = yz - q * t.z;
      float d2 = dx * dx;
      d2 = fmaf(dy, dy, d2);
      d2 = fmaf(dz, dz, d2);
      amax = fmaxf(amax, -d2);
    }
    amax = warp_max(amax);
    float sum = 0.f;
    for (int m = lane; m < M; m += 32) {
      const float4 t = T4[m];
      const float dx = yx - q * t.x, dy = yy - q * t.y, dz = yz - q * t.z;
      float d2 = dx * dx;
      d2 = fmaf(dy, dy, d2);
      d2 = fmaf(dz, dz, d2);
      sum += ex2_approx(-d2 - amax);
    }
    sum = warp_sumf(sum);
    if (lane == 0) {
      const double den = (double)sum * exp2((double)amax) + c;
      if (!(den > 0.0) || !isfinite(den)) {
        atomicExch(&st->status, (int)CPD_ENUMERIC);
      } else {
        const float lid = (float)(-log2(den));
        Yb[n].w = lid;
        if (den_out) den_out[n] = den;
        if (!defer_loglik) atomicAdd(&st->loglik, -0.69314718055994531 * (double)lid);
      }
    }
  }
}

// ------------------------------------------------------------------ pass B
// FP32 pass B: each thread owns kRowsB32 model points as packed pairs; scene
// records are broadcast from shared memory as {(x,x),(y,y)},{(z,z),(l,l)}
// with l = -log2 den_n.  Per pair of Gaussians: 3 sub + 1 mul + 2 fma for the
// distance and 1 sub for the exponent on f32x2, two MUFU ex2, then scalar
// 1 add + 4 fma per Gaussian to accumulate P1, PY (3) and V.
// ROWS < kRowsB32 serves a partial last tile (as COLS in pass A).
// clear_rows = 0 leaves the row list alone, for callers that reduce rows in
// the same pass (and clear the list elsewhere).
template <int ROWS = kRowsB32>
__device__ __forceinline__ void passB_f32_body(const float4* FCPD_RESTRICT T4, int M, const float4* FCPD_RESTRICT Yb, int N,
          int cols_per_chunk, float* FCPD_RESTRICT partB, DevState* FCPD_RESTRICT st, int gate, int bx, int by, int gx, int gy,
          int clear_rows = 1) {
  if (gate && iteration_gated(st)) return;
  static_assert(ROWS % 2 == 0 && ROWS <= kRowsB32, "model points per thread: even, at most kRowsB32");
  // the column list was consumed by fixA (the previous kernel) and the row
  // list is filled only after this kernel: both can be cleared here
  if (bx == 0 && by == 0 && threadIdx.x == 0) {
    st->n_flag_cols = 0;
    if (clear_rows) st->n_flag_rows = 0;
  }
  constexpr int P = ROWS / 2;
  ulonglong2 (*sY)[2] = s_pass_tile;
  const float q = scale_q(st->sigma2);
  const int mbase = bx * (kThreadsB * kRowsB32) + threadIdx.x;
  f2_t tx[P], ty[P], tz[P];
  float p1[2 * P], px[2 * P], py[2 * P], pz[2 * P], v[2 * P];
#pragma unroll
  for (int p = 0; p < P; ++p) {
    float c[2][3];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int m = mbase + (2 * p + h) * kThreadsB;
      if (m < M) {
        const float4 t = T4[m];
        c[h][0] = q * t.x; c[h][1] = q * t.y; c[h][2] = q * t.z;
      } else {
        c[h][0] = c[h][1] = c[h][2] = kFar;
      }
    }
    tx[p] = f2_pack(c[0][0], c[1][0]);
    ty[p] = f2_pack(c[0][1], c[1][1]);
    tz[p] = f2_pack(c[0][2], c[1][2]);
  }
#pragma unroll
  for (int j = 0; j < 2 * P; ++j) p1[j] = px[j] = py[j] = pz[j] = v[j] = 0.f;
  const int c0 = by * cols_per_chunk;
  const int c1 = min(N, c0 + cols_per_chunk);
  // next tile's scene records prefetched into registers (as in pass A)
  static_assert(kTileB <= kThreadsB, "one scene point per thread per tile");
  const float4 far4 = make_float4(-kFar, -kFar, -kFar, 0.f);
  float4 nxt = far4;
  if (threadIdx.x < kTileB && c0 + (int)threadIdx.x < c1) nxt = Yb[c0 + threadIdx.x];
  for (int base = c0; base < c1; base += kTileB) {
    __syncthreads();
    if (threadIdx.x < kTileB) {
      const float4 y = base + (int)threadIdx.x < c1 ? nxt : far4;
      sY[threadIdx.x][0] = make_ulonglong2(f2_pack(y.x, y.x), f2_pack(y.y, y.y));
      sY[threadIdx.x][1] = make_ulonglong2(f2_pack(y.z, y.z), f2_pack(y.w, y.w));
    }
    __syncthreads();
    if (threadIdx.x < kTileB && base + kTileB + (int)threadIdx.x < c1) nxt = Yb[base + kTileB + threadIdx.x];
    const int cnt = min(kTileB, c1 - base);
#pragma unroll kUnrollB
    for (int i = 0; i < cnt; ++i) {
      const ulonglong2 a = sY[i][0], b = sY[i][1];
#pragma unroll
      for (int p = 0; p < P; ++p) {
        const f2_t dx = f2_sub(tx[p], a.x), dy = f2_sub(ty[p], a.y), dz = f2_sub(tz[p], b.x);
        f2_t d2 = f2_mul(dx, dx);
        d2 = f2_fma(dy, dy, d2);
        d2 = f2_fma(dz, dz, d2);
        float e0, e1, q0, q1, yx, yy, yz, lid;
        f2_unpack(f2_sub(b.y, d2), e0, e1);     // register halves: no move
        f2_unpack(d2, q0, q1);
        f2_unpack(a.x, yx, lid);
        f2_unpack(a.y, yy, lid);
        f2_unpack(b.x, yz, lid);
        const float w0 = ex2_approx(e0), w1 = ex2_approx(e1);   // e_mn / den_n
        p1[2 * p] += w0;                         p1[2 * p + 1] += w1;
        px[2 * p] = fmaf(w0, yx, px[2 * p]);     px[2 * p + 1] = fmaf(w1, yx, px[2 * p + 1]);
        py[2 * p] = fmaf(w0, yy, py[2 * p]);     py[2 * p + 1] = fmaf(w1, yy, py[2 * p + 1]);
        pz[2 * p] = fmaf(w0, yz, pz[2 * p]);     pz[2 * p + 1] = fmaf(w1, yz, pz[2 * p + 1]);
        v[2 * p] = fmaf(w0, q0, v[2 * p]);       v[2 * p + 1] = fmaf(w1, q1, v[2 * p + 1]);
      }
    }
  }
  const size_t plane = (size_t)gy * M;
#pragma unroll
  for (int j = 0; j < 2 * P; ++j) {
    const int m = mbase + j * kThreadsB;
    if (m < M) {
      const size_t o = (size_t)by * M + m;
      partB[o] = p1[j];
      partB[o + plane] = px[j];
      partB[o + 2 * plane] = py[j];
      partB[o + 3 * plane] = pz[j];
      partB[o + 4 * plane] = v[j];
    }
  }
}

// ------------------------------------------------ pruned FP32 passes (exact)
// With model and scene points in spatial (Morton) order, each warp owns 128
// consecutive points (4 per thread), so its points fill a small box.  Before
// a shared tile of 128 points of the other set is used, each warp bounds the
// tile pair's exponents by the boxes (per 32-point sub-tile of the staged
// tile): in pass A every exponent is
// -|y' - t'|^2 <= -gap^2, in pass B lid_n - |y' - t'|^2 <= max lid - gap^2
// (gap: distance between the boxes of the scaled points).  ex2.approx.ftz
// returns exactly 0 for exponents below -126 (the result would be
// subnormal), so a tile pair whose bound is below -kPruneExp contributes
// exactly nothing and is skipped: the sums are bit-identical to evaluating
// it.  kPruneExp keeps one unit of margin for the FP32 rounding of the
// scaled coordinates and of the distances (relative 1e-6 of 127).
constexpr float kPruneExp = 127.0f;
constexpr int kPrunePts = 4;                          // points per thread
constexpr int kPruneWarpPts = 32 * kPrunePts;         // consecutive points per warp
constexpr int kPruneTile = kThreadsA * kPrunePts;     // points per block tile (1024)
static_assert(kThreadsA == kThreadsB && kTileA == 128 && kTileB == 128, "pruned passes: 256-thread blocks, 128-point tiles");

__shared__ float s_prune_box[4][8];                   // per staging warp: lo[3], hi[3], max lid

__device__ __forceinline__ void warp_box(float (&lo)[3], float (&hi)[3]) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      lo[d] = fminf(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], o));
      hi[d] = fmaxf(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], o));
    }
}

// Squared gap between two boxes (INF if either is empty).
__device__ __forceinline__ float box_gap2(const float (&alo)[3], const float (&ahi)[3], const float (&blo)[3],
                                          const float (&bhi)[3]) {
  float g2 = 0.f;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float g = fmaxf(0.f, fmaxf(alo[d] - bhi[d], blo[d] - ahi[d]));
    g2 = fmaf(g, g, g2);
  }
  return g2;
}

// Staged tile boxes: threads < 128 hold one point each (valid or not);
// warps 0-3 reduce, so s_prune_box[s] bounds points [32 s, 32 s + 32) of the
// tile (an empty box if none is valid).  Ends with __syncthreads.
__device__ __forceinline__ void stage_tile_box(bool valid, float x, float y, float z, float l) {
  if (threadIdx.x < 128) {
    float a[3] = {valid ? x : INFINITY, valid ? y : INFINITY, valid ? z : INFINITY};
    float b[3] = {valid ? x : -INFINITY, valid ? y : -INFINITY, valid ? z : -INFINITY};
    float m = valid ? l : -INFINITY;
    warp_box(a, b);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) {
      float* w = s_prune_box[threadIdx.x >> 5];
      w[0] = a[0]; w[1] = a[1]; w[2] = a[2]; w[3] = b[0]; w[4] = b[1]; w[5] = b[2]; w[6] = m;
    }
  }
  __syncthreads();
}

// Exponent bound of the pairs of this warp's points with staged sub-tile s:
// max lid - gap^2 (lid = 0 in pass A).  -INF for an empty sub-tile.
__device__ __forceinline__ float sub_tile_bound(const float (&wlo)[3], const float (&whi)[3], int s) {
  const float* b = s_prune_box[s];
  const float lo[3] = {b[0], b[1], b[2]}, hi[3] = {b[3], b[4], b[5]};
  return b[6] - box_gap2(wlo, whi, lo, hi);
}

// Pruned pass A: block (bx, by) = scene points [bx * 1024, +1024) (warp w:
// [.. + 128 w, +128), lane + 32 j) against model rows [by * rows_per_chunk,
// +rows_per_chunk).  Writes partA[by][n] like the dense pass.
__device__ __forceinline__ void passA_f32_pruned_body(const float4* FCPD_RESTRICT T4, int M, int rows_per_chunk,
          const float4* FCPD_RESTRICT Y4, int N, float* FCPD_RESTRICT partA, DevState* FCPD_RESTRICT st, int bx, int by) {
  constexpr int P = kPrunePts / 2;
  ulonglong2 (*sT)[2] = s_pass_tile;
  const bool skip_ok = !(st->prune_ctl & kPruneNoSkip);
  const float q = scale_q(st->sigma2);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nbase = bx * kPruneTile + warp * kPruneWarpPts + lane;
  f2_t yx[P], yy[P], yz[P];
  float acc[2 * P];
  float wlo[3] = {INFINITY, INFINITY, INFINITY}, whi[3] = {-INFINITY, -INFINITY, -INFINITY};
  int nvalid = 0;
#pragma unroll
  for (int p = 0; p < P; ++p) {
    float c[2][3];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int n = nbase + (2 * p + h) * 32;
      if (n < N) {
        const float4 y = Y4[n];
        c[h][0] = q * y.x; c[h][1] = q * y.y; c[h][2] = q * y.z;
#pragma unroll
        for (int d = 0; d < 3; ++d) { wlo[d] = fminf(wlo[d], c[h][d]); whi[d] = fmaxf(whi[d], c[h][d]); }
        ++nvalid;
      } else {
        c[h][0] = c[h][1] = c[h][2] = -kFar;
      }
    }
    yx[p] = f2_pack(c[0][0], c[1][0]);
    yy[p] = f2_pack(c[0][1], c[1][1]);
    yz[p] = f2_pack(c[0][2], c[1][2]);
    acc[2 * p] = acc[2 * p + 1] = 0.f;
  }
  warp_box(wlo, whi);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) nvalid += __shfl_xor_sync(0xffffffffu, nvalid, o);
  unsigned long long evaluated = 0;
  const int r0 = by * rows_per_chunk;
  const int r1 = min(M, r0 + rows_per_chunk);
  for (int base = r0; base < r1; base += kTileA) {
    __syncthreads();
    bool in = false;
    float tx = kFar, ty = kFar, tz = kFar;
    if (threadIdx.x < kTileA) {
      const int m = base + threadIdx.x;
      in = m < r1;
      if (in) {
        const float4 t = T4[m];
        tx = q * t.x; ty = q * t.y; tz = q * t.z;
      }
      sT[threadIdx.x][0] = make_ulonglong2(f2_pack(tx, tx), f2_pack(ty, ty));
      sT[threadIdx.x][1] = make_ulonglong2(f2_pack(tz, tz), 0ull);
    }
    stage_tile_box(in, tx, ty, tz, 0.f);     // its __syncthreads also publishes sT
    const int cnt = min(kTileA, r1 - base);
#pragma unroll 1
    for (int sub = 0; sub * 32 < cnt; ++sub) {
    if (skip_ok && sub_tile_bound(wlo, whi, sub) < -kPruneExp) continue;   // warp-uniform
    const int i1 = min(cnt, sub * 32 + 32);
    evaluated += (unsigned long long)(i1 - sub * 32) * (unsigned long long)nvalid;
#pragma unroll 1
    for (int i = sub * 32; i < i1; ++i) {
      const ulonglong2 a = sT[i][0];
      const f2_t tz2 = sT[i][1].x;
#pragma unroll
      for (int p = 0; p < P; ++p) {
        const f2_t dx = f2_sub(yx[p], a.x), dy = f2_sub(yy[p], a.y), dz = f2_sub(yz[p], tz2);
        f2_t d2 = f2_mul(dx, dx);
        d2 = f2_fma(dy, dy, d2);
        d2 = f2_fma(dz, dz, d2);
        float d0, d1;
        f2_unpack(d2, d0, d1);
        acc[2 * p] += ex2_approx(-d0);
        acc[2 * p + 1] += ex2_approx(-d1);
      }
    }
    }
  }
#pragma unroll
  for (int p = 0; p < P; ++p)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int n = nbase + (2 * p + h) * 32;
      if (n < N) partA[(size_t)by * N + n] = acc[2 * p + h];
    }
  if (lane == 0 && evaluated) atomicAdd(&st->pairs_eval, evaluated);
}

// Pruned pass B: block (bx, by) = model points [bx * 1024, +1024) (warp w:
// [.. + 128 w, +128), lane + 32 j) against scene points [by *
// cols_per_chunk, +cols_per_chunk).  Writes partB like the dense pass (gy =
// number of column chunks).
__device__ __forceinline__ void passB_f32_pruned_body(const float4* FCPD_RESTRICT T4, int M,
          const float4* FCPD_RESTRICT Yb, int N, int cols_per_chunk, float* FCPD_RESTRICT partB,
          DevState* FCPD_RESTRICT st, int bx, int by, int gy) {
  constexpr int P = kPrunePts / 2;
  if (bx == 0 && by == 0 && threadIdx.x == 0) {   // as the dense pass: both lists are free here
    st->n_flag_cols = 0;
    st->n_flag_rows = 0;
  }
  ulonglong2 (*sY)[2] = s_pass_tile;
  const bool skip_ok = !(st->prune_ctl & kPruneNoSkip);
  const float q = scale_q(st->sigma2);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int mbase = bx * kPruneTile + warp * kPruneWarpPts + lane;
  f2_t tx[P], ty[P], tz[P];
  float p1[2 * P], px[2 * P], py[2 * P], pz[2 * P], v[2 * P];
  float wlo[3] = {INFINITY, INFINITY, INFINITY}, whi[3] = {-INFINITY, -INFINITY, -INFINITY};
  int nvalid = 0;
#pragma unroll
  for (int p = 0; p < P; ++p) {
    float c[2][3];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int m = mbase + (2 * p + h) * 32;
      if (m < M) {
        const float4 t = T4[m];
        c[h][0] = q * t.x; c[h][1] = q * t.y; c[h][2] = q * t.z;
#pragma unroll
        for (int d = 0; d < 3; ++d) { wlo[d] = fminf(wlo[d], c[h][d]); whi[d] = fmaxf(whi[d], c[h][d]); }
        ++nvalid;
      } else {
        c[h][0] = c[h][1] = c[h][2] = kFar;
      }
    }
    tx[p] = f2_pack(c[0][0], c[1][0]);
    ty[p] = f2_pack(c[0][1], c[1][1]);
    tz[p] = f2_pack(c[0][2], c[1][2]);
  }
#pragma unroll
  for (int j = 0; j < 2 * P; ++j) p1[j] = px[j] = py[j] = pz[j] = v[j] = 0.f;
  warp_box(wlo, whi);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) nvalid += __shfl_xor_sync(0xffffffffu, nvalid, o);
  unsigned long long evaluated = 0;
  const int c0 = by * cols_per_chunk;
  const int c1 = min(N, c0 + cols_per_chunk);
  for (int base = c0; base < c1; base += kTileB) {
    __syncthreads();
    bool in = false;
    float4 y = make_float4(-kFar, -kFar, -kFar, 0.f);
    if (threadIdx.x < kTileB) {
      const int n = base + threadIdx.x;
      in = n < c1;
      if (in) y = Yb[n];
      sY[threadIdx.x][0] = make_ulonglong2(f2_pack(y.x, y.x), f2_pack(y.y, y.y));
      sY[threadIdx.x][1] = make_ulonglong2(f2_pack(y.z, y.z), f2_pack(y.w, y.w));
    }
    stage_tile_box(in, y.x, y.y, y.z, y.w);   // Yb holds scaled coordinates and lid
    const int cnt = min(kTileB, c1 - base);
#pragma unroll 1
    for (int sub = 0; sub * 32 < cnt; ++sub) {
    if (skip_ok && sub_tile_bound(wlo, whi, sub) < -kPruneExp) continue;   // warp-uniform
    const int i1 = min(cnt, sub * 32 + 32);
    evaluated += (unsigned long long)(i1 - sub * 32) * (unsigned long long)nvalid;
#pragma unroll 1
    for (int i = sub * 32; i < i1; ++i) {
      const ulonglong2 a = sY[i][0], b = sY[i][1];
#pragma unroll
      for (int p = 0; p < P; ++p) {
        const f2_t dx = f2_sub(tx[p], a.x), dy = f2_sub(ty[p], a.y), dz = f2_sub(tz[p], b.x);
        f2_t d2 = f2_mul(dx, dx);
        d2 = f2_fma(dy, dy, d2);
        d2 = f2_fma(dz, dz, d2);
        float e0, e1, q0, q1, yx, yy, yz, lid;
        f2_unpack(f2_sub(b.y, d2), e0, e1);
        f2_unpack(d2, q0, q1);
        f2_unpack(a.x, yx, lid);
        f2_unpack(a.y, yy, lid);
        f2_unpack(b.x, yz, lid);
        const float w0 = ex2_approx(e0), w1 = ex2_approx(e1);
        p1[2 * p] += w0;                         p1[2 * p + 1] += w1;
        px[2 * p] = fmaf(w0, yx, px[2 * p]);     px[2 * p + 1] = fmaf(w1, yx, px[2 * p + 1]);
        py[2 * p] = fmaf(w0, yy, py[2 * p]);     py[2 * p + 1] = fmaf(w1, yy, py[2 * p + 1]);
        pz[2 * p] = fmaf(w0, yz, pz[2 * p]);     pz[2 * p + 1] = fmaf(w1, yz, pz[2 * p + 1]);
        v[2 * p] = fmaf(w0, q0, v[2 * p]);       v[2 * p + 1] = fmaf(w1, q1, v[2 * p + 1]);
      }
    }
    }
  }
  const size_t plane = (size_t)gy * M;
#pragma unroll
  for (int p = 0; p < P; ++p)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int m = mbase + (2 * p + h) * 32;
      const int j = 2 * p + h;
      if (m < M) {
        const size_t o = (size_t)by * M + m;
        partB[o] = p1[j];
        partB[o + plane] = px[j];
        partB[o + 2 * plane] = py[j];
        partB[o + 3 * plane] = pz[j];
        partB[o + 4 * plane] = v[j];
      }
    }
  if (lane == 0 && evaluated) atomicAdd(&st->pairs_eval, evaluated);
}


__device__ __forceinline__ void passB_f64_body(const dvec4* FCPD_RESTRICT T4, int M, const dvec4* FCPD_RESTRICT Yb, int N,
          int cols_per_chunk, double* FCPD_RESTRICT partB, const DevState* FCPD_RESTRICT st, int gate, int bx, int by, int gx, int gy) {
  if (gate && iteration_gated(st)) return;
  __shared__ dvec4 sY[kTileB];
  const double inv2s2 = 1.0 / (2.0 * st->sigma2);
  const int mbase = bx * (kThreadsB * kRowsB64) + threadIdx.x;
  double tx[kRowsB64], ty[kRowsB64], tz[kRowsB64];
  double p1[kRowsB64], px[kRowsB64], py[kRowsB64], pz[kRowsB64], v[kRowsB64];
#pragma unroll
  for (int j = 0; j < kRowsB64; ++j) {
    const int m = mbase + j * kThreadsB;
    const dvec4 t = m < M ? T4[m] : dvec4{0, 0, 0, 0};
    tx[j] = t.x; ty[j] = t.y; tz[j] = t.z;
    p1[j] = px[j] = py[j] = pz[j] = v[j] = 0.0;
  }
  const int c0 = by * cols_per_chunk;
  const int c1 = min(N, c0 + cols_per_chunk);
  for (int base = c0; base < c1; base += kTileB) {
    __syncthreads();
    for (int i = threadIdx.x; i < kTileB; i += kThreadsB) {
      const int n = base + i;
      sY[i] = n < c1 ? Yb[n] : dvec4{0, 0, 0, 0};
    }
    __syncthreads();
    const int cnt = min(kTileB, c1 - base);
    for (int i = 0; i < cnt; ++i) {
      const dvec4 y = sY[i];
#pragma unroll
      for (int j = 0; j < kRowsB64; ++j) {
        const double dx = tx[j] - y.x, dy = ty[j] - y.y, dz = tz[j] - y.z;
        const double d2 = dx * dx + dy * dy + dz * dz;
        const double wv = exp(-d2 * inv2s2) * y.w;      // e_mn / den_n
        p1[j] += wv;
        px[j] += wv * y.x;
        py[j] += wv * y.y;
        pz[j] += wv * y.z;
        v[j] += wv * d2;
      }
    }
  }
  const size_t plane = (size_t)gy * M;
#pragma unroll
  for (int j = 0; j < kRowsB64; ++j) {
    const int m = mbase + j * kThreadsB;
    if (m < M) {
      const size_t o = (size_t)by * M + m;
      partB[o] = p1[j];
      partB[o + plane] = px[j];
      partB[o + 2 * plane] = py[j];
      partB[o + 3 * plane] = pz[j];
      partB[o + 4 * plane] = v[j];
    }
  }
}

// Writes the Eq. 5 outputs of row m from its (possibly rescaled) sums.
template <typename F>
__device__ __forceinline__ void write_row(int m, double p1s, double px, double py, double pz, double v,
                                          double unscale, double unscale2, const typename Vec<F>::t4& x,
                                          typename Vec<F>::t4* FCPD_RESTRICT Yt4,
                                          typename Vec<F>::t4* FCPD_RESTRICT R4, double* vrow_out) {
  const double inv = 1.0 / p1s;                       // one FP64 division per row
  const double yx = px * inv * unscale, yy = py * inv * unscale, yz = pz * inv * unscale;
  const double vrow = v * inv * unscale2;
  using V4 = typename Vec<F>::t4;
  V4 yt;
  yt.x = (F)yx; yt.y = (F)yy; yt.z = (F)yz; yt.w = (F)vrow;
  Yt4[m] = yt;
  if (R4) {
    V4 r;
    r.x = (F)(yx - (double)x.x); r.y = (F)(yy - (double)x.y); r.z = (F)(yz - (double)x.z); r.w = (F)0;
    R4[m] = r;
  }
  *vrow_out = vrow;
}

// --------------------------------------------- pass B reduction + Eq. 5
// Ytil_m = PY_m / P1_m (the corresponding constraint), V_m / P1_m =
// sum_n p^_mn |y_n - t_m|^2, R_m = Ytil_m - x_m.  FP64: a row whose mass is
// 0 or not finite cannot be normalised -> CPD_ENUMERIC.  FP32: rows whose
// mass is below 2^-90 are listed for the exact log-domain path.
// A block owns kRedRows rows; kRedRowSub threads per row each sum a strided
// subset of the chunks for the five quantities of that row (coalesced across
// rows), and the first thread of each row adds the subsets in order.
#ifndef FCPD_RED_ROWS
#define FCPD_RED_ROWS 32
#endif
constexpr int kRedRows = FCPD_RED_ROWS;
constexpr int kRedRowSub = kThreadsR / kRedRows;
static_assert(kRedRows * kRedRowSub == kThreadsR && kRedRows % 32 == 0, "rows per block: a multiple of 32 dividing the block");

template <typename F>
// Returns true in the block that completed the reduction over all gx blocks.
// skip_vsum: the EM iterations, which do not use the Eq. 18 sum of V_m / P1_m
// as such (each row carries its share to the M-step), skip its reduction.
// m_off: row of the first model point this launch reduces (pass B in row
// pieces: X4, Yt4, R4 and P1_out start at that row); the flagged-row list
// holds rows of the whole model.
__device__ __forceinline__ bool reduceB_body(const F* FCPD_RESTRICT partB, int chunks, int M, const typename Vec<F>::t4* FCPD_RESTRICT X4,
        typename Vec<F>::t4* FCPD_RESTRICT Yt4, typename Vec<F>::t4* FCPD_RESTRICT R4,
        double* FCPD_RESTRICT P1_out, double* FCPD_RESTRICT sums, int* FCPD_RESTRICT flag_rows,
        DevState* FCPD_RESTRICT st, int gate, int bx, int by, int gx, int gy, int skip_vsum = 0, int m_off = 0) {
  if (gate && iteration_gated(st)) return false;
  __shared__ double sh[32];
  __shared__ F part[kRedRowSub][5][kRedRows];
  __shared__ bool last;
  const int row = threadIdx.x % kRedRows, sub = threadIdx.x / kRedRows;
  const int m = bx * kRedRows + row;
  const size_t plane = (size_t)chunks * M;
  typename Vec<F>::t4 xm{};                   // x_m, in flight with the partial loads
  if (R4 && sub == 0 && m < M) xm = X4[m];
  F a[5] = {(F)0, (F)0, (F)0, (F)0, (F)0};   // summed in F, fixed order
  if (m < M) {
#pragma unroll 4
    for (int k = sub; k < chunks; k += kRedRowSub) {
      const size_t o = (size_t)k * M + m;
#pragma unroll
      for (int qn = 0; qn < 5; ++qn) a[qn] += __ldcg(partB + o + qn * plane);
    }
  }
#pragma unroll
  for (int qn = 0; qn < 5; ++qn) part[sub][qn][row] = a[qn];
  __syncthreads();
  double vrow = 0.0;
  int bad = 0;
  if (sub == 0 && m < M) {
    F f1 = 0, fx = 0, fy = 0, fz = 0, fv = 0;
#pragma unroll
    for (int j = 0; j < kRedRowSub; ++j) {
      f1 += part[j][0][row]; fx += part[j][1][row]; fy += part[j][2][row];
      fz += part[j][3][row]; fv += part[j][4][row];
    }
    double p1 = f1, px = fx, py = fy, pz = fz, v = fv;
    if constexpr (sizeof(F) == 4) {
      if (!(p1 >= kRowFloor) || !isfinite(p1)) {
        flag_rows[atomicAdd(&st->n_flag_rows, 1)] = m + m_off;
      } else {
        const float qi = 1.0f / scale_q(st->sigma2);
        write_row<F>(m, p1, px, py, pz, v, (double)qi, (double)qi * (double)qi, xm, Yt4, R4, &vrow);
        if (P1_out) P1_out[m] = p1;
      }
    } else {
      if (!(p1 > 0.0) || !isfinite(p1)) {
        bad = 1;
        p1 = 1.0;   // keep outputs finite; the status word reports the failure
      }
      write_row<F>(m, p1, px, py, pz, v, 1.0, 1.0, xm, Yt4, R4, &vrow);
      if (P1_out) P1_out[m] = bad ? 0.0 : p1;
    }
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicExch(&st->status, (int)CPD_ENUMERIC);
  if (skip_vsum) return false;
  const double bs = block_sum(vrow, sh);
  if (threadIdx.x == 0) {
    sums[bx] = bs;
    __threadfence();
    last = atomicAdd(&st->ticket_b, 1u) == gx - 1;
  }
  __syncthreads();
  if (last) {
    __threadfence();
    double vv = 0.0;
    for (int i = threadIdx.x; i < (int)gx; i += blockDim.x) vv += __ldcg(sums + i);
    const double tot = block_sum(vv, sh);
    if (threadIdx.x == 0) {
      st->vsum = tot;
      st->ticket_b = 0;
    }
  }
  return last;
}

// Exact FP32 rows in the log domain for the listed rows: with
// a = max_n (lid_n - d'^2_mn), every sum is taken over 2^(lid_n - d'^2 - a);
// the Eq. 5 ratios do not depend on the shift, and P1_m = 2^a * sum.
// Only listed rows in [m_lo, m_hi) are taken (pass B in row pieces: each
// piece's fix-up leaves the rows of the other pieces alone).
__device__ __forceinline__ void fixB_f32_body(const float4* FCPD_RESTRICT T4, int M, const float4* FCPD_RESTRICT Yb, int N,
         const float4* FCPD_RESTRICT X4, float4* FCPD_RESTRICT Yt4, float4* FCPD_RESTRICT R4,
         double* FCPD_RESTRICT P1_out, const int* FCPD_RESTRICT flag_rows, DevState* FCPD_RESTRICT st, int gate, int bx, int by, int gx, int gy,
         int m_lo = 0, int m_hi = 0x7fffffff) {
  if (gate && iteration_gated(st)) return;
  const int count = st->n_flag_rows;
  if (count == 0) return;
  const float q = scale_q(st->sigma2);
  const int lane = threadIdx.x & 31;
  const int nwarps = gx * (kThreadsF / 32);
  for (int j = bx * (kThreadsF / 32) + (threadIdx.x >> 5); j < count; j += nwarps) {
    const int m = flag_rows[j];
    if (m < m_lo || m >= m_hi) continue;     // another piece's row (same for the whole warp)
    const float4 t = T4[m];
    const float tx = q * t.x, ty = q * t.y, tz = q * t.z;
    float amax = -INFINITY;
    for (int n = lane; n < N; n += 32) {
      const float4 y = Yb[n];
      const float dx = tx - y.x, dy = ty - y.y, dz = tz - y.z;
      float d2 = dx * dx;
      d2 = fmaf(dy, dy, d2);
      d2 = fmaf(dz, dz, d2);
      amax = fmaxf(amax, y.w - d2);
    }
    amax = warp_max(amax);
    float p1 = 0.f, px = 0.f, py = 0.f, pz = 0.f, v = 0.f;
    for (int n = lane; n < N; n += 32) {
      const float4 y = Yb[n];
      const float dx = tx - y.x, dy = ty - y.y, dz = tz - y.z;
      float d2 = dx * dx;
      d2 = fmaf(dy, dy, d2);
      d2 = fmaf(dz, dz, d2);
      const float wv = ex2_approx(y.w - d2 - amax);
      p1 += wv;
      px = fmaf(wv, y.x, px);
      py = fmaf(wv, y.y, py);
      pz = fmaf(wv, y.z, pz);
      v = fmaf(wv, d2, v);
    }
    p1 = warp_sumf(p1); px = warp_sumf(px); py = warp_sumf(py); pz = warp_sumf(pz); v = warp_sumf(v);
    if (lane == 0) {
      const double mass = (double)p1 * exp2((double)amax);
      if (!(mass > 0.0) || !isfinite(mass)) {
        atomicExch(&st->status, (int)CPD_ENUMERIC);    // zero even in double precision
      } else {
        const float qi = 1.0f / q;
        double vrow = 0.0;
        const float4 xf = R4 ? X4[m] : float4{};
        write_row<float>(m, (double)p1, px, py, pz, v, (double)qi, (double)qi * (double)qi, xf, Yt4, R4, &vrow);
        if (P1_out) P1_out[m] = mass;
        atomicAdd(&st->vsum, vrow);
      }
    }
  }
}

}  // namespace dev
}  // namespace fcpd
