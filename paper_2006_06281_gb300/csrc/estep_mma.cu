// E-step passes with tensor-core distance tiles (mixed-precision mode).
//
// The exponent of every Gaussian of a 16 x 8 tile of (row point, column
// point) pairs is one warp-level FP16 tensor-core product with FP32
// accumulation (mma.sync m16n8k16, K = 16):
//     e = 2 r'.c' - |r'|^2 - |c'|^2 (+ lid_c in pass B)
// over the coordinates pre-scaled by q = sqrt(log2(e) / (2 sigma2)), so
// e = -|r' - c'|^2 (+ lid) is the base-2 exponent the FP32 passes compute
// directly.  Each FP32 value v is split into two FP16 parts v1 + v2 (22
// significant bits); the cross products v1w1, v1w2, v2w1 are kept (v2w2 is
// 2^-22 of the product), the norms and lid enter as split terms against an
// exact 1:
//   k  0..8   row side 2 r_d^(i)           col side c_d^(j)   (d, (i, j) in (1,1) (1,2) (2,1))
//   k  9..10  row side -|r'|^2 (split)     col side 1
//   k 11..12  row side 1                   col side -|c'|^2 (split)
//   k 13..14  row side 1                   col side lid (split; 0 in pass A)
//   k 15      0
// Products of FP16 values are exact in FP32; what remains is the FP32
// accumulation of terms as large as |r'|^2 and the 2^-22 split residue,
// both growing with 1 / sigma2 -- so these passes run only while sigma2 >=
// mma_s2min (see kMmaS2PerR2; there q^2 R^2 <= ~2000, well inside FP16's
// range), and the FP32 direct passes take over below it (both are in every
// captured iteration; each steps aside on the device-side test).  The
// exponentials and sums are the FP32 passes' own: ex2.approx.ftz, FP32
// accumulation, split partials reduced in a fixed order.  (A first version
// with three BF16 parts and K = 32 measured the legacy tensor pipe 44 %
// busy in pass A: halving K moves the bound to the exponentials.)
#include "estep_dev.cuh"

#include <cuda_fp16.h>

#include <algorithm>

namespace fcpd {

namespace {

using namespace dev;

constexpr int kMmaThreads = 256;            // 8 warps
constexpr int kMmaTilesPerWarp = 2;         // 16-point row tiles per warp
constexpr int kMmaRowsPerBlock = 8 * 16 * kMmaTilesPerWarp;   // 256 row points per block
constexpr int kMmaStage = 128;              // column points staged per shared tile
constexpr int kAugK = 16;                   // augmented dimension
constexpr int kAugStride = 24;              // halves per staged vector (48 bytes: conflict-free ldmatrix)
constexpr float kPadNorm = -60000.f;        // padding column: exponents far below -126, finite in FP16
static_assert(kAugStride >= kAugK && (kAugStride * 2) % 16 == 0, "staged vectors: K halves, 16-byte rows");

// Row-side and column-side augmented vectors (FP16) of a scaled point.
__device__ __forceinline__ void split2(float v, __half& a, __half& b) {
  a = __float2half_rn(v);
  b = __float2half_rn(v - __half2float(a));
}

// (row part, column part) of the three kept cross products
__device__ __forceinline__ int row_part(int p) { return p == 2 ? 1 : 0; }
__device__ __forceinline__ int col_part(int p) { return p == 1 ? 1 : 0; }

__device__ __forceinline__ void row_vector(float x, float y, float z, bool valid, __half* out) {
  __half s[3][2], nn[2];
  const float v[3] = {x, y, z};
#pragma unroll
  for (int d = 0; d < 3; ++d) split2(valid ? 2.0f * v[d] : 0.f, s[d][0], s[d][1]);
  split2(valid ? -(x * x + y * y + z * z) : 0.f, nn[0], nn[1]);
  const __half one = __float2half_rn(1.0f), zero = __float2half_rn(0.0f);
#pragma unroll
  for (int d = 0; d < 3; ++d)
#pragma unroll
    for (int p = 0; p < 3; ++p) out[3 * d + p] = s[d][row_part(p)];
  out[9] = nn[0]; out[10] = nn[1];
#pragma unroll
  for (int k = 11; k < 15; ++k) out[k] = one;
  out[15] = zero;
}

// Column side; an invalid (padding) point gets a large negative norm so its
// exponents are far below -126 (its Gaussians are exactly 0).
__device__ __forceinline__ void col_vector(float x, float y, float z, float lid, bool valid, __half* out) {
  __half s[3][2], nn[2], ll[2];
  const float v[3] = {x, y, z};
#pragma unroll
  for (int d = 0; d < 3; ++d) split2(valid ? v[d] : 0.f, s[d][0], s[d][1]);
  split2(valid ? -(x * x + y * y + z * z) : kPadNorm, nn[0], nn[1]);
  split2(valid ? lid : 0.f, ll[0], ll[1]);
  const __half one = __float2half_rn(1.0f), zero = __float2half_rn(0.0f);
#pragma unroll
  for (int d = 0; d < 3; ++d)
#pragma unroll
    for (int p = 0; p < 3; ++p) out[3 * d + p] = s[d][col_part(p)];
  out[9] = one; out[10] = one;
  out[11] = nn[0]; out[12] = nn[1];
  out[13] = ll[0]; out[14] = ll[1];
  out[15] = zero;
}

__device__ __forceinline__ unsigned int smem_u32(const void* p) {
  return (unsigned int)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void ldsm_x4(unsigned int addr, unsigned int& r0, unsigned int& r1, unsigned int& r2,
                                        unsigned int& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}

// D = A B: 16 x 8 FP32 from FP16 A (16 x 16, row) and B (16 x 8, col).
__device__ __forceinline__ void mma_f16(const unsigned int (&a)[4], unsigned int b0, unsigned int b1, float (&d)[4]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%10, %11, %12, %13};"
      : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1), "f"(0.f), "f"(0.f), "f"(0.f), "f"(0.f));
}

// Row fragments of a warp: tiles of 16 row points staged as augmented
// vectors in shared memory; A fragments (two K-steps) via ldmatrix.x4.
__device__ __forceinline__ void load_row_frags(const __half (*sRow)[kAugStride], int tile0,
                                               unsigned int (&a)[kMmaTilesPerWarp][4]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int g = 0; g < kMmaTilesPerWarp; ++g) {
    // matrices: (rows 0-7, k 0-7), (rows 8-15, k 0-7), (rows 0-7, k 8-15), (rows 8-15, k 8-15)
    const int mat = lane >> 3, r = lane & 7;
    const int row = 16 * (tile0 + g) + (mat & 1) * 8 + r;
    const int k = (mat >> 1) * 8;
    ldsm_x4(smem_u32(&sRow[row][k]), a[g][0], a[g][1], a[g][2], a[g][3]);
  }
}

// B fragments of two groups of 8 column points (j, j + 8): matrices (cols
// j.., k 0-7), (cols j.., k 8-15), (cols j+8.., k 0-7), (cols j+8.., k 8-15).
__device__ __forceinline__ void load_col_frags(const __half (*sCol)[kAugStride], int j, unsigned int& b00,
                                               unsigned int& b01, unsigned int& b10, unsigned int& b11) {
  const int lane = threadIdx.x & 31;
  const int mat = lane >> 3;
  ldsm_x4(smem_u32(&sCol[j + 8 * (mat >> 1) + (lane & 7)][8 * (mat & 1)]), b00, b01, b10, b11);
}

// ------------------------------------------------------------------ pass A
// Rows: scene points (block: kMmaRowsPerBlock of them); columns: model
// points of the block's row chunk, staged kMmaStage at a time.  Writes the
// split column sums partA[chunk][n] like the FP32 pass A.
__global__ void __launch_bounds__(kMmaThreads)
passA_f32_mma(const float4* __restrict__ T4, int M, int rows_per_chunk, const float4* __restrict__ Y4, int N,
              float* __restrict__ partA, DevState* __restrict__ st, int gate) {
  if ((gate && iteration_gated(st)) || !mma_active(st)) return;
  __shared__ __align__(16) __half sRow[kMmaRowsPerBlock][kAugStride];
  __shared__ __align__(16) __half sCol[kMmaStage][kAugStride];
  const float q = scale_q(st->sigma2);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n0 = blockIdx.x * kMmaRowsPerBlock;
  for (int i = threadIdx.x; i < kMmaRowsPerBlock; i += kMmaThreads) {
    const int n = n0 + i;
    float4 y = make_float4(0.f, 0.f, 0.f, 0.f);
    if (n < N) y = Y4[n];
    row_vector(q * y.x, q * y.y, q * y.z, n < N, sRow[i]);
  }
  __syncthreads();
  unsigned int a[kMmaTilesPerWarp][4];
  load_row_frags(sRow, warp * kMmaTilesPerWarp, a);
  float acc[kMmaTilesPerWarp][2];
#pragma unroll
  for (int g = 0; g < kMmaTilesPerWarp; ++g) acc[g][0] = acc[g][1] = 0.f;
  const int r0 = blockIdx.y * rows_per_chunk;
  const int r1 = min(M, r0 + rows_per_chunk);
  for (int base = r0; base < r1; base += kMmaStage) {
    __syncthreads();
    for (int i = threadIdx.x; i < kMmaStage; i += kMmaThreads) {
      const int m = base + i;
      float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
      if (m < r1) t = T4[m];
      col_vector(q * t.x, q * t.y, q * t.z, 0.f, m < r1, sCol[i]);
    }
    __syncthreads();
    const int cnt = min(kMmaStage, r1 - base);
#pragma unroll 1
    for (int j = 0; j < cnt; j += 16) {       // staged tiles are whole multiples of 16 points
      unsigned int b[2][2];
      load_col_frags(sCol, j, b[0][0], b[0][1], b[1][0], b[1][1]);
#pragma unroll
      for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int g = 0; g < kMmaTilesPerWarp; ++g) {
          float d[4];
          mma_f16(a[g], b[c][0], b[c][1], d);
          acc[g][0] += ex2_approx(d[0]) + ex2_approx(d[1]);   // row lane/4, columns 2(lane%4), +1
          acc[g][1] += ex2_approx(d[2]) + ex2_approx(d[3]);   // row lane/4 + 8
        }
    }
  }
  // the four lanes of a quad hold the same rows: add their column subsets
#pragma unroll
  for (int g = 0; g < kMmaTilesPerWarp; ++g)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float v = acc[g][h];
      v += __shfl_xor_sync(0xffffffffu, v, 1);
      v += __shfl_xor_sync(0xffffffffu, v, 2);
      const int n = n0 + 16 * (warp * kMmaTilesPerWarp + g) + 8 * h + (lane >> 2);
      if ((lane & 3) == 0 && n < N) partA[(size_t)blockIdx.y * N + n] = v;
    }
}

// ------------------------------------------------------------------ pass B
// Rows: model points; columns: scene points of the block's column chunk
// (scaled coordinates and lid from Yb).  Writes partB like the FP32 pass B
// (P1, PY x 3, V = sum_n w d'^2 with d'^2 = lid - e).
__global__ void __launch_bounds__(kMmaThreads)
passB_f32_mma(const float4* __restrict__ T4, int M, const float4* __restrict__ Yb, int N, int cols_per_chunk,
              float* __restrict__ partB, DevState* __restrict__ st, int gate) {
  if ((gate && iteration_gated(st)) || !mma_active(st)) return;
  // the column list was consumed by fixA and the row list is filled after
  // this pass (as in the FP32 pass B)
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
    st->n_flag_cols = 0;
    st->n_flag_rows = 0;
  }
  __shared__ __align__(16) __half sRow[kMmaRowsPerBlock][kAugStride];
  __shared__ __align__(16) __half sCol[kMmaStage][kAugStride];
  __shared__ float4 sY[kMmaStage];
  const float q = scale_q(st->sigma2);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * kMmaRowsPerBlock;
  for (int i = threadIdx.x; i < kMmaRowsPerBlock; i += kMmaThreads) {
    const int m = m0 + i;
    float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
    if (m < M) t = T4[m];
    row_vector(q * t.x, q * t.y, q * t.z, m < M, sRow[i]);
  }
  __syncthreads();
  unsigned int a[kMmaTilesPerWarp][4];
  load_row_frags(sRow, warp * kMmaTilesPerWarp, a);
  // per row (h: lane/4, lane/4 + 8): P1, PX, PY, PZ, V over the thread's
  // columns (scalar: packing two MUFU results would cost moves)
  float p1[kMmaTilesPerWarp][2], px[kMmaTilesPerWarp][2], py[kMmaTilesPerWarp][2], pz[kMmaTilesPerWarp][2],
      v[kMmaTilesPerWarp][2];
#pragma unroll
  for (int g = 0; g < kMmaTilesPerWarp; ++g)
#pragma unroll
    for (int h = 0; h < 2; ++h) p1[g][h] = px[g][h] = py[g][h] = pz[g][h] = v[g][h] = 0.f;
  const int c0 = blockIdx.y * cols_per_chunk;
  const int c1 = min(N, c0 + cols_per_chunk);
  for (int base = c0; base < c1; base += kMmaStage) {
    __syncthreads();
    for (int i = threadIdx.x; i < kMmaStage; i += kMmaThreads) {
      const int n = base + i;
      float4 y = make_float4(0.f, 0.f, 0.f, 0.f);
      if (n < c1) y = Yb[n];           // q-scaled coordinates, lid = -log2 den_n
      sY[i] = y;
      col_vector(y.x, y.y, y.z, y.w, n < c1, sCol[i]);
    }
    __syncthreads();
    const int cnt = min(kMmaStage, c1 - base);
#pragma unroll 1
    for (int j = 0; j < cnt; j += 16) {       // staged tiles are whole multiples of 16 points
      unsigned int b[2][2];
      load_col_frags(sCol, j, b[0][0], b[0][1], b[1][0], b[1][1]);
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        // columns of d[0]/d[2] and d[1]/d[3]
        const float4 ya = sY[j + 8 * c + 2 * (lane & 3)], yb = sY[j + 8 * c + 2 * (lane & 3) + 1];
#pragma unroll
        for (int g = 0; g < kMmaTilesPerWarp; ++g) {
          float d[4];
          mma_f16(a[g], b[c][0], b[c][1], d);
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const float w0 = ex2_approx(d[2 * h]), w1 = ex2_approx(d[2 * h + 1]);   // e_mn / den_n
            p1[g][h] += w0;
            p1[g][h] += w1;
            px[g][h] = fmaf(w1, yb.x, fmaf(w0, ya.x, px[g][h]));
            py[g][h] = fmaf(w1, yb.y, fmaf(w0, ya.y, py[g][h]));
            pz[g][h] = fmaf(w1, yb.z, fmaf(w0, ya.z, pz[g][h]));
            v[g][h] = fmaf(w1, yb.w - d[2 * h + 1], fmaf(w0, ya.w - d[2 * h], v[g][h]));   // d'^2 = lid - e
          }
        }
      }
    }
  }
  const size_t plane = (size_t)gridDim.y * M;
#pragma unroll
  for (int g = 0; g < kMmaTilesPerWarp; ++g)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float s[5] = {p1[g][h], px[g][h], py[g][h], pz[g][h], v[g][h]};
#pragma unroll
      for (int qn = 0; qn < 5; ++qn) {
        s[qn] += __shfl_xor_sync(0xffffffffu, s[qn], 1);
        s[qn] += __shfl_xor_sync(0xffffffffu, s[qn], 2);
      }
      const int m = m0 + 16 * (warp * kMmaTilesPerWarp + g) + 8 * h + (lane >> 2);
      if ((lane & 3) == 0 && m < M) {
        const size_t o = (size_t)blockIdx.y * M + m;
#pragma unroll
        for (int qn = 0; qn < 5; ++qn) partB[o + qn * plane] = s[qn];
      }
    }
}

__global__ void __launch_bounds__(1024) mma_threshold(const float4* __restrict__ X4, int M, const float4* __restrict__ Y4,
                                                     int N, DevState* __restrict__ st) {
  __shared__ float sh[32];
  float r2 = 0.f;
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    const float4 p = X4[i];
    r2 = fmaxf(r2, p.x * p.x + p.y * p.y + p.z * p.z);
  }
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const float4 p = Y4[i];
    r2 = fmaxf(r2, p.x * p.x + p.y * p.y + p.z * p.z);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) r2 = fmaxf(r2, __shfl_xor_sync(0xffffffffu, r2, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = r2;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r2 = fmaxf(r2, sh[w]);
    r2 = fmaxf(r2, sh[0]);
    // the deformation moves T by a fraction of the extent: a 25 % margin
    st->mma_s2min = kMmaS2PerR2 * 1.25 * (double)r2;
  }
}

int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace

void launch_mma_threshold(const float4* X4, int64_t M, const float4* Y4, int64_t N, DevState* st, cudaStream_t s) {
  mma_threshold<<<1, 1024, 0, s>>>(X4, (int)M, Y4, (int)N, st);
}

// Grids of the tensor-core passes: rows in blocks of 256 points, the other
// dimension split into chunks (multiples of the 16-point tile) chosen so the
// blocks fill whole waves of the pass's own occupancy: the cost of a split is
// its number of waves x (chunk length + a per-block overhead), and the
// cheapest split wins (fewer chunks on ties, so fewer partial sums).
namespace {
void split_fill(int64_t L, int64_t tiles, int64_t slots, int& len, int& chunks) {
  constexpr int64_t kGran = 16, kMinLen = 64, kOverhead = 32;
  int64_t best = -1;
  const int64_t cmax = 4 * std::max<int64_t>(1, slots / tiles) + 2;
  for (int64_t c = 1; c <= cmax; ++c) {
    const int64_t ln = std::max(kMinLen, cdiv(cdiv(L, c), kGran) * kGran);
    const int64_t ch = cdiv(L, ln);
    const int64_t cost = cdiv(tiles * ch, slots) * (ln + kOverhead);
    if (best < 0 || cost < best) {
      best = cost;
      len = (int)ln;
      chunks = (int)ch;
    }
  }
}
}  // namespace

void plan_estep_mma(int64_t M, int64_t N, int sms, MmaPlan& p) {
  int occA = 0, occB = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occA, passA_f32_mma, kMmaThreads, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occB, passB_f32_mma, kMmaThreads, 0);
  p.a_row_tiles = (int)cdiv(N, kMmaRowsPerBlock);
  split_fill(M, p.a_row_tiles, (int64_t)sms * std::max(occA, 1), p.a_rows_per_chunk, p.a_chunks);
  p.b_row_tiles = (int)cdiv(M, kMmaRowsPerBlock);
  split_fill(N, p.b_row_tiles, (int64_t)sms * std::max(occB, 1), p.b_cols_per_chunk, p.b_chunks);
}

void launch_passA_mma(const MmaPlan& p, const float4* T4, int64_t M, const float4* Y4, int64_t N, float* partA,
                      DevState* st, int gate, cudaStream_t s) {
  passA_f32_mma<<<dim3(p.a_row_tiles, p.a_chunks), kMmaThreads, 0, s>>>(T4, (int)M, p.a_rows_per_chunk, Y4,
                                                                         (int)N, partA, st, gate);
}

void launch_passB_mma(const MmaPlan& p, const float4* T4, int64_t M, const float4* Yb, int64_t N, float* partB,
                      DevState* st, int gate, cudaStream_t s) {
  passB_f32_mma<<<dim3(p.b_row_tiles, p.b_chunks), kMmaThreads, 0, s>>>(T4, (int)M, Yb, (int)N, p.b_cols_per_chunk,
                                                                         partB, st, gate);
}

}  // namespace fcpd
