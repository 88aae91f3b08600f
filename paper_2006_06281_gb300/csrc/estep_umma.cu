// E-step passes with tcgen05 distance tiles (mixed-precision mode, Eq. 4-5).
//
// The base-2 exponent of every Gaussian of a 128 x 128 tile of (row point,
// column point) pairs is one tcgen05.mma (kind::f16, M = 128, N = 128, K = 16)
// of the points' augmented FP16 vectors (estep_aug.cuh: 2 r'.c' - |r'|^2 -
// |c'|^2 + lid over the q-scaled coordinates, FP32 accumulation), written to
// tensor memory; the epilogue warps read it with tcgen05.ld, one row per
// thread, and spend their issue slots on the per-pair exponential and sums
// only.  The arithmetic, its error and its sigma2 floor are those of the
// augmented vectors; the exponentials (ex2.approx.ftz) and FP32 sums are the
// FP32 passes', and the split partials have their layout, so the reductions
// that follow are shared.
//
//   pass A   rows: 128 scene points y_n; columns: model points t_m of the
//            CTA's chunk; thread (row n) sums 2^e over its columns -> den_n
//            partial (partA[chunk][n]).
//   pass B   rows: 128 model points; columns: scene points of the chunk with
//            lid_n = -log2 den_n folded into the vector; thread (row m) sums
//            w = 2^e, w y_n (3) and w (lid_n - e) = w d'^2 -> P1, PY, V
//            partials (partB, five planes).
//
// CTA: 8 epilogue warps (warp w reads TMEM lanes 32 (w % 4).. and columns
// 64 (w / 4).. of each tile) and one control warp (its lane 0 issues the bulk
// copies of the chunk's column vectors -- prepared for the whole point set by
// prep_cols -- and the MMAs).  Two TMEM accumulators of 128 columns each: the
// MMA of tile j + 1 runs while the epilogue reads tile j (mbarriers tfull /
// tempty).  Operand tiles in shared memory are K-major without swizzle:
// 8-row x 16-byte core matrices, the two K halves of a group of 8 points 128
// bytes apart, groups 256 bytes apart.  Every wait is bounded in wall time;
// on expiry the CTA records CPD_ETIMEOUT, waits (bounded) for its copies and
// MMAs in flight, frees its TMEM and returns.
#include "estep_dev.cuh"
#include "estep_aug.cuh"
#include "tc05.cuh"

#include <algorithm>

namespace fcpd {

namespace {

using namespace dev;
using namespace tc05;

constexpr int kEThreads = 288;              // 8 epilogue warps + 1 control warp
constexpr int kEWarps = 8;
constexpr int kETile = 128;                 // points per operand tile (rows = TMEM lanes, columns)
constexpr int kETileBytes = kETile * 32;    // 128 augmented vectors of 16 FP16 values
constexpr int kEMaxTilesA = 24;             // column tiles per CTA chunk, pass A (96 KB)
constexpr int kEMaxTilesB = 16;             // pass B (64 KB + 32 KB of scene records)
constexpr uint32_t kETmemCols = 256;        // two accumulators of 128 columns
constexpr unsigned long long kEWaitNs = 2000000000ull;

// Byte offset of the 16-byte half h (K values 8h..8h+7) of point r of a tile
// in the no-swizzle K-major core-matrix layout.
__host__ __device__ constexpr int aug_offset(int r, int h) { return (r >> 3) * 256 + h * 128 + (r & 7) * 16; }

__device__ __forceinline__ void store_aug(unsigned char* tile, int r, const __half (&v)[kAugK]) {
  const uint4* src = reinterpret_cast<const uint4*>(v);
  *reinterpret_cast<uint4*>(tile + aug_offset(r, 0)) = src[0];
  *reinterpret_cast<uint4*>(tile + aug_offset(r, 1)) = src[1];
}

// Column vectors of all points, tile by tile (n_pad = points rounded up to
// 128; points >= n are padding with Gaussians exactly 0).  scene = 0: model
// points T4 (scaled by q here, lid 0, pass A); scene = 1: scene records Yb
// (already {q y, lid}, pass B), which are also copied to `rec` pair by pair
// for pass B's packed epilogue: points 2p, 2p+1 as {x x', y y'} {z z', l l'}
// (zero for padding).
__global__ void __launch_bounds__(256)
prep_cols(const float4* __restrict__ P4, int n, int n_pad, int scene, DevState* __restrict__ st, int gate,
          unsigned char* __restrict__ out, float* __restrict__ rec) {
  if ((gate && iteration_gated(st)) || !mma_active(st)) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_pad) return;
  const bool valid = i < n;
  float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
  if (valid) p = P4[i];
  float x = p.x, y = p.y, z = p.z, lid = p.w;
  if (!scene) {
    const float q = scale_q(st->sigma2);
    x *= q; y *= q; z *= q; lid = 0.f;
  }
  __align__(16) __half v[kAugK];
  col_vector(x, y, z, lid, valid, v);
  store_aug(out + (size_t)(i / kETile) * kETileBytes, i % kETile, v);
  if (rec) {
    float* r = rec + (size_t)(i >> 1) * 8 + (i & 1);
    r[0] = valid ? x : 0.f;
    r[2] = valid ? y : 0.f;
    r[4] = valid ? z : 0.f;
    r[6] = valid ? lid : 0.f;
  }
}

// Bounded wait made uniform across a warp (the tcgen05.ld that follows is
// warp-collective): if any lane saw the phase complete, every lane does.
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity) {
  bool ok = mbar_wait(bar, parity, kEWaitNs);
  if (__any_sync(0xffffffffu, ok) && !ok) ok = mbar_wait(bar, parity, 1000000ull);
  return __all_sync(0xffffffffu, ok);
}

template <int PASS> __host__ __device__ constexpr int max_tiles() { return PASS == 0 ? kEMaxTilesA : kEMaxTilesB; }
// Row tiles per CTA and columns per MMA: pass A one 128-row tile, 128
// columns; pass B two row tiles (256 model points) and 64 columns, so each
// scene record an epilogue thread reads from shared memory serves two rows.
// Either way an accumulator buffer is 128 TMEM columns.
template <int PASS> __host__ __device__ constexpr int row_tiles() { return PASS == 0 ? 1 : 2; }
template <int PASS> __host__ __device__ constexpr int mma_cols() { return PASS == 0 ? 128 : 64; }
template <int PASS> constexpr size_t pass_smem_bytes() {
  return 1024 + (size_t)row_tiles<PASS>() * kETileBytes + (size_t)max_tiles<PASS>() * kETileBytes +
         (PASS == 1 ? (size_t)kEMaxTilesB * kETile * sizeof(float4) : 0) + 64 * sizeof(uint64_t);
}
__host__ __device__ constexpr uint32_t idesc_m128(int n) {
  return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

// One pass (PASS 0: A, 1: B).  Rows4: the row points (A: scene Y4, B: model
// T4), cols: prep_cols output for the column points, recs (pass B): the
// scene records paired by prep_cols, read by the epilogue.  Grid: (row blocks of
// 128 row_tiles points, column chunks of `tpc` 128-point tiles).  Writes
// partA[chunk][n] or the five partB planes.
template <int PASS>
__global__ void __launch_bounds__(kEThreads, 2)
pass_umma(const float4* __restrict__ Rows4, int n_rows, const unsigned char* __restrict__ cols, int n_cols,
          const float4* __restrict__ recs, int tpc, float* __restrict__ part, DevState* __restrict__ st, int gate) {
  constexpr int RT = row_tiles<PASS>();
  constexpr int NC = mma_cols<PASS>();
  constexpr int SUB = kETile / NC;                      // MMA column tiles per 128-point operand tile
  constexpr int WC = NC / 2;                            // columns per epilogue warp per row tile
  constexpr uint32_t IDESC = idesc_m128(NC);
  if ((gate && iteration_gated(st)) || !mma_active(st)) return;
  if (PASS == 1 && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
    // the column list was consumed by fixA; the row list is filled after this pass
    st->n_flag_cols = 0;
    st->n_flag_rows = 0;
  }
  extern __shared__ unsigned char smem_raw[];
  // 1024-byte aligned, by an offset from the shared array (an integer round
  // trip would turn later accesses into generic ones)
  unsigned char* smem = smem_raw + ((1024u - (saddr(smem_raw) & 1023u)) & 1023u);
  unsigned char* sA = smem;
  unsigned char* sB = smem + (size_t)RT * kETileBytes;
  float4* sY = reinterpret_cast<float4*>(sB + (size_t)max_tiles<PASS>() * kETileBytes);
  uint64_t* bfull = reinterpret_cast<uint64_t*>(reinterpret_cast<unsigned char*>(sY) +
                                                (PASS == 1 ? (size_t)kEMaxTilesB * kETile * sizeof(float4) : 0));
  uint64_t* tfull = bfull + max_tiles<PASS>();
  uint64_t* tempty = tfull + 2;
  uint64_t* mdone = tempty + 2;
  uint64_t* yfull = mdone + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(yfull + 1);
  __shared__ float red[5][RT * kETile];
  __shared__ volatile int s_fail;
  __shared__ int s_issued;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntc = (n_cols + kETile - 1) / kETile;           // column tiles of the whole point set
  const int c0t = blockIdx.y * tpc;
  const int nt = max(0, min(ntc, c0t + tpc) - c0t);          // >= 1 by the plan
  const int njt = nt * SUB;                                 // MMA column tiles
  const int ncol0 = c0t * kETile;
  const int nvalid = max(0, min(n_cols, ncol0 + nt * kETile) - ncol0);

  if (threadIdx.x == 0) {
    s_fail = 0;
    s_issued = 0;
    for (int j = 0; j < nt; ++j) mbar_init(&bfull[j], 1);
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], kEWarps);
    }
    mbar_init(mdone, 1);
    mbar_init(yfull, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(tmem_slot, kETmemCols);
  // row vectors of the CTA's row points (generic-proxy writes, fenced for
  // the tensor core's async-proxy reads)
  const float q = scale_q(st->sigma2);
  const int row0 = blockIdx.x * (RT * kETile);
  if (threadIdx.x < RT * kETile) {
    const int r = row0 + threadIdx.x;
    float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
    if (r < n_rows) p = Rows4[r];
    __align__(16) __half v[kAugK];
    row_vector(q * p.x, q * p.y, q * p.z, r < n_rows, v);
    store_aug(sA + (size_t)(threadIdx.x / kETile) * kETileBytes, threadIdx.x % kETile, v);
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  f2_t acc2[RT][5];      // packed sums over even / odd columns
#pragma unroll
  for (int t = 0; t < RT; ++t)
#pragma unroll
    for (int k = 0; k < 5; ++k) acc2[t][k] = f2_pack(0.f, 0.f);
  if (warp == kEWarps) {
    if (lane == 0) {
      // copies of the chunk's column vectors (and, pass B, its scene records)
      if (PASS == 1 && nvalid > 0) {   // whole tiles: the padding records are zero
        mbar_expect_tx(yfull, (uint32_t)nt * kETile * 16u);
        bulk_load(sY, recs + ncol0, (uint32_t)nt * kETile * 16u, yfull);
      }
      for (int j = 0; j < nt; ++j) {
        mbar_expect_tx(&bfull[j], (uint32_t)kETileBytes);
        bulk_load(sB + (size_t)j * kETileBytes, cols + (size_t)(c0t + j) * kETileBytes, (uint32_t)kETileBytes,
                  &bfull[j]);
      }
      s_issued = nt;
      // per MMA column tile, one MMA per row tile into the accumulator the
      // epilogue released (row tile t at columns t NC of the buffer)
      for (int j = 0; j < njt; ++j) {
        const int b = j & 1;
        if (s_fail) break;
        if ((j >= 2 && !mbar_wait(&tempty[b], (uint32_t)((j >> 1) - 1) & 1u, kEWaitNs)) ||
            !mbar_wait(&bfull[j / SUB], 0, kEWaitNs)) {
          s_fail = 1;
          break;
        }
        fence_after();
        const uint64_t bdesc = smem_desc_noswz(saddr(sB + (size_t)(j / SUB) * kETileBytes + (j % SUB) * (NC * 32)),
                                               128, 256);
#pragma unroll
        for (int t = 0; t < RT; ++t)
          umma_f16(tmem + (uint32_t)(b * kETile + t * NC), smem_desc_noswz(saddr(sA + (size_t)t * kETileBytes), 128, 256),
                   bdesc, IDESC, 0u);
        umma_commit(&tfull[b]);
      }
      umma_commit(mdone);       // arrives once every MMA issued above has completed
    }
  } else {
    const int quarter = warp & 3, half = warp >> 2;
    const uint32_t lanes = (uint32_t)(quarter * 32) << 16;
    bool ok = true;
    if (PASS == 1 && nvalid > 0) ok = warp_wait(yfull, 0);
    for (int j = 0; j < njt && ok; ++j) {
      const int b = j & 1;
      if (!warp_wait(&tfull[b], (uint32_t)(j >> 1) & 1u)) {
        ok = false;
        break;
      }
      fence_after();
      const uint32_t ta = tmem + lanes + (uint32_t)(b * kETile + half * WC);
      if (PASS == 0) {
        // this warp's 64 columns into registers, the accumulator back to the
        // MMA at once, then column pairs on packed FP32 (one add per two
        // Gaussians)
        uint32_t e0[32], e1[32];
        tmem_ld32_nowait(ta, e0);
        tmem_ld32_nowait(ta + 32u, e1);
        tmem_wait();
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[b]);
#pragma unroll
        for (int i = 0; i < 64; i += 2) {
          const float ea = __uint_as_float(i < 32 ? e0[i] : e1[i - 32]);
          const float eb = __uint_as_float(i < 32 ? e0[i + 1] : e1[i - 31]);
          acc2[0][(i >> 1) & 1] = f2_add(acc2[0][(i >> 1) & 1], f2_pack(ex2_approx(ea), ex2_approx(eb)));
        }
      } else {
        // 16 columns of both row tiles at a time (the other accumulator keeps
        // the MMA busy meanwhile), column pairs on packed FP32; every record
        // pair (two 16-byte broadcasts) serves both rows of the thread
        const ulonglong2* ys2 = reinterpret_cast<const ulonglong2*>(sY) + (size_t)j * NC + half * WC;
#pragma unroll
        for (int c = 0; c < WC / 16; ++c) {
          uint32_t e0[16], e1[16];
          tmem_ld16_nowait(ta + (uint32_t)(c * 16), e0);
          tmem_ld16_nowait(ta + (uint32_t)(NC + c * 16), e1);
          tmem_wait();
#pragma unroll
          for (int i = 0; i < 16; i += 2) {
            const ulonglong2 a = ys2[c * 16 + i], cc = ys2[c * 16 + i + 1];   // {x x', y y'}, {z z', l l'}
#pragma unroll
            for (int t = 0; t < RT; ++t) {
              const float ea = __uint_as_float(t == 0 ? e0[i] : e1[i]);
              const float eb = __uint_as_float(t == 0 ? e0[i + 1] : e1[i + 1]);
              const f2_t w = f2_pack(ex2_approx(ea), ex2_approx(eb));   // e_mn / den_n
              acc2[t][0] = f2_add(acc2[t][0], w);
              acc2[t][1] = f2_fma(w, a.x, acc2[t][1]);
              acc2[t][2] = f2_fma(w, a.y, acc2[t][2]);
              acc2[t][3] = f2_fma(w, cc.x, acc2[t][3]);
              acc2[t][4] = f2_fma(w, f2_sub(cc.y, f2_pack(ea, eb)), acc2[t][4]);   // d'^2 = lid - e
            }
          }
        }
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[b]);
      }
    }
    if (!ok && lane == 0) s_fail = 1;
  }
  float acc[RT][5];
#pragma unroll
  for (int t = 0; t < RT; ++t)
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      float lo, hi;
      f2_unpack(acc2[t][k], lo, hi);
      acc[t][k] = lo + hi;
    }
  if (PASS == 0) {
    float a0, a1, b0, b1;
    f2_unpack(acc2[0][0], a0, a1);
    f2_unpack(acc2[0][1], b0, b1);
    acc[0][0] = (a0 + a1) + (b0 + b1);
  }
  // every MMA has completed (or the CTA gave up) before TMEM is freed
  const bool ok_done = mbar_wait(mdone, 0, kEWaitNs);
  __syncthreads();
  if (!ok_done) s_fail = 1;
  if (warp < kEWarps && (warp >> 2) == 1) {
#pragma unroll
    for (int t = 0; t < RT; ++t) {
      const int r = t * kETile + (warp & 3) * 32 + lane;
#pragma unroll
      for (int k = 0; k < (PASS == 0 ? 1 : 5); ++k) red[k][r] = acc[t][k];
    }
  }
  __syncthreads();
  if (s_fail) {
    if (threadIdx.x == 0) atomicExch(&st->status, (int)CPD_ETIMEOUT);
    if (threadIdx.x == kEWarps * 32) {
      // copies still landing: wait for them before the CTA's memory is released
      for (int j = 0; j < s_issued; ++j) mbar_wait(&bfull[j], 0, kEWaitNs);
      if (PASS == 1 && nvalid > 0 && s_issued > 0) mbar_wait(yfull, 0, kEWaitNs);
    }
  } else if (warp < 4) {
#pragma unroll
    for (int t = 0; t < RT; ++t) {
      const int r = t * kETile + warp * 32 + lane, row = row0 + r;
      if (row < n_rows) {
        if (PASS == 0) {
          part[(size_t)blockIdx.y * n_rows + row] = acc[0][0] + red[0][r];
        } else {
          const size_t plane = (size_t)gridDim.y * n_rows, o = (size_t)blockIdx.y * n_rows + row;
#pragma unroll
          for (int k = 0; k < 5; ++k) part[o + k * plane] = acc[t][k] + red[k][r];
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    tmem_dealloc(tmem, kETmemCols);
  }
}

// sigma2 floor of the tensor-core passes from the largest point norm R of the
// model and scene points: the augmented vectors' FP32 accumulation carries
// terms as large as q^2 R^2, so the passes run while sigma2 >= kMmaS2PerR2 R^2
// (q^2 R^2 <= ~2000, exponent rounding near 1e-3); the FP32 passes below.
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

// Resident CTAs per SM from the kernel's registers and shared memory (the
// occupancy query reported one CTA where two are resident on GB300, so the
// count is taken from the resources themselves; 0 if the shared memory does
// not fit at all).
template <int PASS> int pass_occupancy() {
  static int occ = -1;
  if (occ < 0) {
    occ = 0;
    const int bytes = (int)pass_smem_bytes<PASS>();
    cudaFuncAttributes a;
    int dev = 0, smem_sm = 0, regs_sm = 0, resv = 0;
    if (cudaFuncSetAttribute(pass_umma<PASS>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) == cudaSuccess &&
        cudaFuncSetAttribute(pass_umma<PASS>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared) == cudaSuccess &&
        cudaFuncGetAttributes(&a, pass_umma<PASS>) == cudaSuccess && cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&resv, cudaDevAttrReservedSharedMemoryPerBlock, dev) == cudaSuccess) {
      const int warps = (kEThreads + 31) / 32;
      const int regs_warp = (a.numRegs * 32 + 255) / 256 * 256;
      const int by_regs = regs_sm / std::max(1, regs_warp * warps);
      const int by_smem = smem_sm / std::max(1, (int)a.sharedSizeBytes + bytes + resv);
      occ = std::max(0, std::min(by_regs, by_smem));
    }
    cudaGetLastError();
  }
  return occ;
}

// Column tiles per chunk.  The passes are bound by each SM's issue and
// exponential rate, so the cost of a split is the CTAs on the busiest SM
// times (tiles per CTA + a fixed per-CTA overhead of two tiles); ties go to
// more CTAs (more warps per SM to hide latency).
void split_tiles(int64_t row_tiles, int64_t col_tiles, int64_t sms, int max_tpc, int& tpc, int& chunks) {
  int64_t best = -1;
  for (int64_t c = cdiv(col_tiles, max_tpc); c <= col_tiles; ++c) {
    const int64_t t = cdiv(col_tiles, c);
    const int64_t ch = cdiv(col_tiles, t);
    const int64_t cost = cdiv(row_tiles * ch, sms) * (t + 2);
    if (best < 0 || cost <= best) {
      if (cost == best && ch <= chunks) continue;
      best = cost;
      tpc = (int)t;
      chunks = (int)ch;
    }
    if (ch * row_tiles > 64 * sms) break;
  }
}

}  // namespace

void plan_estep_mma(int64_t M, int64_t N, int sms, MmaPlan& p) {
  p.a_row_tiles = (int)cdiv(N, kETile);
  split_tiles(p.a_row_tiles, cdiv(M, kETile), sms, kEMaxTilesA, p.a_tpc, p.a_chunks);
  p.a_rows_per_chunk = p.a_tpc * kETile;
  p.b_row_tiles = (int)cdiv(M, row_tiles<1>() * kETile);
  split_tiles(p.b_row_tiles, cdiv(N, kETile), sms, kEMaxTilesB, p.b_tpc, p.b_chunks);
  p.b_cols_per_chunk = p.b_tpc * kETile;
  // column vectors (32 bytes per point) of either pass, and pass B's paired
  // scene records (16 bytes per point) after its vectors
  p.prep_floats = std::max(cdiv(M, kETile) * kETile * 8, cdiv(N, kETile) * kETile * 12);
}

void launch_mma_threshold(const float4* X4, int64_t M, const float4* Y4, int64_t N, DevState* st, cudaStream_t s) {
  mma_threshold<<<1, 1024, 0, s>>>(X4, (int)M, Y4, (int)N, st);
}

int estep_mma_occupancy(int pass) { return pass == 0 ? pass_occupancy<0>() : pass_occupancy<1>(); }

bool estep_mma_supported() { return pass_occupancy<0>() > 0 && pass_occupancy<1>() > 0; }

void launch_passA_mma(const MmaPlan& p, const float4* T4, int64_t M, const float4* Y4, int64_t N, float* partA,
                      float* prep, DevState* st, int gate, cudaStream_t s) {
  unsigned char* cols = reinterpret_cast<unsigned char*>(prep);
  const int64_t mpad = cdiv(M, kETile) * kETile;
  prep_cols<<<(unsigned)cdiv(mpad, 256), 256, 0, s>>>(T4, (int)M, (int)mpad, 0, st, gate, cols, nullptr);
  pass_umma<0><<<dim3(p.a_row_tiles, p.a_chunks), kEThreads, pass_smem_bytes<0>(), s>>>(
      Y4, (int)N, cols, (int)M, nullptr, p.a_tpc, partA, st, gate);
}

void launch_passB_mma(const MmaPlan& p, const float4* T4, int64_t M, const float4* Yb, int64_t N, float* partB,
                      float* prep, DevState* st, int gate, cudaStream_t s) {
  unsigned char* cols = reinterpret_cast<unsigned char*>(prep);
  const int64_t npad = cdiv(N, kETile) * kETile;
  float* rec = prep + npad * 8;            // past the column vectors (32 bytes per point)
  prep_cols<<<(unsigned)cdiv(npad, 256), 256, 0, s>>>(Yb, (int)N, (int)npad, 1, st, gate, cols, rec);
  pass_umma<1><<<dim3(p.b_row_tiles, p.b_chunks), kEThreads, pass_smem_bytes<1>(), s>>>(
      T4, (int)M, cols, (int)N, reinterpret_cast<const float4*>(rec), p.b_tpc, partB, st, gate);
}

}  // namespace fcpd
