// M-step of fast CPD on sm_103a: the per-registration kernels (thin wrappers
// over the device bodies in mstep_dev.cuh), their launch plan and launcher.
// See mstep_dev.cuh for the method (Eq. 17, Eq. 20, Eq. 18) and the design.
#include "mstep_dev.cuh"

#include <algorithm>
#include <type_traits>

namespace fcpd {

namespace {

using namespace dev;

// trim: 0 = no spectral trim in this context; 1 = the full M-step of a
// context with the trim (steps aside when the trimmed one runs); 2 = the
// trimmed M-step (runs only then).  trim_now is set once per iteration,
// before the M-step, by the E-step's last launch (fixB_f32).
__device__ __forceinline__ bool trim_skip(const DevState* st, int trim) {
  return trim != 0 && ((trim == 2) != (st->trim_now != 0));
}

template <typename F, typename S>
__global__ void __launch_bounds__(kThreadsP)
colsum(const S* __restrict__ A, int64_t ldA, int rows, int cols, const typename Vec<F>::t4* __restrict__ V,
       int rows_per_chunk, F* __restrict__ part, int64_t ldP, DevState* __restrict__ st, int gate,
       int clear_row_flags, int trim) {
  if (trim_skip(st, trim)) return;
  dev::colsum_body<F, S, kThreadsP>(A, ldA, rows, cols, V, rows_per_chunk, part, ldP, st, gate, clear_row_flags, blockIdx.x, blockIdx.y, gridDim.x, gridDim.y);
}

// ------------------------------------------------- colsum, bulk-copy ring
// The same product and partial-sum layout as colsum, with the rows of A
// streamed into shared memory by the copy engine: one thread issues
// cp.async.bulk copies (a tile row of A per copy, plus the slot's rows of V)
// into a ring of slots, each completing on its own mbarrier, and the block
// consumes slot k while the next slots are in flight.  The bytes in flight
// per SM are then set by the ring rather than by the registers a thread can
// hold loads in.  Thread t owns 16-byte vectors t, t + THREADS, .. of each
// tile row (conflict-free shared-memory reads).  A is read once: its copies
// carry an L2 evict-first hint.  Every wait is bounded (kBulkWaitNs): on
// expiry the block records CPD_ETIMEOUT, waits (bounded) for the copies it
// issued and returns without writing.
// Ring geometry, measured at M = N = 20000 (full basis): an FP32 basis 128
// threads and 3 slots of 32 KB (2 blocks per SM; 6.66 TB/s against 6.36 for
// the register-streaming colsum); an FP16 basis, whose threads do twice the
// arithmetic per byte, 256 threads and 2 slots of 32 KB (3 blocks, 24 warps
// per SM: 6.27 TB/s; 128 threads 4.8, 256 threads x 3 slots 5.6, 512 threads
// 5.8-5.9, 16-24 KB slots 5.6-5.9).
#ifndef FCPD_BULK_THREADS_H
#define FCPD_BULK_THREADS_H 256
#endif
#ifndef FCPD_BULK_STAGES_H
#define FCPD_BULK_STAGES_H 2
#endif
#ifndef FCPD_BULK_SLOT_KB_H
#define FCPD_BULK_SLOT_KB_H 32
#endif
constexpr unsigned long long kBulkWaitNs = 2000000000ull;

template <typename S> struct BulkGeom {
  static constexpr bool H = sizeof(S) == 2;
  static constexpr int THREADS = H ? FCPD_BULK_THREADS_H : 128;
  static constexpr int STAGES = H ? FCPD_BULK_STAGES_H : 3;
  static constexpr int SLOT = (H ? FCPD_BULK_SLOT_KB_H : 32) * 1024;   // bytes of A per slot
  static constexpr int L = L16<S>::W;                  // elements per 16-byte vector
  static constexpr int NV = colsum_vectors<S>();       // vectors per thread and row
  static constexpr int VPR = THREADS * NV;             // vectors per tile row
  static constexpr int COLS = VPR * L;                 // tile columns
  static constexpr int ROWS = SLOT / (VPR * 16);       // tile rows per slot
  static_assert(ROWS >= 1 && SLOT % (VPR * 16) == 0, "a slot holds whole tile rows");
};

template <typename F, typename S> constexpr size_t bulk_smem_bytes() {
  using G = BulkGeom<S>;
  return G::STAGES * ((size_t)G::SLOT + G::ROWS * sizeof(typename Vec<F>::t4)) +
         G::STAGES * sizeof(unsigned long long);
}

__device__ __forceinline__ unsigned int smem_addr(const void* p) {
  return (unsigned int)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned int bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned int parity) {
  unsigned int ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait for the phase of `bar` with the given parity; false after limit_ns.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned int parity,
                                          unsigned long long limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(bar, parity))
    if (global_ns() - t0 > limit_ns) return false;
  return true;
}
// Bulk copy global -> shared (16-byte aligned addresses, size a multiple of
// 16), completion counted on `bar` in bytes.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned int bytes, unsigned long long* bar,
                                         unsigned long long policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::
          "r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(policy)
      : "memory");
}

template <typename F, typename S>
__global__ void __launch_bounds__(BulkGeom<S>::THREADS)
colsum_bulk(const S* __restrict__ A, int64_t ldA, int rows, int cols, const typename Vec<F>::t4* __restrict__ V,
            int rows_per_chunk, F* __restrict__ part, int64_t ldP, DevState* __restrict__ st, int gate,
            int clear_row_flags, int trim) {
  if (trim_skip(st, trim) || (gate && iteration_gated(st))) return;
  if (clear_row_flags && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) st->n_flag_rows = 0;
  using G = BulkGeom<S>;
  using V4 = typename Vec<F>::t4;
  using LT = typename L16<S>::t;
  constexpr int W = G::NV * G::L;
  extern __shared__ __align__(128) unsigned char smem[];
  LT* tiles = reinterpret_cast<LT*>(smem);
  V4* vt = reinterpret_cast<V4*>(smem + (size_t)G::STAGES * G::SLOT);
  unsigned long long* bar =
      reinterpret_cast<unsigned long long*>(smem + (size_t)G::STAGES * (G::SLOT + G::ROWS * sizeof(V4)));
  const int tid = threadIdx.x;
  const int64_t cb = (int64_t)blockIdx.x * G::COLS;
  // 16-byte vectors of a tile row: the columns rounded up to W (<= ldA, a
  // multiple of W)
  const int64_t wcols = ((int64_t)cols + W - 1) / W * W;
  const int64_t lim = (wcols < ldA ? wcols : ldA) - cb;
  const int vecs = (int)(lim / G::L < G::VPR ? lim / G::L : G::VPR);
  const unsigned int row_bytes = (unsigned int)vecs * 16u;
  const int r0 = blockIdx.y * rows_per_chunk;
  const int r1 = min(rows, r0 + rows_per_chunk);
  const int nst = r0 < r1 ? (r1 - r0 + G::ROWS - 1) / G::ROWS : 0;
  const bool fault = (st->prune_ctl & kBulkWaitFault) != 0;
  const unsigned int extra_tx = fault ? 16u : 0u;
  const unsigned long long wait_ns = fault ? kBulkFaultWaitNs : kBulkWaitNs;
  unsigned long long pol_a = 0, pol_v = 0;
  if (tid == 0) {
    for (int k = 0; k < G::STAGES; ++k) mbar_init(&bar[k], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol_a));
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol_v));
  }
  __syncthreads();
  auto issue = [&](int k) {
    const int slot = k % G::STAGES;
    const int ra = r0 + k * G::ROWS;
    const int nr = min(G::ROWS, r1 - ra);
    mbar_expect_tx(&bar[slot], (unsigned int)nr * (row_bytes + (unsigned int)sizeof(V4)) + extra_tx);
    LT* dst = tiles + (size_t)slot * (G::SLOT / 16);
    for (int i = 0; i < nr; ++i)
      bulk_g2s(dst + (size_t)i * G::VPR, A + (size_t)(ra + i) * ldA + cb, row_bytes, &bar[slot], pol_a);
    bulk_g2s(vt + (size_t)slot * G::ROWS, V + ra, (unsigned int)(nr * sizeof(V4)), &bar[slot], pol_v);
  };
  if (tid == 0)
    for (int k = 0; k < min(nst, G::STAGES); ++k) issue(k);
  F acc[W][3];
#pragma unroll
  for (int w = 0; w < W; ++w) acc[w][0] = acc[w][1] = acc[w][2] = (F)0;
  const F scale = (F)lane_scale<S>();
  int failed_at = -1;
  for (int k = 0; k < nst; ++k) {
    const int slot = k % G::STAGES;
    const bool ok = mbar_wait(&bar[slot], (unsigned int)(k / G::STAGES) & 1u, wait_ns);
    const LT* tile = tiles + (size_t)slot * (G::SLOT / 16);
    const V4* vv = vt + (size_t)slot * G::ROWS;
    const int nr = min(G::ROWS, r1 - (r0 + k * G::ROWS));
#pragma unroll 4
    for (int i = 0; i < nr; ++i) {
      LT u[G::NV];
#pragma unroll
      for (int v = 0; v < G::NV; ++v) u[v] = tile[(size_t)i * G::VPR + tid + v * G::THREADS];
      V4 r = vv[i];
      if constexpr (sizeof(S) == 2) {          // exact power-of-two pre-scale (see lane_of)
        r.x *= scale; r.y *= scale; r.z *= scale;
      }
#pragma unroll
      for (int v = 0; v < G::NV; ++v)
#pragma unroll
        for (int l = 0; l < G::L; ++l) {
          const F uw = (F)lane_of(u[v], l);
          F* a = acc[v * G::L + l];
          a[0] = fma(uw, r.x, a[0]);
          a[1] = fma(uw, r.y, a[1]);
          a[2] = fma(uw, r.z, a[2]);
        }
    }
    // every thread is done with the slot (and learns whether any wait expired)
    if (__syncthreads_or(!ok)) {
      failed_at = k;
      break;
    }
    if (tid == 0 && k + G::STAGES < nst) issue(k + G::STAGES);
  }
  if (failed_at >= 0) {
    if (tid == 0) {
      atomicExch(&st->status, (int)CPD_ETIMEOUT);
      // the copies issued and not yet consumed: stages failed_at .. failed_at + G::STAGES - 1
      for (int j = failed_at; j < min(nst, failed_at + G::STAGES); ++j)
        mbar_wait(&bar[j % G::STAGES], (unsigned int)(j / G::STAGES) & 1u, wait_ns);
    }
    __syncthreads();
    return;
  }
#pragma unroll
  for (int v = 0; v < G::NV; ++v) {
    const int vec = tid + v * G::THREADS;
    if (vec >= vecs) continue;
    const int64_t c = cb + (int64_t)vec * G::L;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      F* out = part + ((size_t)blockIdx.y * 3 + d) * ldP + c;
      if constexpr (sizeof(F) == 4) {
#pragma unroll
        for (int q = 0; q < G::L / 4; ++q)
          reinterpret_cast<float4*>(out)[q] = make_float4(acc[v * G::L + 4 * q][d], acc[v * G::L + 4 * q + 1][d],
                                                          acc[v * G::L + 4 * q + 2][d], acc[v * G::L + 4 * q + 3][d]);
      } else {
#pragma unroll
        for (int q = 0; q < G::L / 2; ++q)
          reinterpret_cast<double2*>(out)[q] = make_double2(acc[v * G::L + 2 * q][d], acc[v * G::L + 2 * q + 1][d]);
      }
    }
  }
}

// Diagonal update of the first K columns; columns K .. k_zero - 1 (the
// directions a trimmed M-step drops) get B = C = 0.
template <typename F, int COLS>
__global__ void __launch_bounds__(kThreadsD)
diag_update(const F* __restrict__ partP, int chunks, int64_t ldP, int K, int k_zero, const double* __restrict__ lam,
            typename Vec<F>::t4* __restrict__ B4, typename Vec<F>::t4* __restrict__ C4,
            const DevState* __restrict__ st, int gate, int trim) {
  if (trim_skip(st, trim) || (gate && iteration_gated(st))) return;
  dev::diag_update_body<F, COLS>(partP, chunks, ldP, K, lam, B4, C4, st, 0, blockIdx.x, blockIdx.y, gridDim.x,
                                 gridDim.y);
  const int k = blockIdx.x * COLS + threadIdx.x;
  if (threadIdx.x < COLS && k >= K && k < k_zero) {
    typename Vec<F>::t4 z;
    z.x = z.y = z.z = z.w = (F)0;
    B4[k] = z;
    C4[k] = z;
  }
}

// With EPI (an iteration) a trimmed M-step (trim == 2) is counted in
// st->trim_iters by the block that completes the iteration.
template <typename F, bool EPI>
__global__ void __launch_bounds__(kThreadsD)
expand_finish(const F* __restrict__ partE, int chunks, int64_t ldM, int M,
              const typename Vec<F>::t4* __restrict__ X4, const typename Vec<F>::t4* __restrict__ Yt4,
              typename Vec<F>::t4* __restrict__ Tout, const typename Vec<F>::t4* __restrict__ Yhat4,
              double* __restrict__ sums, DevState* __restrict__ st, int gate, int trim) {
  if (trim_skip(st, trim)) return;
  const bool last = dev::expand_finish_body<F, EPI>(partE, chunks, ldM, M, X4, Yt4, Tout, Yhat4, sums, st, gate,
                                                    blockIdx.x, blockIdx.y, gridDim.x, gridDim.y);
  if (EPI && last && trim == 2 && threadIdx.x == 0) st->trim_iters += 1;
}

// ---------------------------------------- narrow basis: row expansion
// T = X + U B and the Eq. 18 epilogue in ONE launch when the basis is narrow
// (K <= kRowsMaxK: the low-rank and trimmed M-steps).  There the column-
// parallel expansion over U^T (colsum_bulk) is latency-bound -- K rows of
// 16-byte vectors split over few blocks -- and its partials need the
// expand_finish launch.  Here one thread owns one model point: it reads its
// row of U once in 16-byte vectors (eight in flight), multiplies with B from
// shared memory (every thread reads the same element: a broadcast) in a
// fixed order, forms t_m and the row's Eq. 18 terms in FP64 -- the epilogue
// of all 32 rows of a warp in parallel -- and the block sums (FP64) meet in
// the last block to finish (ticket), which ends the iteration as
// expand_finish does.  (Four threads per point, 64 points per block,
// measured slower: 26 against 19 us per launch at M = 20000, K = 200.)
constexpr int kRowsMaxK = 256;
constexpr int kRowsThreads = 128;

__device__ __forceinline__ void row_load(const float* p, float (&u)[8]) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  u[0] = v.x; u[1] = v.y; u[2] = v.z; u[3] = v.w;
}
__device__ __forceinline__ void row_load(const __half* p, float (&u)[8]) {
  const uint4 r = __ldg(reinterpret_cast<const uint4*>(p));
  const __half2* h = reinterpret_cast<const __half2*>(&r);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float2 f = __half22float2(h[i]);
    u[2 * i] = f.x;
    u[2 * i + 1] = f.y;
  }
}

template <typename S, bool EPI>
__global__ void __launch_bounds__(kRowsThreads)
expand_rows(const S* __restrict__ U, int64_t ldU, int M, int K, const float4* __restrict__ B4,
            const float4* __restrict__ X4, const float4* __restrict__ Yt4, float4* __restrict__ Tout,
            const float4* __restrict__ Yhat4, double* __restrict__ sums, DevState* __restrict__ st, int gate,
            int trim) {
  if (trim_skip(st, trim) || (gate && iteration_gated(st))) return;
  constexpr int L = 16 / (int)sizeof(S);       // elements per 16-byte vector
  __shared__ float sB[3][kRowsMaxK + 8];
  __shared__ double sh3[32][3];
  __shared__ bool last;
  const int m = blockIdx.x * kRowsThreads + threadIdx.x;
  const bool row = m < M;
  // the row's inputs, in flight with the basis row
  float4 x = make_float4(0.f, 0.f, 0.f, 0.f), to{}, yt{}, yh{};
  if (row) {
    if (X4) x = X4[m];
    if constexpr (EPI) {
      to = Tout[m];
      yt = Yt4[m];
      if (Yhat4) yh = Yhat4[m];
    }
  }
  for (int k = threadIdx.x; k < kRowsMaxK + 8; k += kRowsThreads) {
    const float4 b = k < K ? B4[k] : make_float4(0.f, 0.f, 0.f, 0.f);
    sB[0][k] = b.x;
    sB[1][k] = b.y;
    sB[2][k] = b.z;
  }
  __syncthreads();
  double contrib = 0.0, dT2 = 0.0, gt2 = 0.0;
  if (row) {
    const int nvec = (K + L - 1) / L;          // 16-byte vectors holding the K columns
    const S* ur = U + (size_t)m * ldU;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f;
#pragma unroll 8
    for (int v = 0; v < nvec; ++v) {
      float u[8];
      row_load(ur + (size_t)v * L, u);
#pragma unroll
      for (int i = 0; i < L; ++i) {
        const int k = v * L + i;                // sB is zero past K (the padding of U never counts)
        const float w = k < K ? u[i] : 0.f;
        a0 = fmaf(w, sB[0][k], a0);
        a1 = fmaf(w, sB[1][k], a1);
        a2 = fmaf(w, sB[2][k], a2);
      }
    }
    float4 tn;
    tn.x = (float)((double)x.x + (double)a0);
    tn.y = (float)((double)x.y + (double)a1);
    tn.z = (float)((double)x.z + (double)a2);
    tn.w = 0.f;
    if constexpr (EPI) point_terms<float4>(to, tn, yt, Yhat4 ? &yh : nullptr, 0, contrib, dT2, gt2);
    Tout[m] = tn;
  }
  if constexpr (EPI) {
    block_sum3(contrib, dT2, gt2, sh3, kRowsThreads / 32);
    if (threadIdx.x == 0) {
      sums[(size_t)blockIdx.x * 3] = contrib;
      sums[(size_t)blockIdx.x * 3 + 1] = dT2;
      sums[(size_t)blockIdx.x * 3 + 2] = gt2;
      __threadfence();
      last = atomicAdd(&st->ticket_e, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last) {
      __threadfence();
      double s0 = 0, s1 = 0, s2 = 0;
      for (int i = threadIdx.x; i < (int)gridDim.x; i += kRowsThreads) {
        s0 += __ldcg(sums + (size_t)i * 3);
        s1 += __ldcg(sums + (size_t)i * 3 + 1);
        s2 += __ldcg(sums + (size_t)i * 3 + 2);
      }
      block_sum3(s0, s1, s2, sh3, kRowsThreads / 32);
      if (threadIdx.x == 0) {
        finish_iteration(st, s0, s1, s2, M);
        st->ticket_e = 0;
        if (trim == 2) st->trim_iters += 1;
      }
    }
  }
}

int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Row chunks for a colsum over a rows x ld matrix: enough blocks to fill the
// GPU, but at least ~256 KB of the matrix per block (a small matrix needs few
// chunks, which keeps the partial sums short).
void plan_colsum(int64_t rows, int64_t ld, int64_t es, int sms, int W, int threads, int& col_tiles, int& chunks,
                 int& rpc) {
  col_tiles = (int)cdiv(ld, (int64_t)threads * W);
  const int64_t target = (int64_t)sms * 8;
  int64_t ch = std::max<int64_t>(1, cdiv(target, col_tiles));
  ch = std::min<int64_t>(ch, std::max<int64_t>(1, rows * ld * es / (256 * 1024)));
  const int64_t r = std::max<int64_t>(32, cdiv(rows, ch));
  rpc = (int)r;
  chunks = (int)cdiv(rows, r);
}

// Grid of colsum_bulk over a rows x ld matrix: one resident wave (slots =
// SMs x resident blocks), the rows of each column tile split into equal
// chunks of whole slots, at least 4 slots of rows per block.
void plan_colsum_bulk(int64_t rows, int64_t ld, int64_t slots, int tile_cols, int slot_rows, int& col_tiles,
                      int& chunks, int& rpc) {
  col_tiles = (int)cdiv(ld, tile_cols);
  int64_t ch = std::max<int64_t>(1, slots / col_tiles);
  ch = std::min<int64_t>(ch, std::max<int64_t>(1, rows / (4 * (int64_t)slot_rows)));
  const int64_t r = cdiv(cdiv(rows, ch), slot_rows) * slot_rows;
  rpc = (int)r;
  chunks = (int)cdiv(rows, r);
}

template <typename F, typename S> int64_t bulk_slots(int sms) {
  const int bytes = (int)bulk_smem_bytes<F, S>();
  cudaFuncSetAttribute(colsum_bulk<F, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, colsum_bulk<F, S>, BulkGeom<S>::THREADS, bytes);
  return (int64_t)sms * std::max(occ, 1);
}

// colsum_bulk for the per-registration launches of FP32 and FP16 bases (the
// register-streaming colsum for FP32 when built with FCPD_COLSUM_REG_F32; FP64
// and the batched kernel always use it).
#ifdef FCPD_COLSUM_REG_F32
constexpr bool kBulkF32 = false;
#else
constexpr bool kBulkF32 = true;
#endif

}  // namespace

namespace {
// Grids of both products over a U with `cols_p` streamed columns (row stride
// of the partials ldPp) and a U^T with `rows_e` streamed rows.
void plan_products(MstepPlan& p, int64_t M, int64_t cols_p, int64_t rows_e, int64_t es, int sms, int W,
                   int colsum_threads) {
  if (p.bulk) {
    const int64_t slots = es == 2 ? bulk_slots<float, __half>(sms) : bulk_slots<float, float>(sms);
    const int tc = es == 2 ? BulkGeom<__half>::COLS : BulkGeom<float>::COLS;
    const int tr = es == 2 ? BulkGeom<__half>::ROWS : BulkGeom<float>::ROWS;
    plan_colsum_bulk(M, p.ldPp, slots, tc, tr, p.p_col_tiles, p.p_row_chunks, p.p_rows_per_chunk);
    plan_colsum_bulk(rows_e, p.ldM, slots, tc, tr, p.e_col_tiles, p.e_row_chunks, p.e_rows_per_chunk);
  } else {
    plan_colsum(M, p.ldPp, es, sms, W, colsum_threads, p.p_col_tiles, p.p_row_chunks, p.p_rows_per_chunk);
    plan_colsum(rows_e, p.ldM, es, sms, W, colsum_threads, p.e_col_tiles, p.e_row_chunks, p.e_rows_per_chunk);
  }
  (void)cols_p;
  p.part_elems = std::max((int64_t)p.p_row_chunks * 3 * p.ldPp, (int64_t)p.e_row_chunks * 3 * p.ldM);
  p.e_blocks = (int)cdiv(M, kMRedCols);
  p.sums_elems = (int64_t)p.e_blocks * 3;
}

int colsum_width(int64_t es) {
  const int nv = es == 2 ? colsum_vectors<__half>() : 2;
  return (int)(16 * nv / es);   // columns per colsum thread; row strides padded to it
}
}  // namespace

MstepPlan plan_mstep(int64_t M, int64_t K, bool fp64, int sms, int colsum_threads, int basis_bytes) {
  MstepPlan p{};
  const int64_t es = basis_bytes > 0 ? basis_bytes : (fp64 ? 8 : 4);
  const int W = colsum_width(es);
  p.K = K;
  p.ldU = cdiv(K, W) * W;
  p.ldPp = p.ldU;
  p.ldM = cdiv(M, W) * W;
  p.bulk = colsum_threads == kThreadsP && (es == 2 || (es == 4 && kBulkF32));
  plan_products(p, M, K, K, es, sms, W, colsum_threads);
  return p;
}

MstepPlan plan_mstep_trim(const MstepPlan& full, int64_t M, int64_t K_cap, bool fp64, int sms, int basis_bytes) {
  MstepPlan p = full;
  p.n_pieces = 0;
  const int64_t es = basis_bytes > 0 ? basis_bytes : (fp64 ? 8 : 4);
  const int W = colsum_width(es);
  p.K = K_cap;
  p.ldPp = std::min(full.ldU, cdiv(K_cap, W) * W);
  plan_products(p, M, K_cap, K_cap, es, sms, W, kThreadsP);
  return p;
}

// Each piece's projection is planned like a whole one over its rows (one
// resident wave when it runs alone); its partial rows follow the previous
// pieces', so the diagonal update sums them all in one launch.
bool plan_mstep_pieces(MstepPlan& p, int64_t M, int sms, int pieces, const int* m0, const int* rows) {
  if (!p.bulk || pieces < 2 || pieces > kMaxPieces || p.K <= kRowsMaxK) return false;
  const int64_t slots = bulk_slots<float, float>(sms);
  // the pieces that run beside pass B: one block per SM, which fits beside
  // two pass B blocks (registers exactly, shared memory with room); planned
  // for two per SM, a side projection that reached the SMs first left room
  // for one pass B block and the split was slower than one piece
  const int64_t side_slots = std::min<int64_t>(slots, (int64_t)sms);
  int off = 0, tiles = 0;
  for (int i = 0; i < pieces; ++i) {
    if (rows[i] < 1 || m0[i] < 0 || (int64_t)m0[i] + rows[i] > M) return false;
    int ch = 0, rpc = 0;
    plan_colsum_bulk(rows[i], p.ldPp, i + 1 < pieces ? side_slots : slots, BulkGeom<float>::COLS,
                     BulkGeom<float>::ROWS, tiles, ch, rpc);
    p.pp_m0[i] = m0[i];
    p.pp_rows[i] = rows[i];
    p.pp_chunks[i] = ch;
    p.pp_rpc[i] = rpc;
    p.pp_off[i] = off;
    off += ch;
  }
  if (tiles != p.p_col_tiles) return false;
  p.n_pieces = pieces;
  p.pp_chunks_total = off;
  p.part_elems = std::max(p.part_elems, (int64_t)off * 3 * p.ldPp);
  return true;
}

void launch_projection_piece(const MstepPlan& pl, int piece, const float* U, const float4* R4, float* part,
                             DevState* st, cudaStream_t s) {
  const int64_t m0 = pl.pp_m0[piece];
  colsum_bulk<float, float><<<dim3(pl.p_col_tiles, pl.pp_chunks[piece]), BulkGeom<float>::THREADS,
                              bulk_smem_bytes<float, float>(), s>>>(
      U + m0 * pl.ldU, pl.ldU, pl.pp_rows[piece], (int)pl.K, R4 + m0, pl.pp_rpc[piece],
      part + (size_t)pl.pp_off[piece] * 3 * pl.ldPp, pl.ldPp, st, 1, 0, 0);
}

// Partials of A^T V over the plan's grid (colsum or colsum_bulk); ldP: row
// stride of the partials.
template <typename F, typename S>
void launch_colsum(const MstepPlan& pl, bool expansion, const S* A, int64_t ldA, int64_t ldP, int64_t rows,
                   int64_t cols, const typename Vec<F>::t4* V, F* part, DevState* st, int gate, int clear_row_flags,
                   int trim, cudaStream_t s) {
  const dim3 grid = expansion ? dim3(pl.e_col_tiles, pl.e_row_chunks) : dim3(pl.p_col_tiles, pl.p_row_chunks);
  const int rpc = expansion ? pl.e_rows_per_chunk : pl.p_rows_per_chunk;
  if (pl.bulk && !std::is_same<F, double>::value)
    colsum_bulk<F, S><<<grid, BulkGeom<S>::THREADS, bulk_smem_bytes<F, S>(), s>>>(
        A, ldA, (int)rows, (int)cols, V, rpc, part, ldP, st, gate, clear_row_flags, trim);
  else
    colsum<F, S><<<grid, kThreadsP, 0, s>>>(A, ldA, (int)rows, (int)cols, V, rpc, part, ldP, st, gate,
                                            clear_row_flags, trim);
}

template <typename F> bool rows_expansion(int64_t K) { return std::is_same<F, float>::value && K <= kRowsMaxK; }

// One thread per model point; the block sums fit the plan's scratch, sized
// for e_blocks = M / 64 blocks.
template <typename F, typename S>
void launch_expand_rows(const S* U, int64_t ldU, int64_t M, int64_t K, const typename Vec<F>::t4* B4,
                        const typename Vec<F>::t4* X4, const typename Vec<F>::t4* Yt4, typename Vec<F>::t4* T4,
                        const typename Vec<F>::t4* Yhat4, double* sums, int e_blocks, DevState* st, int gate,
                        int trim, cudaStream_t s) {
  if constexpr (std::is_same<F, float>::value) {
    const unsigned grid = (unsigned)cdiv(M, kRowsThreads);   // <= e_blocks (64 rows per block there)
    (void)e_blocks;
    expand_rows<S, true><<<grid, kRowsThreads, 0, s>>>(U, ldU, (int)M, (int)K, B4, X4, Yt4, T4, Yhat4, sums, st,
                                                       gate, trim);
  }
}

// diag_update over columns 0 .. k_zero - 1 with as few columns per block as
// keep each thread's share of the `chunks` partial rows at about 8 (64
// columns per block for few chunks, down to 8 for hundreds).
template <typename F>
void launch_diag(const F* part, int chunks, int64_t ldP, int K, int k_zero, const double* lam,
                 typename Vec<F>::t4* B4, typename Vec<F>::t4* C4, const DevState* st, int gate, int trim,
                 cudaStream_t s) {
  const int sub = (chunks + 7) / 8;
  const int cols = sub > 16 ? 8 : sub > 8 ? 16 : sub > 4 ? 32 : 64;
  const unsigned blocks = (unsigned)cdiv(k_zero, cols);
  switch (cols) {
    case 8: diag_update<F, 8><<<blocks, kThreadsD, 0, s>>>(part, chunks, ldP, K, k_zero, lam, B4, C4, st, gate, trim); break;
    case 16: diag_update<F, 16><<<blocks, kThreadsD, 0, s>>>(part, chunks, ldP, K, k_zero, lam, B4, C4, st, gate, trim); break;
    case 32: diag_update<F, 32><<<blocks, kThreadsD, 0, s>>>(part, chunks, ldP, K, k_zero, lam, B4, C4, st, gate, trim); break;
    default: diag_update<F, 64><<<blocks, kThreadsD, 0, s>>>(part, chunks, ldP, K, k_zero, lam, B4, C4, st, gate, trim); break;
  }
}

template <typename F, typename S>
void launch_mstep(const MstepPlan& pl, const S* U, const S* Ut, const double* lam, int64_t M, int64_t K,
                  const typename Vec<F>::t4* X4, const typename Vec<F>::t4* R4,
                  const typename Vec<F>::t4* Yt4, typename Vec<F>::t4* T4,
                  const typename Vec<F>::t4* Yhat4, F* part, double* sums, typename Vec<F>::t4* B4,
                  typename Vec<F>::t4* C4, DevState* st, bool iteration, cudaStream_t s, cudaEvent_t* ev,
                  const MstepPlan* trim, bool projected) {
  const int g = iteration ? 1 : 0;
  const MstepPlan* tr = iteration ? trim : nullptr;
  const int mf = tr ? 1 : 0;      // the full M-step's trim mode
  projected = projected && iteration && !tr && pl.n_pieces > 1;
  if (!projected) {
    if (tr) launch_colsum<F, S>(*tr, false, U, tr->ldU, tr->ldPp, M, tr->K, R4, part, st, g, g, 2, s);
    launch_colsum<F, S>(pl, false, U, pl.ldU, pl.ldPp, M, K, R4, part, st, g, g, mf, s);
  }
  record_after(ev, 0, s);
  if (tr) launch_diag<F>(part, tr->p_row_chunks, tr->ldPp, (int)tr->K, (int)K, lam, B4, C4, st, g, 2, s);
  launch_diag<F>(part, projected ? pl.pp_chunks_total : pl.p_row_chunks, pl.ldPp, (int)K, (int)K, lam, B4, C4, st,
                 g, mf, s);
  record_after(ev, 1, s);
  // narrow bases (FP32 working precision, iterations): the row expansion
  // with its epilogue replaces colsum (U^T) + expand_finish
  const bool rows_tr = iteration && tr && rows_expansion<F>(tr->K);
  const bool rows_pl = iteration && rows_expansion<F>(K);
  if (tr && !rows_tr) launch_colsum<F, S>(*tr, true, Ut, tr->ldM, tr->ldM, tr->K, M, B4, part, st, g, 0, 2, s);
  if (!rows_pl) launch_colsum<F, S>(pl, true, Ut, pl.ldM, pl.ldM, K, M, B4, part, st, g, 0, mf, s);
  record_after(ev, 2, s);
  if (iteration) {
    if (tr) {
      if (rows_tr)
        launch_expand_rows<F, S>(U, tr->ldU, M, tr->K, B4, X4, Yt4, T4, Yhat4, sums, tr->e_blocks, st, g, 2, s);
      else
        expand_finish<F, true><<<tr->e_blocks, kThreadsD, 0, s>>>(part, tr->e_row_chunks, tr->ldM, (int)M, X4,
                                                                  Yt4, T4, Yhat4, sums, st, g, 2);
    }
    if (rows_pl)
      launch_expand_rows<F, S>(U, pl.ldU, M, K, B4, X4, Yt4, T4, Yhat4, sums, pl.e_blocks, st, g, mf, s);
    else
      expand_finish<F, true><<<pl.e_blocks, kThreadsD, 0, s>>>(part, pl.e_row_chunks, pl.ldM, (int)M, X4, Yt4, T4,
                                                               Yhat4, sums, st, g, mf);
  } else {
    expand_finish<F, false><<<pl.e_blocks, kThreadsD, 0, s>>>(part, pl.e_row_chunks, pl.ldM, (int)M, X4, Yt4,
                                                              T4, nullptr, sums, st, 0, 0);
  }
  record_after(ev, 3, s);
}

template <typename F, typename S>
void launch_w(const MstepPlan& pl, const S* Ut, int64_t M, int64_t K, const typename Vec<F>::t4* C4, F* part,
              typename Vec<F>::t4* W4, DevState* st, cudaStream_t s) {
  launch_colsum<F, S>(pl, true, Ut, pl.ldM, pl.ldM, K, M, C4, part, st, 0, 0, 0, s);
  expand_finish<F, false><<<pl.e_blocks, kThreadsD, 0, s>>>(part, pl.e_row_chunks, pl.ldM, (int)M, nullptr,
                                                            nullptr, W4, nullptr, nullptr, st, 0, 0);
}

template void launch_mstep<float, float>(const MstepPlan&, const float*, const float*, const double*, int64_t,
                                         int64_t, const float4*, const float4*, const float4*, float4*,
                                         const float4*, float*, double*, float4*, float4*, DevState*, bool,
                                         cudaStream_t, cudaEvent_t*, const MstepPlan*, bool);
template void launch_mstep<double, double>(const MstepPlan&, const double*, const double*, const double*, int64_t,
                                           int64_t, const dvec4*, const dvec4*, const dvec4*, dvec4*, const dvec4*,
                                           double*, double*, dvec4*, dvec4*, DevState*, bool, cudaStream_t,
                                           cudaEvent_t*, const MstepPlan*, bool);
template void launch_mstep<float, __half>(const MstepPlan&, const __half*, const __half*, const double*, int64_t,
                                          int64_t, const float4*, const float4*, const float4*, float4*,
                                          const float4*, float*, double*, float4*, float4*, DevState*, bool,
                                          cudaStream_t, cudaEvent_t*, const MstepPlan*, bool);
template void launch_w<float, float>(const MstepPlan&, const float*, int64_t, int64_t, const float4*, float*,
                                     float4*, DevState*, cudaStream_t);
template void launch_w<double, double>(const MstepPlan&, const double*, int64_t, int64_t, const dvec4*, double*,
                                       dvec4*, DevState*, cudaStream_t);
template void launch_w<float, __half>(const MstepPlan&, const __half*, int64_t, int64_t, const float4*, float*,
                                      float4*, DevState*, cudaStream_t);

}  // namespace fcpd
