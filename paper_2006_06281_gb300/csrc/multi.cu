// Several registrations against one model (one eigenbasis U, U^T): the
// M-step products of all scenes in one pass over the basis (Eq. 17 with 3S
// right-hand sides), between per-scene E-steps and per-scene diagonal
// updates / Eq. 18 epilogues.
//
// colsum_multi<S> computes, for S right-hand sides at once,
//     part_s[chunk][d][c] = sum_{r in chunk} A[r][c] * V_s[r][d]     (d = 0..2)
// with A's rows streamed into shared memory by the copy engine
// (cp.async.bulk into a ring of slots, one mbarrier each, bounded waits, as
// in the single-scene M-step) and the S rows of V staged beside them.  Each
// thread owns one 16-byte vector (4 columns) of a tile row and 12 S FP32
// accumulators; the basis is read once for all S scenes, so the products
// stay HBM-bound up to S ~ 8 (12 S FMA per 16 bytes).  The partials of
// scene s are laid out exactly like the single-scene kernel's, so the
// per-scene diagonal update and expansion epilogue are the same device
// bodies.
#include "mstep_dev.cuh"

#include <algorithm>

namespace fcpd {

namespace {

using namespace dev;

constexpr int kThreadsMulti = 256;
constexpr int kMultiStages = 3;
constexpr int kMultiSlot = 32 * 1024;                      // bytes of A per slot
constexpr int kMultiVPR = kThreadsMulti;                    // 16-byte vectors per tile row
constexpr int kMultiCols = kMultiVPR * 4;                   // FP32 tile columns
constexpr int kMultiRows = kMultiSlot / (kMultiVPR * 16);   // tile rows per slot (8)
constexpr unsigned long long kMultiWaitNs = 2000000000ull;

template <int S> constexpr size_t multi_smem_bytes() {
  return kMultiStages * ((size_t)kMultiSlot + (size_t)S * kMultiRows * sizeof(float4)) +
         kMultiStages * sizeof(unsigned long long);
}

__device__ __forceinline__ unsigned int saddr(const void* p) { return (unsigned int)__cvta_generic_to_shared(p); }
__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool bar_try(unsigned long long* bar, unsigned int parity) {
  unsigned int ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(saddr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool bar_wait(unsigned long long* bar, unsigned int parity, unsigned long long limit) {
  if (bar_try(bar, parity)) return true;
  const unsigned long long t0 = now_ns();
  while (!bar_try(bar, parity))
    if (now_ns() - t0 > limit) return false;
  return true;
}
__device__ __forceinline__ void copy_g2s(void* dst, const void* src, unsigned int bytes, unsigned long long* bar,
                                         unsigned long long policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::
          "r"(saddr(dst)),
      "l"(src), "r"(bytes), "r"(saddr(bar)), "l"(policy)
      : "memory");
}

// A: rows x ldA (FP32, ldA a multiple of 8); V: S arrays of `rows` float4
// (V + s * ldV); part: S x chunks x 3 x ldP.  Timeouts are recorded in
// *status (CPD_ETIMEOUT).
template <int S>
__global__ void __launch_bounds__(kThreadsMulti)
colsum_multi(const float* __restrict__ A, int64_t ldA, int rows, int cols, const float4* __restrict__ V,
             int64_t ldV, int rows_per_chunk, int chunks, float* __restrict__ part, int64_t ldP,
             int* __restrict__ status) {
  extern __shared__ __align__(128) unsigned char smem[];
  float4* tiles = reinterpret_cast<float4*>(smem);
  float4* vt = reinterpret_cast<float4*>(smem + (size_t)kMultiStages * kMultiSlot);
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(
      smem + (size_t)kMultiStages * (kMultiSlot + (size_t)S * kMultiRows * sizeof(float4)));
  const int tid = threadIdx.x;
  const int64_t cb = (int64_t)blockIdx.x * kMultiCols;
  const int64_t wcols = ((int64_t)cols + 7) / 8 * 8;
  const int64_t lim = (wcols < ldA ? wcols : ldA) - cb;
  const int vecs = (int)(lim / 4 < kMultiVPR ? lim / 4 : kMultiVPR);
  const unsigned int row_bytes = (unsigned int)vecs * 16u;
  const int r0 = blockIdx.y * rows_per_chunk;
  const int r1 = min(rows, r0 + rows_per_chunk);
  const int nst = r0 < r1 ? (r1 - r0 + kMultiRows - 1) / kMultiRows : 0;
  unsigned long long pol_a = 0, pol_v = 0;
  if (tid == 0) {
    for (int k = 0; k < kMultiStages; ++k)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(&bar[k])), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol_a));
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol_v));
  }
  __syncthreads();
  auto issue = [&](int k) {
    const int slot = k % kMultiStages;
    const int ra = r0 + k * kMultiRows;
    const int nr = min(kMultiRows, r1 - ra);
    const unsigned int tx = (unsigned int)nr * (row_bytes + (unsigned int)(S * sizeof(float4)));
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(&bar[slot])), "r"(tx)
                 : "memory");
    float4* dst = tiles + (size_t)slot * (kMultiSlot / 16);
    for (int i = 0; i < nr; ++i)
      copy_g2s(dst + (size_t)i * kMultiVPR, A + (size_t)(ra + i) * ldA + cb, row_bytes, &bar[slot], pol_a);
    for (int s = 0; s < S; ++s)
      copy_g2s(vt + ((size_t)slot * S + s) * kMultiRows, V + (size_t)s * ldV + ra,
               (unsigned int)(nr * sizeof(float4)), &bar[slot], pol_v);
  };
  if (tid == 0)
    for (int k = 0; k < min(nst, kMultiStages); ++k) issue(k);
  float acc[S][3][4];
#pragma unroll
  for (int s = 0; s < S; ++s)
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int l = 0; l < 4; ++l) acc[s][d][l] = 0.f;
  int failed_at = -1;
  for (int k = 0; k < nst; ++k) {
    const int slot = k % kMultiStages;
    const bool ok = bar_wait(&bar[slot], (unsigned int)(k / kMultiStages) & 1u, kMultiWaitNs);
    const float4* tile = tiles + (size_t)slot * (kMultiSlot / 16);
    const float4* vs = vt + (size_t)slot * S * kMultiRows;
    const int nr = min(kMultiRows, r1 - (r0 + k * kMultiRows));
#pragma unroll 2
    for (int i = 0; i < nr; ++i) {
      const float4 u = tile[(size_t)i * kMultiVPR + tid];
#pragma unroll
      for (int s = 0; s < S; ++s) {
        const float4 r = vs[s * kMultiRows + i];
        const float rv[3] = {r.x, r.y, r.z};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          acc[s][d][0] = fmaf(u.x, rv[d], acc[s][d][0]);
          acc[s][d][1] = fmaf(u.y, rv[d], acc[s][d][1]);
          acc[s][d][2] = fmaf(u.z, rv[d], acc[s][d][2]);
          acc[s][d][3] = fmaf(u.w, rv[d], acc[s][d][3]);
        }
      }
    }
    if (__syncthreads_or(!ok)) {
      failed_at = k;
      break;
    }
    if (tid == 0 && k + kMultiStages < nst) issue(k + kMultiStages);
  }
  if (failed_at >= 0) {
    if (tid == 0) {
      atomicExch(status, (int)CPD_ETIMEOUT);
      for (int j = failed_at; j < min(nst, failed_at + kMultiStages); ++j)
        bar_wait(&bar[j % kMultiStages], (unsigned int)(j / kMultiStages) & 1u, kMultiWaitNs);
    }
    __syncthreads();
    return;
  }
  if (tid >= vecs) return;
  const int64_t c = cb + (int64_t)tid * 4;
#pragma unroll
  for (int s = 0; s < S; ++s)
#pragma unroll
    for (int d = 0; d < 3; ++d)
      *reinterpret_cast<float4*>(part + (((size_t)s * chunks + blockIdx.y) * 3 + d) * ldP + c) =
          make_float4(acc[s][d][0], acc[s][d][1], acc[s][d][2], acc[s][d][3]);
}

__global__ void __launch_bounds__(kThreadsD)
diag_update_scene(const float* __restrict__ partP, int chunks, int64_t ldP, int K, const double* __restrict__ lam,
                  float4* __restrict__ B4, float4* __restrict__ C4, const DevState* __restrict__ st) {
  dev::diag_update_body<float>(partP, chunks, ldP, K, lam, B4, C4, st, 1, blockIdx.x, blockIdx.y, gridDim.x,
                               gridDim.y);
}

__global__ void __launch_bounds__(kThreadsD)
expand_finish_scene(const float* __restrict__ partE, int chunks, int64_t ldM, int M, const float4* __restrict__ X4,
                    const float4* __restrict__ Yt4, float4* __restrict__ Tout, double* __restrict__ sums,
                    DevState* __restrict__ st) {
  dev::expand_finish_body<float, true>(partE, chunks, ldM, M, X4, Yt4, Tout, nullptr, sums, st, 1, blockIdx.x,
                                       blockIdx.y, gridDim.x, gridDim.y);
}

int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

template <int S> int multi_occupancy() {
  const int bytes = (int)multi_smem_bytes<S>();
  cudaFuncSetAttribute(colsum_multi<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, colsum_multi<S>, kThreadsMulti, bytes);
  return std::max(occ, 1);
}

int occupancy_for(int S) {
  switch (S) {
    case 1: return multi_occupancy<1>();
    case 2: return multi_occupancy<2>();
    case 3: return multi_occupancy<3>();
    case 4: return multi_occupancy<4>();
    case 5: return multi_occupancy<5>();
    case 6: return multi_occupancy<6>();
    case 7: return multi_occupancy<7>();
    default: return multi_occupancy<8>();
  }
}

// One resident wave of blocks; the rows of each column tile split into
// equal chunks of whole slots, at least 4 slots of rows per block.
void plan_grid(int64_t rows, int64_t ld, int64_t slots, int& col_tiles, int& chunks, int& rpc) {
  col_tiles = (int)cdiv(ld, kMultiCols);
  int64_t ch = std::max<int64_t>(1, slots / col_tiles);
  ch = std::min<int64_t>(ch, std::max<int64_t>(1, rows / (4 * (int64_t)kMultiRows)));
  const int64_t r = cdiv(cdiv(rows, ch), kMultiRows) * kMultiRows;
  rpc = (int)r;
  chunks = (int)cdiv(rows, r);
}

template <int S>
void launch_products(const float* A, int64_t ldA, int64_t rows, int64_t cols, const float4* V, int64_t ldV,
                     int col_tiles, int chunks, int rpc, float* part, int64_t ldP, int* status, cudaStream_t s) {
  colsum_multi<S><<<dim3(col_tiles, chunks), kThreadsMulti, multi_smem_bytes<S>(), s>>>(
      A, ldA, (int)rows, (int)cols, V, ldV, rpc, chunks, part, ldP, status);
}

void products(int S, const float* A, int64_t ldA, int64_t rows, int64_t cols, const float4* V, int64_t ldV,
              int col_tiles, int chunks, int rpc, float* part, int64_t ldP, int* status, cudaStream_t s) {
  switch (S) {
    case 1: launch_products<1>(A, ldA, rows, cols, V, ldV, col_tiles, chunks, rpc, part, ldP, status, s); break;
    case 2: launch_products<2>(A, ldA, rows, cols, V, ldV, col_tiles, chunks, rpc, part, ldP, status, s); break;
    case 3: launch_products<3>(A, ldA, rows, cols, V, ldV, col_tiles, chunks, rpc, part, ldP, status, s); break;
    case 4: launch_products<4>(A, ldA, rows, cols, V, ldV, col_tiles, chunks, rpc, part, ldP, status, s); break;
    case 5: launch_products<5>(A, ldA, rows, cols, V, ldV, col_tiles, chunks, rpc, part, ldP, status, s); break;
    case 6: launch_products<6>(A, ldA, rows, cols, V, ldV, col_tiles, chunks, rpc, part, ldP, status, s); break;
    case 7: launch_products<7>(A, ldA, rows, cols, V, ldV, col_tiles, chunks, rpc, part, ldP, status, s); break;
    default: launch_products<8>(A, ldA, rows, cols, V, ldV, col_tiles, chunks, rpc, part, ldP, status, s); break;
  }
}

}  // namespace

int64_t multi_sums_elems(int64_t M) { return cdiv(M, kMRedCols) * 3; }

MultiPlan plan_multi(int64_t M, int64_t K, int64_t ldU, int64_t ldM, int S, int sms) {
  MultiPlan p{};
  p.S = S;
  const int64_t slots = (int64_t)sms * occupancy_for(S);
  plan_grid(M, ldU, slots, p.p_col_tiles, p.p_chunks, p.p_rpc);
  plan_grid(K, ldM, slots, p.e_col_tiles, p.e_chunks, p.e_rpc);
  p.part_elems = std::max((int64_t)S * p.p_chunks * 3 * ldU, (int64_t)S * p.e_chunks * 3 * ldM);
  p.e_blocks = (int)cdiv(M, kMRedCols);
  p.sums_elems = (int64_t)p.e_blocks * 3;
  return p;
}

void launch_mstep_multi(const MultiPlan& p, const float* U, int64_t ldU, const float* Ut, int64_t ldM,
                        const double* lam, int64_t M, int64_t K, const float4* X4, const float4* R4,
                        const float4* Yt4, float4* T4, float4* B4, float4* C4, DevState* const* st, float* part,
                        double* sums, int* status, cudaStream_t s) {
  const int S = p.S;
  // projection a_s = U^T R_s of every scene (R4 + s M), one pass over U
  products(S, U, ldU, M, K, R4, M, p.p_col_tiles, p.p_chunks, p.p_rpc, part, ldU, status, s);
  for (int i = 0; i < S; ++i)
    diag_update_scene<<<(unsigned)cdiv(K, kMRedCols), kThreadsD, 0, s>>>(
        part + (size_t)i * p.p_chunks * 3 * ldU, p.p_chunks, ldU, (int)K, lam, B4 + (size_t)i * K,
        C4 + (size_t)i * K, st[i]);
  // expansion U B_s of every scene (B4 + s K), one pass over U^T
  products(S, Ut, ldM, K, M, B4, K, p.e_col_tiles, p.e_chunks, p.e_rpc, part, ldM, status, s);
  for (int i = 0; i < S; ++i)
    expand_finish_scene<<<p.e_blocks, kThreadsD, 0, s>>>(part + (size_t)i * p.e_chunks * 3 * ldM, p.e_chunks, ldM,
                                                         (int)M, X4, Yt4 + (size_t)i * M, T4 + (size_t)i * M, sums,
                                                         st[i]);
}

// The same M-step with the products on the tensor cores (umma.cu), for an
// FP16 basis: V is packed from the scenes' right-hand sides (hi / lo FP16
// parts), then one tcgen05 pass over U^T (projection) and one over U
// (expansion); the partials feed the per-scene diagonal updates and Eq. 18
// epilogues above.
cudaError_t launch_mstep_multi_mma(const UmmaPlan& pp, const UmmaPlan& pe, const __half* U, int64_t ldU,
                                   const __half* Ut, int64_t ldM, const double* lam, int64_t M, int64_t K,
                                   const float4* X4, const float4* R4, const float4* Yt4, float4* T4, float4* B4,
                                   float4* C4, DevState* const* st, __half* Vp, __half* Ve, float* part,
                                   double* sums, int* status, bool fault_wait, cudaStream_t s) {
  const int S = pp.S;
  launch_pack_rhs(pp, R4, M, Vp, s);
  cudaError_t e = launch_umma_products(pp, Ut, ldM, Vp, part, ldU, status, fault_wait, s);
  if (e != cudaSuccess) return e;
  for (int i = 0; i < S; ++i)
    diag_update_scene<<<(unsigned)cdiv(K, kMRedCols), kThreadsD, 0, s>>>(
        part + (size_t)i * pp.chunks * 3 * ldU, pp.chunks, ldU, (int)K, lam, B4 + (size_t)i * K, C4 + (size_t)i * K,
        st[i]);
  launch_pack_rhs(pe, B4, K, Ve, s);
  e = launch_umma_products(pe, U, ldU, Ve, part, ldM, status, fault_wait, s);
  if (e != cudaSuccess) return e;
  const unsigned eb = (unsigned)cdiv(M, kMRedCols);
  for (int i = 0; i < S; ++i)
    expand_finish_scene<<<eb, kThreadsD, 0, s>>>(part + (size_t)i * pe.chunks * 3 * ldM, pe.chunks, ldM, (int)M, X4,
                                                 Yt4 + (size_t)i * M, T4 + (size_t)i * M, sums, st[i]);
  return cudaGetLastError();
}

}  // namespace fcpd
