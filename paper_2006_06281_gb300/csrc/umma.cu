// Tensor-core M-step products for several scenes against one model (Eq. 17 /
// Eq. 20 with one eigenbasis for S scenes), on sm_103a's fifth-generation
// tensor cores: tcgen05.mma with operands staged in shared memory by TMA and
// the accumulator in tensor memory (TMEM).
//
// With S scenes the two products of an M-step are
//     projection  a_s = U^T R_s     (K x 3 per scene; R_s = Ytil_s - X)
//     expansion   d_s = U B_s       (M x 3 per scene; B_s = diag(s) a_s)
// i.e. D = A V^T with A the stored FP16 basis (U^T for the projection, U for
// the expansion: both row-major with the contraction index contiguous) and V
// the 3S right-hand sides, transposed so the contraction index is contiguous
// too.  Each right-hand side is split into two FP16 parts, hi = fp16(r) and
// lo = fp16(r - hi): the products of FP16 values are exact in the FP32
// accumulator, so the result carries the FP16 rounding of the basis only
// (the same as the single-scene mixed-precision M-step), not of the scenes.
// V's rows: [0, 3S) hi, [H, H + 3S) lo, the rest zero (H = 3S rounded up to
// 16); NPAD = 2H columns of the MMA, 16 <= NPAD <= 256.
//
// Kernel layout (128 threads, one 128-row tile of D per CTA, a chunk of the
// contraction per blockIdx.y; split-K partials are summed by the per-scene
// reduction kernels that follow, in a fixed order):
//   thread 0    TMA producer: A tile (128 rows x 64 FP16) and V tile (NPAD
//               rows x 64 FP16) per stage, 128-byte swizzle, into a ring of
//               kStages slots, each slot's full barrier completing on the
//               bytes; it refills a slot once the MMAs that read it signal
//               the slot's empty barrier (tcgen05.commit).
//   thread 32   MMA issuer: four tcgen05.mma (M = 128, N = NPAD, K = 16) per
//               stage into one TMEM accumulator, then a commit to the slot's
//               empty barrier; after the last stage a commit to `done`.
//   all warps   epilogue: warp w reads TMEM lanes 32w..32w+31 (its rows) with
//               tcgen05.ld, adds the hi and lo columns of each right-hand
//               side and writes the partials part[s][chunk][d][row].
// Every wait is bounded in wall time (%globaltimer); on expiry the CTA
// records CPD_ETIMEOUT in *status, stops issuing, waits (bounded) for its
// copies and MMAs in flight, frees its TMEM and returns without writing.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "tc05.cuh"

namespace fcpd {

namespace {

using namespace tc05;

constexpr int kUThreads = 128;
constexpr int kUM = 128;                 // rows of D per tile = TMEM lanes
constexpr int kUK = 64;                  // contraction elements per stage (128 bytes of FP16)
constexpr int kUABytes = kUM * kUK * 2;  // 16 KB
constexpr unsigned long long kUWaitNs = 2000000000ull;

__host__ __device__ constexpr int tmem_cols(int n) { return n <= 32 ? 32 : n <= 64 ? 64 : n <= 128 ? 128 : 256; }
template <int NPAD> __host__ __device__ constexpr int stage_bytes() { return kUABytes + NPAD * kUK * 2; }
// Ring depth: 3 slots while two CTAs fit on an SM (one CTA's start-up and
// epilogue overlap the other's streaming), 4 when only one does.
template <int NPAD> __host__ __device__ constexpr int stages() { return stage_bytes<NPAD>() <= 32 * 1024 ? 3 : 4; }
template <int NPAD> constexpr size_t umma_smem_bytes() {
  return (size_t)stages<NPAD>() * stage_bytes<NPAD>() + 1024 /* alignment slack */ + 128 /* barriers, TMEM slot */;
}

// D[row][j] = sum_q A[row][q] V[j][q] for the rows of tile blockIdx.x and the
// contraction stages [blockIdx.y * kspc, ...): partials of scene s written to
// part[((s * chunks + blockIdx.y) * 3 + d) * ldP + row] = D[row][3s+d] +
// D[row][H+3s+d].  extra_tx > 0 (host fault injection only) makes every full
// barrier expect that many bytes more than its copies carry.
template <int NPAD>
__global__ void __launch_bounds__(kUThreads, 1)
umma_products(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmV, int P, int Q,
              int kspc, int chunks, int S, float* __restrict__ part, int64_t ldP, int* __restrict__ status,
              unsigned int extra_tx, unsigned long long wait_ns) {
  constexpr int H = NPAD / 2;
  constexpr int STAGE = stage_bytes<NPAD>();
  constexpr int kUStages = stages<NPAD>();
  constexpr uint32_t COLS = tmem_cols(NPAD);
  constexpr uint32_t IDESC = idesc_f16_m128(NPAD);
  extern __shared__ unsigned char smem_raw[];
  // 1024-byte aligned, by an offset from the shared array (an integer round
  // trip would turn later accesses into generic ones)
  unsigned char* smem = smem_raw + ((1024u - (saddr(smem_raw) & 1023u)) & 1023u);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)kUStages * STAGE);
  uint64_t* empty = full + kUStages;
  uint64_t* done = empty + kUStages;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  __shared__ volatile int s_fail;
  __shared__ int s_consumed;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nk_total = (Q + kUK - 1) / kUK;
  const int k0 = blockIdx.y * kspc;
  const int nk = max(0, min(nk_total, k0 + kspc) - k0);

  if (threadIdx.x == 0) {
    s_fail = 0;
    s_consumed = 0;
    for (int i = 0; i < kUStages; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(tmem_slot)),
                 "r"(COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  int issued = 0;
  if (threadIdx.x == 0) {
    // TMA producer
    uint64_t pol_a, pol_v;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol_a));
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol_v));
    for (int i = 0; i < nk; ++i) {
      const int slot = i % kUStages;
      if (i >= kUStages && !mbar_wait(&empty[slot], (uint32_t)((i / kUStages) - 1) & 1u, wait_ns)) {
        s_fail = 1;
        break;
      }
      if (s_fail) break;
      unsigned char* st = smem + (size_t)slot * STAGE;
      mbar_expect_tx(&full[slot], (uint32_t)STAGE + extra_tx);
      tma_load_2d(st, &tmA, (k0 + i) * kUK, blockIdx.x * kUM, &full[slot], pol_a);
      tma_load_2d(st + kUABytes, &tmV, (k0 + i) * kUK, 0, &full[slot], pol_v);
      issued = i + 1;
    }
  } else if (threadIdx.x == 32) {
    // MMA issuer
    int i = 0;
    for (; i < nk; ++i) {
      const int slot = i % kUStages;
      if (s_fail || !mbar_wait(&full[slot], (uint32_t)(i / kUStages) & 1u, wait_ns)) {
        s_fail = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = saddr(smem + (size_t)slot * STAGE);
      const uint32_t v0 = a0 + kUABytes;
#pragma unroll
      for (int kk = 0; kk < kUK / 16; ++kk)
        umma_f16(tmem, smem_desc_sw128(a0 + kk * 32), smem_desc_sw128(v0 + kk * 32), IDESC,
                 (i > 0 || kk > 0) ? 1u : 0u);
      umma_commit(&empty[slot]);
    }
    s_consumed = i;
    umma_commit(done);      // arrives once every MMA issued above has completed
  }
  // everyone: the accumulator is complete (or the CTA gave up)
  const bool ok_done = mbar_wait(done, 0, wait_ns);
  __syncthreads();
  if (!ok_done) s_fail = 1;
  __syncthreads();
  const bool failed = s_fail != 0;
  if (failed) {
    if (threadIdx.x == 0) {
      atomicExch(status, (int)CPD_ETIMEOUT);
      // copies issued but never consumed are still landing: wait for them
      for (int j = s_consumed; j < issued; ++j) mbar_wait(&full[j % kUStages], (uint32_t)(j / kUStages) & 1u, wait_ns);
    }
  } else {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int row = blockIdx.x * kUM + warp * 32 + lane;
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
    const int nrhs = 3 * S;
    for (int j0 = 0; j0 < nrhs; j0 += 16) {
      float hi[16], lo[16];
      tmem_ld16(trow + (uint32_t)j0, hi);
      tmem_ld16(trow + (uint32_t)(H + j0), lo);
      if (row < P) {
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) {
          const int j = j0 + jj;
          if (j < nrhs) {
            const int s = j / 3, d = j - 3 * s;
            part[(((size_t)s * chunks + blockIdx.y) * 3 + d) * ldP + row] = hi[jj] + lo[jj];
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(COLS) : "memory");
  }
}

// V (NPAD rows x ldq, FP16, row j contiguous over the contraction index q):
// rows 3s+d and H+3s+d hold the hi and lo FP16 parts of component d of
// src[s * ld_src + q] for q < Q.  Padding rows and columns stay as zeroed at
// allocation.
__global__ void pack_rhs_f16(const float4* __restrict__ src, int64_t ld_src, int S, int Q, int H, int64_t ldq,
                             __half* __restrict__ V) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)S * Q) return;
  const int s = (int)(i / Q), q = (int)(i - (int64_t)s * Q);
  const float4 r = src[(size_t)s * ld_src + q];
  const float c[3] = {r.x, r.y, r.z};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const __half h = __float2half_rn(c[d]);
    const __half l = __float2half_rn(c[d] - __half2float(h));
    V[(size_t)(3 * s + d) * ldq + q] = h;
    V[(size_t)(H + 3 * s + d) * ldq + q] = l;
  }
}

int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, []() {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

// Row-major FP16 matrix [rows][cols] with row stride ld elements; box
// {kUK, box_rows}, 128-byte swizzle, zero fill outside.
bool make_map(CUtensorMap* map, const __half* base, int64_t rows, int64_t cols, int64_t ld, int box_rows) {
  return tc05::make_map_2d(map, base, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, rows, cols, ld, box_rows);
}

template <int NPAD> int umma_occupancy() {
  const int bytes = (int)umma_smem_bytes<NPAD>();
  if (cudaFuncSetAttribute(umma_products<NPAD>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess ||
      cudaFuncSetAttribute(umma_products<NPAD>, cudaFuncAttributePreferredSharedMemoryCarveout,
                           cudaSharedmemCarveoutMaxShared) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, umma_products<NPAD>, kUThreads, bytes);
  return occ;
}

int occupancy_for_npad(int npad) {
  switch (npad) {
    case 32: return umma_occupancy<32>();
    case 64: return umma_occupancy<64>();
    case 96: return umma_occupancy<96>();
    case 128: return umma_occupancy<128>();
    case 160: return umma_occupancy<160>();
    case 192: return umma_occupancy<192>();
    case 224: return umma_occupancy<224>();
    default: return umma_occupancy<256>();
  }
}

template <int NPAD>
cudaError_t launch_products_npad(const CUtensorMap& a, const CUtensorMap& v, int P, int Q, int tiles, int chunks,
                                 int kspc, int S, float* part, int64_t ldP, int* status, unsigned int extra_tx,
                                 unsigned long long wait_ns, cudaStream_t s) {
  umma_products<NPAD><<<dim3(tiles, chunks), kUThreads, umma_smem_bytes<NPAD>(), s>>>(
      a, v, P, Q, kspc, chunks, S, part, ldP, status, extra_tx, wait_ns);
  return cudaGetLastError();
}

}  // namespace

bool tc05::make_map_2d(CUtensorMap* map, const void* base, CUtensorMapDataType type, int64_t rows, int64_t cols,
                       int64_t ld, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  const cuuint32_t box[2] = {(cuuint32_t)kUK, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return fn(map, type, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

int umma_npad(int S) {
  const int h = (int)cdiv(3 * S, 16) * 16;
  return 2 * h;
}

bool umma_supported(int S) {
  if (S < 1 || umma_npad(S) > 256) return false;
  return encode_fn() != nullptr;
}

UmmaPlan plan_umma(int64_t P, int64_t Q, int S, int sms) {
  UmmaPlan p{};
  p.P = P;
  p.Q = Q;
  p.S = S;
  p.npad = umma_npad(S);
  p.tiles = (int)cdiv(P, kUM);
  const int64_t nk = cdiv(Q, kUK);
  const int64_t slots = (int64_t)sms * std::max(1, occupancy_for_npad(p.npad));
  // chunks of the contraction: one resident wave costs (stages + fixed
  // per-CTA overhead); pick the split with the least total cost, at least 8
  // stages per CTA so the ring is filled
  double best = 1e300;
  int64_t best_c = 1;
  for (int64_t c = 1; c <= std::max<int64_t>(1, nk / 8); ++c) {
    const int64_t kspc = cdiv(nk, c);
    const int64_t ch = cdiv(nk, kspc);
    const double cost = (double)cdiv((int64_t)p.tiles * ch, slots) * (double)(kspc + 6);
    if (cost < best - 1e-9) {
      best = cost;
      best_c = c;
    }
  }
  p.kspc = (int)cdiv(nk, best_c);
  p.chunks = (int)cdiv(nk, p.kspc);
  p.ldq = cdiv(Q, 8) * 8;
  return p;
}

int64_t umma_rhs_elems(const UmmaPlan& p) { return (int64_t)p.npad * p.ldq; }

void launch_pack_rhs(const UmmaPlan& p, const float4* src, int64_t ld_src, __half* V, cudaStream_t s) {
  const int64_t n = (int64_t)p.S * p.Q;
  pack_rhs_f16<<<(unsigned)cdiv(n, 256), 256, 0, s>>>(src, ld_src, p.S, (int)p.Q, p.npad / 2, p.ldq, V);
}

cudaError_t launch_umma_products(const UmmaPlan& p, const __half* A, int64_t ldA, const __half* V, float* part,
                                 int64_t ldP, int* status, bool fault_wait, cudaStream_t s) {
  CUtensorMap ma, mv;
  if (!make_map(&ma, A, p.P, p.Q, ldA, kUM) || !make_map(&mv, V, p.npad, p.Q, p.ldq, p.npad))
    return cudaErrorInvalidValue;
  const unsigned int extra = fault_wait ? 16u : 0u;
  const unsigned long long wait_ns = fault_wait ? 50000000ull : kUWaitNs;
  const int P = (int)p.P, Q = (int)p.Q;
  switch (p.npad) {
    case 32: return launch_products_npad<32>(ma, mv, P, Q, p.tiles, p.chunks, p.kspc, p.S, part, ldP, status, extra, wait_ns, s);
    case 64: return launch_products_npad<64>(ma, mv, P, Q, p.tiles, p.chunks, p.kspc, p.S, part, ldP, status, extra, wait_ns, s);
    case 96: return launch_products_npad<96>(ma, mv, P, Q, p.tiles, p.chunks, p.kspc, p.S, part, ldP, status, extra, wait_ns, s);
    case 128: return launch_products_npad<128>(ma, mv, P, Q, p.tiles, p.chunks, p.kspc, p.S, part, ldP, status, extra, wait_ns, s);
    case 160: return launch_products_npad<160>(ma, mv, P, Q, p.tiles, p.chunks, p.kspc, p.S, part, ldP, status, extra, wait_ns, s);
    case 192: return launch_products_npad<192>(ma, mv, P, Q, p.tiles, p.chunks, p.kspc, p.S, part, ldP, status, extra, wait_ns, s);
    case 224: return launch_products_npad<224>(ma, mv, P, Q, p.tiles, p.chunks, p.kspc, p.S, part, ldP, status, extra, wait_ns, s);
    case 256: return launch_products_npad<256>(ma, mv, P, Q, p.tiles, p.chunks, p.kspc, p.S, part, ldP, status, extra, wait_ns, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fcpd
