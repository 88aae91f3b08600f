// BF16 tensor-core GEMM of the warm-start network's per-point layers (not
// part of fast CPD): tcgen05.mma kind::f16 with BF16 operands and FP32
// accumulation in tensor memory.
//
//   D[p][n] = sum_q A[p][q] B[n][q]        (A: P x Q, B: N x Q, both BF16 with
//                                           the contraction index contiguous)
//
// One CTA computes a 128-row tile of D over a chunk of the contraction:
// thread 0 streams A and B tiles (64 BF16 of the contraction, 128-byte
// swizzle) by TMA into a 3-slot mbarrier ring; thread 32 issues four
// tcgen05.mma (M = 128, N = NB, K = 16) per slot into one TMEM accumulator
// and hands each slot back with tcgen05.commit; all four warps then read the
// accumulator (tcgen05.ld, one row per thread) and apply the epilogue:
//   split-K mode   the chunk's FP32 partial, out[chunk][p][n] (summed in a
//                  fixed order afterwards);
//   full mode      + bias[n], then ReLU or the ReLU-derivative mask
//                  (mask[p][n] > 0), written as FP32 out[p][n] and, when
//                  asked, as BF16 row-major and BF16 transposed [n][p]
//                  copies -- the operands of the next GEMMs.
// Every wait is bounded in wall time; on expiry the CTA records
// CPD_ETIMEOUT in *status, waits (bounded) for its copies and MMAs, frees
// its TMEM and returns without writing.  extra_tx > 0 (host fault injection
// only) makes every full barrier expect more bytes than its copies carry,
// so the waits run out (after wait_ns) while every copy still lands.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "tc05.cuh"

namespace fcpd {

namespace {

using namespace tc05;

constexpr int kGThreads = 128;
constexpr int kGM = 128;                  // rows of D per CTA (TMEM lanes)
constexpr int kGK = 64;                   // contraction per stage (128 bytes of BF16)
constexpr int kGABytes = kGM * kGK * 2;   // 16 KB
constexpr int kGStages = 3;
constexpr unsigned long long kGWaitNs = 2000000000ull;

template <int NB> __host__ __device__ constexpr int g_stage_bytes() { return kGABytes + NB * kGK * 2; }
template <int NB> constexpr size_t g_smem_bytes() { return (size_t)kGStages * g_stage_bytes<NB>() + 1024 + 128; }
// kind::f16 instruction descriptor: D FP32, A and B BF16, both K-major,
// N = NB, M = 128.
template <int NB> __host__ __device__ constexpr uint32_t g_idesc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NB >> 3) << 17) | ((uint32_t)(kGM >> 4) << 24);
}

struct GemmOut {
  float* out;                 // FP32 result (full mode) or partials (split-K mode)
  int64_t ldo;                // row stride of out
  int64_t chunk_stride;       // split-K: elements between chunks' partials (0: full mode)
  const float* bias;          // full mode, optional: + bias[n]
  int relu;                   // full mode: max(0, .)
  const float* mask;          // full mode, optional: 0 where mask[p][n] <= 0
  int64_t ldm;
  __nv_bfloat16* out_bf;      // optional BF16 copy [p][n]
  int64_t ldb;
  __nv_bfloat16* out_t;       // optional BF16 transposed copy [n][p]
  int64_t ldt;
};

template <int NB>
__global__ void __launch_bounds__(kGThreads, 1)
gemm_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int P, int Q, int kspc,
        GemmOut o, int* __restrict__ status, unsigned int extra_tx, unsigned long long wait_ns) {
  constexpr int STAGE = g_stage_bytes<NB>();
  constexpr uint32_t COLS = NB;           // 128 or 256 TMEM columns
  constexpr uint32_t IDESC = g_idesc<NB>();
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((1024u - (saddr(smem_raw) & 1023u)) & 1023u);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)kGStages * STAGE);
  uint64_t* empty = full + kGStages;
  uint64_t* done = empty + kGStages;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  __shared__ volatile int s_fail;
  __shared__ int s_consumed;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nk_total = (Q + kGK - 1) / kGK;
  const int k0 = blockIdx.y * kspc;
  const int nk = max(0, min(nk_total, k0 + kspc) - k0);

  if (threadIdx.x == 0) {
    s_fail = 0;
    s_consumed = 0;
    for (int i = 0; i < kGStages; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(tmem_slot, COLS);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  int issued = 0;
  if (threadIdx.x == 0) {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    for (int i = 0; i < nk; ++i) {
      const int slot = i % kGStages;
      if (i >= kGStages && !mbar_wait(&empty[slot], (uint32_t)((i / kGStages) - 1) & 1u, wait_ns)) {
        s_fail = 1;
        break;
      }
      if (s_fail) break;
      unsigned char* st = smem + (size_t)slot * STAGE;
      mbar_expect_tx(&full[slot], (uint32_t)STAGE + extra_tx);
      tma_load_2d(st, &tmA, (k0 + i) * kGK, blockIdx.x * kGM, &full[slot], pol);
      tma_load_2d(st + kGABytes, &tmB, (k0 + i) * kGK, 0, &full[slot], pol);
      issued = i + 1;
    }
  } else if (threadIdx.x == 32) {
    int i = 0;
    for (; i < nk; ++i) {
      const int slot = i % kGStages;
      if (s_fail || !mbar_wait(&full[slot], (uint32_t)(i / kGStages) & 1u, wait_ns)) {
        s_fail = 1;
        break;
      }
      fence_after();
      const uint32_t a0 = saddr(smem + (size_t)slot * STAGE);
      const uint32_t b0 = a0 + kGABytes;
#pragma unroll
      for (int kk = 0; kk < kGK / 16; ++kk)
        umma_f16(tmem, smem_desc_sw128(a0 + kk * 32), smem_desc_sw128(b0 + kk * 32), IDESC,
                 (i > 0 || kk > 0) ? 1u : 0u);
      umma_commit(&empty[slot]);
    }
    s_consumed = i;
    umma_commit(done);
  }
  const bool ok_done = mbar_wait(done, 0, wait_ns);
  __syncthreads();
  if (!ok_done) s_fail = 1;
  __syncthreads();
  if (s_fail || nk == 0) {
    if (s_fail && threadIdx.x == 0) {
      atomicExch(status, (int)CPD_ETIMEOUT);
      for (int j = s_consumed; j < issued; ++j) mbar_wait(&full[j % kGStages], (uint32_t)(j / kGStages) & 1u, wait_ns);
    }
  } else {
    fence_after();
    const int row = blockIdx.x * kGM + warp * 32 + lane;
    const bool live = row < P;
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
    float* out = o.out + (size_t)blockIdx.y * o.chunk_stride;
    for (int c0 = 0; c0 < NB; c0 += 16) {
      float v[16];
      tmem_ld16(trow + (uint32_t)c0, v);
      if (!live) continue;
      if (o.chunk_stride == 0) {
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) {
          float x = v[jj];
          if (o.bias) x += o.bias[c0 + jj];
          if (o.relu) x = fmaxf(x, 0.f);
          v[jj] = x;
        }
        if (o.mask) {
          const float4* mk = reinterpret_cast<const float4*>(o.mask + (size_t)row * o.ldm + c0);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float4 m4 = mk[q];
            if (!(m4.x > 0.f)) v[4 * q] = 0.f;
            if (!(m4.y > 0.f)) v[4 * q + 1] = 0.f;
            if (!(m4.z > 0.f)) v[4 * q + 2] = 0.f;
            if (!(m4.w > 0.f)) v[4 * q + 3] = 0.f;
          }
        }
      }
      float4* dst = reinterpret_cast<float4*>(out + (size_t)row * o.ldo + c0);
#pragma unroll
      for (int q = 0; q < 4; ++q) dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
      if (o.out_bf) {
        __align__(16) __nv_bfloat162 h[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) h[q] = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
        uint4* bd = reinterpret_cast<uint4*>(o.out_bf + (size_t)row * o.ldb + c0);
        bd[0] = reinterpret_cast<const uint4*>(h)[0];
        bd[1] = reinterpret_cast<const uint4*>(h)[1];
      }
      if (o.out_t) {
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) o.out_t[(size_t)(c0 + jj) * o.ldt + row] = __float2bfloat16_rn(v[jj]);
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    tmem_dealloc(tmem, COLS);
  }
}

// FP32 [R][C] -> BF16 row-major [R][C] (optional) and transposed [C][ldt]
// (optional), through a 32 x 32 shared tile so both writes are coalesced.
__global__ void to_bf16(const float* __restrict__ X, int64_t R, int C, __nv_bfloat16* __restrict__ row,
                        __nv_bfloat16* __restrict__ tr, int64_t ldt) {
  __shared__ float tile[32][33];
  const int64_t r0 = (int64_t)blockIdx.x * 32;
  const int c0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int64_t r = r0 + i;
    const int c = c0 + threadIdx.x;
    float v = 0.f;
    if (r < R && c < C) v = X[r * C + c];
    tile[i][threadIdx.x] = v;
    if (row && r < R && c < C) row[r * C + c] = __float2bfloat16_rn(v);
  }
  __syncthreads();
  if (!tr) return;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = c0 + i;
    const int64_t r = r0 + threadIdx.x;
    if (c < C && r < R) tr[(int64_t)c * ldt + r] = __float2bfloat16_rn(tile[threadIdx.x][i]);
  }
}

// W (fi x fo, row-major FP32) -> BF16 W (fi x fo) and W^T (fo x fi).
__global__ void weights_bf16(const float* __restrict__ W, int fi, int fo, __nv_bfloat16* __restrict__ w,
                             __nv_bfloat16* __restrict__ wt) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= fi * fo) return;
  const int i = e / fo, o = e % fo;
  const __nv_bfloat16 b = __float2bfloat16_rn(W[e]);
  if (w) w[e] = b;
  if (wt) wt[(int64_t)o * fi + i] = b;
}

int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

template <int NB> bool gemm_smem_ready() {
  static int ok = -1;
  if (ok < 0) {
    ok = cudaFuncSetAttribute(gemm_tc<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g_smem_bytes<NB>()) ==
                 cudaSuccess
             ? 1
             : 0;
    cudaGetLastError();
  }
  return ok == 1;
}

}  // namespace

// D = A B^T (A: P x Q with row stride lda, B: N x Q with row stride ldb, both
// BF16, N = 128 or 256) on the tensor cores; `chunks` > 1 splits the
// contraction (split-K mode: o.out receives chunks partials of P x N, o.ldo
// = N, o.chunk_stride = P x N; nothing else of o is used).
cudaError_t launch_gemm_tc(const __nv_bfloat16* A, int64_t lda, const __nv_bfloat16* B, int64_t ldb, int P, int N,
                           int Q, int chunks, const float* bias, bool relu, const float* mask, int64_t ldm,
                           float* out, int64_t ldo, __nv_bfloat16* out_bf, int64_t ld_bf, __nv_bfloat16* out_t,
                           int64_t ld_t, int* status, bool fault_wait, cudaStream_t s) {
  if (N != 128 && N != 256) return cudaErrorInvalidValue;
  const unsigned int extra_tx = fault_wait ? 16u : 0u;
  const unsigned long long wait_ns = fault_wait ? 50000000ull : kGWaitNs;
  CUtensorMap ma, mb;
  if (!make_map_2d(&ma, A, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, P, Q, lda, kGM) ||
      !make_map_2d(&mb, B, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, N, Q, ldb, N))
    return cudaErrorInvalidValue;
  const int nk = (int)cdiv(Q, kGK);
  chunks = std::max(1, std::min(chunks, nk));
  const int kspc = (int)cdiv(nk, chunks);
  chunks = (int)cdiv(nk, kspc);
  GemmOut o{};
  o.out = out;
  o.ldo = ldo;
  if (chunks > 1) {
    o.chunk_stride = (int64_t)P * ldo;
  } else {
    o.bias = bias;
    o.relu = relu ? 1 : 0;
    o.mask = mask;
    o.ldm = ldm;
    o.out_bf = out_bf;
    o.ldb = ld_bf;
    o.out_t = out_t;
    o.ldt = ld_t;
  }
  const dim3 grid((unsigned)cdiv(P, kGM), (unsigned)chunks);
  if (N == 128) {
    if (!gemm_smem_ready<128>()) return cudaErrorInvalidValue;
    gemm_tc<128><<<grid, kGThreads, g_smem_bytes<128>(), s>>>(ma, mb, P, Q, kspc, o, status, extra_tx, wait_ns);
  } else {
    if (!gemm_smem_ready<256>()) return cudaErrorInvalidValue;
    gemm_tc<256><<<grid, kGThreads, g_smem_bytes<256>(), s>>>(ma, mb, P, Q, kspc, o, status, extra_tx, wait_ns);
  }
  return cudaGetLastError();
}

// Chunks actually used for a split-K contraction of length Q.
int gemm_tc_chunks(int Q, int chunks) {
  const int nk = (int)cdiv(Q, kGK);
  chunks = std::max(1, std::min(chunks, nk));
  const int kspc = (int)cdiv(nk, chunks);
  return (int)cdiv(nk, kspc);
}

void launch_to_bf16(const float* X, int64_t R, int C, __nv_bfloat16* row, __nv_bfloat16* tr, int64_t ldt,
                    cudaStream_t s) {
  to_bf16<<<dim3((unsigned)cdiv(R, 32), (unsigned)cdiv(C, 32)), dim3(32, 8), 0, s>>>(X, R, C, row, tr, ldt);
}

void launch_weights_bf16(const float* W, int fi, int fo, __nv_bfloat16* w, __nv_bfloat16* wt, cudaStream_t s) {
  weights_bf16<<<(unsigned)cdiv((int64_t)fi * fo, 256), 256, 0, s>>>(W, fi, fo, w, wt);
}

}  // namespace fcpd
