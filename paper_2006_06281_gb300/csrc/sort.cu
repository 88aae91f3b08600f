// Spatial ordering of point sets, and the permuted copies between the
// caller's order and the sorted order.
//
// Points are ordered by a 12-bit Morton key: the bounding box is cut into
// 16 x 16 x 16 cells and the cell indices' bits are interleaved, so points
// that are consecutive in the sorted order are close in space.  The E-step
// relies on that only for speed (exact pruning of far tile pairs); no result
// depends on the order beyond summation order.
//
// The sort is a stable counting sort on the device: one warp per tile of
// 1024 points counts its keys, an exclusive scan over (key, tile) gives every
// tile's first slot per key, and the warp scatters its points in their
// original order (ranks among equal keys within a round of 32 come from
// __match_any_sync), so the result is deterministic.
#include "common.cuh"

namespace fcpd {

namespace {

constexpr int kKeys = 4096;          // 2^12 Morton cells
constexpr int kTile = 1024;          // points per sorting warp
constexpr int kScanThreads = 1024;

int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

__device__ __forceinline__ unsigned int spread4(unsigned int v) {
  // bits b3 b2 b1 b0 -> b3 0 0 b2 0 0 b1 0 0 b0
  return (v & 1u) | ((v & 2u) << 2) | ((v & 4u) << 4) | ((v & 8u) << 6);
}

__device__ __forceinline__ int cell(float v, float lo, float inv) {
  const int c = (int)((v - lo) * inv);
  return c < 0 ? 0 : c > 15 ? 15 : c;
}

__device__ __forceinline__ unsigned int morton_key(const float4& p, const float* box) {
  const int cx = cell(p.x, box[0], box[3]), cy = cell(p.y, box[1], box[4]), cz = cell(p.z, box[2], box[5]);
  return spread4(cx) | (spread4(cy) << 1) | (spread4(cz) << 2);
}

// box[0..2] = lower corner, box[3..5] = 16 / extent per axis (0 for a flat axis).
__global__ void __launch_bounds__(1024) bounding_box(const float4* __restrict__ P, int64_t n, float* __restrict__ box) {
  __shared__ float sh[6][32];
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const float4 p = P[i];
    lo[0] = fminf(lo[0], p.x); lo[1] = fminf(lo[1], p.y); lo[2] = fminf(lo[2], p.z);
    hi[0] = fmaxf(hi[0], p.x); hi[1] = fmaxf(hi[1], p.y); hi[2] = fmaxf(hi[2], p.z);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      lo[d] = fminf(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], o));
      hi[d] = fmaxf(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], o));
    }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0)
    for (int d = 0; d < 3; ++d) { sh[d][w] = lo[d]; sh[3 + d][w] = hi[d]; }
  __syncthreads();
  if (threadIdx.x < 3) {
    const int d = threadIdx.x;
    float a = INFINITY, b = -INFINITY;
    for (int j = 0; j < (int)(blockDim.x >> 5); ++j) { a = fminf(a, sh[d][j]); b = fmaxf(b, sh[3 + d][j]); }
    box[d] = a;
    box[3 + d] = b > a ? 16.0f / (b - a) : 0.0f;
  }
}

// Per tile: count of each key, written key-major (hist[key * tiles + tile]).
__global__ void __launch_bounds__(32) count_keys(const float4* __restrict__ P, int64_t n, const float* __restrict__ box,
                                                 int* __restrict__ hist, int tiles) {
  __shared__ int cnt[kKeys];
  __shared__ float sbox[6];
  const int lane = threadIdx.x;
  if (lane < 6) sbox[lane] = box[lane];
  for (int k = lane; k < kKeys; k += 32) cnt[k] = 0;
  __syncwarp();
  const int64_t t0 = (int64_t)blockIdx.x * kTile;
  const int64_t t1 = t0 + kTile < n ? t0 + kTile : n;
  for (int64_t i = t0 + lane; i < t1; i += 32) atomicAdd(&cnt[morton_key(P[i], sbox)], 1);
  __syncwarp();
  for (int k = lane; k < kKeys; k += 32) hist[(int64_t)k * tiles + blockIdx.x] = cnt[k];
}

// Exclusive scan of `len` ints in place, one block.
__global__ void __launch_bounds__(kScanThreads) exclusive_scan(int* __restrict__ a, int64_t len) {
  __shared__ int part[kScanThreads];
  const int64_t seg = (len + kScanThreads - 1) / kScanThreads;
  const int64_t b = threadIdx.x * seg;
  const int64_t e = b + seg < len ? b + seg : len;
  int s = 0;
  for (int64_t i = b; i < e; ++i) s += a[i];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int o = 1; o < kScanThreads; o <<= 1) {     // Hillis-Steele over the segment sums
    const int v = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  int run = threadIdx.x ? part[threadIdx.x - 1] : 0;
  for (int64_t i = b; i < e; ++i) {
    const int v = a[i];
    a[i] = run;
    run += v;
  }
}

// Stable scatter: points of each tile go to their key's slots in original order.
__global__ void __launch_bounds__(32) scatter_keys(const float4* __restrict__ P, int64_t n,
                                                   const float* __restrict__ box, const int* __restrict__ offs,
                                                   int tiles, float4* __restrict__ out, int* __restrict__ perm) {
  __shared__ int cur[kKeys];
  __shared__ float sbox[6];
  const int lane = threadIdx.x;
  if (lane < 6) sbox[lane] = box[lane];
  for (int k = lane; k < kKeys; k += 32) cur[k] = offs[(int64_t)k * tiles + blockIdx.x];
  __syncwarp();
  const int64_t t0 = (int64_t)blockIdx.x * kTile;
  const int64_t t1 = t0 + kTile < n ? t0 + kTile : n;
  for (int64_t base = t0; base < t1; base += 32) {
    const int64_t i = base + lane;
    const unsigned int valid = __ballot_sync(0xffffffffu, i < t1);
    if (i < t1) {
      const float4 p = P[i];
      const unsigned int key = morton_key(p, sbox);
      const unsigned int peers = __match_any_sync(valid, key);
      const int rank = __popc(peers & ((1u << lane) - 1u));
      const int pos = cur[key] + rank;
      __syncwarp(valid);
      if (rank == 0) cur[key] += __popc(peers);
      out[pos] = p;
      if (perm) perm[pos] = (int)i;
    }
    __syncwarp();
  }
}

__global__ void invert_perm(const int* __restrict__ perm, int64_t n, int* __restrict__ inv) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n) inv[perm[s]] = (int)s;
}

template <typename F>
__global__ void pack_gather(const F* __restrict__ src, const int* __restrict__ perm, int64_t n,
                            typename Vec<F>::t4* __restrict__ dst, int with_norm) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int64_t i = perm[s];
  typename Vec<F>::t4 v;
  v.x = src[3 * i]; v.y = src[3 * i + 1]; v.z = src[3 * i + 2];
  v.w = with_norm ? v.x * v.x + v.y * v.y + v.z * v.z : (F)0;
  dst[s] = v;
}

template <typename F>
__global__ void unpack_gather(const typename Vec<F>::t4* __restrict__ src, const int* __restrict__ inv, int64_t n,
                              F* __restrict__ dst) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const typename Vec<F>::t4 v = src[inv[i]];
  dst[3 * i] = v.x; dst[3 * i + 1] = v.y; dst[3 * i + 2] = v.z;
}

__global__ void gather_rows_f32(const float* __restrict__ src, int64_t ld_src, const int* __restrict__ inv, int64_t n,
                                int64_t cols, float* __restrict__ dst) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * cols) return;
  const int64_t i = e / cols, k = e % cols;
  dst[e] = src[(int64_t)inv[i] * ld_src + k];
}

}  // namespace

int64_t spatial_sort_scratch_bytes(int64_t n) {
  const int64_t tiles = cdiv(n, kTile);
  return 64 + (int64_t)kKeys * tiles * (int64_t)sizeof(int);
}

bool spatial_sort_supported(int64_t n) { return n >= 1 && n <= kMaxSortPoints; }

cudaError_t launch_spatial_sort(const float4* in, int64_t n, float4* out, int* perm, void* scratch, cudaStream_t s) {
  const int tiles = (int)cdiv(n, kTile);
  float* box = static_cast<float*>(scratch);
  int* hist = reinterpret_cast<int*>(static_cast<char*>(scratch) + 64);
  bounding_box<<<1, 1024, 0, s>>>(in, n, box);
  count_keys<<<tiles, 32, 0, s>>>(in, n, box, hist, tiles);
  exclusive_scan<<<1, kScanThreads, 0, s>>>(hist, (int64_t)kKeys * tiles);
  scatter_keys<<<tiles, 32, 0, s>>>(in, n, box, hist, tiles, out, perm);
  return cudaGetLastError();
}

void launch_invert_perm(const int* perm, int64_t n, int* inv, cudaStream_t s) {
  invert_perm<<<(unsigned)cdiv(n, 256), 256, 0, s>>>(perm, n, inv);
}

template <typename F>
void launch_pack_gather(const F* src, const int* perm, int64_t n, typename Vec<F>::t4* dst, bool with_norm,
                        cudaStream_t s) {
  pack_gather<F><<<(unsigned)cdiv(n, 256), 256, 0, s>>>(src, perm, n, dst, with_norm ? 1 : 0);
}

template <typename F>
void launch_unpack_gather(const typename Vec<F>::t4* src, const int* inv, int64_t n, F* dst, cudaStream_t s) {
  unpack_gather<F><<<(unsigned)cdiv(n, 256), 256, 0, s>>>(src, inv, n, dst);
}

void launch_gather_rows_f32(const float* src, int64_t ld_src, const int* inv, int64_t n, int64_t cols, float* dst,
                            cudaStream_t s) {
  gather_rows_f32<<<(unsigned)cdiv(n * cols, 256), 256, 0, s>>>(src, ld_src, inv, n, cols, dst);
}

template void launch_pack_gather<float>(const float*, const int*, int64_t, float4*, bool, cudaStream_t);
template void launch_unpack_gather<float>(const float4*, const int*, int64_t, float*, cudaStream_t);

}  // namespace fcpd
