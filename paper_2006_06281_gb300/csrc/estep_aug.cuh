// Augmented FP16 vectors of the tensor-core distance tiles (mixed-precision
// E-step): for a row point r' and a column point c' (coordinates pre-scaled
// by q) the K = 16 dot product of their vectors is
//     2 r'.c' - |r'|^2 - |c'|^2 + lid_c  =  lid_c - |r' - c'|^2,
// the base-2 exponent of the Gaussian (lid_c = -log2 den_c in pass B, 0 in
// pass A).  Each FP32 value v is split into two FP16 parts v1 + v2 (22
// significant bits); the cross products v1 w1, v1 w2, v2 w1 are kept (v2 w2 is
// 2^-22 of the product), the norms and lid enter as split terms against an
// exact 1:
//   k  0..8   row side 2 r_d^(i)           col side c_d^(j)   (d, (i, j) in (1,1) (1,2) (2,1))
//   k  9..10  row side -|r'|^2 (split)     col side 1
//   k 11..12  row side 1                   col side -|c'|^2 (split)
//   k 13..14  row side 1                   col side lid (split; 0 in pass A)
//   k 15      0
#pragma once

#include <cuda_fp16.h>

namespace fcpd {
namespace dev {

constexpr int kAugK = 16;                   // augmented dimension
constexpr float kPadNorm = -60000.f;        // padding column: exponents far below -126, finite in FP16

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

}  // namespace dev
}  // namespace fcpd
