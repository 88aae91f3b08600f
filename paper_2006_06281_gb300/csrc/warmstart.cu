// Learned warm start (not part of fast CPD): a point-set network that
// predicts where the EM loop will end -- the leading eigen-coefficients of
// the displacement T - X in the context's basis and log sigma2 -- so a
// registration can start there instead of at W = 0.  The paper's EM loop
// itself is unchanged; a start from W = 0 stays the fallback.
//
// Network (the layout of the FP64 reference in the tests): a per-point MLP
// 3 -> 128 -> 128 -> 256 (ReLU) shared by all points, the maximum over the
// points of each feature, and a head 256 -> 256 (ReLU) -> n_out.  Every step
// of training and inference runs in the kernels below: a tiled FP32 GEMM
// with optional operand transposes, fused bias and ReLU (split over K with a
// fixed-order reduction for the weight gradients, whose reduction runs over
// all B x N points), max-pool forward/backward, ReLU masks, column sums, the
// mean-squared-error gradient and Adam.  FP32 throughout (results are
// deterministic: no atomics in any sum).
//
// BF16 precision (cpd_net_create_ex): the two wide per-point layers
// (128 -> 128 and 128 -> 256, over all B x N points) and their three
// backward products each (the activation gradient and the weight gradient)
// run on the tensor cores -- tcgen05 BF16 x BF16 -> FP32 (gemm_tc.cu) with
// bias, ReLU and the ReLU-derivative mask in the epilogue, which also writes
// the BF16 row-major and transposed operands of the next product.  Master
// weights, Adam moments, biases, the first layer (3 inputs), the head and all
// reductions stay FP32.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <random>
#include <string>
#include <vector>

#include "common.cuh"

using namespace fcpd;

namespace {

constexpr int kGT = 64;       // GEMM tile (rows and columns of C per block)
constexpr int kGK = 16;       // K step
constexpr int kGThreads = 256;
constexpr int kSplitK = 64;   // K splits of the weight-gradient GEMMs
constexpr int kTcChunks = 128;  // contraction chunks of the BF16 weight-gradient products

int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// C_z = op(A) op(B) (+ bias[col], ReLU) over K range z of a split; C_z = C + z * strideC.
__global__ void __launch_bounds__(kGThreads)
sgemm(const float* __restrict__ A, int64_t lda, int ta, const float* __restrict__ B, int64_t ldb, int tb,
      float* __restrict__ C, int64_t ldc, int64_t strideC, int M, int N, int K, int kchunk,
      const float* __restrict__ bias, int relu) {
  __shared__ float As[kGK][kGT + 4];
  __shared__ float Bs[kGK][kGT + 4];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int i0 = blockIdx.y * kGT, j0 = blockIdx.x * kGT;
  const int kb = blockIdx.z * kchunk;
  const int ke = min(K, kb + kchunk);
  float acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = 0.f;
  for (int k0 = kb; k0 < ke; k0 += kGK) {
    for (int e = threadIdx.x; e < kGT * kGK; e += kGThreads) {
      int ii, kk;
      if (ta) { kk = e / kGT; ii = e % kGT; } else { ii = e / kGK; kk = e % kGK; }
      const int gi = i0 + ii, gk = k0 + kk;
      float v = 0.f;
      if (gi < M && gk < ke) v = ta ? A[(int64_t)gk * lda + gi] : A[(int64_t)gi * lda + gk];
      As[kk][ii] = v;
    }
    for (int e = threadIdx.x; e < kGT * kGK; e += kGThreads) {
      int jj, kk;
      if (tb) { jj = e / kGK; kk = e % kGK; } else { kk = e / kGT; jj = e % kGT; }
      const int gj = j0 + jj, gk = k0 + kk;
      float v = 0.f;
      if (gj < N && gk < ke) v = tb ? B[(int64_t)gj * ldb + gk] : B[(int64_t)gk * ldb + gj];
      Bs[kk][jj] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kGK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[kk][ty + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = Bs[kk][tx + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(a[r], b[c], acc[r][c]);
    }
    __syncthreads();
  }
  float* Cz = C + (int64_t)blockIdx.z * strideC;
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int i = i0 + ty + 16 * r, j = j0 + tx + 16 * c;
      if (i < M && j < N) {
        float v = acc[r][c];
        if (bias) v += bias[j];
        if (relu) v = fmaxf(v, 0.f);
        Cz[(int64_t)i * ldc + j] = v;
      }
    }
}

// out[e] = sum_z part[z * n + e] (z in order).
__global__ void sum_splits(const float* __restrict__ part, int S, int64_t n, float* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  float s = 0.f;
  for (int z = 0; z < S; ++z) s += part[(int64_t)z * n + e];
  out[e] = s;
}

// part[z][c] = sum of rows [z * rows_per, ...) of column c; then sum_splits.
__global__ void col_sum_part(const float* __restrict__ X, int64_t R, int C, int64_t rows_per, float* __restrict__ part) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  const int64_t r0 = (int64_t)blockIdx.y * rows_per;
  const int64_t r1 = r0 + rows_per < R ? r0 + rows_per : R;
  float s = 0.f;
  for (int64_t r = r0; r < r1; ++r) s += X[r * C + c];
  part[(int64_t)blockIdx.y * C + c] = s;
}

__global__ void relu_mask(float* __restrict__ d, const float* __restrict__ h, int64_t n) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n && !(h[e] > 0.f)) d[e] = 0.f;
}

// g[b][f] = max over the points of h[b][n][f]; arg = first index of the maximum.
__global__ void maxpool_fwd(const float* __restrict__ h, int N, int F, float* __restrict__ g, int* __restrict__ arg) {
  const int b = blockIdx.x, f = threadIdx.x;
  if (f >= F) return;
  const float* hb = h + (int64_t)b * N * F;
  float best = hb[f];
  int bi = 0;
  for (int n = 1; n < N; ++n) {
    const float v = hb[(int64_t)n * F + f];
    if (v > best) { best = v; bi = n; }
  }
  g[b * F + f] = best;
  arg[b * F + f] = bi;
}

__global__ void maxpool_bwd(const float* __restrict__ dg, const int* __restrict__ arg, int N, int F,
                            float* __restrict__ dh) {
  const int b = blockIdx.x, f = threadIdx.x;
  if (f >= F) return;
  dh[((int64_t)b * N + arg[b * F + f]) * F + f] = dg[b * F + f];
}

// dpred = 2 (pred - target) / count; loss = mean of squares (one block, fixed order).
__global__ void __launch_bounds__(1024) mse_grad(const float* __restrict__ pred, const float* __restrict__ tgt, int n,
                                                 float* __restrict__ dpred, float* __restrict__ loss) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const float d = pred[e] - tgt[e];
    dpred[e] = 2.0f * d / (float)n;
    s += (double)d * d;
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) *loss = (float)(s / n);
}

__global__ void adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                     int64_t n, float lr_t, float b1, float b2, float eps) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const float gi = g[e];
  const float mi = b1 * m[e] + (1.f - b1) * gi;
  const float vi = b2 * v[e] + (1.f - b2) * gi * gi;
  m[e] = mi;
  v[e] = vi;
  p[e] -= lr_t * mi / (sqrtf(vi) + eps);
}

// Basis element as float (FP32 basis, or the FP16 basis of the mixed mode).
__device__ __forceinline__ float basis_f(float u) { return u; }
__device__ __forceinline__ float basis_f(__half u) { return __half2float(u); }

// c[k][d] = sum_m U[m][k] (T[m] - X[m])_d, one block per k, fixed order.
template <typename B>
__global__ void __launch_bounds__(256) coefficients(const B* __restrict__ U, int64_t ldU, int M,
                                                    const float4* __restrict__ T4, const float4* __restrict__ X4,
                                                    float* __restrict__ c) {
  __shared__ double sh[32];
  const int k = blockIdx.x;
  double s[3] = {0.0, 0.0, 0.0};
  for (int m = threadIdx.x; m < M; m += blockDim.x) {
    const double u = basis_f(U[(int64_t)m * ldU + k]);
    const float4 t = T4[m], x = X4[m];
    s[0] += u * ((double)t.x - x.x);
    s[1] += u * ((double)t.y - x.y);
    s[2] += u * ((double)t.z - x.z);
  }
  for (int d = 0; d < 3; ++d) {
    const double v = block_sum(s[d], sh);
    if (threadIdx.x == 0) c[3 * k + d] = (float)v;
  }
}

// T[m] = X[m] + sum_{k < nc} U[m][k] c[k].
template <typename B>
__global__ void warm_start_T(const B* __restrict__ U, int64_t ldU, int M, int nc, const float* __restrict__ c,
                             const float4* __restrict__ X4, float4* __restrict__ T4) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  float4 x = X4[m];
  float a0 = 0.f, a1 = 0.f, a2 = 0.f;
  for (int k = 0; k < nc; ++k) {
    const float u = basis_f(U[(int64_t)m * ldU + k]);
    a0 = fmaf(u, c[3 * k], a0);
    a1 = fmaf(u, c[3 * k + 1], a1);
    a2 = fmaf(u, c[3 * k + 2], a2);
  }
  T4[m] = make_float4(x.x + a0, x.y + a1, x.z + a2, 0.f);
}

struct DevBuf {
  void* p = nullptr;
  size_t n = 0;
  bool alloc(size_t bytes) {
    if (bytes <= n) return true;
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    n = bytes;
    return true;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  template <typename T> T* as() const { return static_cast<T*>(p); }
};

cpd_status fail(cpd_status s, const std::string& m) {
  set_last_error(m);
  return s;
}

}  // namespace

struct cpd_net {
  int dev = 0;
  int n_out = 0, max_batch = 0, n_points = 0;
  cudaStream_t stream = nullptr;
  int64_t np = 0;
  int64_t w_off[5], b_off[5];
  int fin[5], fout[5];
  int64_t step = 0;
  DevBuf params, grads, m, v, h1, h2, h3, g, arg, z, pred, dpred, dz, dg, dh3, dh2, dh1, part, loss, tgt;
  // BF16 precision only: operand copies (row-major [R][F], transposed
  // [F][ldt]), BF16 weights and the tensor-core kernels' status word.
  int precision = CPD_NET_FP32;
  int64_t ldt = 0;
  bool launch_failed = false;
  DevBuf h1b, h1t, h2b, h2t, dh3b, dh3t, dh2b, dh2t, wbf, gstat;
  ~cpd_net() {
    for (DevBuf* b : {&params, &grads, &m, &v, &h1, &h2, &h3, &g, &arg, &z, &pred, &dpred, &dz, &dg, &dh3, &dh2,
                      &dh1, &part, &loss, &tgt, &h1b, &h1t, &h2b, &h2t, &dh3b, &dh3t, &dh2b, &dh2t, &wbf, &gstat})
      b->release();
  }
};

namespace {

void gemm(cpd_net* net, const float* A, int64_t lda, bool ta, const float* B, int64_t ldb, bool tb, float* C,
          int64_t ldc, int M, int N, int K, const float* bias, bool relu) {
  dim3 grid((unsigned)cdiv(N, kGT), (unsigned)cdiv(M, kGT), 1);
  sgemm<<<grid, kGThreads, 0, net->stream>>>(A, lda, ta ? 1 : 0, B, ldb, tb ? 1 : 0, C, ldc, 0, M, N, K, K, bias,
                                               relu ? 1 : 0);
}

// C (M x N) = op(A) op(B) with K split kSplitK ways into net->part, then summed.
void gemm_splitk(cpd_net* net, const float* A, int64_t lda, bool ta, const float* B, int64_t ldb, bool tb, float* C,
                 int M, int N, int K) {
  const int kchunk = (int)(cdiv(cdiv(K, kSplitK), kGK) * kGK);
  const int S = (int)cdiv(K, kchunk);
  dim3 grid((unsigned)cdiv(N, kGT), (unsigned)cdiv(M, kGT), (unsigned)S);
  sgemm<<<grid, kGThreads, 0, net->stream>>>(A, lda, ta ? 1 : 0, B, ldb, tb ? 1 : 0, net->part.as<float>(), N,
                                               (int64_t)M * N, M, N, K, kchunk, nullptr, 0);
  sum_splits<<<(unsigned)cdiv((int64_t)M * N, 256), 256, 0, net->stream>>>(net->part.as<float>(), S, (int64_t)M * N, C);
}

void col_sum(cpd_net* net, const float* X, int64_t R, int C, float* out) {
  const int S = (int)std::min<int64_t>(kSplitK, std::max<int64_t>(1, R / 64));
  const int64_t rows_per = cdiv(R, S);
  dim3 grid((unsigned)cdiv(C, 256), (unsigned)S);
  col_sum_part<<<grid, 256, 0, net->stream>>>(X, R, C, rows_per, net->part.as<float>());
  sum_splits<<<(unsigned)cdiv(C, 256), 256, 0, net->stream>>>(net->part.as<float>(), S, C, out);
}

void mask(cpd_net* net, float* d, const float* h, int64_t n) {
  relu_mask<<<(unsigned)cdiv(n, 256), 256, 0, net->stream>>>(d, h, n);
}

float* W(cpd_net* n, DevBuf& b, int l) { return b.as<float>() + n->w_off[l]; }
float* Bv(cpd_net* n, DevBuf& b, int l) { return b.as<float>() + n->b_off[l]; }

__nv_bfloat16* bf(DevBuf& b) { return b.as<__nv_bfloat16>(); }
// BF16 weight copies: W2 (128 x 128), W2^T, W3 (128 x 256), W3^T (256 x 128).
__nv_bfloat16* w2_bf(cpd_net* n) { return bf(n->wbf); }
__nv_bfloat16* w2t_bf(cpd_net* n) { return bf(n->wbf) + 128 * 128; }
__nv_bfloat16* w3_bf(cpd_net* n) { return bf(n->wbf) + 2 * 128 * 128; }
__nv_bfloat16* w3t_bf(cpd_net* n) { return bf(n->wbf) + 2 * 128 * 128 + 128 * 256; }

// CPD_FAULT=gemm_wait (host fault injection): the tensor-core GEMMs' waits
// run out, exercising their bounded waits and the CPD_ETIMEOUT report.
bool gemm_fault() {
  const char* f = std::getenv("CPD_FAULT");
  return f && std::strcmp(f, "gemm_wait") == 0;
}

// out (R x N) = epilogue(A B^T) on the tensor cores, A: R x Q, B: N x Q (BF16).
void tc(cpd_net* n, const __nv_bfloat16* A, int64_t lda, const __nv_bfloat16* B, int64_t ldb, int64_t R, int N, int Q,
        const float* bias, bool relu, const float* mask_by, float* out, __nv_bfloat16* out_bf, __nv_bfloat16* out_t) {
  if (launch_gemm_tc(A, lda, B, ldb, (int)R, N, Q, 1, bias, relu, mask_by, N, out, N, out_bf, N, out_t, n->ldt,
                     n->gstat.as<int>(), gemm_fault(), n->stream) != cudaSuccess)
    n->launch_failed = true;
}

// C (P x N) = A B^T over a long contraction (all points): kTcChunks partials,
// summed in order.
void tc_splitk(cpd_net* n, const __nv_bfloat16* A, const __nv_bfloat16* B, int P, int N, int64_t Q, float* C) {
  const int S = gemm_tc_chunks((int)Q, kTcChunks);
  if (launch_gemm_tc(A, n->ldt, B, n->ldt, P, N, (int)Q, S, nullptr, false, nullptr, 0, n->part.as<float>(), N,
                     nullptr, 0, nullptr, 0, n->gstat.as<int>(), gemm_fault(), n->stream) != cudaSuccess)
    n->launch_failed = true;
  sum_splits<<<(unsigned)cdiv((int64_t)P * N, 256), 256, 0, n->stream>>>(n->part.as<float>(), S, (int64_t)P * N, C);
}

// train: also write the transposed BF16 activations the weight gradients read.
void forward(cpd_net* n, const float* Y, int B, bool train) {
  const int64_t R = (int64_t)B * n->n_points;
  gemm(n, Y, 3, false, W(n, n->params, 0), 128, false, n->h1.as<float>(), 128, (int)R, 128, 3, Bv(n, n->params, 0), true);
  if (n->precision == CPD_NET_BF16) {
    launch_weights_bf16(W(n, n->params, 1), 128, 128, w2_bf(n), w2t_bf(n), n->stream);
    launch_weights_bf16(W(n, n->params, 2), 128, 256, w3_bf(n), w3t_bf(n), n->stream);
    launch_to_bf16(n->h1.as<float>(), R, 128, bf(n->h1b), train ? bf(n->h1t) : nullptr, n->ldt, n->stream);
    tc(n, bf(n->h1b), 128, w2t_bf(n), 128, R, 128, 128, Bv(n, n->params, 1), true, nullptr, n->h2.as<float>(),
       bf(n->h2b), train ? bf(n->h2t) : nullptr);
    tc(n, bf(n->h2b), 128, w3t_bf(n), 128, R, 256, 128, Bv(n, n->params, 2), true, nullptr, n->h3.as<float>(), nullptr,
       nullptr);
  } else {
    gemm(n, n->h1.as<float>(), 128, false, W(n, n->params, 1), 128, false, n->h2.as<float>(), 128, (int)R, 128, 128,
         Bv(n, n->params, 1), true);
    gemm(n, n->h2.as<float>(), 128, false, W(n, n->params, 2), 256, false, n->h3.as<float>(), 256, (int)R, 256, 128,
         Bv(n, n->params, 2), true);
  }
  maxpool_fwd<<<B, 256, 0, n->stream>>>(n->h3.as<float>(), n->n_points, 256, n->g.as<float>(), n->arg.as<int>());
  gemm(n, n->g.as<float>(), 256, false, W(n, n->params, 3), 256, false, n->z.as<float>(), 256, B, 256, 256,
       Bv(n, n->params, 3), true);
  gemm(n, n->z.as<float>(), 256, false, W(n, n->params, 4), n->n_out, false, n->pred.as<float>(), n->n_out, B,
       n->n_out, 256, Bv(n, n->params, 4), false);
}

// Gradients of the mean-squared error into n->grads (after forward).
void backward(cpd_net* n, const float* Y, const float* tgt, int B) {
  const int64_t R = (int64_t)B * n->n_points;
  const int no = n->n_out;
  mse_grad<<<1, 1024, 0, n->stream>>>(n->pred.as<float>(), tgt, B * no, n->dpred.as<float>(), n->loss.as<float>());
  gemm(n, n->z.as<float>(), 256, true, n->dpred.as<float>(), no, false, W(n, n->grads, 4), no, 256, no, B, nullptr, false);
  col_sum(n, n->dpred.as<float>(), B, no, Bv(n, n->grads, 4));
  gemm(n, n->dpred.as<float>(), no, false, W(n, n->params, 4), no, true, n->dz.as<float>(), 256, B, 256, no, nullptr, false);
  mask(n, n->dz.as<float>(), n->z.as<float>(), (int64_t)B * 256);
  gemm(n, n->g.as<float>(), 256, true, n->dz.as<float>(), 256, false, W(n, n->grads, 3), 256, 256, 256, B, nullptr, false);
  col_sum(n, n->dz.as<float>(), B, 256, Bv(n, n->grads, 3));
  gemm(n, n->dz.as<float>(), 256, false, W(n, n->params, 3), 256, true, n->dg.as<float>(), 256, B, 256, 256, nullptr, false);
  cudaMemsetAsync(n->dh3.p, 0, (size_t)R * 256 * sizeof(float), n->stream);
  maxpool_bwd<<<B, 256, 0, n->stream>>>(n->dg.as<float>(), n->arg.as<int>(), n->n_points, 256, n->dh3.as<float>());
  mask(n, n->dh3.as<float>(), n->h3.as<float>(), R * 256);
  if (n->precision == CPD_NET_BF16) {
    launch_to_bf16(n->dh3.as<float>(), R, 256, bf(n->dh3b), bf(n->dh3t), n->ldt, n->stream);
    tc_splitk(n, bf(n->h2t), bf(n->dh3t), 128, 256, R, W(n, n->grads, 2));
    col_sum(n, n->dh3.as<float>(), R, 256, Bv(n, n->grads, 2));
    tc(n, bf(n->dh3b), 256, w3_bf(n), 256, R, 128, 256, nullptr, false, n->h2.as<float>(), n->dh2.as<float>(),
       bf(n->dh2b), bf(n->dh2t));
    tc_splitk(n, bf(n->h1t), bf(n->dh2t), 128, 128, R, W(n, n->grads, 1));
    col_sum(n, n->dh2.as<float>(), R, 128, Bv(n, n->grads, 1));
    tc(n, bf(n->dh2b), 128, w2_bf(n), 128, R, 128, 128, nullptr, false, n->h1.as<float>(), n->dh1.as<float>(), nullptr,
       nullptr);
  } else {
    gemm_splitk(n, n->h2.as<float>(), 128, true, n->dh3.as<float>(), 256, false, W(n, n->grads, 2), 128, 256, (int)R);
    col_sum(n, n->dh3.as<float>(), R, 256, Bv(n, n->grads, 2));
    gemm(n, n->dh3.as<float>(), 256, false, W(n, n->params, 2), 256, true, n->dh2.as<float>(), 128, (int)R, 128, 256,
         nullptr, false);
    mask(n, n->dh2.as<float>(), n->h2.as<float>(), R * 128);
    gemm_splitk(n, n->h1.as<float>(), 128, true, n->dh2.as<float>(), 128, false, W(n, n->grads, 1), 128, 128, (int)R);
    col_sum(n, n->dh2.as<float>(), R, 128, Bv(n, n->grads, 1));
    gemm(n, n->dh2.as<float>(), 128, false, W(n, n->params, 1), 128, true, n->dh1.as<float>(), 128, (int)R, 128, 128,
         nullptr, false);
    mask(n, n->dh1.as<float>(), n->h1.as<float>(), R * 128);
  }
  gemm_splitk(n, Y, 3, true, n->dh1.as<float>(), 128, false, W(n, n->grads, 0), 3, 128, (int)R);
  col_sum(n, n->dh1.as<float>(), R, 128, Bv(n, n->grads, 0));
}

// After a synchronisation: a failed tensor-core launch, or a status word
// that a kernel set (a bounded wait that expired), fails the call.
cpd_status net_status(cpd_net* n) {
  if (n->launch_failed) {
    n->launch_failed = false;
    return fail(CPD_ECUDA, "a tensor-core GEMM of the network could not be launched");
  }
  if (n->precision != CPD_NET_BF16) return CPD_OK;
  int st = 0;
  if (cudaMemcpy(&st, n->gstat.p, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(CPD_ECUDA, "read of the network status failed");
  if (st != 0) {
    cudaMemset(n->gstat.p, 0, sizeof(int));
    return fail((cpd_status)st, "a tensor-core GEMM of the network timed out waiting on its pipeline");
  }
  return CPD_OK;
}

bool on_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" {

cpd_status cpd_net_create(int32_t n_out, int32_t max_batch, int32_t n_points, uint64_t seed, void* stream,
                          cpd_net** out) {
  return cpd_net_create_ex(n_out, max_batch, n_points, seed, CPD_NET_FP32, stream, out);
}

cpd_status cpd_net_create_ex(int32_t n_out, int32_t max_batch, int32_t n_points, uint64_t seed, int32_t precision,
                             void* stream, cpd_net** out) {
  set_last_error("");
  if (!out) return fail(CPD_EINVAL, "out is NULL");
  if (precision != CPD_NET_FP32 && precision != CPD_NET_BF16)
    return fail(CPD_EINVAL, "precision must be CPD_NET_FP32 or CPD_NET_BF16");
  if (n_out < 1 || n_out > 4096) return fail(CPD_EINVAL, "n_out must be in [1, 4096]");
  if (max_batch < 1 || max_batch > 1024) return fail(CPD_EINVAL, "max_batch must be in [1, 1024]");
  if (n_points < 1 || (int64_t)max_batch * n_points > (1LL << 24))
    return fail(CPD_EINVAL, "n_points must be >= 1 with max_batch * n_points <= 2^24");
  cpd_net* n = new (std::nothrow) cpd_net();
  if (!n) return fail(CPD_ENOMEM, "host allocation failed");
  n->n_out = n_out;
  n->max_batch = max_batch;
  n->n_points = n_points;
  n->stream = (cudaStream_t)stream;
  if (cudaGetDevice(&n->dev) != cudaSuccess) { delete n; return fail(CPD_ECUDA, "no CUDA device"); }
  const int fi[5] = {3, 128, 128, 256, 256}, fo[5] = {128, 128, 256, 256, n_out};
  int64_t o = 0;
  for (int l = 0; l < 5; ++l) {
    n->fin[l] = fi[l];
    n->fout[l] = fo[l];
    n->w_off[l] = o;
    o += (int64_t)fi[l] * fo[l];
    n->b_off[l] = o;
    o += fo[l];
  }
  n->np = o;
  const int64_t R = (int64_t)max_batch * n_points;
  const int64_t part = std::max<int64_t>((int64_t)kSplitK * 256 * 256, (int64_t)kSplitK * 4096);
  bool ok = n->params.alloc(o * 4) && n->grads.alloc(o * 4) && n->m.alloc(o * 4) && n->v.alloc(o * 4) &&
            n->h1.alloc(R * 128 * 4) && n->h2.alloc(R * 128 * 4) && n->h3.alloc(R * 256 * 4) &&
            n->g.alloc((int64_t)max_batch * 256 * 4) && n->arg.alloc((int64_t)max_batch * 256 * 4) &&
            n->z.alloc((int64_t)max_batch * 256 * 4) && n->pred.alloc((int64_t)max_batch * n_out * 4) &&
            n->dpred.alloc((int64_t)max_batch * n_out * 4) && n->dz.alloc((int64_t)max_batch * 256 * 4) &&
            n->dg.alloc((int64_t)max_batch * 256 * 4) && n->dh3.alloc(R * 256 * 4) && n->dh2.alloc(R * 128 * 4) &&
            n->dh1.alloc(R * 128 * 4) && n->part.alloc(part * 4) && n->loss.alloc(4) &&
            n->tgt.alloc((int64_t)max_batch * n_out * 4);
  if (ok && precision == CPD_NET_BF16) {
    int cc_major = 0;
    cudaDeviceGetAttribute(&cc_major, cudaDevAttrComputeCapabilityMajor, n->dev);
    if (cc_major != 10) { delete n; return fail(CPD_EINVAL, "BF16 precision needs tcgen05 (compute capability 10.x)"); }
    n->precision = CPD_NET_BF16;
    n->ldt = (R + 7) / 8 * 8;  // transposed rows start on 16-byte boundaries (TMA strides)
    const int64_t bf = 2;
    ok = n->h1b.alloc(R * 128 * bf) && n->h1t.alloc(128 * n->ldt * bf) && n->h2b.alloc(R * 128 * bf) &&
         n->h2t.alloc(128 * n->ldt * bf) && n->dh3b.alloc(R * 256 * bf) && n->dh3t.alloc(256 * n->ldt * bf) &&
         n->dh2b.alloc(R * 128 * bf) && n->dh2t.alloc(128 * n->ldt * bf) &&
         n->wbf.alloc((2 * 128 * 128 + 2 * 128 * 256) * bf) && n->gstat.alloc(sizeof(int)) &&
         cudaMemsetAsync(n->gstat.p, 0, sizeof(int), n->stream) == cudaSuccess;
  }
  if (!ok) { delete n; return fail(CPD_ENOMEM, "device allocation for the network failed"); }
  // He-style initialisation from a seeded generator (host, once)
  std::vector<float> h((size_t)o, 0.f);
  std::mt19937_64 rng(seed);
  for (int l = 0; l < 5; ++l) {
    std::normal_distribution<float> nd(0.f, std::sqrt(2.f / (float)fi[l]) * (l == 4 ? 0.1f : 1.f));
    for (int64_t e = 0; e < (int64_t)fi[l] * fo[l]; ++e) h[n->w_off[l] + e] = nd(rng);
  }
  if (cudaMemcpyAsync(n->params.p, h.data(), o * 4, cudaMemcpyHostToDevice, n->stream) != cudaSuccess ||
      cudaMemsetAsync(n->m.p, 0, o * 4, n->stream) != cudaSuccess ||
      cudaMemsetAsync(n->v.p, 0, o * 4, n->stream) != cudaSuccess || cudaStreamSynchronize(n->stream) != cudaSuccess) {
    delete n;
    return fail(CPD_ECUDA, "network initialisation failed");
  }
  *out = n;
  return CPD_OK;
}

int64_t cpd_net_num_params(const cpd_net* n) { return n ? n->np : 0; }

int32_t cpd_net_precision(const cpd_net* n) { return n ? n->precision : -1; }

cpd_status cpd_net_get_params(cpd_net* n, float* out) {
  if (!n || !out) return fail(CPD_EINVAL, "net and out are required");
  if (cudaMemcpyAsync(out, n->params.p, n->np * 4, cudaMemcpyDefault, n->stream) != cudaSuccess ||
      cudaStreamSynchronize(n->stream) != cudaSuccess)
    return fail(CPD_ECUDA, "copy of the parameters failed");
  return CPD_OK;
}

cpd_status cpd_net_set_params(cpd_net* n, const float* in) {
  if (!n || !in) return fail(CPD_EINVAL, "net and in are required");
  if (cudaMemcpyAsync(n->params.p, in, n->np * 4, cudaMemcpyDefault, n->stream) != cudaSuccess ||
      cudaMemsetAsync(n->m.p, 0, n->np * 4, n->stream) != cudaSuccess ||
      cudaMemsetAsync(n->v.p, 0, n->np * 4, n->stream) != cudaSuccess ||
      cudaStreamSynchronize(n->stream) != cudaSuccess)
    return fail(CPD_ECUDA, "copy of the parameters failed");
  n->step = 0;
  return CPD_OK;
}

cpd_status cpd_net_forward(cpd_net* n, const float* Y, int32_t B, float* pred_out) {
  if (!n || !Y || !pred_out) return fail(CPD_EINVAL, "net, Y and pred_out are required");
  if (B < 1 || B > n->max_batch) return fail(CPD_EINVAL, "B must be in [1, max_batch]");
  if (!on_device(Y)) return fail(CPD_EINVAL, "Y must be device memory (B x n_points x 3 floats)");
  forward(n, Y, B, false);
  if (cudaMemcpyAsync(pred_out, n->pred.p, (size_t)B * n->n_out * 4, cudaMemcpyDefault, n->stream) != cudaSuccess ||
      cudaStreamSynchronize(n->stream) != cudaSuccess || cudaGetLastError() != cudaSuccess)
    return fail(CPD_ECUDA, "forward pass failed");
  return net_status(n);
}

cpd_status cpd_net_gradients(cpd_net* n, const float* Y, const float* target, int32_t B, float* grad_out,
                             float* loss_out) {
  if (!n || !Y || !target) return fail(CPD_EINVAL, "net, Y and target are required");
  if (B < 1 || B > n->max_batch) return fail(CPD_EINVAL, "B must be in [1, max_batch]");
  if (!on_device(Y)) return fail(CPD_EINVAL, "Y must be device memory (B x n_points x 3 floats)");
  if (cudaMemcpyAsync(n->tgt.p, target, (size_t)B * n->n_out * 4, cudaMemcpyDefault, n->stream) != cudaSuccess)
    return fail(CPD_ECUDA, "copy of the target failed");
  forward(n, Y, B, true);
  backward(n, Y, n->tgt.as<float>(), B);
  if (grad_out && cudaMemcpyAsync(grad_out, n->grads.p, n->np * 4, cudaMemcpyDefault, n->stream) != cudaSuccess)
    return fail(CPD_ECUDA, "copy of the gradients failed");
  if (loss_out && cudaMemcpyAsync(loss_out, n->loss.p, 4, cudaMemcpyDefault, n->stream) != cudaSuccess)
    return fail(CPD_ECUDA, "copy of the loss failed");
  if (cudaStreamSynchronize(n->stream) != cudaSuccess || cudaGetLastError() != cudaSuccess)
    return fail(CPD_ECUDA, "backward pass failed");
  return net_status(n);
}

cpd_status cpd_net_train_step(cpd_net* n, const float* Y, const float* target, int32_t B, float lr, float* loss_out) {
  if (!(lr > 0.f)) return fail(CPD_EINVAL, "lr must be > 0");
  // the gradients, then Adam (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected step)
  if (!n || !Y || !target) return fail(CPD_EINVAL, "net, Y and target are required");
  if (B < 1 || B > n->max_batch) return fail(CPD_EINVAL, "B must be in [1, max_batch]");
  if (!on_device(Y)) return fail(CPD_EINVAL, "Y must be device memory (B x n_points x 3 floats)");
  if (cudaMemcpyAsync(n->tgt.p, target, (size_t)B * n->n_out * 4, cudaMemcpyDefault, n->stream) != cudaSuccess)
    return fail(CPD_ECUDA, "copy of the target failed");
  forward(n, Y, B, true);
  backward(n, Y, n->tgt.as<float>(), B);
  ++n->step;
  const float b1 = 0.9f, b2 = 0.999f;
  const float lr_t = lr * std::sqrt(1.f - std::pow(b2, (float)n->step)) / (1.f - std::pow(b1, (float)n->step));
  adam<<<(unsigned)cdiv(n->np, 256), 256, 0, n->stream>>>(n->params.as<float>(), n->grads.as<float>(), n->m.as<float>(),
                                                          n->v.as<float>(), n->np, lr_t, b1, b2, 1e-8f);
  if (loss_out && cudaMemcpyAsync(loss_out, n->loss.p, 4, cudaMemcpyDefault, n->stream) != cudaSuccess)
    return fail(CPD_ECUDA, "copy of the loss failed");
  if (cudaStreamSynchronize(n->stream) != cudaSuccess || cudaGetLastError() != cudaSuccess)
    return fail(CPD_ECUDA, "training step failed");
  return net_status(n);
}

void cpd_net_destroy(cpd_net* n) {
  if (!n) return;
  cudaStreamSynchronize(n->stream);
  delete n;
}

}  // extern "C"

// ------------------------------------------------ context side (fcpd_abi.cu)
namespace fcpd {
template <typename B>
void launch_coefficients(const B* U, int64_t ldU, int64_t M, int64_t K, const float4* T4, const float4* X4, float* c,
                         cudaStream_t s) {
  coefficients<B><<<(unsigned)K, 256, 0, s>>>(U, ldU, (int)M, T4, X4, c);
}
template <typename B>
void launch_warm_start_T(const B* U, int64_t ldU, int64_t M, int64_t nc, const float* c, const float4* X4,
                         float4* T4, cudaStream_t s) {
  warm_start_T<B><<<(unsigned)cdiv(M, 256), 256, 0, s>>>(U, ldU, (int)M, (int)nc, c, X4, T4);
}
template void launch_coefficients<float>(const float*, int64_t, int64_t, int64_t, const float4*, const float4*,
                                         float*, cudaStream_t);
template void launch_coefficients<__half>(const __half*, int64_t, int64_t, int64_t, const float4*, const float4*,
                                          float*, cudaStream_t);
template void launch_warm_start_T<float>(const float*, int64_t, int64_t, int64_t, const float*, const float4*,
                                         float4*, cudaStream_t);
template void launch_warm_start_T<__half>(const __half*, int64_t, int64_t, int64_t, const float*, const float4*,
                                          float4*, cudaStream_t);
}  // namespace fcpd
