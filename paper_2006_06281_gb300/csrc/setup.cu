// One-time setup kernels of fast CPD (Sec. III, Eq. 11, Eq. 16, Eq. 19) and
// small per-call helpers: packing caller arrays into 4-vectors, the initial
// variance, and device-state updates.
#include "common.cuh"

#include <math.h>

namespace fcpd {

namespace {

constexpr int kThreads = 256;

int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

template <typename F>
__global__ void pack(const F* __restrict__ src, int64_t n, typename Vec<F>::t4* __restrict__ dst, int with_norm) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  typename Vec<F>::t4 v;
  v.x = src[3 * i];
  v.y = src[3 * i + 1];
  v.z = src[3 * i + 2];
  v.w = with_norm ? v.x * v.x + v.y * v.y + v.z * v.z : (F)0;
  dst[i] = v;
}

template <typename F>
__global__ void unpack(const typename Vec<F>::t4* __restrict__ src, int64_t n, F* __restrict__ dst) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const typename Vec<F>::t4 v = src[i];
  dst[3 * i] = v.x;
  dst[3 * i + 1] = v.y;
  dst[3 * i + 2] = v.z;
}

// Eq. 11: Phi_ij = exp(-|x_i - x_j|^2 / (2 beta^2)) in FP64 (symmetric, so the
// row-major result is also the column-major matrix the eigensolver reads).
template <typename V4>
__global__ void gram_f64(const V4* __restrict__ X4, int M, double inv2b2, double* __restrict__ Phi) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  if (j >= M) return;
  const V4 a = X4[i], b = X4[j];
  const double dx = (double)a.x - (double)b.x, dy = (double)a.y - (double)b.y, dz = (double)a.z - (double)b.z;
  Phi[(size_t)i * M + j] = exp(-(dx * dx + dy * dy + dz * dz) * inv2b2);
}

// The eigensolvers return eigenvalues ascending and eigenvectors as columns of
// a column-major M x nv matrix V (nv = M for the full solver).  The basis kept
// here is descending (Eq. 19 keeps the K largest), stored row-major:
// U[m * ldU + k] = V[m, nv-1-k], with zero padding for K <= k < ldU.  Tiled
// transpose through shared memory.
template <typename F> __device__ __forceinline__ F to_basis(double v) { return (F)v; }
template <> __device__ __forceinline__ __half to_basis<__half>(double v) { return __double2half(v); }

template <typename F>
__global__ void extract_basis(const double* __restrict__ V, int M, int nv, int K, F* __restrict__ U, int64_t ldU) {
  __shared__ double tile[32][33];
  const int k0 = blockIdx.x * 32, m0 = blockIdx.y * 32;
  // read: for output columns k0..k0+31, source column M-1-k is contiguous in m
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int k = k0 + r, m = m0 + threadIdx.x;
    double v = 0.0;
    if (k < K && m < M) v = V[(size_t)(nv - 1 - k) * M + m];
    tile[r][threadIdx.x] = v;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int m = m0 + r, k = k0 + threadIdx.x;
    if (m < M && k < ldU) U[(size_t)m * ldU + k] = to_basis<F>(tile[threadIdx.x][r]);
  }
}

// U^T row k is eigenvector nv-1-k: a contiguous column of V, cast to F, with
// zero padding for M <= m < ldM.
template <typename F>
__global__ void extract_basis_t(const double* __restrict__ V, int M, int nv, int K, F* __restrict__ Ut, int64_t ldM) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)K * ldM) return;
  const int k = (int)(i / ldM), m = (int)(i % ldM);
  Ut[i] = to_basis<F>(m < M ? V[(size_t)(nv - 1 - k) * M + m] : 0.0);
}

__global__ void extract_lambda(const double* __restrict__ w, int nv, int K, double* __restrict__ lam) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < K) lam[k] = fmax(w[nv - 1 - k], 0.0);   // clamp: Phi is PSD, rounding-level noise can be < 0
}

// sigma2_0 = sum_m sum_n |y_n - x_m|^2 / (D M N), evaluated in closed form
// about the two centroids (FP64):
//   N sum_m |x_m - mx|^2 + M sum_n |y_n - my|^2 + M N |mx - my|^2.
template <typename V4>
__global__ void sigma2_init_k(const V4* __restrict__ X4, int M, const V4* __restrict__ Y4, int N,
                              DevState* __restrict__ st) {
  __shared__ double sh[32];
  double sx[3] = {0, 0, 0}, sy[3] = {0, 0, 0};
  for (int i = threadIdx.x; i < M; i += blockDim.x) { sx[0] += X4[i].x; sx[1] += X4[i].y; sx[2] += X4[i].z; }
  for (int i = threadIdx.x; i < N; i += blockDim.x) { sy[0] += Y4[i].x; sy[1] += Y4[i].y; sy[2] += Y4[i].z; }
  __shared__ double mean[6];
  for (int d = 0; d < 3; ++d) {
    double a = block_sum(sx[d], sh);
    if (threadIdx.x == 0) mean[d] = a / M;
    double b = block_sum(sy[d], sh);
    if (threadIdx.x == 0) mean[3 + d] = b / N;
  }
  __syncthreads();
  double cx = 0.0, cy = 0.0;
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    const double a = X4[i].x - mean[0], b = X4[i].y - mean[1], c = X4[i].z - mean[2];
    cx += a * a + b * b + c * c;
  }
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const double a = Y4[i].x - mean[3], b = Y4[i].y - mean[4], c = Y4[i].z - mean[5];
    cy += a * a + b * b + c * c;
  }
  const double tx = block_sum(cx, sh);
  const double ty = block_sum(cy, sh);
  if (threadIdx.x == 0) {
    const double dmx = mean[0] - mean[3], dmy = mean[1] - mean[4], dmz = mean[2] - mean[5];
    const double tot = (double)N * tx + (double)M * ty + (double)M * (double)N * (dmx * dmx + dmy * dmy + dmz * dmz);
    st->sigma2 = tot / (3.0 * (double)M * (double)N);
  }
}

__global__ void begin_iterations(DevState* st, int n_iter) { st->iter_target = st->iter + n_iter; }

// Condition of the device-side iteration loop: run another iteration while
// the target is not reached, no tolerance stopped the registration and no
// failure was recorded.
__global__ void loop_control(const DevState* st, cudaGraphConditionalHandle h) {
  const bool more = st->iter < st->iter_target && !st->done && st->status == 0;
  cudaGraphSetConditional(h, more ? 1u : 0u);
}

__global__ void state_params(DevState* st, double w, double lambda, double tol, double gt_tol, int has_gt,
                             double* hist, int M, int N, int K) {
  st->w = w;
  st->lambda = lambda;
  st->tol = tol;
  st->gt_tol = gt_tol;
  st->has_gt = has_gt;
  st->hist = hist;
  st->M = M;
  st->N = N;
  st->K = K;
}

template <typename V4>
__global__ void residual(const V4* __restrict__ Yt4, const V4* __restrict__ X4, V4* __restrict__ R4, int M) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  const V4 a = Yt4[m], b = X4[m];
  V4 r;
  r.x = a.x - b.x; r.y = a.y - b.y; r.z = a.z - b.z; r.w = 0;
  R4[m] = r;
}

__global__ void state_init(DevState* st, double sigma2) {
  st->sigma2 = sigma2;
  st->loglik = 0.0;
  st->last_dT2 = 0.0;
  st->last_rmse = nan("");
  st->vsum = 0.0;
  st->iter = 0;
  st->iter_target = 0;
  st->status = 0;
  st->done = 0;
  st->n_flag_cols = st->n_flag_rows = 0;
  st->ticket_a = st->ticket_b = st->ticket_m = st->ticket_e = 0;
  st->pairs_eval = 0;
  st->last_eval_frac = 1.0;
  st->prune_r2 = 0.f;
  st->prune_ctl = 0;
  st->mma_s2min = INFINITY;
  st->trim_lam = -1.0;
  st->trim_now = 0;
  st->trim_iters = 0;
}

__global__ void state_trim(DevState* st, double trim_lam) { st->trim_lam = trim_lam; }

__global__ void state_prune(DevState* st, float r2, int ctl) {
  st->prune_r2 = r2;
  st->prune_ctl = ctl;
}

}  // namespace

template <typename F>
void launch_pack(const F* src, int64_t n, typename Vec<F>::t4* dst, bool with_norm, cudaStream_t s) {
  if (n <= 0) return;
  pack<F><<<(unsigned)cdiv(n, kThreads), kThreads, 0, s>>>(src, n, dst, with_norm ? 1 : 0);
}
template <typename F>
void launch_unpack(const typename Vec<F>::t4* src, int64_t n, F* dst, cudaStream_t s) {
  if (n <= 0) return;
  unpack<F><<<(unsigned)cdiv(n, kThreads), kThreads, 0, s>>>(src, n, dst);
}

void launch_gram_f64(const void* X4, bool x_fp64, int64_t M, double beta, double* Phi, cudaStream_t s) {
  const double inv2b2 = 1.0 / (2.0 * beta * beta);
  dim3 grid((unsigned)cdiv(M, kThreads), (unsigned)M);
  if (x_fp64) gram_f64<dvec4><<<grid, kThreads, 0, s>>>((const dvec4*)X4, (int)M, inv2b2, Phi);
  else gram_f64<float4><<<grid, kThreads, 0, s>>>((const float4*)X4, (int)M, inv2b2, Phi);
}

template <typename F>
void launch_extract_basis(const double* V, int64_t M, int64_t nv, int64_t K, F* U, int64_t ldU, F* Ut, int64_t ldM,
                          const double* w, double* lam, cudaStream_t s) {
  dim3 grid((unsigned)cdiv(ldU, 32), (unsigned)cdiv(M, 32));
  extract_basis<F><<<grid, dim3(32, 8), 0, s>>>(V, (int)M, (int)nv, (int)K, U, ldU);
  extract_basis_t<F><<<(unsigned)cdiv(K * ldM, kThreads), kThreads, 0, s>>>(V, (int)M, (int)nv, (int)K, Ut, ldM);
  extract_lambda<<<(unsigned)cdiv(K, kThreads), kThreads, 0, s>>>(w, (int)nv, (int)K, lam);
}

template <typename F>
void launch_sigma2_init(const typename Vec<F>::t4* X4, int64_t M, const typename Vec<F>::t4* Y4, int64_t N,
                        double* /*scratch*/, DevState* st, cudaStream_t s) {
  sigma2_init_k<typename Vec<F>::t4><<<1, 1024, 0, s>>>(X4, (int)M, Y4, (int)N, st);
}

void launch_begin_iterations(DevState* st, int n_iter, cudaStream_t s) { begin_iterations<<<1, 1, 0, s>>>(st, n_iter); }
void launch_loop_control(const DevState* st, cudaGraphConditionalHandle h, cudaStream_t s) {
  loop_control<<<1, 1, 0, s>>>(st, h);
}
void launch_state_params(DevState* st, double w, double lambda, double tol, double gt_tol, int has_gt,
                         double* hist, int64_t M, int64_t N, int64_t K, cudaStream_t s) {
  state_params<<<1, 1, 0, s>>>(st, w, lambda, tol, gt_tol, has_gt, hist, (int)M, (int)N, (int)K);
}
template <typename F>
void launch_residual(const typename Vec<F>::t4* Yt4, const typename Vec<F>::t4* X4, typename Vec<F>::t4* R4,
                     int64_t M, cudaStream_t s) {
  residual<typename Vec<F>::t4><<<(unsigned)cdiv(M, kThreads), kThreads, 0, s>>>(Yt4, X4, R4, (int)M);
}
template void launch_residual<float>(const float4*, const float4*, float4*, int64_t, cudaStream_t);
template void launch_residual<double>(const dvec4*, const dvec4*, dvec4*, int64_t, cudaStream_t);
void launch_state_init(DevState* st, double sigma2, cudaStream_t s) { state_init<<<1, 1, 0, s>>>(st, sigma2); }
void launch_state_trim(DevState* st, double trim_lam, cudaStream_t s) { state_trim<<<1, 1, 0, s>>>(st, trim_lam); }
void launch_state_prune(DevState* st, float prune_r2, int prune_ctl, cudaStream_t s) {
  state_prune<<<1, 1, 0, s>>>(st, prune_r2, prune_ctl);
}

namespace {
__global__ void basis_to_f32(const __half* __restrict__ U, int64_t M, int64_t K, int64_t ldU, float* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M * K) return;
  out[i] = __half2float(U[(i / K) * ldU + i % K]);
}
}  // namespace

void launch_basis_to_f32(const __half* U, int64_t M, int64_t K, int64_t ldU, float* out, cudaStream_t s) {
  basis_to_f32<<<(unsigned)cdiv(M * K, kThreads), kThreads, 0, s>>>(U, M, K, ldU, out);
}

template void launch_pack<float>(const float*, int64_t, float4*, bool, cudaStream_t);
template void launch_pack<double>(const double*, int64_t, dvec4*, bool, cudaStream_t);
template void launch_unpack<float>(const float4*, int64_t, float*, cudaStream_t);
template void launch_unpack<double>(const dvec4*, int64_t, double*, cudaStream_t);
template void launch_extract_basis<float>(const double*, int64_t, int64_t, int64_t, float*, int64_t, float*, int64_t,
                                          const double*, double*, cudaStream_t);
template void launch_extract_basis<double>(const double*, int64_t, int64_t, int64_t, double*, int64_t, double*, int64_t,
                                           const double*, double*, cudaStream_t);
template void launch_extract_basis<__half>(const double*, int64_t, int64_t, int64_t, __half*, int64_t, __half*, int64_t,
                                           const double*, double*, cudaStream_t);
template void launch_sigma2_init<float>(const float4*, int64_t, const float4*, int64_t, double*, DevState*,
                                        cudaStream_t);
template void launch_sigma2_init<double>(const dvec4*, int64_t, const dvec4*, int64_t, double*, DevState*,
                                         cudaStream_t);

}  // namespace fcpd
