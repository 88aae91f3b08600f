// Top-K eigenpairs of the Gaussian Gram matrix for the low-rank basis
// (Eq. 19): subspace iteration with a Rayleigh-Ritz step, in FP64.
//
// The paper takes the K largest eigenpairs of Phi (Eq. 19-20) and counts the
// one-time eigendecomposition as t_eig.  A full symmetric eigensolver spends
// O(M^3) on all M pairs; for K << M this routine works in a block of
// L = K + p directions (p oversampling columns) instead:
//   A   = orth(Phi Omega)                    Omega: M x L, seeded uniform
//   repeat:
//     Z = Phi A,  B = A^T Z                  (L x L, symmetric)
//     B = V diag(theta) V^T                  (small dense eigensolver)
//     U = A V,  Phi U = Z V                  (Ritz pairs (theta_i, u_i))
//     stop when |Phi u_i - theta_i u_i| <= tol * theta_max for the top K
//     A   = orth(Phi U)
// (Rutishauser's subspace iteration with Rayleigh-Ritz projection, started
// from a random block as in Halko, Martinsson and Tropp, SIAM Review 53,
// 2011.)  The spectrum of a Gaussian Gram matrix decays fast, so the top K
// pairs converge in a few steps; each step costs one M x M x L product.
// Products are cuBLAS DGEMMs and the orthogonalisation / small eigenproblem
// are cuSOLVER routines: all of it runs once, at setup.
#include <cublas_v2.h>
#include <cusolverDn.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "common.cuh"

namespace fcpd {

namespace {

constexpr int kThreads = 256;

// SplitMix64 (Steele, Lea, Flood 2014): a counter-based generator, so every
// element of the start block is a pure function of (seed, index).
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void fill_uniform(double* __restrict__ a, int64_t n, unsigned long long seed) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const unsigned long long h = splitmix64(seed + (unsigned long long)i);
  a[i] = (double)(h >> 11) * 0x1p-53 * 2.0 - 1.0;      // uniform in [-1, 1)
}

// res[j - j0] = |P[:, j] - w[j] U[:, j]| for columns j0 <= j < L (column-major, M rows).
__global__ void ritz_residuals(const double* __restrict__ U, const double* __restrict__ P,
                               const double* __restrict__ w, int64_t M, int j0, double* __restrict__ res) {
  __shared__ double sh[32];
  const int j = j0 + blockIdx.x;
  const double th = w[j];
  const double* u = U + (size_t)j * M;
  const double* p = P + (size_t)j * M;
  double s = 0.0;
  for (int64_t m = threadIdx.x; m < M; m += blockDim.x) {
    const double r = p[m] - th * u[m];
    s += r * r;
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) res[blockIdx.x] = sqrt(s);
}

struct DevBufs {
  std::vector<void*> ptrs;
  ~DevBufs() {
    for (void* p : ptrs) cudaFree(p);
  }
  template <typename T> cudaError_t get(T** out, size_t count) {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) {
      cudaGetLastError();
      return e;
    }
    ptrs.push_back(p);
    *out = static_cast<T*>(p);
    return cudaSuccess;
  }
  void release(void* p) {
    auto it = std::find(ptrs.begin(), ptrs.end(), p);
    if (it != ptrs.end()) ptrs.erase(it);
  }
};

}  // namespace

int topk_oversampling(int64_t K) { return (int)std::max<int64_t>(16, (K + 3) / 4); }

bool topk_eig_applies(int64_t M, int64_t K) {
  return K > 0 && K < M && 2 * (K + topk_oversampling(K)) <= M;
}

int topk_eigh(const double* Phi, int64_t M, int64_t K, double tol, int max_steps, cudaStream_t s,
              double** V_out, double** w_out, int64_t* nv_out, int* steps_out, std::string* err) {
  const int64_t L = std::min<int64_t>(M, K + topk_oversampling(K));
  const int m = (int)M, l = (int)L, k = (int)K;
  DevBufs bufs;
  double *A = nullptr, *Z = nullptr, *U = nullptr, *P = nullptr, *B = nullptr, *w = nullptr, *tau = nullptr,
         *res = nullptr, *work = nullptr;
  int* info = nullptr;
  auto oom = [&](const char* what) {
    *err = std::string("top-K eigensolver: cannot allocate ") + what;
    return (int)CPD_ENOMEM;
  };
  if (bufs.get(&A, (size_t)M * L) != cudaSuccess) return oom("the subspace block");
  if (bufs.get(&Z, (size_t)M * L) != cudaSuccess) return oom("the product block");
  if (bufs.get(&U, (size_t)M * L) != cudaSuccess) return oom("the Ritz vectors");
  if (bufs.get(&P, (size_t)M * L) != cudaSuccess) return oom("the Ritz products");
  if (bufs.get(&B, (size_t)L * L) != cudaSuccess) return oom("the projected matrix");
  if (bufs.get(&w, (size_t)L) != cudaSuccess || bufs.get(&tau, (size_t)L) != cudaSuccess ||
      bufs.get(&res, (size_t)L) != cudaSuccess || bufs.get(&info, 1) != cudaSuccess)
    return oom("small vectors");

  cublasHandle_t hb = nullptr;
  cusolverDnHandle_t hs = nullptr;
  if (cublasCreate(&hb) != CUBLAS_STATUS_SUCCESS) {
    *err = "cublasCreate failed";
    return (int)CPD_ESOLVER;
  }
  if (cusolverDnCreate(&hs) != CUSOLVER_STATUS_SUCCESS) {
    cublasDestroy(hb);
    *err = "cusolverDnCreate failed";
    return (int)CPD_ESOLVER;
  }
  struct Handles {
    cublasHandle_t b;
    cusolverDnHandle_t s;
    ~Handles() {
      cusolverDnDestroy(s);
      cublasDestroy(b);
    }
  } handles{hb, hs};
  cublasSetStream(hb, s);
  cublasSetMathMode(hb, CUBLAS_DEFAULT_MATH);        // plain FP64 arithmetic
  cusolverDnSetStream(hs, s);

  int lw_qr = 0, lw_og = 0, lw_ev = 0;
  if (cusolverDnDgeqrf_bufferSize(hs, m, l, A, m, &lw_qr) != CUSOLVER_STATUS_SUCCESS ||
      cusolverDnDorgqr_bufferSize(hs, m, l, l, A, m, tau, &lw_og) != CUSOLVER_STATUS_SUCCESS ||
      cusolverDnDsyevd_bufferSize(hs, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, l, B, l, w, &lw_ev) !=
          CUSOLVER_STATUS_SUCCESS) {
    *err = "top-K eigensolver: workspace query failed";
    return (int)CPD_ESOLVER;
  }
  const int lwork = std::max(std::max(lw_qr, lw_og), std::max(lw_ev, 1));
  if (bufs.get(&work, (size_t)lwork) != cudaSuccess) return oom("the solver workspace");

  const double one = 1.0, zero = 0.0;
  int hinfo = 0;
  auto orth = [&](double* X) -> bool {      // X (M x L) <- Q of its thin QR
    if (cusolverDnDgeqrf(hs, m, l, X, m, tau, work, lwork, info) != CUSOLVER_STATUS_SUCCESS) return false;
    if (cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return false;
    if (cusolverDnDorgqr(hs, m, l, l, X, m, tau, work, lwork, info) != CUSOLVER_STATUS_SUCCESS) return false;
    int i2 = 0;
    if (cudaMemcpyAsync(&i2, info, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return false;
    if (cudaStreamSynchronize(s) != cudaSuccess) return false;
    return hinfo == 0 && i2 == 0;
  };
  auto gemm = [&](cublasOperation_t ta, int rows, int cols, int inner, const double* X, int ldx, const double* Y,
                  int ldy, double* out, int ldo) {
    return cublasDgemm(hb, ta, CUBLAS_OP_N, rows, cols, inner, &one, X, ldx, Y, ldy, &zero, out, ldo) ==
           CUBLAS_STATUS_SUCCESS;
  };

  // start block: A = orth(Phi Omega)
  fill_uniform<<<(unsigned)((M * L + kThreads - 1) / kThreads), kThreads, 0, s>>>(U, M * L, 0x5EEDull);
  if (!gemm(CUBLAS_OP_N, m, l, m, Phi, m, U, m, A, m) || !orth(A)) {
    *err = "top-K eigensolver: start block failed";
    return (int)CPD_ESOLVER;
  }
  std::vector<double> hres((size_t)K), hw((size_t)L);
  for (int step = 1; step <= max_steps; ++step) {
    // Rayleigh-Ritz on span(A)
    if (!gemm(CUBLAS_OP_N, m, l, m, Phi, m, A, m, Z, m) || !gemm(CUBLAS_OP_T, l, l, m, A, m, Z, m, B, l) ||
        cusolverDnDsyevd(hs, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, l, B, l, w, work, lwork, info) !=
            CUSOLVER_STATUS_SUCCESS ||
        !gemm(CUBLAS_OP_N, m, l, l, A, m, B, l, U, m) || !gemm(CUBLAS_OP_N, m, l, l, Z, m, B, l, P, m)) {
      *err = "top-K eigensolver: Rayleigh-Ritz step failed";
      return (int)CPD_ESOLVER;
    }
    // residuals of the K largest Ritz pairs (the last K columns: ascending order)
    ritz_residuals<<<k, kThreads, 0, s>>>(U, P, w, M, l - k, res);
    if (cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(hres.data(), res, (size_t)K * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(hw.data(), w, (size_t)L * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess || hinfo != 0) {
      *err = "top-K eigensolver: small eigenproblem failed (info " + std::to_string(hinfo) + ")";
      return (int)CPD_ESOLVER;
    }
    const double scale = std::max(std::fabs(hw[(size_t)L - 1]), 1e-300);
    const double worst = *std::max_element(hres.begin(), hres.end());
    if (worst <= tol * scale) {
      bufs.release(U);
      bufs.release(w);
      *V_out = U;
      *w_out = w;
      *nv_out = L;
      *steps_out = step;
      return (int)CPD_OK;
    }
    std::swap(A, P);                          // next block: orth(Phi U)
    if (!orth(A)) {
      *err = "top-K eigensolver: orthogonalisation failed";
      return (int)CPD_ESOLVER;
    }
  }
  *err = "top-K eigensolver: no convergence in " + std::to_string(max_steps) + " steps";
  *steps_out = max_steps;
  return -1;                                  // caller falls back to the full eigensolver
}

}  // namespace fcpd
