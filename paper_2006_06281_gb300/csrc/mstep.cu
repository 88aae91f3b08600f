// M-step of fast CPD on sm_103a: the per-registration kernels (thin wrappers
// over the device bodies in mstep_dev.cuh), their launch plan and launcher.
// See mstep_dev.cuh for the method (Eq. 17, Eq. 20, Eq. 18) and the design.
#include "mstep_dev.cuh"

#include <algorithm>

namespace fcpd {

namespace {

using namespace dev;

template <typename F, typename S>
__global__ void __launch_bounds__(kThreadsP)
colsum(const S* __restrict__ A, int64_t ldA, int rows, int cols, const typename Vec<F>::t4* __restrict__ V,
       int rows_per_chunk, F* __restrict__ part, int64_t ldP, DevState* __restrict__ st, int gate,
       int clear_row_flags) {
  dev::colsum_body<F, S, kThreadsP>(A, ldA, rows, cols, V, rows_per_chunk, part, ldP, st, gate, clear_row_flags, blockIdx.x, blockIdx.y, gridDim.x, gridDim.y);
}

template <typename F>
__global__ void __launch_bounds__(kThreadsD)
diag_update(const F* __restrict__ partP, int chunks, int64_t ldU, int K, const double* __restrict__ lam,
            typename Vec<F>::t4* __restrict__ B4, typename Vec<F>::t4* __restrict__ C4,
            const DevState* __restrict__ st, int gate) {
  dev::diag_update_body<F>(partP, chunks, ldU, K, lam, B4, C4, st, gate, blockIdx.x, blockIdx.y, gridDim.x, gridDim.y);
}

template <typename F, bool EPI>
__global__ void __launch_bounds__(kThreadsD)
expand_finish(const F* __restrict__ partE, int chunks, int64_t ldM, int M,
              const typename Vec<F>::t4* __restrict__ X4, const typename Vec<F>::t4* __restrict__ Yt4,
              typename Vec<F>::t4* __restrict__ Tout, const typename Vec<F>::t4* __restrict__ Yhat4,
              double* __restrict__ sums, DevState* __restrict__ st, int gate) {
  dev::expand_finish_body<F, EPI>(partE, chunks, ldM, M, X4, Yt4, Tout, Yhat4, sums, st, gate, blockIdx.x, blockIdx.y, gridDim.x, gridDim.y);
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

}  // namespace

MstepPlan plan_mstep(int64_t M, int64_t K, bool fp64, int sms, int colsum_threads, int basis_bytes) {
  MstepPlan p{};
  const int64_t es = basis_bytes > 0 ? basis_bytes : (fp64 ? 8 : 4);
  const int nv = es == 2 ? colsum_vectors<__half>() : 2;
  const int W = (int)(16 * nv / es);   // columns per colsum thread; row strides padded to it
  p.ldU = cdiv(K, W) * W;
  p.ldM = cdiv(M, W) * W;
  plan_colsum(M, p.ldU, es, sms, W, colsum_threads, p.p_col_tiles, p.p_row_chunks, p.p_rows_per_chunk);
  plan_colsum(K, p.ldM, es, sms, W, colsum_threads, p.e_col_tiles, p.e_row_chunks, p.e_rows_per_chunk);
  p.part_elems = std::max((int64_t)p.p_row_chunks * 3 * p.ldU, (int64_t)p.e_row_chunks * 3 * p.ldM);
  p.e_blocks = (int)cdiv(M, kMRedCols);
  p.sums_elems = (int64_t)p.e_blocks * 3;
  return p;
}

template <typename F, typename S>
void launch_mstep(const MstepPlan& pl, const S* U, const S* Ut, const double* lam, int64_t M, int64_t K,
                  const typename Vec<F>::t4* X4, const typename Vec<F>::t4* R4,
                  const typename Vec<F>::t4* Yt4, typename Vec<F>::t4* T4,
                  const typename Vec<F>::t4* Yhat4, F* part, double* sums, typename Vec<F>::t4* B4,
                  typename Vec<F>::t4* C4, DevState* st, bool iteration, cudaStream_t s, cudaEvent_t* ev) {
  const int g = iteration ? 1 : 0;
  colsum<F, S><<<dim3(pl.p_col_tiles, pl.p_row_chunks), kThreadsP, 0, s>>>(U, pl.ldU, (int)M, (int)K, R4,
                                                                      pl.p_rows_per_chunk, part, pl.ldU, st, g,
                                                                      g);
  record_after(ev, 0, s);
  diag_update<F><<<(unsigned)cdiv(K, kMRedCols), kThreadsD, 0, s>>>(part, pl.p_row_chunks, pl.ldU, (int)K, lam,
                                                                   B4, C4, st, g);
  record_after(ev, 1, s);
  colsum<F, S><<<dim3(pl.e_col_tiles, pl.e_row_chunks), kThreadsP, 0, s>>>(Ut, pl.ldM, (int)K, (int)M, B4,
                                                                      pl.e_rows_per_chunk, part, pl.ldM, st, g,
                                                                      0);
  record_after(ev, 2, s);
  if (iteration) {
    expand_finish<F, true><<<pl.e_blocks, kThreadsD, 0, s>>>(part, pl.e_row_chunks, pl.ldM, (int)M, X4, Yt4, T4,
                                                             Yhat4, sums, st, g);
  } else {
    expand_finish<F, false><<<pl.e_blocks, kThreadsD, 0, s>>>(part, pl.e_row_chunks, pl.ldM, (int)M, X4, Yt4,
                                                              T4, nullptr, sums, st, 0);
  }
  record_after(ev, 3, s);
}

template <typename F, typename S>
void launch_w(const MstepPlan& pl, const S* Ut, int64_t M, int64_t K, const typename Vec<F>::t4* C4, F* part,
              typename Vec<F>::t4* W4, DevState* st, cudaStream_t s) {
  colsum<F, S><<<dim3(pl.e_col_tiles, pl.e_row_chunks), kThreadsP, 0, s>>>(Ut, pl.ldM, (int)K, (int)M, C4,
                                                                      pl.e_rows_per_chunk, part, pl.ldM, st, 0, 0);
  expand_finish<F, false><<<pl.e_blocks, kThreadsD, 0, s>>>(part, pl.e_row_chunks, pl.ldM, (int)M, nullptr,
                                                            nullptr, W4, nullptr, nullptr, st, 0);
}

template void launch_mstep<float, float>(const MstepPlan&, const float*, const float*, const double*, int64_t,
                                         int64_t, const float4*, const float4*, const float4*, float4*,
                                         const float4*, float*, double*, float4*, float4*, DevState*, bool,
                                         cudaStream_t, cudaEvent_t*);
template void launch_mstep<double, double>(const MstepPlan&, const double*, const double*, const double*, int64_t,
                                           int64_t, const dvec4*, const dvec4*, const dvec4*, dvec4*, const dvec4*,
                                           double*, double*, dvec4*, dvec4*, DevState*, bool, cudaStream_t,
                                           cudaEvent_t*);
template void launch_mstep<float, __half>(const MstepPlan&, const __half*, const __half*, const double*, int64_t,
                                          int64_t, const float4*, const float4*, const float4*, float4*,
                                          const float4*, float*, double*, float4*, float4*, DevState*, bool,
                                          cudaStream_t, cudaEvent_t*);
template void launch_w<float, float>(const MstepPlan&, const float*, int64_t, int64_t, const float4*, float*,
                                     float4*, DevState*, cudaStream_t);
template void launch_w<double, double>(const MstepPlan&, const double*, int64_t, int64_t, const dvec4*, double*,
                                       dvec4*, DevState*, cudaStream_t);
template void launch_w<float, __half>(const MstepPlan&, const __half*, int64_t, int64_t, const float4*, float*,
                                      float4*, DevState*, cudaStream_t);

}  // namespace fcpd
