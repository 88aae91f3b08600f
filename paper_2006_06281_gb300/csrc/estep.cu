// E-step of fast CPD on sm_103a: the per-registration kernels (thin wrappers
// over the device bodies in estep_dev.cuh), their launch plan and launcher.
// See estep_dev.cuh for the method (Eq. 4, Eq. 5) and the kernels' design.
#include "estep_dev.cuh"

#include <algorithm>

namespace fcpd {

namespace {

using namespace dev;

// Resident blocks per SM that pass B's register budget is fitted to: 2 (96
// registers); 3 (80 registers, no spills) measured 0.194 against 0.168 ms at
// M = N = 20000 -- the extra warps do not pay for the tighter schedule.
#ifndef FCPD_EB_MINB
#define FCPD_EB_MINB 2
#endif

// The dense FP32 passes step aside (return at once) in iterations that use
// the pruned layout, and the pruned ones in all others; both are in every
// captured iteration.
__global__ void __launch_bounds__(kThreadsA)
passA_f32(const float4* __restrict__ T4, int M, int rows_per_chunk, const float4* __restrict__ Y4,
          int N, float* __restrict__ partA, DevState* __restrict__ st, int gate) {
  if (prune_active(st) || mma_active(st)) return;
  dev::passA_f32_body(T4, M, rows_per_chunk, Y4, N, partA, st, gate, blockIdx.x, blockIdx.y, gridDim.x, gridDim.y);
}

__global__ void __launch_bounds__(kThreadsA)
passA_f32_pruned(const float4* __restrict__ T4, int M, int rows_per_chunk, const float4* __restrict__ Y4,
                 int N, float* __restrict__ partA, DevState* __restrict__ st, int gate) {
  if ((gate && iteration_gated(st)) || !prune_active(st)) return;
  dev::passA_f32_pruned_body(T4, M, rows_per_chunk, Y4, N, partA, st, blockIdx.x, blockIdx.y);
}

__global__ void __launch_bounds__(kThreadsA)
passA_f64(const dvec4* __restrict__ T4, int M, int rows_per_chunk, const dvec4* __restrict__ Y4,
          int N, double* __restrict__ partA, const DevState* __restrict__ st, int gate) {
  dev::passA_f64_body(T4, M, rows_per_chunk, Y4, N, partA, st, gate, blockIdx.x, blockIdx.y, gridDim.x, gridDim.y);
}

// chunks_pruned: chunk count of the pruned layout (used when it ran).
template <typename F>
__global__ void __launch_bounds__(kThreadsR)
reduceA(const F* __restrict__ partA, int chunks, int chunks_pruned, int chunks_mma, int M, const typename Vec<F>::t4* __restrict__ Y4,
        int N, typename Vec<F>::t4* __restrict__ Yb, double* __restrict__ den_out,
        double* __restrict__ sums, int* __restrict__ flag_cols, DevState* __restrict__ st, int gate, int defer) {
  const int ch = mma_active(st) ? chunks_mma : prune_active(st) ? chunks_pruned : chunks;
  dev::reduceA_body<F>(partA, ch, M, Y4, N, Yb, den_out, sums, flag_cols, st, gate, blockIdx.x, blockIdx.y, gridDim.x,
                       gridDim.y, defer);
}

// Eq. 3 in the deferred form: one block, launched on a side stream after
// fixA so that it overlaps pass B.  FP32: the sum of ln den_n =
// -ln 2 * (-log2 den_n) over the exponent offsets that reduceA and fixA
// left in Yb; FP64: the sum of reduceA's block sums (with fixA's nothing
// to add).  Fixed summation order.
// 1024 threads, four independent partial sums per thread (loads in flight
// together rather than one per dependent add).
constexpr int kThreadsL = 1024;
template <typename F>
__global__ void __launch_bounds__(kThreadsL)
loglik_finish(const double* __restrict__ sums, int nsums, const typename Vec<F>::t4* __restrict__ Yb,
              DevState* __restrict__ st, int M, int N, int gate) {
  if (gate && iteration_gated(st)) return;
  __shared__ double sh[32];
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  const int n = sizeof(F) == 4 ? N : nsums;
  for (int i0 = threadIdx.x; i0 < n; i0 += 4 * kThreadsL) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int i = i0 + j * kThreadsL;
      if (i < n) {
        if constexpr (sizeof(F) == 4)
          v[j] += (double)Yb[i].w;
        else
          v[j] += __ldcg(sums + i);
      }
    }
  }
  double t = (v[0] + v[1]) + (v[2] + v[3]);
  if constexpr (sizeof(F) == 4) t *= -0.69314718055994531;
  const double tot = block_sum(t, sh);
  if (threadIdx.x == 0) {
    const double s2 = st->sigma2, w = st->w;
    st->loglik += tot + (double)N * log((1.0 - w) / (double)M) - 1.5 * (double)N * log(2.0 * kPi * s2);
  }
}

__global__ void __launch_bounds__(kThreadsF)
fixA_f32(const float4* __restrict__ T4, int M, const float4* __restrict__ Y4, int N,
         float4* __restrict__ Yb, double* __restrict__ den_out, const int* __restrict__ flag_cols,
         DevState* __restrict__ st, int gate, int defer) {
  dev::fixA_f32_body(T4, M, Y4, N, Yb, den_out, flag_cols, st, gate, blockIdx.x, blockIdx.y, gridDim.x, gridDim.y,
                     defer);
}

__global__ void __launch_bounds__(kThreadsB, FCPD_EB_MINB)
passB_f32(const float4* __restrict__ T4, int M, const float4* __restrict__ Yb, int N,
          int cols_per_chunk, float* __restrict__ partB, DevState* __restrict__ st, int gate, int clear_rows) {
  if (prune_active(st) || mma_active(st)) return;
  dev::passB_f32_body(T4, M, Yb, N, cols_per_chunk, partB, st, gate, blockIdx.x, blockIdx.y, gridDim.x, gridDim.y,
                      clear_rows);
}

__global__ void __launch_bounds__(kThreadsB)
passB_f32_pruned(const float4* __restrict__ T4, int M, const float4* __restrict__ Yb, int N,
                 int cols_per_chunk, float* __restrict__ partB, DevState* __restrict__ st, int gate) {
  if ((gate && iteration_gated(st)) || !prune_active(st)) return;
  dev::passB_f32_pruned_body(T4, M, Yb, N, cols_per_chunk, partB, st, blockIdx.x, blockIdx.y, gridDim.y);
}

__global__ void __launch_bounds__(kThreadsB)
passB_f64(const dvec4* __restrict__ T4, int M, const dvec4* __restrict__ Yb, int N,
          int cols_per_chunk, double* __restrict__ partB, const DevState* __restrict__ st, int gate) {
  dev::passB_f64_body(T4, M, Yb, N, cols_per_chunk, partB, st, gate, blockIdx.x, blockIdx.y, gridDim.x, gridDim.y);
}

template <typename F>
__global__ void __launch_bounds__(kThreadsR)
reduceB(const F* __restrict__ partB, int chunks, int chunks_pruned, int chunks_mma, int M, const typename Vec<F>::t4* __restrict__ X4,
        typename Vec<F>::t4* __restrict__ Yt4, typename Vec<F>::t4* __restrict__ R4,
        double* __restrict__ P1_out, double* __restrict__ sums, int* __restrict__ flag_rows,
        DevState* __restrict__ st, int gate, int skip_vsum, int m_off) {
  const int ch = mma_active(st) ? chunks_mma : prune_active(st) ? chunks_pruned : chunks;
  dev::reduceB_body<F>(partB, ch, M, X4, Yt4, R4, P1_out, sums, flag_rows, st, gate, blockIdx.x, blockIdx.y,
                       gridDim.x, gridDim.y, skip_vsum, m_off);
}

__global__ void __launch_bounds__(kThreadsF)
fixB_f32(const float4* __restrict__ T4, int M, const float4* __restrict__ Yb, int N,
         const float4* __restrict__ X4, float4* __restrict__ Yt4, float4* __restrict__ R4,
         double* __restrict__ P1_out, const int* __restrict__ flag_rows, DevState* __restrict__ st, int gate,
         int m_lo, int m_hi) {
  // the E-step's last launch also takes the iteration's spectral-trim
  // decision for the M-step that follows (sigma2 is the same in both)
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0 && !(gate && iteration_gated(st)))
    st->trim_now = trim_active(st) ? 1 : 0;
  dev::fixB_f32_body(T4, M, Yb, N, X4, Yt4, R4, P1_out, flag_rows, st, gate, blockIdx.x, blockIdx.y, gridDim.x, gridDim.y,
                     m_lo, m_hi);
}

int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace

// Grids for passes A and B: all blocks resident in one wave (blocks <= SMs x
// resident blocks per SM from the occupancy calculator), with the split of
// the long dimension chosen so every block gets the same amount of work.
EstepPlan plan_estep(int64_t M, int64_t N, bool fp64, int sms, bool with_pruned, bool with_mma) {
  EstepPlan p{};
  int occA = 0, occB = 0;
  if (fp64) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occA, passA_f64, kThreadsA, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occB, passB_f64, kThreadsB, 0);
  } else {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occA, passA_f32, kThreadsA, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occB, passB_f32, kThreadsB, 0);
  }
  const int64_t slotsA = (int64_t)sms * std::max(occA, 1);
  const int64_t slotsB = (int64_t)sms * std::max(occB, 1);
  const int64_t colsA = kThreadsA * (fp64 ? kColsA64 : kColsA32);
  p.a_col_tiles = (int)cdiv(N, colsA);
  int64_t want = std::max<int64_t>(1, slotsA / p.a_col_tiles);
  int64_t rpc = std::max<int64_t>(32, cdiv(M, want));
  p.a_rows_per_chunk = (int)rpc;
  p.a_row_chunks = (int)cdiv(M, rpc);
  const int64_t rowsB = kThreadsB * (fp64 ? kRowsB64 : kRowsB32);
  p.b_row_tiles = (int)cdiv(M, rowsB);
  want = std::max<int64_t>(1, slotsB / p.b_row_tiles);
  int64_t cpc = std::max<int64_t>(32, cdiv(N, want));
  p.b_cols_per_chunk = (int)cpc;
  p.b_col_chunks = (int)cdiv(N, cpc);
  p.partA_elems = (int64_t)p.a_row_chunks * N;
  p.partB_elems = (int64_t)5 * p.b_col_chunks * M;
  // pruned layout: 1024-point tiles of the owning set; pass A chunks of 256
  // model rows, pass B chunks of 512 scene points (2 and 4 shared tiles):
  // small enough that work concentrates where the boxes meet, and the
  // hardware block scheduler balances the many short blocks.
  p.pruned = with_pruned && !fp64;
  p.pa_col_tiles = (int)cdiv(N, kPruneTile);
  p.pa_rows_per_chunk = 2 * kTileA;
  p.pa_row_chunks = (int)cdiv(M, p.pa_rows_per_chunk);
  p.pb_row_tiles = (int)cdiv(M, kPruneTile);
  p.pb_cols_per_chunk = 4 * kTileB;
  p.pb_col_chunks = (int)cdiv(N, p.pb_cols_per_chunk);
  if (p.pruned) {
    p.partA_elems = std::max(p.partA_elems, (int64_t)p.pa_row_chunks * N);
    p.partB_elems = std::max(p.partB_elems, (int64_t)5 * p.pb_col_chunks * M);
  } else {
    p.pa_row_chunks = p.a_row_chunks;          // never used: prune_active is false
    p.pb_col_chunks = p.b_col_chunks;
  }
  p.mma = with_mma && !fp64 && estep_mma_supported();
  if (p.mma) {
    plan_estep_mma(M, N, sms, p.mm);
    p.partA_elems = std::max(p.partA_elems, (int64_t)p.mm.a_chunks * N);
    p.partB_elems = std::max(p.partB_elems, (int64_t)5 * p.mm.b_chunks * M);
  } else {
    p.mm = MmaPlan{};
    p.mm.a_chunks = p.a_row_chunks;            // never used: mma_active is false
    p.mm.b_chunks = p.b_col_chunks;
  }
  // column-vector scratch of the tensor-core passes: past every layout's
  // pass B partials (pass A does not use that buffer; pass B writes only
  // the partials in front of it)
  p.mm.prep_off = 0;
  if (p.mma) {
    p.mm.prep_off = cdiv(p.partB_elems, 32) * 32;
    p.partB_elems = p.mm.prep_off + p.mm.prep_floats;
  }
  p.redA_blocks = cdiv(N, kRedCols);
  p.redB_blocks = cdiv(M, kRedRows);
  p.sums_elems = std::max(p.redA_blocks, p.redB_blocks);
  p.flags_elems = M + N;
  return p;
}

int split_rows(int64_t M, int pieces, int* m0, int* rows) {
  const int64_t tile = (int64_t)kThreadsB * kRowsB32;
  const int64_t tiles = cdiv(M, tile);
  const int n = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)pieces, tiles, (int64_t)kMaxPieces}));
  int64_t start = 0;
  for (int i = 0; i < n; ++i) {
    const int64_t t1 = tiles * (i + 1) / n;          // tiles [t0, t1) of piece i
    const int64_t end = std::min(M, t1 * tile);
    m0[i] = (int)start;
    rows[i] = (int)(end - start);
    start = end;
  }
  return n;
}

// Each piece's pass B fills the GPU on its own (same rule as plan_estep):
// fewer row tiles per piece, so more scene-point chunks.
void plan_estep_pieces(EstepPlan& p, int64_t N, int sms, int pieces, const int* m0, const int* rows) {
  int occB = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occB, passB_f32, kThreadsB, 0);
  const int64_t slotsB = (int64_t)sms * std::max(occB, 1);
  const int64_t rowsB = (int64_t)kThreadsB * kRowsB32;
  p.n_pieces = pieces;
  for (int i = 0; i < pieces; ++i) {
    BPiece& b = p.piece[i];
    b.m0 = m0[i];
    b.rows = rows[i];
    b.row_tiles = (int)cdiv(b.rows, rowsB);
    const int64_t want = std::max<int64_t>(1, slotsB / b.row_tiles);
    b.cols_per_chunk = (int)std::max<int64_t>(32, cdiv(N, want));
    b.col_chunks = (int)cdiv(N, b.cols_per_chunk);
    b.red_blocks = (int)cdiv(b.rows, kRedRows);
    p.partB_elems = std::max(p.partB_elems, (int64_t)5 * b.col_chunks * b.rows);
  }
}

template <typename F>
bool launch_estep(const EstepPlan& pl, const typename Vec<F>::t4* T4, const typename Vec<F>::t4* X4,
                  int64_t M, const typename Vec<F>::t4* Y4, typename Vec<F>::t4* Yb, int64_t N,
                  F* partA, F* partB, double* sums, int* flags, typename Vec<F>::t4* Yt4,
                  typename Vec<F>::t4* R4, double* P1_out, double* den_out, DevState* st,
                  bool gate, cudaStream_t s, cudaEvent_t* ev, const EstepSide* side, const EstepPieces* pieces) {
  const int g = gate ? 1 : 0;
  const int defer = side ? 1 : 0;
  dim3 ga(pl.a_col_tiles, pl.a_row_chunks);
  dim3 gb(pl.b_row_tiles, pl.b_col_chunks);
  int* flag_rows = flags;
  int* flag_cols = flags + M;
  if constexpr (sizeof(F) == 4) {
    passA_f32<<<ga, kThreadsA, 0, s>>>(T4, (int)M, pl.a_rows_per_chunk, Y4, (int)N, partA, st, g);
    if (pl.pruned)
      passA_f32_pruned<<<dim3(pl.pa_col_tiles, pl.pa_row_chunks), kThreadsA, 0, s>>>(
          T4, (int)M, pl.pa_rows_per_chunk, Y4, (int)N, partA, st, g);
    if (pl.mma) launch_passA_mma(pl.mm, T4, M, Y4, N, partA, partB + pl.mm.prep_off, st, g, s);
  } else {
    passA_f64<<<ga, kThreadsA, 0, s>>>(T4, (int)M, pl.a_rows_per_chunk, Y4, (int)N, partA, st, g);
  }
  record_after(ev, 0, s);
  reduceA<F><<<(unsigned)pl.redA_blocks, kThreadsR, 0, s>>>(partA, pl.a_row_chunks, pl.pa_row_chunks, pl.mm.a_chunks, (int)M, Y4,
                                                            (int)N, Yb, den_out, sums, flag_cols, st, g, defer);
  if constexpr (sizeof(F) == 4) {
    fixA_f32<<<304, kThreadsF, 0, s>>>(T4, (int)M, Y4, (int)N, Yb, den_out, flag_cols, st, g, defer);
  }
  if (side) {
    // the log-likelihood's total on the side stream, beside pass B
    cudaEventRecord(side->fork, s);
    cudaStreamWaitEvent(side->s, side->fork, 0);
    loglik_finish<F><<<1, kThreadsL, 0, side->s>>>(sums, (int)pl.redA_blocks, Yb, st, (int)M, (int)N, g);
    cudaEventRecord(side->join, side->s);
  }
  record_after(ev, 1, s);
  if constexpr (sizeof(F) == 4) {
    if (pieces && side && pl.n_pieces > 1 && !pl.pruned && !pl.mma) {
      // pass B in row pieces; the caller enqueues each piece's projection
      // and joins the side stream
      for (int i = 0; i < pl.n_pieces; ++i) {
        const BPiece& b = pl.piece[i];
        passB_f32<<<dim3(b.row_tiles, b.col_chunks), kThreadsB, 0, s>>>(T4 + b.m0, b.rows, Yb, (int)N,
                                                                        b.cols_per_chunk, partB, st, g, i == 0);
        reduceB<F><<<(unsigned)b.red_blocks, kThreadsR, 0, s>>>(
            partB, b.col_chunks, b.col_chunks, b.col_chunks, b.rows, X4 + b.m0, Yt4 + b.m0, R4 + b.m0,
            P1_out ? P1_out + b.m0 : nullptr, sums, flag_rows, st, g, 1, b.m0);
        fixB_f32<<<304, kThreadsF, 0, s>>>(T4, (int)M, Yb, (int)N, X4, Yt4, R4, P1_out, flag_rows, st, g, b.m0,
                                           b.m0 + b.rows);
        pieces->after_piece(pieces->user, i);
      }
      return true;
    }
    passB_f32<<<gb, kThreadsB, 0, s>>>(T4, (int)M, Yb, (int)N, pl.b_cols_per_chunk, partB, st, g, 1);
    if (pl.pruned)
      passB_f32_pruned<<<dim3(pl.pb_row_tiles, pl.pb_col_chunks), kThreadsB, 0, s>>>(
          T4, (int)M, Yb, (int)N, pl.pb_cols_per_chunk, partB, st, g);
    if (pl.mma) launch_passB_mma(pl.mm, T4, M, Yb, N, partB, partB + pl.mm.prep_off, st, g, s);
  } else {
    passB_f64<<<gb, kThreadsB, 0, s>>>(T4, (int)M, Yb, (int)N, pl.b_cols_per_chunk, partB, st, g);
  }
  record_after(ev, 2, s);
  reduceB<F><<<(unsigned)pl.redB_blocks, kThreadsR, 0, s>>>(partB, pl.b_col_chunks, pl.pb_col_chunks, pl.mm.b_chunks, (int)M, X4,
                                                            Yt4, R4, P1_out, sums, flag_rows, st, g, defer, 0);
  if constexpr (sizeof(F) == 4) {
    fixB_f32<<<304, kThreadsF, 0, s>>>(T4, (int)M, Yb, (int)N, X4, Yt4, R4, P1_out, flag_rows, st, g, 0,
                                       0x7fffffff);
  }
  if (side) cudaStreamWaitEvent(s, side->join, 0);
  record_after(ev, 3, s);
  return false;
}

template bool launch_estep<float>(const EstepPlan&, const float4*, const float4*, int64_t, const float4*,
                                  float4*, int64_t, float*, float*, double*, int*, float4*, float4*, double*,
                                  double*, DevState*, bool, cudaStream_t, cudaEvent_t*, const EstepSide*,
                                  const EstepPieces*);
template bool launch_estep<double>(const EstepPlan&, const dvec4*, const dvec4*, int64_t, const dvec4*,
                                   dvec4*, int64_t, double*, double*, double*, int*, dvec4*, dvec4*, double*,
                                   double*, DevState*, bool, cudaStream_t, cudaEvent_t*, const EstepSide*,
                                   const EstepPieces*);

}  // namespace fcpd
