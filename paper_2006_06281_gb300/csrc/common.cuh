// Internal declarations of the sm_103a fast-CPD library (not part of the ABI).
//
// Device data layout (all buffers owned by a context, sized at setup /
// first iterate):
//   X4, T4    M model points as 4-vectors {x, y, z, 0}       (FP32: float4, FP64: dvec4)
//   Y4        N scene points {x, y, z, |y|^2}
//   Yb        N scene points prepared for E-pass B: {q y, -log2 den_n} (FP32) or
//             {y, 1/den_n} (FP64)
//   U         M x ldU row-major eigenbasis, ldU = K rounded up to 16 bytes;
//             column k is the k-th largest eigenvector of Phi (Eq. 16, 19)
//   lam       K eigenvalues (double), descending, clamped at 0
//   Yt4       M rows {Ytil_m (3), V_m / P1_m} after the E-step (Eq. 5)
//   R4        M rows {Ytil_m - x_m (3), 0}: the M-step right-hand side (Eq. 17)
//   B4, C4    K rows s_k A_k and A_k / (l_k + lambda sigma2)
//   partials  split-reduction scratch of the E-step and the M-step
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

// Pointer qualifier of the device bodies' arguments.  A translation unit whose
// kernel writes and later reads the same buffers within one launch (the
// batched persistent kernel) defines it empty before including this header,
// so the compiler never turns those loads into non-coherent cache loads.
#ifndef FCPD_RESTRICT
#define FCPD_RESTRICT __restrict__
#endif

#include "../../include/fcpd.h"

namespace fcpd {

constexpr double kLog2e = 1.4426950408889634074;
constexpr double kPi = 3.14159265358979323846;
constexpr int kHistCap = 65536;

struct __align__(32) dvec4 {
  double x, y, z, w;
};

template <typename F> struct Vec;
template <> struct Vec<float> { using t4 = float4; };
template <> struct Vec<double> { using t4 = dvec4; };

// Registration state kept on the device so that iterations need no host sync.
struct DevState {
  double sigma2;        // variance used by the next E-step / M-step
  double loglik;        // Eq. 3 at the last E-step
  double last_dT2;      // sum_m |T_k - T_(k-1)|^2 of the last iteration
  double last_rmse;     // Eq. 22 of the last iteration (NaN without ground truth)
  double w;             // outlier weight
  double lambda;        // regulariser
  double tol;           // RMS(T_k - T_(k-1)) stop threshold (0: off)
  double gt_tol;        // RMSE stop threshold (0: off)
  double vsum;          // sum_m V_m / P1_m of the last E-step (Eq. 18 numerator at T)
  double* hist;         // 4 x kHistCap: sigma2, log-likelihood, RMSE, evaluated-pair fraction per iteration
  int iter;             // iterations completed
  int iter_target;      // iterations run until iter == iter_target
  int status;           // cpd_status of a device-side failure (0 = none)
  int done;             // tolerance reached
  int has_gt;           // ground truth present
  int M, N, K;
  int n_flag_cols;      // FP32: columns whose Gaussian sum needs the exact log-domain path
  int n_flag_rows;      // FP32: rows whose mass needs the exact log-domain path
  unsigned int ticket_a;  // last-block counters (reset by their last block)
  unsigned int ticket_b;
  unsigned int ticket_m;
  unsigned int ticket_e;
  unsigned long long pairs_eval;  // Gaussian pairs evaluated by the pruned passes this iteration
  double last_eval_frac;          // fraction of the 2 M N pairs of passes A+B evaluated last iteration
  float prune_r2;                 // pruned passes run while 127 / kappa (FP32 cutoff radius^2) < this
  int prune_ctl;                  // kPrune* / kMmaAllowed / kBulkWaitFault bits (0: dense passes only)
  double mma_s2min;               // tensor-core passes run while sigma2 >= this
  double trim_lam;                // spectral trim: largest eigenvalue the trimmed M-step drops (< 0: off)
  int trim_now;                   // the trimmed M-step runs in this iteration (set by fixB_f32)
  int trim_iters;                 // iterations of this registration that ran the trimmed M-step
};

static_assert(sizeof(DevState) == 184, "DevState layout changed: update the benchmark's transfer count");

// DevState::prune_ctl bits.
constexpr int kPruneAllowed = 1;   // points are in spatial order: the pruned passes may run
constexpr int kPruneAlways = 2;    // run the pruned passes whatever sigma2 (verification)
constexpr int kPruneNoSkip = 4;    // pruned passes evaluate every tile pair (verification)
constexpr int kMmaAllowed = 8;     // mixed precision: tensor-core distance passes while sigma2 is large
// Verification of the M-step's bounded waits (host fault injection): the
// bulk-copy colsum expects 16 bytes more than it copies, so no slot's phase
// completes and every wait runs out after kBulkFaultWaitNs; the kernel
// records CPD_ETIMEOUT.  All its copies land; none is left in flight.
constexpr int kBulkWaitFault = 16;
constexpr unsigned long long kBulkFaultWaitNs = 50000000ull;   // 50 ms
// The tensor-core passes accumulate exponent terms as large as q^2 |p|^2 in
// FP32: they run while q^2 R^2 <= ~2000 (R = largest point norm), i.e.
// sigma2 >= kMmaS2PerR2 * R^2, which keeps the exponent's rounding near 1e-3.
constexpr double kMmaS2PerR2 = 3.5e-4;

// Spectral trim of the M-step (Eq. 17 with only the leading directions):
// a direction k enters T through s_k a_k, s_k = l_k / (l_k + lambda sigma2).
// When every dropped direction has s_k < kTrimEps, the dropped part of
// U diag(s) U^T R has norm <= kTrimEps |R| (U orthonormal) -- below one FP32
// rounding of T -- and the trimmed M-step over the top K_cap columns runs.
constexpr double kTrimEps = 0x1p-24;
__device__ __forceinline__ bool trim_active(const DevState* st) {
  const double l = st->trim_lam;
  return l >= 0.0 && l < kTrimEps * (l + st->lambda * st->sigma2);
}

// The tensor-core passes' layout is used this iteration (same answer in
// every kernel of an E-step: sigma2 does not change within it).
__device__ __forceinline__ bool mma_active(const DevState* st) {
  return (st->prune_ctl & kMmaAllowed) && st->sigma2 >= st->mma_s2min;
}

// The pruned passes' layout is used this iteration.
__device__ __forceinline__ bool prune_active(const DevState* st) {
  const int c = st->prune_ctl;
  if (!(c & kPruneAllowed) || mma_active(st)) return false;
  if (c & kPruneAlways) return true;
  const double r2 = 127.0 * 2.0 * st->sigma2 / 1.4426950408889634;   // 127 / kappa, kappa = log2(e) / (2 sigma2)
  return r2 < (double)st->prune_r2;
}

// True when the current iteration must not run (target reached, converged,
// or a device failure recorded).  Read once per block at kernel entry.
__device__ __forceinline__ bool iteration_gated(const DevState* st) {
  return st->iter >= st->iter_target || st->done || st->status != 0;
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Sum of a double over a block (blockDim.x multiple of 32, <= 1024).
// Result valid in thread 0.  `sh` holds >= 32 doubles.
__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double r = 0.0;
  if (warp == 0) {
    r = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
  }
  return r;
}

// Sums of three doubles over the first `warps` warps of a block (the other
// warps' values are ignored; every thread of the block must call it).  One
// pair of barriers for the three sums; fixed order.  Results valid in
// thread 0.  `sh` holds >= 32 x 3 doubles.
__device__ __forceinline__ void block_sum3(double& a, double& b, double& c, double (*sh)[3], int warps) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp < warps) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
      c += __shfl_xor_sync(0xffffffffu, c, o);
    }
  }
  __syncthreads();
  if (warp < warps && lane == 0) {
    sh[warp][0] = a;
    sh[warp][1] = b;
    sh[warp][2] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    a = sh[0][0]; b = sh[0][1]; c = sh[0][2];
    for (int w = 1; w < warps; ++w) {
      a += sh[w][0];
      b += sh[w][1];
      c += sh[w][2];
    }
  }
}

// ---------------------------------------------------------- spatial order
// Largest point set the spatial sort handles (larger sets stay unsorted and
// the E-step does not prune).
constexpr int64_t kMaxSortPoints = (int64_t)1 << 20;
bool spatial_sort_supported(int64_t n);
int64_t spatial_sort_scratch_bytes(int64_t n);
// out[s] = in[perm[s]] in Morton order (stable); perm may be null.
cudaError_t launch_spatial_sort(const float4* in, int64_t n, float4* out, int* perm, void* scratch, cudaStream_t s);
void launch_invert_perm(const int* perm, int64_t n, int* inv, cudaStream_t s);
// dst[s] = (src point perm[s], |.|^2 or 0): caller order -> sorted order
template <typename F>
void launch_pack_gather(const F* src, const int* perm, int64_t n, typename Vec<F>::t4* dst, bool with_norm,
                        cudaStream_t s);
// dst point i = src[inv[i]]: sorted order -> caller order
template <typename F>
void launch_unpack_gather(const typename Vec<F>::t4* src, const int* inv, int64_t n, F* dst, cudaStream_t s);
// dst row i (cols floats) = src row inv[i] (stride ld_src)
void launch_gather_rows_f32(const float* src, int64_t ld_src, const int* inv, int64_t n, int64_t cols, float* dst,
                            cudaStream_t s);

// ---------------------------------------------------------- warm start
// c[k][d] = sum_m U[m][k] (T[m] - X[m])_d for k < K (basis stored as B:
// float, or __half in the mixed-precision mode).
template <typename B>
void launch_coefficients(const B* U, int64_t ldU, int64_t M, int64_t K, const float4* T4, const float4* X4, float* c,
                         cudaStream_t s);
// T[m] = X[m] + sum_{k < nc} U[m][k] c[k].
template <typename B>
void launch_warm_start_T(const B* U, int64_t ldU, int64_t M, int64_t nc, const float* c, const float4* X4,
                         float4* T4, cudaStream_t s);

// Message returned by cpd_last_error() on the calling thread.
void set_last_error(const std::string& msg);

// ---------------------------------------------------------------- launchers
struct MmaPlan {
  int a_row_tiles, a_chunks, a_rows_per_chunk;       // pass A: 128-point scene tiles x model-point chunks
  int b_row_tiles, b_chunks, b_cols_per_chunk;       // pass B: 128-point model tiles x scene-point chunks
  int a_tpc, b_tpc;                                  // 128-point column tiles per chunk
  int64_t prep_floats;                               // column-vector scratch (floats) of either pass
  int64_t prep_off;                                  // its offset in the pass B partials buffer
};
void plan_estep_mma(int64_t M, int64_t N, int sms, MmaPlan& p);
// The tcgen05 passes can run on this device (their shared memory fits).
bool estep_mma_supported();
int estep_mma_occupancy(int pass);      // resident CTAs per SM of pass 0 (A) or 1 (B)
// prep: prep_floats of scratch for the column vectors (in the pass B
// partials buffer past the partials; unused by pass A's own partials).
void launch_passA_mma(const MmaPlan& p, const float4* T4, int64_t M, const float4* Y4, int64_t N, float* partA,
                      float* prep, DevState* st, int gate, cudaStream_t s);
void launch_passB_mma(const MmaPlan& p, const float4* T4, int64_t M, const float4* Yb, int64_t N, float* partB,
                      float* prep, DevState* st, int gate, cudaStream_t s);
// sigma2 floor of the tensor-core passes from the largest point norm of X and Y.
void launch_mma_threshold(const float4* X4, int64_t M, const float4* Y4, int64_t N, DevState* st, cudaStream_t s);

// Pass B of an FP32 iteration split into row pieces, so that the M-step's
// projection of the rows a piece has finished (on a side stream) runs beside
// the next piece's pass B: the projection streams U from HBM while pass B
// keeps the FP32 pipes busy.  Piece i covers model rows [m0, m0 + rows).
constexpr int kMaxPieces = 4;
struct BPiece {
  int m0, rows;                                      // model rows of the piece
  int row_tiles, col_chunks, cols_per_chunk;         // its pass B grid
  int red_blocks;                                    // its row-reduction grid
};

struct EstepPlan {
  int a_col_tiles, a_row_chunks, a_rows_per_chunk;   // pass A grid
  int b_row_tiles, b_col_chunks, b_cols_per_chunk;   // pass B grid
  int n_pieces;                                      // > 1: pass B in row pieces (see BPiece)
  BPiece piece[kMaxPieces];
  int64_t partA_elems, partB_elems;                  // scratch sizes (elements of F)
  int64_t redA_blocks, redB_blocks;                  // reduce grids
  int64_t sums_elems;                                // double scratch for block sums
  int64_t flags_elems;                               // int scratch: flagged rows + columns
  // pruned FP32 layout (spatially ordered inputs; see estep_dev.cuh)
  bool pruned;                                       // launch the pruned passes too
  int pa_col_tiles, pa_row_chunks, pa_rows_per_chunk;
  int pb_row_tiles, pb_col_chunks, pb_cols_per_chunk;
  // tensor-core layout (mixed precision; see estep_mma.cu)
  bool mma;                                          // launch the tensor-core passes too
  MmaPlan mm;
};
// with_pruned / with_mma: also plan those layouts (partial buffers sized for all).
EstepPlan plan_estep(int64_t M, int64_t N, bool fp64, int sms, bool with_pruned = false, bool with_mma = false);
// Row boundaries of `pieces` pass B pieces over M rows: whole pass B row
// tiles, as even as they go; returns the number of pieces (fewer when M has
// fewer tiles).
int split_rows(int64_t M, int pieces, int* m0, int* rows);
// Pass B grids of the pieces (FP32 only); enlarges the partial-sum and
// block-sum sizes where a piece needs more.
void plan_estep_pieces(EstepPlan& p, int64_t N, int sms, int pieces, const int* m0, const int* rows);

struct MstepPlan {
  int64_t ldU, ldM;                                  // row strides of U (M x ldU) and U^T (K x ldM)
  int p_col_tiles, p_row_chunks, p_rows_per_chunk;   // projection U^T R grid
  int e_col_tiles, e_row_chunks, e_rows_per_chunk;   // expansion U B grid
  int e_blocks;                                      // expansion reduction grid
  int64_t part_elems;                                // scratch (elements of F), shared by both
  int64_t sums_elems;                                // double scratch for block sums
  bool bulk;                                         // products by colsum_bulk (bulk-copy ring)
  int64_t K;                                         // basis columns the plan streams
  int64_t ldPp;                                      // row stride of the projection partials
  // projection in row pieces (with the E-step's pass B pieces): piece i
  // streams rows [pp_m0, pp_m0 + pp_rows) into partial rows from pp_off on
  int n_pieces;
  int pp_m0[kMaxPieces], pp_rows[kMaxPieces], pp_chunks[kMaxPieces], pp_rpc[kMaxPieces], pp_off[kMaxPieces];
  int pp_chunks_total;
};
// `colsum_threads`: block size of the streaming kernel the plan is for (128
// for the per-pair launches, 256 inside the batched persistent kernel).
// basis_bytes: element size of the stored basis (0: that of the working
// precision; 2 for the FP16 basis of the mixed-precision mode).
MstepPlan plan_mstep(int64_t M, int64_t K, bool fp64, int sms, int colsum_threads = 128, int basis_bytes = 0);
// Plan of the trimmed M-step: the leading K_cap columns of the basis laid
// out by `full` (same row strides).
MstepPlan plan_mstep_trim(const MstepPlan& full, int64_t M, int64_t K_cap, bool fp64, int sms, int basis_bytes);
// Projection grids of row pieces (FP32 basis streamed by colsum_bulk, wide
// bases only): the last piece, which runs alone, gets one resident wave; the
// others one block per SM, the room left beside two pass B blocks.
// Enlarges part_elems.  False (no pieces) where the plan cannot be split.
bool plan_mstep_pieces(MstepPlan& p, int64_t M, int sms, int pieces, const int* m0, const int* rows);

// ------------------------------------------------------------ batched mode
// One registration inside the batched persistent kernel: its sizes, plans
// and buffers (all device pointers).
struct BatchPair {
  int M, N, K;
  EstepPlan ep;
  MstepPlan mp;
  const float4* X4;
  float4* T4;
  const void* U;              // float, or __half with half_basis (mixed precision)
  const void* Ut;
  int half_basis;
  const double* lam;
  float4* Yt4;
  float4* R4;
  float4* B4;
  float4* C4;
  const float4* Y4;
  float4* Yb;
  const float4* Yhat4;
  float* partA;
  float* partB;
  float* partP;
  double* sums;
  int* flags;
  DevState* st;
  unsigned int* tix;          // completion tickets of the pair's tiles (batch_tickets entries, zeroed)
  unsigned int* done;         // phases completed in the current launch, one counter per phase (zeroed per launch)
  int narrow;                 // projection by the row-split body (K <= 128)
};
struct BatchItem {
  int pair, bx, by;
};
// Control block of one persistent launch (zeroed before each launch).
struct BatchCtl {
  unsigned long long next;           // next work item of the launch (iteration-major)
  int status;                 // CPD_ETIMEOUT if a wait for a pair's previous phase gave up
  int pad;
  unsigned long long t_start;        // block 0's clock at the start of the launch
  unsigned long long t_end;          // latest clock at which a block ran out of work items
  unsigned long long wait_ns[16];    // per phase: time blocks spent waiting for a pair's previous phase
  unsigned long long busy_ns[16];    // per phase: time all blocks spent inside work items
};
// Resident blocks of the persistent kernel on `sms` SMs (0 on failure).
int batch_resident_blocks(int sms);
// Fills ep, mp and narrow of every pair from its M, N, K (work-item sizes:
// see batch.cu; the defaults are the untuned plan).
void plan_batch(BatchPair* pairs_host, int n_pairs, int resident, int e_items_per_block = 4, int proj_kbytes = 512);
// Work items of every phase (phase ph owns items [phase_off[ph], phase_off[ph+1])).
void batch_items(const BatchPair* pairs_host, int n_pairs, std::vector<BatchItem>& items, std::vector<int>& phase_off);
// Completion tickets a pair needs (after plan_batch), and the phases per iteration.
int batch_tickets(const BatchPair& p);
int batch_phases();
// Zeroes ctl and the pairs' phase counters (done: 4 per pair), then runs
// n_iter iterations of every pair in one cooperative launch of `grid`
// blocks.  barrier_extra > 0 makes every wait for a pair's previous phase
// ask for one phase more than will ever complete (host-side fault injection
// for the timeout path).
cudaError_t launch_batch(const BatchPair* pairs_dev, int n_pairs, const BatchItem* items, const int* phase_off,
                         BatchCtl* ctl, unsigned int* done, int grid, int n_iter, double wait_limit_s, int barrier_extra,
                         cudaStream_t s);
// Copies every pair's device state into out[0..n_pairs).
void launch_batch_states(const BatchPair* pairs_dev, int n_pairs, DevState* out, cudaStream_t s);


// Optional `ev` arrays: an event is recorded (as an external event-record
// node when captured) after each kernel: 4 for the E-step (pass A, its
// reduction, pass B, its reduction), 4 for the M-step (projection, diagonal
// update, expansion, its reduction + Eq. 18).
inline void record_after(cudaEvent_t* ev, int i, cudaStream_t s) {
  if (!ev) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cs);
  if (cs == cudaStreamCaptureStatusActive) cudaEventRecordWithFlags(ev[i], s, cudaEventRecordExternal);
  else cudaEventRecord(ev[i], s);
}

// Side stream of an iteration's E-step: the log-likelihood total is formed
// there, beside pass B (fork after the column fix-up, join at the E-step's
// end); the iterations then also skip the sum of V_m / P1_m.
struct EstepSide {
  cudaStream_t s;
  cudaEvent_t fork, join;
};

// E-step: passes A and B with their reductions.  Reads T4, Y4 and st->sigma2;
// writes Yt4, R4 (R4 needs X4; may be null to skip) and per-row P1 (double,
// optional), per-column den (double, optional).  Gated by `gate` (iteration mode)
// or always run (standalone).  Without `side`, st->loglik and st->vsum are
// complete when the last kernel ends.
// With `pieces` (FP32 iterations with `side`, plan with n_pieces > 1) pass B
// runs piece by piece and after_piece(user, i) is called once piece i's rows
// of Yt4 / R4 are enqueued on `s`; the side stream is then left for the
// caller to join.  Returns true when pass B ran in pieces.
struct EstepPieces {
  void (*after_piece)(void* user, int piece);
  void* user;
};
template <typename F>
bool launch_estep(const EstepPlan& pl, const typename Vec<F>::t4* T4, const typename Vec<F>::t4* X4,
                  int64_t M, const typename Vec<F>::t4* Y4, typename Vec<F>::t4* Yb, int64_t N,
                  F* partA, F* partB, double* sums, int* flags, typename Vec<F>::t4* Yt4,
                  typename Vec<F>::t4* R4, double* P1_out, double* den_out, DevState* st,
                  bool gate, cudaStream_t s, cudaEvent_t* ev = nullptr, const EstepSide* side = nullptr,
                  const EstepPieces* pieces = nullptr);

// M-step: projection a = U^T R, diagonal update, expansion T = X + U B and
// the Eq. 18 variance in the epilogue.  U is M x ldU, Ut = U^T is K x ldM.
// With `iteration` false the state is not advanced (standalone M-step:
// T4 receives T, no sigma2 update, st supplies sigma2 and lambda).
// S: storage type of the basis (F, or __half in the mixed-precision mode).
// With `trim` (an iteration of a context with the spectral trim) the device
// state's trim_now -- set by the E-step's last launch -- selects the trimmed
// M-step (plan *trim) or the full one (pl) for this iteration; both are
// enqueued, step by step, and the other steps aside.  The trimmed M-step sets B and C to 0 for the
// dropped directions.
// projected: the projection already ran in the plan's row pieces
// (launch_projection_piece); the M-step starts at the diagonal update.
template <typename F, typename S = F>
void launch_mstep(const MstepPlan& pl, const S* U, const S* Ut, const double* lam, int64_t M, int64_t K,
                  const typename Vec<F>::t4* X4, const typename Vec<F>::t4* R4,
                  const typename Vec<F>::t4* Yt4, typename Vec<F>::t4* T4,
                  const typename Vec<F>::t4* Yhat4, F* part, double* sums,
                  typename Vec<F>::t4* B4, typename Vec<F>::t4* C4, DevState* st,
                  bool iteration, cudaStream_t s, cudaEvent_t* ev = nullptr, const MstepPlan* trim = nullptr,
                  bool projected = false);
// Projection partials of piece `piece` of an iteration (FP32 basis).
void launch_projection_piece(const MstepPlan& pl, int piece, const float* U, const float4* R4, float* part,
                             DevState* st, cudaStream_t s);

// Several registrations against one model (multi.cu): the M-step of S
// scenes with both products in one pass over U and U^T each (FP32 basis).
struct MultiPlan {
  int S;                                             // scenes per pass (1..8)
  int p_col_tiles, p_chunks, p_rpc;                  // projection grid (rows of U)
  int e_col_tiles, e_chunks, e_rpc;                  // expansion grid (rows of U^T)
  int e_blocks;                                      // per-scene epilogue grid
  int64_t part_elems, sums_elems;                    // scratch (floats, doubles)
};
constexpr int kMaxScenesPerPass = 8;
MultiPlan plan_multi(int64_t M, int64_t K, int64_t ldU, int64_t ldM, int S, int sms);
// R4, Yt4, T4: S x M rows; B4, C4: S x K rows; st: S device states (host
// array of device pointers); status: device int receiving CPD_ETIMEOUT if a
// bounded wait of the streaming kernel runs out.
void launch_mstep_multi(const MultiPlan& p, const float* U, int64_t ldU, const float* Ut, int64_t ldM,
                        const double* lam, int64_t M, int64_t K, const float4* X4, const float4* R4,
                        const float4* Yt4, float4* T4, float4* B4, float4* C4, DevState* const* st, float* part,
                        double* sums, int* status, cudaStream_t s);

// Tensor-core products for S scenes against one FP16 basis (umma.cu):
// partials part[s][chunk][d][row] of D = A V^T, A the basis (P rows x Q,
// row stride ldA, FP16), V the scenes' right-hand sides split into FP16
// hi / lo parts (npad x ldq, built by launch_pack_rhs from S float4 arrays
// of Q entries, scene stride ld_src).  The partial layout is that of the
// single-scene products, so the per-scene reductions are shared.
struct UmmaPlan {
  int64_t P, Q;          // rows of D, contraction length
  int S, npad;           // scenes, MMA columns (2 x 3S rounded up to 16)
  int tiles, chunks;     // 128-row tiles x contraction chunks (the grid)
  int kspc;              // 64-element stages per chunk
  int64_t ldq;           // row stride of V
};
int umma_npad(int S);
// The tensor-core products can run for S scenes (npad <= 256, the driver's
// tensor-map encoder found).
bool umma_supported(int S);
UmmaPlan plan_umma(int64_t P, int64_t Q, int S, int sms);
int64_t umma_rhs_elems(const UmmaPlan& p);
void launch_pack_rhs(const UmmaPlan& p, const float4* src, int64_t ld_src, __half* V, cudaStream_t s);
// fault_wait: host fault injection (every full barrier expects 16 bytes more
// than its copies: each wait runs out after 50 ms and *status becomes
// CPD_ETIMEOUT).
cudaError_t launch_umma_products(const UmmaPlan& p, const __half* A, int64_t ldA, const __half* V, float* part,
                                 int64_t ldP, int* status, bool fault_wait, cudaStream_t s);
constexpr int kMaxScenesPerPassMma = 32;
// doubles of block sums the per-scene Eq. 18 epilogue needs for M points
int64_t multi_sums_elems(int64_t M);
// The shared-model M-step with tensor-core products (multi.cu): Vp (pp.npad
// x pp.ldq) and Ve (pe.npad x pe.ldq) zeroed before the first use; part
// holds max(S chunks 3 ldU (projection), S chunks 3 ldM (expansion)) floats.
cudaError_t launch_mstep_multi_mma(const UmmaPlan& pp, const UmmaPlan& pe, const __half* U, int64_t ldU,
                                   const __half* Ut, int64_t ldM, const double* lam, int64_t M, int64_t K,
                                   const float4* X4, const float4* R4, const float4* Yt4, float4* T4, float4* B4,
                                   float4* C4, DevState* const* st, __half* Vp, __half* Ve, float* part,
                                   double* sums, int* status, bool fault_wait, cudaStream_t s);

// BF16 tensor-core GEMM of the warm-start network (gemm_tc.cu): D = A B^T,
// A (P x Q, row stride lda) and B (N x Q, row stride ldb) BF16 with the
// contraction contiguous, N = 128 or 256, FP32 accumulation.  chunks > 1:
// split-K partials out[chunk][P][ldo] (to be summed in order); else the
// epilogue + bias, ReLU or the mask (0 where mask[p][n] <= 0) and the FP32
// result out[P][ldo] with optional BF16 copies (row-major, transposed [N][ld_t]).
// fault_wait (host fault injection only): every pipeline wait runs out
// after 50 ms and *status receives CPD_ETIMEOUT.
cudaError_t launch_gemm_tc(const __nv_bfloat16* A, int64_t lda, const __nv_bfloat16* B, int64_t ldb, int P, int N,
                           int Q, int chunks, const float* bias, bool relu, const float* mask, int64_t ldm,
                           float* out, int64_t ldo, __nv_bfloat16* out_bf, int64_t ld_bf, __nv_bfloat16* out_t,
                           int64_t ld_t, int* status, bool fault_wait, cudaStream_t s);
int gemm_tc_chunks(int Q, int chunks);
void launch_to_bf16(const float* X, int64_t R, int C, __nv_bfloat16* row, __nv_bfloat16* tr, int64_t ldt,
                    cudaStream_t s);
void launch_weights_bf16(const float* W, int fi, int fo, __nv_bfloat16* w, __nv_bfloat16* wt, cudaStream_t s);

// W = U C (C from the last M-step), written as 4-vectors.
template <typename F, typename S = F>
void launch_w(const MstepPlan& pl, const S* Ut, int64_t M, int64_t K, const typename Vec<F>::t4* C4, F* part,
              typename Vec<F>::t4* W4, DevState* st, cudaStream_t s);

// Setup helpers.
void launch_gram_f64(const void* X4, bool x_fp64, int64_t M, double beta, double* Phi, cudaStream_t s);
// V: M x nv column-major eigenvectors with eigenvalues w[nv] ascending (the
// eigensolvers' order); the K largest pairs are kept, descending.
template <typename F>
void launch_extract_basis(const double* V, int64_t M, int64_t nv, int64_t K, F* U, int64_t ldU, F* Ut, int64_t ldM,
                          const double* w, double* lam, cudaStream_t s);

// Top-K eigenpairs of the M x M FP64 Gram matrix Phi (eig.cu: subspace
// iteration with Rayleigh-Ritz steps, FP64, cuBLAS / cuSOLVER).  Used when
// topk_eig_applies(M, K).  On CPD_OK: *V_out (M x *nv_out column-major,
// device, cudaMalloc'd, freed by the caller with cudaFree) and *w_out (*nv_out
// device doubles, ascending) hold Ritz pairs whose largest K have residuals
// |Phi u - theta u| <= tol * theta_max; *steps_out = Rayleigh-Ritz steps.
// Returns a cpd_status, or -1 if max_steps were not enough (the caller then
// uses the full eigensolver).  Synchronises `s`.
bool topk_eig_applies(int64_t M, int64_t K);
int topk_oversampling(int64_t K);
int topk_eigh(const double* Phi, int64_t M, int64_t K, double tol, int max_steps, cudaStream_t s, double** V_out,
              double** w_out, int64_t* nv_out, int* steps_out, std::string* err);
// FP16 basis (mixed-precision mode) -> M x K FP32, row-major, unpadded.
void launch_basis_to_f32(const __half* U, int64_t M, int64_t K, int64_t ldU, float* out, cudaStream_t s);
template <typename F>
void launch_sigma2_init(const typename Vec<F>::t4* X4, int64_t M, const typename Vec<F>::t4* Y4,
                        int64_t N, double* scratch, DevState* st, cudaStream_t s);

// Packing between caller arrays (row-major n x 3, float or double) and 4-vectors.
// `with_norm` stores |p|^2 in the 4th lane, else 0.
template <typename F>
void launch_pack(const F* src, int64_t n, typename Vec<F>::t4* dst, bool with_norm, cudaStream_t s);
template <typename F>
void launch_unpack(const typename Vec<F>::t4* src, int64_t n, F* dst, cudaStream_t s);
void launch_begin_iterations(DevState* st, int n_iter, cudaStream_t s);
// Sets the WHILE condition h of a conditional graph node: 1 while another
// iteration should run (target not reached, no tolerance stop, no failure).
void launch_loop_control(const DevState* st, cudaGraphConditionalHandle h, cudaStream_t s);
void launch_state_init(DevState* st, double sigma2, cudaStream_t s);
// Pruning configuration of a context (kept across state_init, which turns it off).
void launch_state_prune(DevState* st, float prune_r2, int prune_ctl, cudaStream_t s);
// Spectral trim threshold of a registration (the largest dropped eigenvalue;
// < 0 switches the trim off).
void launch_state_trim(DevState* st, double trim_lam, cudaStream_t s);
void launch_state_params(DevState* st, double w, double lambda, double tol, double gt_tol, int has_gt,
                         double* hist, int64_t M, int64_t N, int64_t K, cudaStream_t s);
template <typename F>
void launch_residual(const typename Vec<F>::t4* Yt4, const typename Vec<F>::t4* X4, typename Vec<F>::t4* R4,
                     int64_t M, cudaStream_t s);


}  // namespace fcpd
