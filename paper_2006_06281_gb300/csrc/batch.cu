// Batched registrations: many independent (X_i, Y_i) pairs of uneven sizes
// run their EM iterations in ONE persistent cooperative kernel launch.
//
// Every iteration of every pair runs the same arithmetic as the per-pair
// path (estep_dev.cuh / mstep_dev.cuh) in four phases:
//   A  E pass A tiles; the last row chunk of a column tile to finish reduces
//      that tile's columns (den, Eq. 4), and the block completing a pair's
//      columns runs the FP32 log-domain fix-up of its flagged columns;
//   B  E pass B tiles; likewise the row reduction (Eq. 5) per row tile and
//      the row fix-up per pair;
//   P  projection U^T (Ytil - X) by row chunks; the last chunk of a pair
//      runs the diagonal update;
//   E  expansion with U^T by (column tile, row chunk); the last row chunk of
//      a column tile forms T for those columns, and the block completing a
//      pair's columns updates sigma2 (Eq. 18).
// "Last" is decided by per-tile completion tickets (an atomic counter per
// tile, reset by the block that completes it).  For each phase the host
// lists the work items of all pairs -- (pair, block coordinates), largest
// pairs first -- and the resident blocks take items from one atomic counter
// running over every iteration's phases in order, so small and large pairs
// share the GPU without per-pair launches.  Phases are ordered per pair, not
// by grid barriers: the block that completes a pair's phase (its last
// reduction, diagonal update or expansion tile) bumps the pair's counter for
// that phase, and an item of the next phase waits for it -- so pass B items
// of a pair whose columns are done run while other pairs' pass A items are
// still in flight.  The items a block waits for were taken from the counter
// before its own by running blocks, so the wait always ends; it is bounded
// in wall time all the same: past the limit the kernel records CPD_ETIMEOUT
// in the control block and every block returns (no GPU hang); the host
// reports the status.
//
// Buffers such as T, Yb and the partial sums are written in one phase and
// read in a later one of the same launch, so no argument of the device bodies
// is __restrict__ here (only U and U^T, constant for the launch, go through
// the read-only path).  The E-step bodies are compiled with 8 scene points
// (pass A) and 8 model points (pass B) per thread: 2048-point tiles, whose
// partial last tile runs with 2, 4 or 6 points per thread (the fewest that
// cover it) so that small pairs stay lightly padded, where the per-pair
// launches use 16 and 8 for scenes of tens of thousands of points.  At 256
// pairs of 500..8000 points 8 per thread took 0.40 s per 100 iterations
// against 0.42 s with 4 (pass A's shared-memory reads are then shared by
// twice the Gaussians); FCPD_BATCH_PTS_A / _B set the counts.  The
// reduction bodies give each thread a whole column (row) of chunk partials:
// a pair has only a few chunks here, and a reduction block's fixed latency
// (dependent loads, block sums, the completion ticket) is paid per 256
// columns instead of per 32 or 64.
#define FCPD_RESTRICT
#ifndef FCPD_BATCH_PTS_A
#define FCPD_BATCH_PTS_A 8
#endif
#ifndef FCPD_BATCH_PTS_B
#define FCPD_BATCH_PTS_B 8
#endif
#define FCPD_EA_COLS FCPD_BATCH_PTS_A
#define FCPD_EB_ROWS FCPD_BATCH_PTS_B
#define FCPD_RED_COLS 256
#define FCPD_RED_ROWS 256
#define FCPD_MRED_COLS 256
#include "estep_dev.cuh"
#include "mstep_dev.cuh"

#include <algorithm>
#include <vector>

namespace fcpd {

namespace {

constexpr int kThreadsBatch = 256;
constexpr int kNarrowGroups = 16;                               // 8-column groups of a narrow basis
constexpr int kNarrowLanes = kThreadsBatch / kNarrowGroups;     // row lanes
constexpr int kNarrowMaxK = kNarrowGroups * 8;                  // widest basis of the narrow projection

enum Phase { PH_A = 0, PH_B, PH_P, PH_E, kPhases };

constexpr int kTileColsA = dev::kThreadsA * dev::kColsA32;   // scene points per pass-A tile
constexpr int kTileRowsB = dev::kThreadsB * dev::kRowsB32;   // model points per pass-B tile
constexpr int kTileColsE = kThreadsBatch * 8;                // columns of U^T per expansion tile
static_assert(kTileColsA % dev::kRedCols == 0 && kTileRowsB % dev::kRedRows == 0 &&
                  kTileColsE % dev::kMRedCols == 0,
              "a tile holds whole reduction blocks");

static_assert(dev::kThreadsA == kThreadsBatch && dev::kThreadsB == kThreadsBatch && dev::kThreadsR == kThreadsBatch &&
                  dev::kThreadsF == kThreadsBatch && dev::kThreadsD == kThreadsBatch,
              "the persistent kernel runs every phase with one block size");
static_assert(kPhases <= 16, "BatchCtl holds 16 item counters");

int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Thread 0: waits until pair P's phase `need_ph` has completed `need` times
// in this launch (or P's iterations are gated: then the item does nothing
// and needs nothing).  False (CPD_ETIMEOUT recorded unless another failure
// is) past limit_ns, or at once if another block has failed.
__device__ bool wait_phase(const BatchPair& P, int need_ph, unsigned int need, BatchCtl* ctl,
                           unsigned long long limit_ns) {
  volatile unsigned int* c = P.done + need_ph;
  if (*c >= need || iteration_gated(P.st)) return true;
  const unsigned long long t0 = global_ns();
  for (;;) {
    __nanosleep(64);
    if (*c >= need) return true;
    const volatile DevState* st = P.st;
    if (st->iter >= st->iter_target || st->done || st->status != 0) return true;
    if (*(volatile int*)&ctl->status != 0) return false;
    if (global_ns() - t0 > limit_ns) {
      atomicCAS(&ctl->status, 0, (int)CPD_ETIMEOUT);
      return false;
    }
  }
}

// Called by every thread of the block that completed pair P's phase ph.
__device__ __forceinline__ void phase_done(const BatchPair& P, int ph) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(P.done + ph, 1u);
  }
}

// Eight consecutive basis elements as floats (16-byte aligned): FP32, or the
// FP16 basis of the mixed-precision mode.
__device__ __forceinline__ void load8(const float* p, float (&u)[8]) {
  const float4 a = __ldg(reinterpret_cast<const float4*>(p)), b = __ldg(reinterpret_cast<const float4*>(p) + 1);
  u[0] = a.x; u[1] = a.y; u[2] = a.z; u[3] = a.w; u[4] = b.x; u[5] = b.y; u[6] = b.z; u[7] = b.w;
}
__device__ __forceinline__ void load8(const __half* p, float (&u)[8]) {
  const uint4 r = __ldg(reinterpret_cast<const uint4*>(p));
  const __half2* h = reinterpret_cast<const __half2*>(&r);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float2 f = __half22float2(h[i]);
    u[2 * i] = f.x;
    u[2 * i + 1] = f.y;
  }
}

// Projection A = U^T R for a basis of at most 128 columns: 16 groups of 8
// columns x 16 row lanes, the lanes combined in a fixed order through shared
// memory.  Writes the same chunk partials as colsum_body (row chunk `by`).
template <typename B>
__device__ __forceinline__ void proj_narrow_body(const B* U, int64_t ldU, int M, int K, const float4* R4,
                                                 int rows_per_chunk, float* part, int64_t ldP, DevState* st,
                                                 int by) {
  if (iteration_gated(st)) return;
  // the E-step's row list was consumed by fixB before this phase
  if (by == 0 && threadIdx.x == 0) st->n_flag_rows = 0;
  __shared__ float red[kNarrowLanes][kNarrowMaxK];
  const int g = threadIdx.x % kNarrowGroups, lane = threadIdx.x / kNarrowGroups;
  const int c0 = g * 8;
  const int r0 = by * rows_per_chunk;
  const int r1 = min(M, r0 + rows_per_chunk);
  float acc[8][3];
#pragma unroll
  for (int w = 0; w < 8; ++w) acc[w][0] = acc[w][1] = acc[w][2] = 0.f;
  if (c0 < K) {
#pragma unroll 4
    for (int m = r0 + lane; m < r1; m += kNarrowLanes) {
      float u[8];
      load8(U + (size_t)m * ldU + c0, u);
      const float4 r = R4[m];
#pragma unroll
      for (int w = 0; w < 8; ++w) {
        acc[w][0] = fmaf(u[w], r.x, acc[w][0]);
        acc[w][1] = fmaf(u[w], r.y, acc[w][1]);
        acc[w][2] = fmaf(u[w], r.z, acc[w][2]);
      }
    }
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    __syncthreads();
#pragma unroll
    for (int w = 0; w < 8; ++w) red[lane][c0 + w] = acc[w][d];
    __syncthreads();
    if (threadIdx.x < K) {
      float s = 0.f;
#pragma unroll
      for (int l = 0; l < kNarrowLanes; ++l) s += red[l][threadIdx.x];
      part[((size_t)by * 3 + d) * ldP + threadIdx.x] = s;
    }
  }
}

// Expansion of a narrow basis (K <= kNarrowMaxK) fused with T and Eq. 18: one
// item is a tile of kNarrowTileE = 256 model points; lane l of every warp
// owns points 8l..8l+7 of the tile (32-byte loads of a row of U^T) and warp w
// takes the rows k = w, w + 8, .. of U^T, so each thread has K / 8 rows to
// stream instead of K; the eight warps' partial sums meet in shared memory
// (added in warp order), after which thread t forms point t's t_m and Eq. 18
// terms -- the FP64 epilogue of 256 points in parallel.  A per-pair ticket
// over the tiles lets the block that completes the pair finish the iteration.
constexpr int kNarrowTileE = 256;
static_assert(kNarrowTileE == 32 * 8 && kThreadsBatch == kNarrowTileE, "one point per thread in the epilogue");
// the warps' partial sums: [warp][coordinate][point w of a lane][lane],
// padded; one array for both basis types
__shared__ float s_narrow_red[kThreadsBatch / 32][3][8][33];
template <typename B>
__device__ __forceinline__ bool expand_narrow_body(const B* Ut, int64_t ldM, int K, int M, const float4* B4,
                                                   const float4* X4, const float4* Yt4, float4* T4,
                                                   const float4* Yhat4, double* sums, DevState* st, int bx, int gx) {
  if (iteration_gated(st)) return false;
  constexpr int NW = kThreadsBatch / 32;
  __shared__ float4 sB[kNarrowMaxK];
  float (*red)[3][8][33] = s_narrow_red;
  __shared__ double sh3[32][3];
  __shared__ bool last;
  // the epilogue's inputs of point t, in flight with the expansion
  const int m = bx * kNarrowTileE + threadIdx.x;
  float4 x{}, to{}, yt{};
  if (m < M) {
    x = X4[m];
    to = T4[m];
    yt = Yt4[m];
  }
  for (int i = threadIdx.x; i < K; i += kThreadsBatch) sB[i] = B4[i];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c0 = bx * kNarrowTileE + lane * 8;
  float acc[8][3];
#pragma unroll
  for (int w = 0; w < 8; ++w) acc[w][0] = acc[w][1] = acc[w][2] = 0.f;
  if (c0 < M) {                                 // c0 + 8 <= ldM: rows of U^T are padded to 8
#pragma unroll 4
    for (int k = warp; k < K; k += NW) {
      float u[8];
      load8(Ut + (size_t)k * ldM + c0, u);
      const float4 b = sB[k];
#pragma unroll
      for (int w = 0; w < 8; ++w) {
        acc[w][0] = fmaf(u[w], b.x, acc[w][0]);
        acc[w][1] = fmaf(u[w], b.y, acc[w][1]);
        acc[w][2] = fmaf(u[w], b.z, acc[w][2]);
      }
    }
  }
#pragma unroll
  for (int w = 0; w < 8; ++w)
#pragma unroll
    for (int d = 0; d < 3; ++d) red[warp][d][w][lane] = acc[w][d];
  __syncthreads();
  const int lp = threadIdx.x >> 3, wp = threadIdx.x & 7;   // point t = 8 * lane' + w
  double contrib = 0.0, dT2 = 0.0, gt2 = 0.0;
  if (m < M) {
    float a0 = 0.f, a1 = 0.f, a2 = 0.f;
#pragma unroll
    for (int j = 0; j < NW; ++j) {
      a0 += red[j][0][wp][lp];
      a1 += red[j][1][wp][lp];
      a2 += red[j][2][wp][lp];
    }
    float4 tn;
    tn.x = (float)((double)x.x + (double)a0);
    tn.y = (float)((double)x.y + (double)a1);
    tn.z = (float)((double)x.z + (double)a2);
    tn.w = 0.f;
    dev::point_terms<float4>(to, tn, yt, Yhat4, m, contrib, dT2, gt2);
    T4[m] = tn;
  }
  block_sum3(contrib, dT2, gt2, sh3, NW);
  if (threadIdx.x == 0) {
    sums[(size_t)bx * 3] = contrib;
    sums[(size_t)bx * 3 + 1] = dT2;
    sums[(size_t)bx * 3 + 2] = gt2;
    __threadfence();
    last = atomicAdd(&st->ticket_e, 1u) == (unsigned)gx - 1;
  }
  __syncthreads();
  if (last) {
    __threadfence();
    double a0 = 0, a1 = 0, a2 = 0;
    for (int i = threadIdx.x; i < gx; i += kThreadsBatch) {
      a0 += __ldcg(sums + (size_t)i * 3);
      a1 += __ldcg(sums + (size_t)i * 3 + 1);
      a2 += __ldcg(sums + (size_t)i * 3 + 2);
    }
    block_sum3(a0, a1, a2, sh3, NW);
    if (threadIdx.x == 0) {
      dev::finish_iteration(st, a0, a1, a2, M);
      st->ticket_e = 0;
    }
  }
  return last;
}

// Pass A (B) of one tile with the fewest points per thread that cover the
// points left in it: a partial last tile runs with 2, 4, 6 (or, with wider
// tiles, 8 and 12) per thread.
__device__ __forceinline__ void passA_tile(const BatchPair& P, int bx, int by) {
  using namespace dev;
  const EstepPlan& e = P.ep;
  const int rem = P.N - bx * kTileColsA;
#define FCPD_PASS_A_PART(C)                                                                                  \
  if constexpr (kColsA32 > C) {                                                                              \
    if (rem <= kThreadsA * C) {                                                                              \
      passA_f32_body<C>(P.T4, P.M, e.a_rows_per_chunk, P.Y4, P.N, P.partA, P.st, 1, bx, by, e.a_col_tiles,   \
                        e.a_row_chunks);                                                                     \
      return;                                                                                                \
    }                                                                                                        \
  }
  FCPD_PASS_A_PART(2)
  FCPD_PASS_A_PART(4)
  FCPD_PASS_A_PART(6)
  FCPD_PASS_A_PART(8)
  FCPD_PASS_A_PART(12)
#undef FCPD_PASS_A_PART
  passA_f32_body(P.T4, P.M, e.a_rows_per_chunk, P.Y4, P.N, P.partA, P.st, 1, bx, by, e.a_col_tiles, e.a_row_chunks);
}

// The row list is cleared in phase P: rows of tiles finished during this
// phase are listed while other tiles still run, so pass B leaves it alone.
__device__ __forceinline__ void passB_tile(const BatchPair& P, int bx, int by) {
  using namespace dev;
  const EstepPlan& e = P.ep;
  const int rem = P.M - bx * kTileRowsB;
  if (rem <= kThreadsB * 2) {
    passB_f32_body<2>(P.T4, P.M, P.Yb, P.N, e.b_cols_per_chunk, P.partB, P.st, 1, bx, by, e.b_row_tiles,
                      e.b_col_chunks, 0);
    return;
  }
  if constexpr (kRowsB32 > 4) {
    if (rem <= kThreadsB * 4) {
      passB_f32_body<4>(P.T4, P.M, P.Yb, P.N, e.b_cols_per_chunk, P.partB, P.st, 1, bx, by, e.b_row_tiles,
                        e.b_col_chunks, 0);
      return;
    }
  }
  if constexpr (kRowsB32 > 6) {
    if (rem <= kThreadsB * 6) {
      passB_f32_body<6>(P.T4, P.M, P.Yb, P.N, e.b_cols_per_chunk, P.partB, P.st, 1, bx, by, e.b_row_tiles,
                        e.b_col_chunks, 0);
      return;
    }
  }
  passB_f32_body(P.T4, P.M, P.Yb, P.N, e.b_cols_per_chunk, P.partB, P.st, 1, bx, by, e.b_row_tiles, e.b_col_chunks,
                 0);
}

// Completion ticket of a tile of n work items: true in the block that
// finished the tile's last item (after which the tile's results written by
// the other blocks are visible to it).  Called by every thread of the block.
__device__ __forceinline__ bool tile_done(unsigned int* ticket, unsigned int n) {
  __shared__ int s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const bool last = atomicAdd(ticket, 1u) == n - 1;
    if (last) *ticket = 0;         // every item has arrived: rewind for the next iteration
    s_last = last;
  }
  __syncthreads();
  const bool last = s_last != 0;
  if (last) __threadfence();
  return last;
}

// One work item of phase ph for pair P: block coordinates (bx, by) of the
// per-pair kernel it stands for.
__device__ void run_item(int ph, const BatchPair& P, int bx, int by) {
  using namespace dev;
  const EstepPlan& e = P.ep;
  const MstepPlan& m = P.mp;
  unsigned int* tA = P.tix;
  unsigned int* tB = tA + e.a_col_tiles;
  unsigned int* tP = tB + e.b_row_tiles;
  unsigned int* tE = tP + 1;
  switch (ph) {
    case PH_A: {
      passA_tile(P, bx, by);
      if (!tile_done(tA + bx, (unsigned)e.a_row_chunks)) break;
      const int u1 = min((bx + 1) * (kTileColsA / kRedCols), (int)e.redA_blocks);
      for (int u = bx * (kTileColsA / kRedCols); u < u1; ++u) {
        const bool pair_done = reduceA_body<float>(P.partA, e.a_row_chunks, P.M, P.Y4, P.N, P.Yb, nullptr, P.sums,
                                                   P.flags + P.M, P.st, 1, u, 0, (int)e.redA_blocks, 1);
        __syncthreads();
        if (pair_done) {
          __threadfence();
          fixA_f32_body(P.T4, P.M, P.Y4, P.N, P.Yb, nullptr, P.flags + P.M, P.st, 1, 0, 0, 1, 1);
          phase_done(P, PH_A);
        }
      }
      break;
    }
    case PH_B: {
      passB_tile(P, bx, by);
      if (!tile_done(tB + bx, (unsigned)e.b_col_chunks)) break;
      const int u1 = min((bx + 1) * (kTileRowsB / kRedRows), (int)e.redB_blocks);
      for (int u = bx * (kTileRowsB / kRedRows); u < u1; ++u) {
        const bool pair_done = reduceB_body<float>(P.partB, e.b_col_chunks, P.M, P.X4, P.Yt4, P.R4, nullptr, P.sums,
                                                   P.flags, P.st, 1, u, 0, (int)e.redB_blocks, 1);
        __syncthreads();
        if (pair_done) {
          __threadfence();
          fixB_f32_body(P.T4, P.M, P.Yb, P.N, P.X4, P.Yt4, P.R4, nullptr, P.flags, P.st, 1, 0, 0, 1, 1);
          phase_done(P, PH_B);
        }
      }
      break;
    }
    case PH_P: {
      if (P.narrow && P.half_basis)
        proj_narrow_body(static_cast<const __half*>(P.U), m.ldU, P.M, P.K, P.R4, m.p_rows_per_chunk, P.partP, m.ldU,
                         P.st, by);
      else if (P.narrow)
        proj_narrow_body(static_cast<const float*>(P.U), m.ldU, P.M, P.K, P.R4, m.p_rows_per_chunk, P.partP, m.ldU,
                         P.st, by);
      else if (P.half_basis)
        colsum_body<float, __half, kThreadsBatch>(static_cast<const __half*>(P.U), m.ldU, P.M, P.K, P.R4,
                                                  m.p_rows_per_chunk, P.partP, m.ldU, P.st, 1, 1, bx, by,
                                                  m.p_col_tiles, m.p_row_chunks);
      else
        colsum_body<float, float, kThreadsBatch>(static_cast<const float*>(P.U), m.ldU, P.M, P.K, P.R4,
                                                 m.p_rows_per_chunk, P.partP, m.ldU, P.st, 1, 1, bx, by,
                                                 m.p_col_tiles, m.p_row_chunks);
      if (!tile_done(tP, (unsigned)(m.p_col_tiles * m.p_row_chunks))) break;
      const int nu = (P.K + kMRedCols - 1) / kMRedCols;
      for (int u = 0; u < nu; ++u) {
        diag_update_body<float>(P.partP, m.p_row_chunks, m.ldU, P.K, P.lam, P.B4, P.C4, P.st, 1, u, 0, nu, 1);
        __syncthreads();
      }
      phase_done(P, PH_P);
      break;
    }
    case PH_E: {
      if (P.narrow) {
        const bool last =
            P.half_basis
                ? expand_narrow_body(static_cast<const __half*>(P.Ut), m.ldM, P.K, P.M, P.B4, P.X4, P.Yt4, P.T4,
                                     P.Yhat4, P.sums, P.st, bx, m.e_col_tiles)
                : expand_narrow_body(static_cast<const float*>(P.Ut), m.ldM, P.K, P.M, P.B4, P.X4, P.Yt4, P.T4,
                                     P.Yhat4, P.sums, P.st, bx, m.e_col_tiles);
        if (last) phase_done(P, PH_E);
        break;
      }
      if (P.half_basis)
        colsum_body<float, __half, kThreadsBatch>(static_cast<const __half*>(P.Ut), m.ldM, P.K, P.M, P.B4,
                                                  m.e_rows_per_chunk, P.partP, m.ldM, P.st, 1, 0, bx, by,
                                                  m.e_col_tiles, m.e_row_chunks);
      else
        colsum_body<float, float, kThreadsBatch>(static_cast<const float*>(P.Ut), m.ldM, P.K, P.M, P.B4,
                                                 m.e_rows_per_chunk, P.partP, m.ldM, P.st, 1, 0, bx, by,
                                                 m.e_col_tiles, m.e_row_chunks);
      if (!tile_done(tE + bx, (unsigned)m.e_row_chunks)) break;
      const int u1 = min((bx + 1) * (kTileColsE / kMRedCols), m.e_blocks);
      for (int u = bx * (kTileColsE / kMRedCols); u < u1; ++u) {
        const bool last = expand_finish_body<float, true>(P.partP, m.e_row_chunks, m.ldM, P.M, P.X4, P.Yt4, P.T4,
                                                          P.Yhat4, P.sums, P.st, 1, u, 0, m.e_blocks, 1);
        __syncthreads();
        if (last) phase_done(P, PH_E);
      }
      break;
    }
  }
}

__global__ void __launch_bounds__(kThreadsBatch)
batch_iterations(const BatchPair* __restrict__ pairs, const BatchItem* __restrict__ items,
                 const int* __restrict__ phase_off, BatchCtl* __restrict__ ctl, int n_iter,
                 unsigned long long limit_ns, int barrier_extra) {
  __shared__ unsigned long long s_idx;
  __shared__ int s_ok;
  if (blockIdx.x == 0 && threadIdx.x == 0) ctl->t_start = global_ns();
  const int n_items = phase_off[kPhases];
  const unsigned long long total = (unsigned long long)n_iter * (unsigned long long)n_items;
  unsigned long long busy[kPhases] = {}, waited[kPhases] = {};
  for (;;) {
    if (threadIdx.x == 0) s_idx = *(volatile int*)&ctl->status != 0 ? total : atomicAdd(&ctl->next, 1ull);
    __syncthreads();
    const unsigned long long idx = s_idx;
    if (idx >= total) break;
    const int it = (int)(idx / (unsigned long long)n_items);
    const int j = (int)(idx % (unsigned long long)n_items);
    int ph = 0;
    while (ph + 1 < kPhases && j >= phase_off[ph + 1]) ++ph;
    const BatchItem itm = items[j];
    const BatchPair& P = pairs[itm.pair];
    // the pair's previous phase: the expansion of the previous iteration
    // before pass A (none in the launch's first iteration), else the phase
    // before in this iteration
    if (threadIdx.x == 0) {
      const unsigned long long t0 = global_ns();
      s_ok = 1;
      if (ph != PH_A || it > 0) {
        const int need_ph = ph == PH_A ? PH_E : ph - 1;
        const unsigned int need = (unsigned int)(ph == PH_A ? it : it + 1) + (unsigned int)barrier_extra;
        s_ok = wait_phase(P, need_ph, need, ctl, limit_ns) ? 1 : 0;
      }
      __threadfence();
      waited[ph] += global_ns() - t0;
    }
    __syncthreads();
    if (!s_ok) break;
    const unsigned long long t1 = threadIdx.x == 0 ? global_ns() : 0ull;
    run_item(ph, P, itm.bx, itm.by);
    __syncthreads();
    if (threadIdx.x == 0) busy[ph] += global_ns() - t1;
  }
  if (threadIdx.x == 0) {
    for (int ph = 0; ph < kPhases; ++ph) {
      if (busy[ph]) atomicAdd(&ctl->busy_ns[ph], busy[ph]);
      if (waited[ph]) atomicAdd(&ctl->wait_ns[ph], waited[ph]);
    }
    atomicMax(&ctl->t_end, global_ns());
  }
}

__global__ void batch_begin(const BatchPair* pairs, int n_pairs, int n_iter) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_pairs) pairs[i].st->iter_target = pairs[i].st->iter + n_iter;
}

__global__ void batch_states(const BatchPair* pairs, int n_pairs, DevState* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_pairs) out[i] = *pairs[i].st;
}

}  // namespace

int batch_resident_blocks(int sms) {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batch_iterations, kThreadsBatch, 0) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return occ * sms;
}

// Work-item sizes.  Target: about `e_items_per_block` E-step items per
// resident block over the whole batch (largest items first, so the queue
// balances), each item a full 1024-point tile by a run of the other
// dimension; projection items of about `proj_kbytes` KB of the basis, other
// M-step items of about 256 KB.  cpd_batch_autotune picks the two numbers by
// timing.
void plan_batch(BatchPair* P, int n_pairs, int resident, int e_items_per_block, int proj_kbytes) {
  double total = 0.0;
  for (int i = 0; i < n_pairs; ++i) total += (double)P[i].M * P[i].N;
  const int64_t tileA = (int64_t)dev::kThreadsA * dev::kColsA32;
  const int64_t tileB = (int64_t)dev::kThreadsB * dev::kRowsB32;
  const double per_item = std::max(total / ((double)std::max(e_items_per_block, 1) * std::max(resident, 1)),
                                    (double)tileA * dev::kTileA);
  for (int i = 0; i < n_pairs; ++i) {
    BatchPair& p = P[i];
    const int64_t M = p.M, N = p.N, K = p.K;
    EstepPlan e{};
    e.a_col_tiles = (int)cdiv(N, tileA);
    int64_t run = std::max<int64_t>(32, (int64_t)(per_item / (double)tileA));
    e.a_row_chunks = (int)cdiv(M, run);
    e.a_rows_per_chunk = (int)cdiv(M, e.a_row_chunks);
    e.b_row_tiles = (int)cdiv(M, tileB);
    run = std::max<int64_t>(32, (int64_t)(per_item / (double)tileB));
    e.b_col_chunks = (int)cdiv(N, run);
    e.b_cols_per_chunk = (int)cdiv(N, e.b_col_chunks);
    e.partA_elems = (int64_t)e.a_row_chunks * N;
    e.partB_elems = (int64_t)5 * e.b_col_chunks * M;
    e.redA_blocks = cdiv(N, dev::kRedCols);
    e.redB_blocks = cdiv(M, dev::kRedRows);
    e.sums_elems = std::max(e.redA_blocks, e.redB_blocks);
    e.flags_elems = M + N;
    p.ep = e;

    MstepPlan m{};
    m.ldU = cdiv(K, 8) * 8;              // as plan_mstep lays out the FP32 basis
    m.ldM = cdiv(M, 8) * 8;
    p.narrow = K <= kNarrowMaxK ? 1 : 0;
    const int64_t colsC = (int64_t)kThreadsBatch * 8;     // columns of one colsum tile
    if (p.narrow) {
      m.p_col_tiles = 1;
      const int64_t rows = std::max<int64_t>(64, ((int64_t)proj_kbytes * 1024) / (m.ldU * 4));
      m.p_row_chunks = (int)cdiv(M, rows);
    } else {
      m.p_col_tiles = (int)cdiv(m.ldU, colsC);
      const int64_t rows = std::max<int64_t>(32, (256 * 1024) / (std::min(m.ldU, colsC) * 4));
      m.p_row_chunks = (int)cdiv(M, rows);
    }
    m.p_rows_per_chunk = (int)cdiv(M, m.p_row_chunks);
    m.e_col_tiles = (int)cdiv(p.narrow ? M : m.ldM, p.narrow ? (int64_t)kNarrowTileE : colsC);
    if (p.narrow) {
      m.e_row_chunks = 1;                // the fused expansion takes all K rows per tile
      m.e_rows_per_chunk = (int)K;
    } else {
      const int64_t erows = std::max<int64_t>(32, (256 * 1024) / (std::min(m.ldM, colsC) * 4));
      m.e_row_chunks = (int)cdiv(K, erows);
      m.e_rows_per_chunk = (int)cdiv(K, m.e_row_chunks);
    }
    m.part_elems = std::max((int64_t)m.p_row_chunks * 3 * m.ldU, (int64_t)m.e_row_chunks * 3 * m.ldM);
    m.e_blocks = (int)cdiv(M, dev::kMRedCols);
    m.sums_elems = (int64_t)m.e_blocks * 3;
    p.mp = m;
  }
}

void batch_items(const BatchPair* pairs_host, int n_pairs, std::vector<BatchItem>& items, std::vector<int>& phase_off) {
  // pairs in decreasing work order within every phase (largest items first)
  std::vector<int> order(n_pairs);
  for (int i = 0; i < n_pairs; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return (double)pairs_host[a].M * pairs_host[a].N > (double)pairs_host[b].M * pairs_host[b].N;
  });
  items.clear();
  phase_off.assign(kPhases + 1, 0);
  for (int ph = 0; ph < kPhases; ++ph) {
    phase_off[ph] = (int)items.size();
    for (int i : order) {
      const BatchPair& P = pairs_host[i];
      int gx = 1, gy = 1;
      switch (ph) {
        case PH_A: gx = P.ep.a_col_tiles; gy = P.ep.a_row_chunks; break;
        case PH_B: gx = P.ep.b_row_tiles; gy = P.ep.b_col_chunks; break;
        case PH_P: gx = P.mp.p_col_tiles; gy = P.mp.p_row_chunks; break;
        case PH_E: gx = P.mp.e_col_tiles; gy = P.mp.e_row_chunks; break;
      }
      for (int by = 0; by < gy; ++by)
        for (int bx = 0; bx < gx; ++bx) items.push_back(BatchItem{i, bx, by});
    }
  }
  phase_off[kPhases] = (int)items.size();
}

int batch_tickets(const BatchPair& p) { return p.ep.a_col_tiles + p.ep.b_row_tiles + 1 + p.mp.e_col_tiles; }

int batch_phases() { return kPhases; }

cudaError_t launch_batch(const BatchPair* pairs_dev, int n_pairs, const BatchItem* items, const int* phase_off,
                         BatchCtl* ctl, unsigned int* done, int grid, int n_iter, double wait_limit_s, int barrier_extra,
                         cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(ctl, 0, sizeof(BatchCtl), s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(done, 0, sizeof(unsigned int) * kPhases * (size_t)n_pairs, s);
  if (e != cudaSuccess) return e;
  batch_begin<<<(n_pairs + 255) / 256, 256, 0, s>>>(pairs_dev, n_pairs, n_iter);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kThreadsBatch);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const unsigned long long limit_ns = (unsigned long long)(wait_limit_s * 1e9);
  return cudaLaunchKernelEx(&cfg, batch_iterations, pairs_dev, items, phase_off, ctl, n_iter, limit_ns,
                            barrier_extra);
}

void launch_batch_states(const BatchPair* pairs_dev, int n_pairs, DevState* out, cudaStream_t s) {
  batch_states<<<(n_pairs + 127) / 128, 128, 0, s>>>(pairs_dev, n_pairs, out);
}

}  // namespace fcpd
