// Batched registrations: many independent (X_i, Y_i) pairs of uneven sizes
// run their EM iterations in ONE persistent cooperative kernel launch.
//
// Every iteration of every pair is the same sequence of phases as the
// per-pair path (estep_dev.cuh / mstep_dev.cuh): pass A, its reduction, the
// FP32 log-domain fix-up of columns, pass B, its reduction, the row fix-up,
// projection U^T R, diagonal update, expansion with U^T, and the expansion's
// reduction with Eq. 18.  For each phase the host lists the work items of all
// pairs -- (pair, block coordinates), largest pairs first -- and the resident
// blocks take items from an atomic counter, so small and large pairs share
// the GPU without per-pair launches.  Phases are separated by a grid-wide
// barrier.  The barrier's wait is bounded in wall time: if it does not
// complete within the limit the kernel records CPD_ETIMEOUT in the control
// block and every block returns (no GPU hang); the host reports the status.
//
// Buffers such as T, Yb and the partial sums are written in one phase and
// read in a later one of the same launch, so no argument of the device bodies
// is __restrict__ here (only U and U^T, constant for the launch, go through
// the read-only path).  The E-step bodies are compiled with 4 scene points
// (pass A) and 4 model points (pass B) per thread: tiles of 1024 points keep
// the padding of small pairs (a few hundred points) low, where the per-pair
// launches use 16 and 8 for scenes of tens of thousands of points.
#define FCPD_RESTRICT
#define FCPD_EA_COLS 4
#define FCPD_EB_ROWS 4
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

enum Phase { PH_PASSA = 0, PH_REDA, PH_FIXA, PH_PASSB, PH_REDB, PH_FIXB, PH_PROJ, PH_DIAG, PH_EXPD, PH_FIN, kPhases };

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

// Grid-wide barrier over all co-resident blocks.  Returns false (and leaves
// CPD_ETIMEOUT in ctl->status) if another block failed or the wait exceeded
// limit_ns of wall time.
__device__ bool grid_barrier(BatchCtl* ctl, unsigned int nblocks, unsigned long long limit_ns) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned int* genp = &ctl->barrier_gen;
    const unsigned int gen = *genp;
    __threadfence();
    const unsigned int arrived = atomicAdd(&ctl->barrier_count, 1u);
    if (arrived == nblocks - 1) {
      ctl->barrier_count = 0;
      __threadfence();
      atomicAdd(&ctl->barrier_gen, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      while (*genp == gen) {
        if (*(volatile int*)&ctl->status != 0) { ok = 0; break; }
        __nanosleep(128);
        if (global_ns() - t0 > limit_ns) {
          atomicExch(&ctl->status, (int)CPD_ETIMEOUT);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

// Projection A = U^T R for a basis of at most 128 columns: 16 groups of 8
// columns x 16 row lanes, the lanes combined in a fixed order through shared
// memory.  Writes the same chunk partials as colsum_body (row chunk `by`).
__device__ __forceinline__ void proj_narrow_body(const float* U, int64_t ldU, int M, int K, const float4* R4,
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
      const float4* row = reinterpret_cast<const float4*>(U + (size_t)m * ldU + c0);
      const float4 u0 = __ldg(row), u1 = __ldg(row + 1);
      const float4 r = R4[m];
      const float u[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
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

// One work item.  For the reduction phases (REDA, REDB, DIAG, FIN) an item is
// `by` consecutive reduction blocks starting at `bx`.
__device__ void run_item(int ph, const BatchPair& P, int bx, int by) {
  using namespace dev;
  const EstepPlan& e = P.ep;
  const MstepPlan& m = P.mp;
  switch (ph) {
    case PH_PASSA:
      passA_f32_body(P.T4, P.M, e.a_rows_per_chunk, P.Y4, P.N, P.partA, P.st, 1, bx, by, e.a_col_tiles, e.a_row_chunks);
      break;
    case PH_REDA:
      for (int u = bx; u < bx + by; ++u) {
        reduceA_body<float>(P.partA, e.a_row_chunks, P.M, P.Y4, P.N, P.Yb, nullptr, P.sums, P.flags + P.M, P.st, 1, u,
                            0, (int)e.redA_blocks, 1);
        __syncthreads();
      }
      break;
    case PH_FIXA:
      fixA_f32_body(P.T4, P.M, P.Y4, P.N, P.Yb, nullptr, P.flags + P.M, P.st, 1, bx, 0, kFixItems, 1);
      break;
    case PH_PASSB:
      passB_f32_body(P.T4, P.M, P.Yb, P.N, e.b_cols_per_chunk, P.partB, P.st, 1, bx, by, e.b_row_tiles, e.b_col_chunks);
      break;
    case PH_REDB:
      for (int u = bx; u < bx + by; ++u) {
        reduceB_body<float>(P.partB, e.b_col_chunks, P.M, P.X4, P.Yt4, P.R4, nullptr, P.sums, P.flags, P.st, 1, u, 0,
                            (int)e.redB_blocks, 1);
        __syncthreads();
      }
      break;
    case PH_FIXB:
      fixB_f32_body(P.T4, P.M, P.Yb, P.N, P.X4, P.Yt4, P.R4, nullptr, P.flags, P.st, 1, bx, 0, kFixItems, 1);
      break;
    case PH_PROJ:
      if (P.narrow)
        proj_narrow_body(P.U, m.ldU, P.M, P.K, P.R4, m.p_rows_per_chunk, P.partP, m.ldU, P.st, by);
      else
        colsum_body<float, kThreadsBatch>(P.U, m.ldU, P.M, P.K, P.R4, m.p_rows_per_chunk, P.partP, m.ldU, P.st, 1, 1,
                                          bx, by, m.p_col_tiles, m.p_row_chunks);
      break;
    case PH_DIAG:
      for (int u = bx; u < bx + by; ++u) {
        diag_update_body<float>(P.partP, m.p_row_chunks, m.ldU, P.K, P.lam, P.B4, P.C4, P.st, 1, u, 0,
                                (P.K + kMRedCols - 1) / kMRedCols, 1);
        __syncthreads();
      }
      break;
    case PH_EXPD:
      colsum_body<float, kThreadsBatch>(P.Ut, m.ldM, P.K, P.M, P.B4, m.e_rows_per_chunk, P.partP, m.ldM, P.st, 1, 0, bx,
                                        by, m.e_col_tiles, m.e_row_chunks);
      break;
    case PH_FIN:
      for (int u = bx; u < bx + by; ++u) {
        expand_finish_body<float, true>(P.partP, m.e_row_chunks, m.ldM, P.M, P.X4, P.Yt4, P.T4, P.Yhat4, P.sums, P.st,
                                        1, u, 0, m.e_blocks, 1);
        __syncthreads();
      }
      break;
  }
}

__global__ void __launch_bounds__(kThreadsBatch)
batch_iterations(const BatchPair* __restrict__ pairs, const BatchItem* __restrict__ items,
                 const int* __restrict__ phase_off, BatchCtl* __restrict__ ctl, int n_iter,
                 unsigned long long limit_ns, int barrier_extra) {
  __shared__ int s_idx;
  for (int it = 0; it < n_iter; ++it) {
    for (int ph = 0; ph < kPhases; ++ph) {
      const int lo = phase_off[ph], hi = phase_off[ph + 1];
      for (;;) {
        if (threadIdx.x == 0) s_idx = lo + (int)atomicAdd(&ctl->next_item[ph], 1u);
        __syncthreads();
        const int idx = s_idx;
        if (idx >= hi) break;
        const BatchItem itm = items[idx];
        run_item(ph, pairs[itm.pair], itm.bx, itm.by);
        __syncthreads();
      }
      if (!grid_barrier(ctl, gridDim.x + (unsigned int)barrier_extra, limit_ns)) return;
      // every block has left phase ph: its item counter can be rewound
      if (blockIdx.x == 0 && threadIdx.x == 0) ctl->next_item[ph] = 0;
    }
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

// Work-item sizes.  Target: about four E-step items per resident block over
// the whole batch (largest items first, so the queue balances), each item a
// full 1024-point tile by a run of the other dimension; M-step items of about
// 128-256 KB of the basis.
void plan_batch(BatchPair* P, int n_pairs, int resident) {
  double total = 0.0;
  for (int i = 0; i < n_pairs; ++i) total += (double)P[i].M * P[i].N;
  const int64_t tileA = (int64_t)dev::kThreadsA * dev::kColsA32;
  const int64_t tileB = (int64_t)dev::kThreadsB * dev::kRowsB32;
  const double per_item = std::max(total / (4.0 * std::max(resident, 1)), (double)tileA * dev::kTileA);
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
      const int64_t rows = std::max<int64_t>(64, (128 * 1024) / (m.ldU * 4));
      m.p_row_chunks = (int)cdiv(M, rows);
    } else {
      m.p_col_tiles = (int)cdiv(m.ldU, colsC);
      const int64_t rows = std::max<int64_t>(32, (256 * 1024) / (std::min(m.ldU, colsC) * 4));
      m.p_row_chunks = (int)cdiv(M, rows);
    }
    m.p_rows_per_chunk = (int)cdiv(M, m.p_row_chunks);
    m.e_col_tiles = (int)cdiv(m.ldM, colsC);
    const int64_t erows = std::max<int64_t>(32, (256 * 1024) / (std::min(m.ldM, colsC) * 4));
    m.e_row_chunks = (int)cdiv(K, erows);
    m.e_rows_per_chunk = (int)cdiv(K, m.e_row_chunks);
    m.part_elems = std::max((int64_t)m.p_row_chunks * 3 * m.ldU, (int64_t)m.e_row_chunks * 3 * m.ldM);
    m.e_blocks = (int)cdiv(M, dev::kMRedCols);
    m.sums_elems = (int64_t)m.e_blocks * 3;
    p.mp = m;
  }
}

void batch_items(const BatchPair* pairs_host, int n_pairs, int resident, std::vector<BatchItem>& items,
                 std::vector<int>& phase_off) {
  // pairs in decreasing work order within every phase (largest items first)
  std::vector<int> order(n_pairs);
  for (int i = 0; i < n_pairs; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return (double)pairs_host[a].M * pairs_host[a].N > (double)pairs_host[b].M * pairs_host[b].N;
  });
  auto units = [&](const BatchPair& P, int ph) -> int64_t {
    switch (ph) {
      case PH_REDA: return P.ep.redA_blocks;
      case PH_REDB: return P.ep.redB_blocks;
      case PH_DIAG: return cdiv(P.K, dev::kMRedCols);
      case PH_FIN: return P.mp.e_blocks;
      default: return 0;
    }
  };
  items.clear();
  phase_off.assign(kPhases + 1, 0);
  for (int ph = 0; ph < kPhases; ++ph) {
    phase_off[ph] = (int)items.size();
    const bool grouped = ph == PH_REDA || ph == PH_REDB || ph == PH_DIAG || ph == PH_FIN;
    int64_t group = 1;
    if (grouped) {
      // about two items per resident block over the batch
      int64_t tot = 0;
      for (int i = 0; i < n_pairs; ++i) tot += units(pairs_host[i], ph);
      group = std::max<int64_t>(1, cdiv(tot, 2 * (int64_t)std::max(resident, 1)));
    }
    for (int i : order) {
      const BatchPair& P = pairs_host[i];
      if (grouped) {
        const int64_t u = units(P, ph);
        for (int64_t b = 0; b < u; b += group)
          items.push_back(BatchItem{i, (int)b, (int)std::min(group, u - b)});
        continue;
      }
      int gx = 1, gy = 1;
      switch (ph) {
        case PH_PASSA: gx = P.ep.a_col_tiles; gy = P.ep.a_row_chunks; break;
        case PH_FIXA: gx = kFixItems; break;
        case PH_PASSB: gx = P.ep.b_row_tiles; gy = P.ep.b_col_chunks; break;
        case PH_FIXB: gx = kFixItems; break;
        case PH_PROJ: gx = P.mp.p_col_tiles; gy = P.mp.p_row_chunks; break;
        case PH_EXPD: gx = P.mp.e_col_tiles; gy = P.mp.e_row_chunks; break;
      }
      for (int by = 0; by < gy; ++by)
        for (int bx = 0; bx < gx; ++bx) items.push_back(BatchItem{i, bx, by});
    }
  }
  phase_off[kPhases] = (int)items.size();
}

cudaError_t launch_batch(const BatchPair* pairs_dev, int n_pairs, const BatchItem* items, const int* phase_off,
                         BatchCtl* ctl, int grid, int n_iter, double wait_limit_s, int barrier_extra,
                         cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(ctl, 0, sizeof(BatchCtl), s);
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
