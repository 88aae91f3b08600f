// C ABI of the GB300 fast-CPD EM loop (declared in include/fcpd.h).
//
// Host side only: argument validation, device buffers of a context, staging of
// host arrays, the one-time eigendecomposition (cuSOLVER, FP64), and the
// replay of captured per-iteration CUDA graphs.  Every arithmetic step of the
// EM loop runs in the kernels of estep.cu / mstep.cu / setup.cu.
#include <cusolverDn.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"

using namespace fcpd;

namespace {

thread_local std::string g_err;

cpd_status fail(cpd_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

bool fault_enabled(const char* what) {
  const char* f = std::getenv("CPD_FAULT");
  return f && std::strcmp(f, what) == 0;
}

#define CUDA_TRY(call)                                                                                   \
  do {                                                                                                   \
    cudaError_t e_ = (call);                                                                             \
    if (e_ != cudaSuccess) {                                                                             \
      return fail(e_ == cudaErrorMemoryAllocation ? CPD_ENOMEM : CPD_ECUDA,                              \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                                   \
    }                                                                                                    \
  } while (0)

#define STATUS_TRY(call)              \
  do {                                \
    cpd_status s_ = (call);           \
    if (s_ != CPD_OK) return s_;      \
  } while (0)

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}


struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (dev >= 0 && dev != prev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

// Device buffer that grows on demand.
struct Buf {
  void* p = nullptr;
  size_t bytes = 0;
  cpd_status ensure(size_t want) {
    if (want <= bytes) return CPD_OK;
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
    cudaError_t e = cudaMalloc(&p, want);
    if (e != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      return fail(CPD_ENOMEM, std::string("cudaMalloc(") + std::to_string(want) + "): " + cudaGetErrorString(e));
    }
    bytes = want;
    return CPD_OK;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  template <typename T> T* as() const { return static_cast<T*>(p); }
};

constexpr int32_t kPruneFlags = CPD_FLAG_PRUNE | CPD_FLAG_PRUNE_ALWAYS | CPD_FLAG_PRUNE_NOSKIP;

cpd_status validate_params(const cpd_params* p) {
  if (!p) return fail(CPD_EINVAL, "params is NULL");
  if (p->D != 3) return fail(CPD_EINVAL, "only D = 3 is implemented");
  if (p->precision != CPD_FP64 && p->precision != CPD_FP32 && p->precision != CPD_MIXED)
    return fail(CPD_EINVAL, "unknown precision");
  if (!(p->w >= 0.0 && p->w < 1.0)) return fail(CPD_EINVAL, "w must satisfy 0 <= w < 1");
  if (!(p->beta > 0.0) || !std::isfinite(p->beta)) return fail(CPD_EINVAL, "beta must be > 0");
  if (!(p->lambda > 0.0) || !std::isfinite(p->lambda)) return fail(CPD_EINVAL, "lambda must be > 0");
  if (std::isnan(p->sigma2_init) || std::isinf(p->sigma2_init)) return fail(CPD_EINVAL, "sigma2_init not finite");
  if (p->K < 0) return fail(CPD_EINVAL, "K must be >= 0");
  if (p->max_iter < 0) return fail(CPD_EINVAL, "max_iter must be >= 0");
  if (p->flags & ~(CPD_FLAG_PRUNE | CPD_FLAG_PRUNE_ALWAYS | CPD_FLAG_PRUNE_NOSKIP | CPD_FLAG_SPECTRAL_TRIM |
                   CPD_FLAG_FULL_EIG))
    return fail(CPD_EINVAL, "unknown bits in flags");
  if ((p->flags & CPD_FLAG_SPECTRAL_TRIM) && p->precision == CPD_FP64)
    return fail(CPD_EINVAL, "the spectral trim bounds its error at FP32 rounding: not for CPD_FP64");
  if (!(p->tol >= 0.0) || !std::isfinite(p->tol)) return fail(CPD_EINVAL, "tol must be >= 0");
  return CPD_OK;
}

constexpr int64_t kMaxM = 46340;
// Subspace iteration for the top-K basis: residual |Phi u - theta u| of every
// kept Ritz pair below kTopkTol x the largest eigenvalue (rounding level of
// an FP64 product with Phi), at most kTopkMaxSteps Rayleigh-Ritz steps.
constexpr double kTopkTol = 1e-13;
constexpr int kTopkMaxSteps = 100;          // M*M doubles indexable by the 32-bit eigensolver API
constexpr int64_t kMaxN = 1LL << 30;

}  // namespace

void fcpd::set_last_error(const std::string& msg) { g_err = msg; }

struct cpd_ctx {
  cpd_params p{};
  int dev = 0;
  int sms = 0;
  bool fp64 = false;
  bool half_basis = false;       // CPD_MIXED: U, U^T stored in FP16
  size_t es = 4;                 // element size of the working precision
  size_t bes = 4;                // element size of the stored basis
  size_t v4 = 16;                // bytes of one 4-vector
  int64_t M = 0, K = 0, ldU = 0, N = 0;
  cudaStream_t stream = nullptr; // caller's stream
  cudaStream_t cap = nullptr;    // internal stream used only for graph capture
  EstepSide side{};              // captured side branch of each iteration's E-step
  cudaEvent_t piece_ev[kMaxPieces] = {};   // pass B piece i done: its projection may start (side stream)
  Buf X4, T4, U, Ut, lam, Yt4, R4, B4, C4, Yhat4, W4, hist;
  Buf st, st_aux;
  Buf Y4, Yb, partA, partB, partP, sums, flags, stage;
  Buf auxT4, auxR4, auxB4, auxC4;
  // spatial order (FP32 paths): model points sorted at setup, scenes at upload
  bool sorted_model = false;     // X4, T4, U rows ... are in Morton order
  bool scene_sorted = false;     // the current scene is in Morton order
  Buf permX, invX;               // sorted -> caller index, caller -> sorted index
  Buf sort_scratch, sort_tmp;
  float prune_r2 = 0.f;          // pruned passes below this squared FP32 cutoff radius
  EstepPlan ep{};
  MstepPlan mp{};
  MstepPlan mp_trim{};           // spectral trim: the M-step over the leading k_cap directions
  int64_t k_cap = 0;             // > 0: the trimmed M-step is captured beside the full one
  double trim_lam = -1.0;        // largest eigenvalue the trimmed M-step drops
  int eig_method = 0;            // 0: full eigensolver, 1: top-K subspace iteration
  int eig_steps = 0;             // Rayleigh-Ritz steps of the subspace iteration
  cudaGraphExec_t graph[2] = {nullptr, nullptr};   // 1 iteration, kBatch iterations
  cudaGraphExec_t loop_graph = nullptr;             // device-side loop until the target or a tolerance stop
  cudaGraphExec_t prof_graph = nullptr;             // n iterations with timing events
  int prof_iters = 0;
  std::vector<cudaEvent_t> prof_ev;                 // 9 per sampled iteration
  bool started = false;
  bool has_gt = false;
  double gt_tol = 0.0;
  static constexpr int kBatch = 8;

  ~cpd_ctx() {
    drop_graphs();
    for (Buf* b : {&X4, &T4, &U, &Ut, &lam, &Yt4, &R4, &B4, &C4, &Yhat4, &W4, &hist, &st, &st_aux, &Y4, &Yb,
                   &partA, &partB, &partP, &sums, &flags, &stage, &auxT4, &auxR4, &auxB4, &auxC4, &permX, &invX,
                   &sort_scratch, &sort_tmp})
      b->release();
    if (cap) cudaStreamDestroy(cap);
    if (side.s) cudaStreamDestroy(side.s);
    if (side.fork) cudaEventDestroy(side.fork);
    if (side.join) cudaEventDestroy(side.join);
    for (cudaEvent_t e : piece_ev)
      if (e) cudaEventDestroy(e);
  }
  void drop_graphs() {
    for (auto& g : graph)
      if (g) {
        cudaGraphExecDestroy(g);
        g = nullptr;
      }
    if (loop_graph) cudaGraphExecDestroy(loop_graph);
    loop_graph = nullptr;
    if (prof_graph) cudaGraphExecDestroy(prof_graph);
    prof_graph = nullptr;
    prof_iters = 0;
    for (cudaEvent_t e : prof_ev) cudaEventDestroy(e);
    prof_ev.clear();
  }
  DevState* dst() const { return st.as<DevState>(); }
};

namespace {

// Copies a caller point array (n x 3 of the context precision, host or device)
// into 4-vectors `dst` (4th lane |p|^2 if with_norm).
cpd_status upload_points(cpd_ctx* c, const void* src, int64_t n, void* dst, bool with_norm, Buf& stage,
                         bool fp64, cudaStream_t s) {
  const size_t es = fp64 ? 8 : 4;
  const void* dev = src;
  if (!is_device_ptr(src)) {
    STATUS_TRY(stage.ensure((size_t)n * 3 * es));
    CUDA_TRY(cudaMemcpyAsync(stage.p, src, (size_t)n * 3 * es, cudaMemcpyHostToDevice, s));
    dev = stage.p;
  }
  (void)c;
  if (fp64) launch_pack<double>((const double*)dev, n, (dvec4*)dst, with_norm, s);
  else launch_pack<float>((const float*)dev, n, (float4*)dst, with_norm, s);
  CUDA_TRY(cudaGetLastError());
  return CPD_OK;
}

// Writes 4-vectors `src` to a caller array (n x 3, host or device).  Host
// destinations synchronise `s` (unless `sync` is false: the caller then
// synchronises before it returns).
cpd_status download_points(const void* src, int64_t n, void* dst, Buf& stage, bool fp64, cudaStream_t s,
                           bool sync = true) {
  const size_t es = fp64 ? 8 : 4;
  const bool dev = is_device_ptr(dst);
  void* out = dst;
  if (!dev) {
    STATUS_TRY(stage.ensure((size_t)n * 3 * es));
    out = stage.p;
  }
  if (fp64) launch_unpack<double>((const dvec4*)src, n, (double*)out, s);
  else launch_unpack<float>((const float4*)src, n, (float*)out, s);
  CUDA_TRY(cudaGetLastError());
  if (!dev) {
    CUDA_TRY(cudaMemcpyAsync(dst, stage.p, (size_t)n * 3 * es, cudaMemcpyDeviceToHost, s));
    if (sync) CUDA_TRY(cudaStreamSynchronize(s));
  }
  return CPD_OK;
}

// Per-model-point arrays in the caller's order <-> the context's (sorted)
// order.  Without spatial order these are upload_points / download_points.
cpd_status upload_model(cpd_ctx* c, const void* src, void* dst4) {
  if (!c->sorted_model) return upload_points(c, src, c->M, dst4, false, c->stage, c->fp64, c->stream);
  const float* dev = static_cast<const float*>(src);
  if (!is_device_ptr(src)) {
    STATUS_TRY(c->stage.ensure((size_t)c->M * 3 * sizeof(float)));
    CUDA_TRY(cudaMemcpyAsync(c->stage.p, src, (size_t)c->M * 3 * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    dev = c->stage.as<float>();
  }
  launch_pack_gather<float>(dev, c->permX.as<int>(), c->M, static_cast<float4*>(dst4), false, c->stream);
  CUDA_TRY(cudaGetLastError());
  return CPD_OK;
}

cpd_status download_model(cpd_ctx* c, const void* src4, void* dst, bool sync = true) {
  if (!c->sorted_model) return download_points(src4, c->M, dst, c->stage, c->fp64, c->stream, sync);
  const bool dev = is_device_ptr(dst);
  float* out = static_cast<float*>(dst);
  if (!dev) {
    STATUS_TRY(c->stage.ensure((size_t)c->M * 3 * sizeof(float)));
    out = c->stage.as<float>();
  }
  launch_unpack_gather<float>(static_cast<const float4*>(src4), c->invX.as<int>(), c->M, out, c->stream);
  CUDA_TRY(cudaGetLastError());
  if (!dev) {
    CUDA_TRY(cudaMemcpyAsync(dst, out, (size_t)c->M * 3 * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    if (sync) CUDA_TRY(cudaStreamSynchronize(c->stream));
  }
  return CPD_OK;
}

// Sorts n float4 points in place (Morton order); perm (sorted -> original)
// may be null.
cpd_status sort_points(cpd_ctx* c, void* pts4, int64_t n, int* perm) {
  STATUS_TRY(c->sort_scratch.ensure((size_t)spatial_sort_scratch_bytes(n)));
  STATUS_TRY(c->sort_tmp.ensure((size_t)n * sizeof(float4)));
  CUDA_TRY(launch_spatial_sort(static_cast<const float4*>(pts4), n, c->sort_tmp.as<float4>(), perm,
                               c->sort_scratch.p, c->stream));
  CUDA_TRY(cudaMemcpyAsync(pts4, c->sort_tmp.p, (size_t)n * sizeof(float4), cudaMemcpyDeviceToDevice, c->stream));
  return CPD_OK;
}

// Pass B in row pieces beside the projection (see after_piece): FP32 with a
// wide FP32 basis, no spatial order and no spectral trim; 3 pieces from
// kSplitMinM model points (measured at M = N = 20000, full basis: 1291 EM
// it/s in one piece, 1334 in 2, 1352 in 3).  FCPD_SPLIT_B sets the number
// of pieces (1: off).
constexpr int kSplitPieces = 3;
constexpr int64_t kSplitMinM = 8192;
int pieces_wanted(int64_t M) {
  const char* v = std::getenv("FCPD_SPLIT_B");
  if (v && *v) return std::atoi(v);
  return M >= kSplitMinM ? kSplitPieces : 1;
}
void plan_pieces(cpd_ctx* c) {
  c->mp.n_pieces = 0;
  if (c->fp64 || c->half_basis || c->sorted_model || c->k_cap > 0) return;
  const int want = pieces_wanted(c->M);
  if (want < 2) return;
  int m0[kMaxPieces], rows[kMaxPieces];
  const int n = split_rows(c->M, want, m0, rows);
  if (n >= 2) plan_mstep_pieces(c->mp, c->M, c->sms, n, m0, rows);
}

// E-step layout control of the context for the current scene: pruning
// (spatially ordered points) and, in the mixed-precision mode, the
// tensor-core passes with their sigma2 floor from the current points.
void apply_prune(cpd_ctx* c) {
  int ctl = 0;
  if (c->sorted_model && c->scene_sorted) {
    ctl = kPruneAllowed;
    if (c->p.flags & CPD_FLAG_PRUNE_ALWAYS) ctl |= kPruneAlways;
    if (c->p.flags & CPD_FLAG_PRUNE_NOSKIP) ctl |= kPruneNoSkip;
  }
  if (c->half_basis) ctl |= kMmaAllowed;
  if (fault_enabled("bulk_wait")) ctl |= kBulkWaitFault;
  launch_state_prune(c->dst(), c->prune_r2, ctl, c->stream);
  if (c->k_cap > 0) launch_state_trim(c->dst(), c->trim_lam, c->stream);   // state_init switched it off
  if (c->half_basis) launch_mma_threshold(c->X4.as<float4>(), c->M, c->Y4.as<float4>(), c->N, c->dst(), c->stream);
}

// Spectral trim: the leading directions kept by the trimmed M-step.  With
// the variance floor s2f = kTrimFloor x the model points' variance per axis,
// every direction with l_k >= kTrimEps lambda s2f / (1 - kTrimEps) is kept
// (rounded up to 16 columns); the dropped ones then have s_k < kTrimEps in
// every iteration whose sigma2 >= s2f, and iterations further below run the
// full M-step (the device test uses the largest dropped eigenvalue).
constexpr double kTrimFloor = 1e-4;
cpd_status plan_trim(cpd_ctx* c) {
  std::vector<double> lam((size_t)c->K);
  std::vector<float4> x((size_t)c->M);
  CUDA_TRY(cudaMemcpyAsync(lam.data(), c->lam.p, lam.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaMemcpyAsync(x.data(), c->X4.p, x.size() * sizeof(float4), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  double mean[3] = {0, 0, 0}, var = 0;
  for (const float4& v : x) { mean[0] += v.x; mean[1] += v.y; mean[2] += v.z; }
  for (double& m : mean) m /= (double)c->M;
  for (const float4& v : x) {
    const double dx = v.x - mean[0], dy = v.y - mean[1], dz = v.z - mean[2];
    var += dx * dx + dy * dy + dz * dz;
  }
  var /= 3.0 * (double)c->M;
  const double thr = kTrimEps * c->p.lambda * kTrimFloor * var / (1.0 - kTrimEps);
  int64_t n = 0;
  while (n < c->K && lam[(size_t)n] >= thr) ++n;
  const int64_t kcap = std::max<int64_t>(16, (n + 15) / 16 * 16);
  if (kcap >= c->K) return CPD_OK;                 // nothing to drop
  c->k_cap = kcap;
  c->trim_lam = lam[(size_t)kcap];
  c->mp_trim = plan_mstep_trim(c->mp, c->M, kcap, c->fp64, c->sms, (int)c->bes);
  return CPD_OK;
}

// Up to kMaxScenesPerPass registrations of scenes against the context's
// model: fresh registrations (T = X, sigma2_0 from each scene) of n_iter
// iterations each; per-scene E-steps, the M-step products of all scenes in
// one pass over U and U^T (multi.cu), per-scene diagonal updates and Eq. 18.
struct ScratchSet {
  std::vector<Buf> b;
  explicit ScratchSet(size_t n) : b(n) {}
  ~ScratchSet() {
    for (Buf& x : b) x.release();
  }
};

// One group of S scenes.  FP32 contexts: the products of the group by the
// SIMT streaming kernel (multi.cu, S <= 8).  Mixed-precision contexts (FP16
// basis): the products on the tensor cores (umma.cu, S <= 32) and the
// mixed E-step (tensor-core distance passes while sigma2 is large).  One
// iteration of the group is captured once into a CUDA graph and replayed.
cpd_status shared_group(cpd_ctx* c, int S, const void* const* Y, const int64_t* N, int n_iter, void* const* T_out,
                        double* s2_out) {
  const int64_t M = c->M, K = c->K;
  const bool mixed = c->half_basis;
  MultiPlan mp{};
  UmmaPlan pp{}, pe{};
  int64_t part_elems = 0, sums_elems = 0;
  if (mixed) {
    pp = plan_umma(K, M, S, c->sms);
    pe = plan_umma(M, K, S, c->sms);
    part_elems = std::max((int64_t)S * pp.chunks * 3 * c->ldU, (int64_t)S * pe.chunks * 3 * c->mp.ldM);
    sums_elems = multi_sums_elems(M);
  } else {
    mp = plan_multi(M, K, c->ldU, c->mp.ldM, S, c->sms);
    part_elems = mp.part_elems;
    sums_elems = mp.sums_elems;
  }
  std::vector<EstepPlan> ep((size_t)S);
  std::vector<int64_t> yoff((size_t)S);
  int64_t pa = 0, pb = 0, sm = sums_elems, fl = 0, nmax = 0, ytot = 0;
  for (int i = 0; i < S; ++i) {
    ep[(size_t)i] = plan_estep(M, N[i], false, c->sms, false, mixed);
    pa = std::max(pa, ep[(size_t)i].partA_elems);
    pb = std::max(pb, ep[(size_t)i].partB_elems);
    sm = std::max(sm, ep[(size_t)i].sums_elems);
    fl = std::max(fl, ep[(size_t)i].flags_elems);
    nmax = std::max(nmax, N[i]);
    yoff[(size_t)i] = ytot;
    ytot += N[i];
  }
  enum { kY4, kYb, kPA, kPB, kPP, kSums, kFlags, kT4, kYt4, kR4, kB4, kC4, kSt, kStatus, kVp, kVe, kCount };
  ScratchSet sc(kCount);
  Buf* b = sc.b.data();
  STATUS_TRY(b[kY4].ensure((size_t)ytot * sizeof(float4)));
  STATUS_TRY(b[kYb].ensure((size_t)nmax * sizeof(float4)));
  STATUS_TRY(b[kPA].ensure((size_t)pa * sizeof(float)));
  STATUS_TRY(b[kPB].ensure((size_t)pb * sizeof(float)));
  STATUS_TRY(b[kPP].ensure((size_t)part_elems * sizeof(float)));
  STATUS_TRY(b[kSums].ensure((size_t)sm * sizeof(double)));
  STATUS_TRY(b[kFlags].ensure((size_t)fl * sizeof(int)));
  for (int k : {(int)kT4, (int)kYt4, (int)kR4}) STATUS_TRY(b[k].ensure((size_t)S * M * sizeof(float4)));
  for (int k : {(int)kB4, (int)kC4}) STATUS_TRY(b[k].ensure((size_t)S * K * sizeof(float4)));
  STATUS_TRY(b[kSt].ensure((size_t)S * sizeof(DevState)));
  STATUS_TRY(b[kStatus].ensure(sizeof(int)));
  cudaStream_t s = c->stream;
  if (mixed) {
    STATUS_TRY(b[kVp].ensure((size_t)umma_rhs_elems(pp) * sizeof(__half)));
    STATUS_TRY(b[kVe].ensure((size_t)umma_rhs_elems(pe) * sizeof(__half)));
    CUDA_TRY(cudaMemsetAsync(b[kVp].p, 0, (size_t)umma_rhs_elems(pp) * sizeof(__half), s));
    CUDA_TRY(cudaMemsetAsync(b[kVe].p, 0, (size_t)umma_rhs_elems(pe) * sizeof(__half), s));
  }
  CUDA_TRY(cudaMemsetAsync(b[kStatus].p, 0, sizeof(int), s));
  float4* Y4 = b[kY4].as<float4>();
  float4* T4 = b[kT4].as<float4>();
  std::vector<DevState*> st((size_t)S);
  for (int i = 0; i < S; ++i) {
    st[(size_t)i] = b[kSt].as<DevState>() + i;
    STATUS_TRY(upload_points(c, Y[i], N[i], Y4 + yoff[(size_t)i], true, c->stage, false, s));
    CUDA_TRY(cudaMemcpyAsync(T4 + (size_t)i * M, c->X4.p, (size_t)M * sizeof(float4), cudaMemcpyDeviceToDevice, s));
    const bool from_data = !(c->p.sigma2_init > 0.0);
    launch_state_init(st[(size_t)i], from_data ? 0.0 : c->p.sigma2_init, s);
    launch_state_params(st[(size_t)i], c->p.w, c->p.lambda, 0.0, 0.0, 0, nullptr, M, N[i], K, s);
    if (from_data) launch_sigma2_init<float>(c->X4.as<float4>(), M, Y4 + yoff[(size_t)i], N[i], nullptr,
                                             st[(size_t)i], s);
    if (mixed) {
      launch_state_prune(st[(size_t)i], 0.f, kMmaAllowed, s);
      launch_mma_threshold(c->X4.as<float4>(), M, Y4 + yoff[(size_t)i], N[i], st[(size_t)i], s);
    }
    launch_begin_iterations(st[(size_t)i], n_iter, s);
  }
  CUDA_TRY(cudaGetLastError());
  const bool fault = fault_enabled("umma_wait");
  // one iteration of the whole group, captured once
  cudaError_t le = cudaSuccess;
  CUDA_TRY(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeRelaxed));
  for (int i = 0; i < S; ++i)
    launch_estep<float>(ep[(size_t)i], T4 + (size_t)i * M, c->X4.as<float4>(), M, Y4 + yoff[(size_t)i],
                        b[kYb].as<float4>(), N[i], b[kPA].as<float>(), b[kPB].as<float>(), b[kSums].as<double>(),
                        b[kFlags].as<int>(), b[kYt4].as<float4>() + (size_t)i * M,
                        b[kR4].as<float4>() + (size_t)i * M, nullptr, nullptr, st[(size_t)i], true, c->cap,
                        nullptr, &c->side);
  if (mixed)
    le = launch_mstep_multi_mma(pp, pe, c->U.as<__half>(), c->ldU, c->Ut.as<__half>(), c->mp.ldM, c->lam.as<double>(),
                                M, K, c->X4.as<float4>(), b[kR4].as<float4>(), b[kYt4].as<float4>(), T4,
                                b[kB4].as<float4>(), b[kC4].as<float4>(), st.data(), b[kVp].as<__half>(),
                                b[kVe].as<__half>(), b[kPP].as<float>(), b[kSums].as<double>(), b[kStatus].as<int>(),
                                fault, c->cap);
  else
    launch_mstep_multi(mp, c->U.as<float>(), c->ldU, c->Ut.as<float>(), c->mp.ldM, c->lam.as<double>(), M, K,
                       c->X4.as<float4>(), b[kR4].as<float4>(), b[kYt4].as<float4>(), T4, b[kB4].as<float4>(),
                       b[kC4].as<float4>(), st.data(), b[kPP].as<float>(), b[kSums].as<double>(),
                       b[kStatus].as<int>(), c->cap);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(c->cap, &g);
  if (le != cudaSuccess || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return fail(CPD_ECUDA, std::string("capture of the shared-model iteration: ") +
                               cudaGetErrorString(le != cudaSuccess ? le : e));
  }
  cudaGraphExec_t ge = nullptr;
  e = cudaGraphInstantiate(&ge, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(CPD_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  for (int it = 0; it < n_iter && e == cudaSuccess; ++it) e = cudaGraphLaunch(ge, s);
  cudaStreamSynchronize(s);
  cudaGraphExecDestroy(ge);
  if (e != cudaSuccess) return fail(CPD_ECUDA, std::string("graph launch: ") + cudaGetErrorString(e));
  CUDA_TRY(cudaGetLastError());
  for (int i = 0; i < S; ++i) STATUS_TRY(download_points(T4 + (size_t)i * M, M, T_out[i], c->stage, false, s));
  std::vector<DevState> h((size_t)S);
  int status = 0;
  CUDA_TRY(cudaMemcpyAsync(h.data(), b[kSt].p, (size_t)S * sizeof(DevState), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaMemcpyAsync(&status, b[kStatus].p, sizeof(int), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  if (status != 0)
    return fail((cpd_status)status, std::string("a bounded wait of the shared-model M-step ran out") +
                                        (fault ? " (injected: CPD_FAULT=umma_wait)" : ""));
  for (int i = 0; i < S; ++i) {
    if (h[(size_t)i].status != 0)
      return fail((cpd_status)h[(size_t)i].status, "scene " + std::to_string(i) + ": the device reported a failure");
    s2_out[i] = h[(size_t)i].sigma2;
  }
  return CPD_OK;
}

cpd_status read_state(cpd_ctx* c, DevState* h) {
  CUDA_TRY(cudaMemcpyAsync(h, c->st.p, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return CPD_OK;
}

// M-step launches of an FP32-point context, for either basis storage.
void mstep_f32(cpd_ctx* c, const float4* R4, const float4* Yt4, float4* T4, const float4* Yhat4, float4* B4,
               float4* C4, DevState* st, bool iteration, cudaStream_t s, cudaEvent_t* ev = nullptr,
               bool projected = false) {
  const MstepPlan* trim = iteration && c->k_cap > 0 ? &c->mp_trim : nullptr;
  if (c->half_basis)
    launch_mstep<float, __half>(c->mp, c->U.as<__half>(), c->Ut.as<__half>(), c->lam.as<double>(), c->M, c->K,
                                c->X4.as<float4>(), R4, Yt4, T4, Yhat4, c->partP.as<float>(), c->sums.as<double>(),
                                B4, C4, st, iteration, s, ev, trim);
  else
    launch_mstep<float>(c->mp, c->U.as<float>(), c->Ut.as<float>(), c->lam.as<double>(), c->M, c->K,
                        c->X4.as<float4>(), R4, Yt4, T4, Yhat4, c->partP.as<float>(), c->sums.as<double>(), B4, C4,
                        st, iteration, s, ev, trim, projected);
}

// Pass B in row pieces: once piece i's rows of R are enqueued, their share
// of the projection U^T R follows -- on the side stream for every piece but
// the last, so that it streams U while the next piece's pass B computes.
struct PieceLaunch {
  cpd_ctx* c;
  cudaStream_t s;
  DevState* st;
};
void after_piece(void* user, int i) {
  const PieceLaunch* pl = static_cast<const PieceLaunch*>(user);
  cpd_ctx* c = pl->c;
  cudaStream_t ps = pl->s;
  if (i + 1 < c->mp.n_pieces) {
    cudaEventRecord(c->piece_ev[i], pl->s);
    cudaStreamWaitEvent(c->side.s, c->piece_ev[i], 0);
    ps = c->side.s;
  }
  launch_projection_piece(c->mp, i, c->U.as<float>(), c->R4.as<float4>(), c->partP.as<float>(), pl->st, ps);
}

void w_f32(cpd_ctx* c, const float4* C4, float4* W4, cudaStream_t s) {
  if (c->half_basis)
    launch_w<float, __half>(c->mp, c->Ut.as<__half>(), c->M, c->K, C4, c->partP.as<float>(), W4,
                            c->st_aux.as<DevState>(), s);
  else
    launch_w<float>(c->mp, c->Ut.as<float>(), c->M, c->K, C4, c->partP.as<float>(), W4, c->st_aux.as<DevState>(), s);
}

// The kernels of one EM iteration, enqueued on `s` (used only under capture).
// With `ev` (kEvPerIter = 9 events) the iteration is bracketed by timing
// events: ev[0] before pass A, ev[1..4] after the E-step kernels, ev[5..8]
// after the M-step kernels.
void enqueue_iteration(cpd_ctx* c, cudaStream_t s, cudaEvent_t* ev = nullptr) {
  if (ev) cudaEventRecordWithFlags(ev[0], s, cudaEventRecordExternal);
  cudaEvent_t* ee = ev ? ev + 1 : nullptr;
  cudaEvent_t* em = ev ? ev + 5 : nullptr;
  DevState* st = c->dst();
  if (c->fp64) {
    launch_estep<double>(c->ep, c->T4.as<dvec4>(), c->X4.as<dvec4>(), c->M, c->Y4.as<dvec4>(), c->Yb.as<dvec4>(),
                         c->N, c->partA.as<double>(), c->partB.as<double>(), c->sums.as<double>(), c->flags.as<int>(),
                         c->Yt4.as<dvec4>(), c->R4.as<dvec4>(), nullptr, nullptr, st, true, s, ee, &c->side);
    launch_mstep<double>(c->mp, c->U.as<double>(), c->Ut.as<double>(), c->lam.as<double>(), c->M, c->K,
                         c->X4.as<dvec4>(), c->R4.as<dvec4>(), c->Yt4.as<dvec4>(), c->T4.as<dvec4>(),
                         c->has_gt ? c->Yhat4.as<dvec4>() : nullptr, c->partP.as<double>(), c->sums.as<double>(),
                         c->B4.as<dvec4>(), c->C4.as<dvec4>(), st, true, s, em);
  } else if (!ev && c->ep.n_pieces > 1 && c->ep.n_pieces == c->mp.n_pieces) {
    PieceLaunch pl{c, s, st};
    const EstepPieces hook{&after_piece, &pl};
    const bool split = launch_estep<float>(c->ep, c->T4.as<float4>(), c->X4.as<float4>(), c->M, c->Y4.as<float4>(),
                                           c->Yb.as<float4>(), c->N, c->partA.as<float>(), c->partB.as<float>(),
                                           c->sums.as<double>(), c->flags.as<int>(), c->Yt4.as<float4>(),
                                           c->R4.as<float4>(), nullptr, nullptr, st, true, s, nullptr, &c->side,
                                           &hook);
    if (split) {
      cudaEventRecord(c->side.join, c->side.s);     // log-likelihood and the side projections
      cudaStreamWaitEvent(s, c->side.join, 0);
    }
    mstep_f32(c, c->R4.as<float4>(), c->Yt4.as<float4>(), c->T4.as<float4>(),
              c->has_gt ? c->Yhat4.as<float4>() : nullptr, c->B4.as<float4>(), c->C4.as<float4>(), st, true, s,
              nullptr, split);
  } else {
    launch_estep<float>(c->ep, c->T4.as<float4>(), c->X4.as<float4>(), c->M, c->Y4.as<float4>(), c->Yb.as<float4>(),
                        c->N, c->partA.as<float>(), c->partB.as<float>(), c->sums.as<double>(), c->flags.as<int>(),
                        c->Yt4.as<float4>(), c->R4.as<float4>(), nullptr, nullptr, st, true, s, ee, &c->side);
    mstep_f32(c, c->R4.as<float4>(), c->Yt4.as<float4>(), c->T4.as<float4>(),
              c->has_gt ? c->Yhat4.as<float4>() : nullptr, c->B4.as<float4>(), c->C4.as<float4>(), st, true, s, em);
  }
}

cpd_status capture_graph(cpd_ctx* c, int which) {
  const int iters = which == 0 ? 1 : cpd_ctx::kBatch;
  CUDA_TRY(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeRelaxed));
  for (int i = 0; i < iters; ++i) enqueue_iteration(c, c->cap);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(c->cap, &g);
  if (e != cudaSuccess) return fail(CPD_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(&c->graph[which], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(CPD_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  return CPD_OK;
}

// A graph whose one node is a conditional WHILE loop over one captured
// iteration followed by loop_control: the device runs iterations until the
// target is reached or a tolerance stops the registration, with no host
// round trip and no launches of iterations that would step aside.
cpd_status capture_loop_graph(cpd_ctx* c) {
  cudaGraph_t g = nullptr;
  CUDA_TRY(cudaGraphCreate(&g, 0));
  struct GraphGuard {
    cudaGraph_t g;
    ~GraphGuard() { cudaGraphDestroy(g); }
  } guard{g};
  cudaGraphConditionalHandle h;
  CUDA_TRY(cudaGraphConditionalHandleCreate(&h, g, 1u, cudaGraphCondAssignDefault));
  // the parameter union has no usable default constructor: zeroed storage
  alignas(cudaGraphNodeParams) unsigned char npbuf[sizeof(cudaGraphNodeParams)];
  std::memset(npbuf, 0, sizeof(npbuf));
  cudaGraphNodeParams* np = reinterpret_cast<cudaGraphNodeParams*>(npbuf);
  np->type = cudaGraphNodeTypeConditional;
  np->conditional.handle = h;
  np->conditional.type = cudaGraphCondTypeWhile;
  np->conditional.size = 1;
  cudaGraphNode_t node = nullptr;
  CUDA_TRY(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, np));
  cudaGraph_t body = np->conditional.phGraph_out[0];
  CUDA_TRY(cudaStreamBeginCaptureToGraph(c->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  enqueue_iteration(c, c->cap);
  launch_loop_control(c->dst(), h, c->cap);
  cudaGraph_t out = nullptr;
  cudaError_t e = cudaStreamEndCapture(c->cap, &out);
  if (e != cudaSuccess) return fail(CPD_ECUDA, std::string("loop graph capture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(&c->loop_graph, g, 0);
  if (e != cudaSuccess) {
    c->loop_graph = nullptr;
    return fail(CPD_ECUDA, std::string("loop graph instantiate: ") + cudaGetErrorString(e));
  }
  return CPD_OK;
}

// Sizes the scene-dependent buffers for N scene points.
cpd_status ensure_scene(cpd_ctx* c, int64_t N) {
  if (N == c->N) return CPD_OK;
  c->drop_graphs();
  c->ep = plan_estep(c->M, N, c->fp64, c->sms, c->sorted_model, c->half_basis);
  if (c->mp.n_pieces > 1 && !c->ep.pruned && !c->ep.mma)
    plan_estep_pieces(c->ep, N, c->sms, c->mp.n_pieces, c->mp.pp_m0, c->mp.pp_rows);
  STATUS_TRY(c->Y4.ensure((size_t)N * c->v4));
  STATUS_TRY(c->Yb.ensure((size_t)N * c->v4));
  STATUS_TRY(c->partA.ensure((size_t)c->ep.partA_elems * c->es));
  STATUS_TRY(c->partB.ensure((size_t)c->ep.partB_elems * c->es));
  STATUS_TRY(c->sums.ensure((size_t)std::max(c->ep.sums_elems, c->mp.sums_elems) * sizeof(double)));
  STATUS_TRY(c->flags.ensure((size_t)c->ep.flags_elems * sizeof(int)));
  c->N = N;
  launch_state_params(c->dst(), c->p.w, c->p.lambda, c->p.tol, c->gt_tol, c->has_gt ? 1 : 0,
                      c->hist.as<double>(), c->M, N, c->K, c->stream);
  CUDA_TRY(cudaGetLastError());
  return CPD_OK;
}


// A fresh registration against the uploaded scene: T = X, iteration count 0
// and the initial variance (given, or the mean squared distance over all
// model/scene pairs, evaluated on the device).
cpd_status start_registration(cpd_ctx* c) {
  CUDA_TRY(cudaMemcpyAsync(c->T4.p, c->X4.p, (size_t)c->M * c->v4, cudaMemcpyDeviceToDevice, c->stream));
  if (fault_enabled("nan_sigma")) {
    launch_state_init(c->dst(), std::nan(""), c->stream);
  } else if (c->p.sigma2_init > 0.0) {
    launch_state_init(c->dst(), c->p.sigma2_init, c->stream);
  } else {
    launch_state_init(c->dst(), 0.0, c->stream);
    if (c->fp64) launch_sigma2_init<double>(c->X4.as<dvec4>(), c->M, c->Y4.as<dvec4>(), c->N, nullptr, c->dst(), c->stream);
    else launch_sigma2_init<float>(c->X4.as<float4>(), c->M, c->Y4.as<float4>(), c->N, nullptr, c->dst(), c->stream);
  }
  apply_prune(c);
  CUDA_TRY(cudaGetLastError());
  c->started = true;
  return CPD_OK;
}

// Scene upload and, for a fresh registration, T = X and the initial variance.
cpd_status prepare_iterate(cpd_ctx* c, const void* Y, int64_t N) {
  STATUS_TRY(ensure_scene(c, N));
  STATUS_TRY(upload_points(c, Y, N, c->Y4.p, true, c->stage, c->fp64, c->stream));
  c->scene_sorted = c->sorted_model && spatial_sort_supported(N);
  if (c->scene_sorted) STATUS_TRY(sort_points(c, c->Y4.p, N, nullptr));
  if (!c->started) STATUS_TRY(start_registration(c));
  else apply_prune(c);
  return CPD_OK;
}

// Iterations that carry timing events: every kProfEvery-th and the last.
constexpr int kProfEvery = 10;
constexpr int kEvPerIter = 9;
constexpr int kPhases = kEvPerIter - 1;
bool profiled_iteration(int i, int n_iter) { return i % kProfEvery == 0 || i == n_iter - 1; }

cpd_status capture_profiled(cpd_ctx* c, int n_iter) {
  if (c->prof_graph) cudaGraphExecDestroy(c->prof_graph);
  c->prof_graph = nullptr;
  for (cudaEvent_t e : c->prof_ev) cudaEventDestroy(e);
  int sampled = 0;
  for (int i = 0; i < n_iter; ++i) sampled += profiled_iteration(i, n_iter) ? 1 : 0;
  c->prof_ev.assign((size_t)kEvPerIter * sampled, nullptr);
  for (auto& e : c->prof_ev) CUDA_TRY(cudaEventCreate(&e));
  CUDA_TRY(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeRelaxed));
  for (int i = 0, j = 0; i < n_iter; ++i) {
    if (profiled_iteration(i, n_iter)) enqueue_iteration(c, c->cap, &c->prof_ev[(size_t)kEvPerIter * j++]);
    else enqueue_iteration(c, c->cap, nullptr);
  }
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(c->cap, &g);
  if (e != cudaSuccess) return fail(CPD_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(&c->prof_graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(CPD_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  c->prof_iters = n_iter;
  return CPD_OK;
}
}  // namespace

extern "C" {

int32_t cpd_abi_version(void) { return FCPD_ABI_VERSION; }

const char* cpd_status_string(cpd_status s) {
  switch (s) {
    case CPD_OK: return "CPD_OK";
    case CPD_EINVAL: return "CPD_EINVAL";
    case CPD_ENOMEM: return "CPD_ENOMEM";
    case CPD_ECUDA: return "CPD_ECUDA";
    case CPD_ESOLVER: return "CPD_ESOLVER";
    case CPD_ENUMERIC: return "CPD_ENUMERIC";
    case CPD_ETIMEOUT: return "CPD_ETIMEOUT";
    case CPD_ESTATE: return "CPD_ESTATE";
  }
  return "CPD_UNKNOWN";
}

const char* cpd_last_error(void) { return g_err.c_str(); }

void cpd_params_default(cpd_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->D = 3;
  p->precision = CPD_FP32;
  p->w = 0.1;
  p->beta = 2.0;
  p->lambda = 2.0;
  p->sigma2_init = 0.0;
  p->K = 0;
  p->max_iter = 50;
  p->flags = 0;
  p->tol = 0.0;
}

int64_t cpd_basis_rank(const cpd_ctx* ctx) { return ctx ? ctx->K : 0; }

cpd_status cpd_eig_info(const cpd_ctx* c, int32_t* method, int32_t* steps) {
  if (!c) return fail(CPD_EINVAL, "ctx is NULL");
  if (method) *method = c->eig_method;
  if (steps) *steps = c->eig_steps;
  return CPD_OK;
}

cpd_status cpd_setup(const void* X, int64_t M, const cpd_params* p, void* stream, cpd_ctx** out) {
  g_err.clear();
  STATUS_TRY(validate_params(p));
  if (!X) return fail(CPD_EINVAL, "X is NULL");
  if (!out) return fail(CPD_EINVAL, "out is NULL");
  if (M < 1 || M > kMaxM) return fail(CPD_EINVAL, "M must be in [1, 46340]");
  if (p->K > M) return fail(CPD_EINVAL, "K must not exceed M");
  if (fault_enabled("alloc")) return fail(CPD_ENOMEM, "injected allocation failure (CPD_FAULT=alloc)");

  cpd_ctx* c = new (std::nothrow) cpd_ctx();
  if (!c) return fail(CPD_ENOMEM, "host allocation failed");
  auto bail = [&](cpd_status s) {
    if (c->stream) cudaStreamSynchronize(c->stream);
    delete c;
    return s;
  };
  c->p = *p;
  c->fp64 = p->precision == CPD_FP64;
  c->half_basis = p->precision == CPD_MIXED;
  c->es = c->fp64 ? 8 : 4;
  c->bes = c->fp64 ? 8 : c->half_basis ? 2 : 4;
  c->v4 = c->fp64 ? sizeof(dvec4) : sizeof(float4);
  c->M = M;
  c->K = (p->K == 0 || p->K >= M) ? M : p->K;
  c->stream = (cudaStream_t)stream;
  if (cudaGetDevice(&c->dev) != cudaSuccess) return bail(fail(CPD_ECUDA, "no CUDA device"));
  if (cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->dev) != cudaSuccess)
    return bail(fail(CPD_ECUDA, "cannot query the SM count"));
  if (cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->side.s, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->side.fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->side.join, cudaEventDisableTiming) != cudaSuccess)
    return bail(fail(CPD_ECUDA, "cannot create the capture streams"));
  for (cudaEvent_t& e : c->piece_ev)
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
      return bail(fail(CPD_ECUDA, "cannot create the capture events"));

  cpd_status s;
  if ((s = c->X4.ensure((size_t)M * c->v4)) != CPD_OK) return bail(s);
  if ((s = c->T4.ensure((size_t)M * c->v4)) != CPD_OK) return bail(s);
  if ((s = c->st.ensure(sizeof(DevState))) != CPD_OK) return bail(s);
  if ((s = c->st_aux.ensure(sizeof(DevState))) != CPD_OK) return bail(s);
  if ((s = c->hist.ensure((size_t)4 * kHistCap * sizeof(double))) != CPD_OK) return bail(s);
  if ((s = upload_points(c, X, M, c->X4.p, false, c->stage, c->fp64, c->stream)) != CPD_OK) return bail(s);
  // FP32 paths: model points in spatial order (the E-step prunes far tile
  // pairs exactly); every per-model-point input and output is permuted.
  if (!c->fp64 && (p->flags & kPruneFlags) && spatial_sort_supported(M)) {
    if ((s = c->permX.ensure((size_t)M * sizeof(int))) != CPD_OK) return bail(s);
    if ((s = c->invX.ensure((size_t)M * sizeof(int))) != CPD_OK) return bail(s);
    if ((s = sort_points(c, c->X4.p, M, c->permX.as<int>())) != CPD_OK) return bail(s);
    launch_invert_perm(c->permX.as<int>(), M, c->invX.as<int>(), c->stream);
    float box[6];
    if (cudaMemcpyAsync(box, c->sort_scratch.p, sizeof(box), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
      return bail(fail(CPD_ECUDA, "spatial sort of the model points failed"));
    // pruned passes once the FP32 cutoff radius is below a quarter of the
    // model's largest extent (box[3..5] = 16 / extent, 0 for a flat axis)
    float ext = 0.f;
    for (int d = 0; d < 3; ++d)
      if (box[3 + d] > 0.f) ext = std::max(ext, 16.f / box[3 + d]);
    c->prune_r2 = 0.0625f * ext * ext;
    c->sorted_model = true;
  }

  // The long-lived basis is allocated before the setup temporaries.
  c->mp = plan_mstep(M, c->K, c->fp64, c->sms, 128, (int)c->bes);
  c->ldU = c->mp.ldU;
  if ((s = c->U.ensure((size_t)M * c->ldU * c->bes)) != CPD_OK) return bail(s);
  if ((s = c->Ut.ensure((size_t)c->K * c->mp.ldM * c->bes)) != CPD_OK) return bail(s);
  if ((s = c->lam.ensure((size_t)c->K * sizeof(double))) != CPD_OK) return bail(s);

  // Eq. 11 in FP64, then Eq. 16 by the FP64 symmetric eigensolver.
  Buf phi, wv, info, work;
  auto free_setup = [&]() { phi.release(); wv.release(); info.release(); work.release(); };
  if ((s = phi.ensure((size_t)M * M * sizeof(double))) != CPD_OK) return bail(s);
  launch_gram_f64(c->X4.p, c->fp64, M, p->beta, phi.as<double>(), c->stream);
  const double* V = phi.as<double>();     // eigenvectors (columns, ascending) ...
  const double* wasc = nullptr;           // ... and their eigenvalues
  int64_t nv = M;
  double* topV = nullptr;
  double* topw = nullptr;
  auto free_top = [&]() {
    if (topV) cudaFree(topV);
    if (topw) cudaFree(topw);
    topV = topw = nullptr;
  };
  // Eq. 19 with K << M: the K largest pairs by subspace iteration (eig.cu);
  // otherwise (or if it does not converge) the full FP64 eigensolver.
  c->eig_method = 0;
  c->eig_steps = 0;
  if (!(p->flags & CPD_FLAG_FULL_EIG) && topk_eig_applies(M, c->K) && !fault_enabled("solver")) {
    std::string msg;
    int steps = 0;
    const int r = topk_eigh(phi.as<double>(), M, c->K, kTopkTol, kTopkMaxSteps, c->stream, &topV, &topw, &nv,
                            &steps, &msg);
    if (r == CPD_OK) {
      V = topV;
      wasc = topw;
      c->eig_method = 1;
      c->eig_steps = steps;
    } else if (r != -1) {
      free_top();
      free_setup();
      return bail(fail((cpd_status)r, msg));
    } else {
      free_top();
      nv = M;
      c->eig_steps = steps;
    }
  }
  if (c->eig_method == 0) {
    if ((s = wv.ensure((size_t)M * sizeof(double))) != CPD_OK) { free_setup(); return bail(s); }
    if ((s = info.ensure(sizeof(int))) != CPD_OK) { free_setup(); return bail(s); }
    cusolverDnHandle_t h = nullptr;
    if (cusolverDnCreate(&h) != CUSOLVER_STATUS_SUCCESS) { free_setup(); return bail(fail(CPD_ESOLVER, "cusolverDnCreate failed")); }
    cusolverDnSetStream(h, c->stream);
    int lwork = 0;
    cusolverStatus_t cs = cusolverDnDsyevd_bufferSize(h, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, (int)M,
                                                      phi.as<double>(), (int)M, wv.as<double>(), &lwork);
    if (cs == CUSOLVER_STATUS_SUCCESS) {
      if ((s = work.ensure((size_t)std::max(lwork, 1) * sizeof(double))) != CPD_OK) {
        cusolverDnDestroy(h); free_setup(); return bail(s);
      }
      cs = cusolverDnDsyevd(h, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, (int)M, phi.as<double>(), (int)M,
                            wv.as<double>(), work.as<double>(), lwork, info.as<int>());
    }
    int hinfo = 0;
    if (cs == CUSOLVER_STATUS_SUCCESS) {
      cudaMemcpyAsync(&hinfo, info.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
      cudaStreamSynchronize(c->stream);
    }
    cusolverDnDestroy(h);
    work.release();
    if (cs != CUSOLVER_STATUS_SUCCESS || hinfo != 0 || fault_enabled("solver")) {
      free_setup();
      return bail(fail(CPD_ESOLVER, "eigensolver failed (status " + std::to_string((int)cs) + ", info " +
                                        std::to_string(hinfo) + (fault_enabled("solver") ? ", injected" : "") + ")"));
    }
    wasc = wv.as<double>();
  }
  if (c->fp64) launch_extract_basis<double>(V, M, nv, c->K, c->U.as<double>(), c->ldU, c->Ut.as<double>(),
                                            c->mp.ldM, wasc, c->lam.as<double>(), c->stream);
  else if (c->half_basis)
    launch_extract_basis<__half>(V, M, nv, c->K, c->U.as<__half>(), c->ldU, c->Ut.as<__half>(),
                                 c->mp.ldM, wasc, c->lam.as<double>(), c->stream);
  else launch_extract_basis<float>(V, M, nv, c->K, c->U.as<float>(), c->ldU, c->Ut.as<float>(),
                                   c->mp.ldM, wasc, c->lam.as<double>(), c->stream);
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) { free_top(); free_setup(); return bail(fail(CPD_ECUDA, "setup kernels failed")); }
  free_top();
  free_setup();
  if ((p->flags & CPD_FLAG_SPECTRAL_TRIM) && (s = plan_trim(c)) != CPD_OK) return bail(s);
  plan_pieces(c);

  if ((s = c->Yt4.ensure((size_t)M * c->v4)) != CPD_OK) return bail(s);
  if ((s = c->R4.ensure((size_t)M * c->v4)) != CPD_OK) return bail(s);
  if ((s = c->B4.ensure((size_t)c->K * c->v4)) != CPD_OK) return bail(s);
  if ((s = c->C4.ensure((size_t)c->K * c->v4)) != CPD_OK) return bail(s);
  if ((s = c->partP.ensure((size_t)std::max(c->mp.part_elems, c->k_cap > 0 ? c->mp_trim.part_elems : 0) * c->es)) !=
      CPD_OK)
    return bail(s);
  if ((s = c->sums.ensure((size_t)c->mp.sums_elems * sizeof(double))) != CPD_OK) return bail(s);
  launch_state_init(c->dst(), 0.0, c->stream);
  launch_state_params(c->dst(), p->w, p->lambda, p->tol, 0.0, 0, c->hist.as<double>(), M, 0, c->K, c->stream);
  launch_state_init(c->st_aux.as<DevState>(), 0.0, c->stream);
  launch_state_params(c->st_aux.as<DevState>(), p->w, p->lambda, 0.0, 0.0, 0, nullptr, M, 0, c->K, c->stream);
  if (cudaStreamSynchronize(c->stream) != cudaSuccess || cudaGetLastError() != cudaSuccess)
    return bail(fail(CPD_ECUDA, "setup failed"));
  *out = c;
  return CPD_OK;
}

cpd_status cpd_reset(cpd_ctx* c) {
  if (!c) return fail(CPD_EINVAL, "ctx is NULL");
  c->started = false;
  return CPD_OK;
}

cpd_status cpd_iterate(cpd_ctx* c, const void* Y, int64_t N, int32_t n_iter, void* T_out, double* sigma2_out,
                       int32_t* iters_done) {
  g_err.clear();
  if (!c) return fail(CPD_EINVAL, "ctx is NULL");
  if (!Y) return fail(CPD_EINVAL, "Y is NULL");
  if (N < 1 || N > kMaxN) return fail(CPD_EINVAL, "N must be in [1, 2^30]");
  if (n_iter < 0) return fail(CPD_EINVAL, "n_iter must be >= 0");
  DeviceGuard guard(c->dev);
  STATUS_TRY(prepare_iterate(c, Y, N));
  if (n_iter > 0) {
    launch_begin_iterations(c->dst(), n_iter, c->stream);
    CUDA_TRY(cudaGetLastError());
    if (c->p.tol > 0.0 || (c->has_gt && c->gt_tol > 0.0)) {
      // a tolerance may stop the registration early: loop on the device
      if (!c->loop_graph) STATUS_TRY(capture_loop_graph(c));
      CUDA_TRY(cudaGraphLaunch(c->loop_graph, c->stream));
    } else {
      const int nb = n_iter / cpd_ctx::kBatch, n1 = n_iter % cpd_ctx::kBatch;
      if (nb > 0 && !c->graph[1]) STATUS_TRY(capture_graph(c, 1));
      if (n1 > 0 && !c->graph[0]) STATUS_TRY(capture_graph(c, 0));
      for (int i = 0; i < nb; ++i) CUDA_TRY(cudaGraphLaunch(c->graph[1], c->stream));
      for (int i = 0; i < n1; ++i) CUDA_TRY(cudaGraphLaunch(c->graph[0], c->stream));
    }
  }
  // a host T_out is followed by the state read, whose synchronisation
  // covers the copy of T as well
  const bool host_T = T_out && !is_device_ptr(T_out);
  if (T_out) STATUS_TRY(download_model(c, c->T4.p, T_out, !host_T));
  if (sigma2_out || iters_done || host_T) {
    DevState h;
    STATUS_TRY(read_state(c, &h));
    if (sigma2_out) *sigma2_out = h.sigma2;
    if (iters_done) *iters_done = h.iter;
    if (h.status != 0) return fail((cpd_status)h.status, "the device reported a failure during the iterations");
  }
  return CPD_OK;
}

cpd_status cpd_iterate_profiled(cpd_ctx* c, const void* Y, int64_t N, int32_t n_iter, float* phase_ms) {
  g_err.clear();
  if (!c) return fail(CPD_EINVAL, "ctx is NULL");
  if (!Y || !phase_ms) return fail(CPD_EINVAL, "Y and phase_ms are required");
  if (N < 1 || N > kMaxN) return fail(CPD_EINVAL, "N must be in [1, 2^30]");
  if (n_iter < 1 || n_iter > 4096) return fail(CPD_EINVAL, "n_iter must be in [1, 4096]");
  DeviceGuard guard(c->dev);
  STATUS_TRY(prepare_iterate(c, Y, N));
  launch_begin_iterations(c->dst(), n_iter, c->stream);
  CUDA_TRY(cudaGetLastError());
  if (!c->prof_graph || c->prof_iters != n_iter) STATUS_TRY(capture_profiled(c, n_iter));
  CUDA_TRY(cudaGraphLaunch(c->prof_graph, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  for (int p = 0; p <= kPhases; ++p) phase_ms[p] = 0.f;
  const int sampled = (int)(c->prof_ev.size() / kEvPerIter);
  for (int j = 0; j < sampled; ++j) {
    const cudaEvent_t* ev = &c->prof_ev[(size_t)kEvPerIter * j];
    for (int p = 0; p < kPhases; ++p) {
      float ms = 0.f;
      CUDA_TRY(cudaEventElapsedTime(&ms, ev[p], ev[p + 1]));
      phase_ms[p] += ms / (float)sampled;
    }
  }
  float total = 0.f;
  CUDA_TRY(cudaEventElapsedTime(&total, c->prof_ev[0], c->prof_ev.back()));
  phase_ms[kPhases] = total;
  DevState h;
  STATUS_TRY(read_state(c, &h));
  if (h.status != 0) return fail((cpd_status)h.status, "the device reported a failure during the iterations");
  return CPD_OK;
}

cpd_status cpd_set_ground_truth(cpd_ctx* c, const void* Yhat, double rmse_tol) {
  g_err.clear();
  if (!c) return fail(CPD_EINVAL, "ctx is NULL");
  if (!(rmse_tol >= 0.0) || !std::isfinite(rmse_tol)) return fail(CPD_EINVAL, "rmse_tol must be >= 0");
  DeviceGuard guard(c->dev);
  // the captured iterations hold the ground-truth pointer (or none): they
  // are re-captured only when that changes
  const bool had_gt = c->has_gt;
  const void* old_gt = c->Yhat4.p;
  if (Yhat) {
    STATUS_TRY(c->Yhat4.ensure((size_t)c->M * c->v4));
    STATUS_TRY(upload_model(c, Yhat, c->Yhat4.p));
    c->has_gt = true;
    c->gt_tol = rmse_tol;
  } else {
    c->has_gt = false;
    c->gt_tol = 0.0;
  }
  if (had_gt != c->has_gt || old_gt != c->Yhat4.p) c->drop_graphs();
  launch_state_params(c->dst(), c->p.w, c->p.lambda, c->p.tol, c->gt_tol, c->has_gt ? 1 : 0, c->hist.as<double>(),
                      c->M, c->N, c->K, c->stream);
  CUDA_TRY(cudaGetLastError());
  return CPD_OK;
}

cpd_status cpd_get_state(cpd_ctx* c, double* sigma2, int32_t* iters, int32_t* device_status) {
  if (!c) return fail(CPD_EINVAL, "ctx is NULL");
  DeviceGuard guard(c->dev);
  DevState h;
  STATUS_TRY(read_state(c, &h));
  if (sigma2) *sigma2 = h.sigma2;
  if (iters) *iters = h.iter;
  if (device_status) *device_status = h.status;
  return CPD_OK;
}

cpd_status cpd_get_history(cpd_ctx* c, int32_t n, double* s2h, double* llh, double* rmh) {
  if (!c) return fail(CPD_EINVAL, "ctx is NULL");
  DeviceGuard guard(c->dev);
  DevState h;
  STATUS_TRY(read_state(c, &h));
  if (n < 0 || n > h.iter || n > kHistCap) return fail(CPD_EINVAL, "n exceeds the recorded iterations");
  if (n == 0) return CPD_OK;
  const double* base = c->hist.as<double>();
  if (s2h) CUDA_TRY(cudaMemcpy(s2h, base, n * sizeof(double), cudaMemcpyDefault));
  if (llh) CUDA_TRY(cudaMemcpy(llh, base + kHistCap, n * sizeof(double), cudaMemcpyDefault));
  if (rmh) CUDA_TRY(cudaMemcpy(rmh, base + 2 * kHistCap, n * sizeof(double), cudaMemcpyDefault));
  return CPD_OK;
}

cpd_status cpd_get_W(cpd_ctx* c, void* W_out) {
  g_err.clear();
  if (!c) return fail(CPD_EINVAL, "ctx is NULL");
  if (!W_out) return fail(CPD_EINVAL, "W_out is NULL");
  DeviceGuard guard(c->dev);
  DevState h;
  STATUS_TRY(read_state(c, &h));
  if (!c->started || h.iter == 0) return fail(CPD_ESTATE, "no M-step has run yet");
  STATUS_TRY(c->W4.ensure((size_t)c->M * c->v4));
  if (c->fp64) launch_w<double>(c->mp, c->Ut.as<double>(), c->M, c->K, c->C4.as<dvec4>(), c->partP.as<double>(),
                                c->W4.as<dvec4>(), c->st_aux.as<DevState>(), c->stream);
  else w_f32(c, c->C4.as<float4>(), c->W4.as<float4>(), c->stream);
  CUDA_TRY(cudaGetLastError());
  return download_model(c, c->W4.p, W_out);
}

cpd_status cpd_get_basis(cpd_ctx* c, void* U_out, double* lam_out) {
  if (!c) return fail(CPD_EINVAL, "ctx is NULL");
  DeviceGuard guard(c->dev);
  if (U_out && !c->sorted_model && !c->half_basis) {
    CUDA_TRY(cudaMemcpy2DAsync(U_out, (size_t)c->K * c->es, c->U.p, (size_t)c->ldU * c->es, (size_t)c->K * c->es,
                               (size_t)c->M, cudaMemcpyDefault, c->stream));
  } else if (U_out) {
    // float rows (FP16 converted), then in the caller's point order
    Buf conv, stage;
    const float* rows = c->U.as<float>();
    int64_t ld = c->ldU;
    if (c->half_basis) {
      STATUS_TRY(conv.ensure((size_t)c->M * c->K * sizeof(float)));
      launch_basis_to_f32(c->U.as<__half>(), c->M, c->K, c->ldU, conv.as<float>(), c->stream);
      rows = conv.as<float>();
      ld = c->K;
    }
    const bool dev_out = is_device_ptr(U_out);
    float* dst = static_cast<float*>(U_out);
    if (!dev_out) {
      STATUS_TRY(stage.ensure((size_t)c->M * c->K * sizeof(float)));
      dst = stage.as<float>();
    }
    if (c->sorted_model)
      launch_gather_rows_f32(rows, ld, c->invX.as<int>(), c->M, c->K, dst, c->stream);
    else
      CUDA_TRY(cudaMemcpyAsync(dst, rows, (size_t)c->M * c->K * sizeof(float), cudaMemcpyDeviceToDevice, c->stream));
    CUDA_TRY(cudaGetLastError());
    if (!dev_out)
      CUDA_TRY(cudaMemcpyAsync(U_out, dst, (size_t)c->M * c->K * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
  }
  if (lam_out)
    CUDA_TRY(cudaMemcpyAsync(lam_out, c->lam.p, (size_t)c->K * sizeof(double), cudaMemcpyDefault, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return CPD_OK;
}

cpd_status cpd_get_work(cpd_ctx* c, int32_t n, double* eval_frac) {
  if (!c || !eval_frac) return fail(CPD_EINVAL, "ctx and eval_frac are required");
  DeviceGuard guard(c->dev);
  DevState h;
  STATUS_TRY(read_state(c, &h));
  if (n < 0 || n > h.iter || n > kHistCap) return fail(CPD_EINVAL, "n exceeds the recorded iterations");
  if (n > 0) CUDA_TRY(cudaMemcpy(eval_frac, c->hist.as<double>() + 3 * kHistCap, n * sizeof(double), cudaMemcpyDefault));
  return CPD_OK;
}

int32_t cpd_spatial_order(const cpd_ctx* c) { return c && c->sorted_model ? 1 : 0; }

cpd_status cpd_iterate_shared(cpd_ctx* c, int32_t n_scenes, const void* const* Y, const int64_t* N, int32_t n_iter,
                              void* const* T_out, double* sigma2_out) {
  g_err.clear();
  if (!c) return fail(CPD_EINVAL, "ctx is NULL");
  if (n_scenes < 1 || n_scenes > 4096) return fail(CPD_EINVAL, "n_scenes must be in [1, 4096]");
  if (!Y || !N || !T_out || !sigma2_out) return fail(CPD_EINVAL, "Y, N, T_out and sigma2_out are required");
  if (n_iter < 1 || n_iter > 100000) return fail(CPD_EINVAL, "n_iter must be in [1, 100000]");
  if (c->fp64 || c->sorted_model || c->k_cap > 0)
    return fail(CPD_EINVAL, "shared-model registrations need a CPD_FP32 or CPD_MIXED context without flags");
  if (c->half_basis && !umma_supported(1))
    return fail(CPD_ECUDA, "the tensor-map encoder of the driver is unavailable");
  for (int i = 0; i < n_scenes; ++i) {
    if (!Y[i] || !T_out[i]) return fail(CPD_EINVAL, "scene " + std::to_string(i) + ": Y or T_out is NULL");
    if (N[i] < 1 || N[i] > kMaxN) return fail(CPD_EINVAL, "scene " + std::to_string(i) + ": N must be in [1, 2^30]");
  }
  DeviceGuard guard(c->dev);
  const int per_pass = c->half_basis ? kMaxScenesPerPassMma : kMaxScenesPerPass;
  for (int g0 = 0; g0 < n_scenes; g0 += per_pass) {
    const int S = std::min(per_pass, n_scenes - g0);
    STATUS_TRY(shared_group(c, S, Y + g0, N + g0, n_iter, T_out + g0, sigma2_out + g0));
  }
  return CPD_OK;
}

cpd_status cpd_pass_b_pieces(cpd_ctx* c, int32_t* pieces) {
  g_err.clear();
  if (!c || !pieces) return fail(CPD_EINVAL, "ctx and pieces are required");
  *pieces = c->mp.n_pieces > 1 ? c->mp.n_pieces : 1;
  return CPD_OK;
}

cpd_status cpd_get_trim(cpd_ctx* c, int64_t* k_cap, int32_t* trimmed_iters) {
  g_err.clear();
  if (!c || !k_cap || !trimmed_iters) return fail(CPD_EINVAL, "ctx, k_cap and trimmed_iters are required");
  *k_cap = c->k_cap;
  *trimmed_iters = 0;
  if (!c->started) return CPD_OK;
  DeviceGuard guard(c->dev);
  DevState h;
  STATUS_TRY(read_state(c, &h));
  *trimmed_iters = h.trim_iters;
  return CPD_OK;
}

cpd_status cpd_coefficients(cpd_ctx* c, int32_t n_coef, void* coef_out) {
  g_err.clear();
  if (!c || !coef_out) return fail(CPD_EINVAL, "ctx and coef_out are required");
  if (c->fp64) return fail(CPD_EINVAL, "coefficients need a CPD_FP32 or CPD_MIXED context");
  if (n_coef < 1 || n_coef > c->K) return fail(CPD_EINVAL, "n_coef must be in [1, K]");
  if (!c->started) return fail(CPD_ESTATE, "no registration has started");
  DeviceGuard guard(c->dev);
  Buf tmp;
  STATUS_TRY(tmp.ensure((size_t)n_coef * 3 * sizeof(float)));
  if (c->half_basis)
    launch_coefficients<__half>(c->U.as<__half>(), c->ldU, c->M, n_coef, c->T4.as<float4>(), c->X4.as<float4>(),
                                tmp.as<float>(), c->stream);
  else
    launch_coefficients<float>(c->U.as<float>(), c->ldU, c->M, n_coef, c->T4.as<float4>(), c->X4.as<float4>(),
                               tmp.as<float>(), c->stream);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemcpyAsync(coef_out, tmp.p, (size_t)n_coef * 3 * sizeof(float), cudaMemcpyDefault, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return CPD_OK;
}

cpd_status cpd_coefficients_of(cpd_ctx* c, int32_t n_coef, const void* T, void* coef_out) {
  g_err.clear();
  if (!c || !T || !coef_out) return fail(CPD_EINVAL, "ctx, T and coef_out are required");
  if (c->fp64) return fail(CPD_EINVAL, "coefficients need a CPD_FP32 or CPD_MIXED context");
  if (n_coef < 1 || n_coef > c->K) return fail(CPD_EINVAL, "n_coef must be in [1, K]");
  DeviceGuard guard(c->dev);
  Buf tmp, t4;
  STATUS_TRY(tmp.ensure((size_t)n_coef * 3 * sizeof(float)));
  STATUS_TRY(t4.ensure((size_t)c->M * sizeof(float4)));
  STATUS_TRY(upload_model(c, T, t4.p));
  if (c->half_basis)
    launch_coefficients<__half>(c->U.as<__half>(), c->ldU, c->M, n_coef, t4.as<float4>(), c->X4.as<float4>(),
                                tmp.as<float>(), c->stream);
  else
    launch_coefficients<float>(c->U.as<float>(), c->ldU, c->M, n_coef, t4.as<float4>(), c->X4.as<float4>(),
                               tmp.as<float>(), c->stream);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemcpyAsync(coef_out, tmp.p, (size_t)n_coef * 3 * sizeof(float), cudaMemcpyDefault, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return CPD_OK;
}

cpd_status cpd_warm_start(cpd_ctx* c, int32_t n_coef, const void* coef, double sigma2_0) {
  g_err.clear();
  if (!c || !coef) return fail(CPD_EINVAL, "ctx and coef are required");
  if (c->fp64) return fail(CPD_EINVAL, "a warm start needs a CPD_FP32 or CPD_MIXED context");
  if (n_coef < 0 || n_coef > c->K) return fail(CPD_EINVAL, "n_coef must be in [0, K]");
  if (!(sigma2_0 > 0.0) || !std::isfinite(sigma2_0)) return fail(CPD_EINVAL, "sigma2_0 must be > 0");
  DeviceGuard guard(c->dev);
  Buf tmp;
  STATUS_TRY(tmp.ensure((size_t)std::max(n_coef, 1) * 3 * sizeof(float)));
  if (n_coef > 0)
    CUDA_TRY(cudaMemcpyAsync(tmp.p, coef, (size_t)n_coef * 3 * sizeof(float), cudaMemcpyDefault, c->stream));
  if (c->half_basis)
    launch_warm_start_T<__half>(c->U.as<__half>(), c->ldU, c->M, n_coef, tmp.as<float>(), c->X4.as<float4>(),
                                c->T4.as<float4>(), c->stream);
  else
    launch_warm_start_T<float>(c->U.as<float>(), c->ldU, c->M, n_coef, tmp.as<float>(), c->X4.as<float4>(),
                               c->T4.as<float4>(), c->stream);
  launch_state_init(c->dst(), sigma2_0, c->stream);
  if (c->N > 0) apply_prune(c);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaStreamSynchronize(c->stream));       // tmp is freed on return
  c->started = true;
  return CPD_OK;
}

cpd_status cpd_mstep(cpd_ctx* c, const void* Ytil, double sigma2, void* T_out, void* W_out) {
  g_err.clear();
  if (!c) return fail(CPD_EINVAL, "ctx is NULL");
  if (!Ytil || !T_out) return fail(CPD_EINVAL, "Ytil and T_out are required");
  if (!(sigma2 > 0.0) || !std::isfinite(sigma2)) return fail(CPD_EINVAL, "sigma2 must be > 0");
  DeviceGuard guard(c->dev);
  STATUS_TRY(c->auxT4.ensure((size_t)c->M * c->v4));
  STATUS_TRY(c->auxR4.ensure((size_t)c->M * c->v4));
  STATUS_TRY(c->auxB4.ensure((size_t)c->K * c->v4));
  STATUS_TRY(c->auxC4.ensure((size_t)c->K * c->v4));
  STATUS_TRY(upload_model(c, Ytil, c->auxT4.p));
  DevState* sa = c->st_aux.as<DevState>();
  launch_state_init(sa, sigma2, c->stream);
  if (c->fp64) {
    launch_residual<double>(c->auxT4.as<dvec4>(), c->X4.as<dvec4>(), c->auxR4.as<dvec4>(), c->M, c->stream);
    launch_mstep<double>(c->mp, c->U.as<double>(), c->Ut.as<double>(), c->lam.as<double>(), c->M, c->K,
                         c->X4.as<dvec4>(), c->auxR4.as<dvec4>(), nullptr, c->auxT4.as<dvec4>(), nullptr, c->partP.as<double>(),
                         c->sums.as<double>(), c->auxB4.as<dvec4>(), c->auxC4.as<dvec4>(), sa, false, c->stream);
  } else {
    launch_residual<float>(c->auxT4.as<float4>(), c->X4.as<float4>(), c->auxR4.as<float4>(), c->M, c->stream);
    mstep_f32(c, c->auxR4.as<float4>(), nullptr, c->auxT4.as<float4>(), nullptr, c->auxB4.as<float4>(),
              c->auxC4.as<float4>(), sa, false, c->stream);
  }
  CUDA_TRY(cudaGetLastError());
  STATUS_TRY(download_model(c, c->auxT4.p, T_out));
  if (W_out) {
    if (c->fp64) launch_w<double>(c->mp, c->Ut.as<double>(), c->M, c->K, c->auxC4.as<dvec4>(), c->partP.as<double>(),
                                  c->auxR4.as<dvec4>(), c->st_aux.as<DevState>(), c->stream);
    else w_f32(c, c->auxC4.as<float4>(), c->auxR4.as<float4>(), c->stream);
    CUDA_TRY(cudaGetLastError());
    STATUS_TRY(download_model(c, c->auxR4.p, W_out));
  }
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return CPD_OK;
}

cpd_status cpd_estep(const void* T, int64_t M, const void* Y, int64_t N, int32_t precision, double sigma2, double w,
                     void* Ytil_out, void* P1_out, void* den_out, double* sums_out, void* stream) {
  g_err.clear();
  if (!T || !Y || !Ytil_out) return fail(CPD_EINVAL, "T, Y and Ytil_out are required");
  if (M < 1 || M > kMaxN || N < 1 || N > kMaxN) return fail(CPD_EINVAL, "M and N must be in [1, 2^30]");
  if (precision != CPD_FP64 && precision != CPD_FP32 && precision != CPD_MIXED)
    return fail(CPD_EINVAL, "unknown precision");
  const bool mixed = precision == CPD_MIXED;   // FP32 E-step with tensor-core passes while sigma2 allows
  if (mixed) precision = CPD_FP32;
  if (!(sigma2 > 0.0) || !std::isfinite(sigma2)) return fail(CPD_EINVAL, "sigma2 must be > 0");
  if (!(w >= 0.0 && w < 1.0)) return fail(CPD_EINVAL, "w must satisfy 0 <= w < 1");
  cudaStream_t s = (cudaStream_t)stream;
  const bool fp64 = precision == CPD_FP64;
  const size_t es = fp64 ? 8 : 4, v4 = fp64 ? sizeof(dvec4) : sizeof(float4);
  int dev = 0, sms = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const EstepPlan ep = plan_estep(M, N, fp64, sms, false, mixed);
  Buf T4, Y4, Yb, Yt4, pA, pB, sums, flags, P1, den, st, stage;
  auto release = [&]() {
    for (Buf* b : {&T4, &Y4, &Yb, &Yt4, &pA, &pB, &sums, &flags, &P1, &den, &st, &stage}) b->release();
  };
  auto run = [&]() -> cpd_status {
    STATUS_TRY(T4.ensure((size_t)M * v4));
    STATUS_TRY(Y4.ensure((size_t)N * v4));
    STATUS_TRY(Yb.ensure((size_t)N * v4));
    STATUS_TRY(Yt4.ensure((size_t)M * v4));
    STATUS_TRY(pA.ensure((size_t)ep.partA_elems * es));
    STATUS_TRY(pB.ensure((size_t)ep.partB_elems * es));
    STATUS_TRY(sums.ensure((size_t)ep.sums_elems * sizeof(double)));
    STATUS_TRY(flags.ensure((size_t)ep.flags_elems * sizeof(int)));
    STATUS_TRY(P1.ensure((size_t)M * sizeof(double)));
    STATUS_TRY(den.ensure((size_t)N * sizeof(double)));
    STATUS_TRY(st.ensure(sizeof(DevState)));
    STATUS_TRY(upload_points(nullptr, T, M, T4.p, false, stage, fp64, s));
    STATUS_TRY(upload_points(nullptr, Y, N, Y4.p, true, stage, fp64, s));
    launch_state_init(st.as<DevState>(), sigma2, s);
    launch_state_params(st.as<DevState>(), w, 1.0, 0.0, 0.0, 0, nullptr, M, N, 0, s);
    if (mixed) {
      launch_state_prune(st.as<DevState>(), 0.f, kMmaAllowed, s);
      launch_mma_threshold(T4.as<float4>(), M, Y4.as<float4>(), N, st.as<DevState>(), s);
    }
    if (fp64)
      launch_estep<double>(ep, T4.as<dvec4>(), nullptr, M, Y4.as<dvec4>(), Yb.as<dvec4>(), N, pA.as<double>(),
                           pB.as<double>(), sums.as<double>(), flags.as<int>(), Yt4.as<dvec4>(), nullptr, P1.as<double>(),
                           den.as<double>(), st.as<DevState>(), false, s);
    else
      launch_estep<float>(ep, T4.as<float4>(), nullptr, M, Y4.as<float4>(), Yb.as<float4>(), N, pA.as<float>(),
                          pB.as<float>(), sums.as<double>(), flags.as<int>(), Yt4.as<float4>(), nullptr, P1.as<double>(),
                          den.as<double>(), st.as<DevState>(), false, s);
    CUDA_TRY(cudaGetLastError());
    STATUS_TRY(download_points(Yt4.p, M, Ytil_out, stage, fp64, s));
    if (P1_out) CUDA_TRY(cudaMemcpyAsync(P1_out, P1.p, (size_t)M * sizeof(double), cudaMemcpyDefault, s));
    if (den_out) CUDA_TRY(cudaMemcpyAsync(den_out, den.p, (size_t)N * sizeof(double), cudaMemcpyDefault, s));
    DevState h;
    CUDA_TRY(cudaMemcpyAsync(&h, st.p, sizeof(DevState), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (sums_out) {
      sums_out[0] = h.vsum;
      sums_out[1] = h.loglik;
    }
    if (h.status != 0) return fail((cpd_status)h.status, "the device reported a failure during the iterations");
    return CPD_OK;
  };
  const cpd_status r = run();
  cudaStreamSynchronize(s);
  release();
  return r;
}

cpd_status cpd_register(const void* X, int64_t M, const void* Y, int64_t N, const cpd_params* p, void* stream,
                        void* T_out, void* W_out, double* sigma2_out, int32_t* iters_done) {
  g_err.clear();
  if (!T_out) return fail(CPD_EINVAL, "T_out is NULL");
  if (!Y) return fail(CPD_EINVAL, "Y is NULL");
  if (N < 1 || N > kMaxN) return fail(CPD_EINVAL, "N must be in [1, 2^30]");
  cpd_ctx* c = nullptr;
  STATUS_TRY(cpd_setup(X, M, p, stream, &c));
  cpd_status s = cpd_iterate(c, Y, N, p->max_iter, T_out, sigma2_out, iters_done);
  if (s == CPD_OK && W_out) s = cpd_get_W(c, W_out);
  const std::string keep = g_err;
  cpd_destroy(c);
  g_err = keep;
  return s;
}

void cpd_destroy(cpd_ctx* c) {
  if (!c) return;
  DeviceGuard guard(c->dev);
  cudaStreamSynchronize(c->stream);
  delete c;
}

}  // extern "C"

// ------------------------------------------------------------------ batched registrations
// Many independent registrations (X_i, Y_i) advanced together by one
// persistent kernel launch per call (batch.cu).  Each pair keeps a full
// context (its own eigenbasis and state); the batch adds the work-item lists
// of the persistent kernel, its control block and a CUDA graph of the launch.
struct cpd_batch {
  int dev = 0;
  int sms = 0;
  int n = 0;
  int grid = 0;
  double wait_s = 5.0;
  cudaStream_t stream = nullptr;
  cudaStream_t cap = nullptr;
  std::vector<cpd_ctx*> ctx;
  std::vector<BatchPair> pairs;
  std::vector<int> phase_off_host;
  Buf pairs_dev, items, phase_off, ctl, states, tickets, done;
  int n_items = 0;
  cudaGraphExec_t graph = nullptr;
  int graph_iters = -1;
  int graph_extra = -1;
  BatchCtl last{};            // control block after the last call
  int last_iters = 0;
  size_t n_tickets = 0;
  int tune_e = 0, tune_p = 0; // work-item plan in use (see plan_batch)

  ~cpd_batch() {
    if (graph) cudaGraphExecDestroy(graph);
    for (cpd_ctx* c : ctx) delete c;
    for (Buf* b : {&pairs_dev, &items, &phase_off, &ctl, &states, &tickets, &done}) b->release();
    if (cap) cudaStreamDestroy(cap);
  }
};

namespace {

constexpr int kMaxBatch = 1 << 16;
constexpr int kBatchDefaultItems = 4;      // untuned plan: E-step items per resident block
constexpr int kBatchDefaultProjKB = 512;   // untuned plan: KB of the basis per projection item

// Scene of one pair: buffers, upload, state parameters.
cpd_status batch_load_scene(cpd_ctx* c, int64_t N, const void* Y) {
  c->drop_graphs();
  STATUS_TRY(c->Y4.ensure((size_t)N * c->v4));
  STATUS_TRY(c->Yb.ensure((size_t)N * c->v4));
  c->N = N;
  launch_state_params(c->dst(), c->p.w, c->p.lambda, c->p.tol, 0.0, 0, c->hist.as<double>(), c->M, N, c->K,
                      c->stream);
  return upload_points(c, Y, N, c->Y4.p, true, c->stage, false, c->stream);
}

// Per-pair scratch sized for a batched plan.
cpd_status batch_size_pair(cpd_ctx* c, const BatchPair& bp) {
  if (bp.mp.ldU != c->mp.ldU || bp.mp.ldM != c->mp.ldM)
    return fail(CPD_ECUDA, "internal: batched basis layout differs from the context's");
  c->ep = bp.ep;
  c->mp = bp.mp;
  STATUS_TRY(c->partA.ensure((size_t)c->ep.partA_elems * c->es));
  STATUS_TRY(c->partB.ensure((size_t)c->ep.partB_elems * c->es));
  STATUS_TRY(c->partP.ensure((size_t)c->mp.part_elems * c->es));
  STATUS_TRY(c->sums.ensure((size_t)std::max(c->ep.sums_elems, c->mp.sums_elems) * sizeof(double)));
  STATUS_TRY(c->flags.ensure((size_t)c->ep.flags_elems * sizeof(int)));
  return CPD_OK;
}

BatchPair batch_pointers(cpd_ctx* c, const BatchPair& plan) {
  BatchPair b = plan;
  b.X4 = c->X4.as<float4>();
  b.T4 = c->T4.as<float4>();
  b.U = c->U.p;
  b.Ut = c->Ut.p;
  b.half_basis = c->half_basis ? 1 : 0;
  b.lam = c->lam.as<double>();
  b.Yt4 = c->Yt4.as<float4>();
  b.R4 = c->R4.as<float4>();
  b.B4 = c->B4.as<float4>();
  b.C4 = c->C4.as<float4>();
  b.Y4 = c->Y4.as<float4>();
  b.Yb = c->Yb.as<float4>();
  b.Yhat4 = nullptr;
  b.partA = c->partA.as<float>();
  b.partB = c->partB.as<float>();
  b.partP = c->partP.as<float>();
  b.sums = c->sums.as<double>();
  b.flags = c->flags.as<int>();
  b.st = c->dst();
  return b;
}

// Work-item plan (item sizes e_items per resident block / proj_kb KB, see
// plan_batch): per-pair scratch, device pair table, item lists, tickets.
// Invalidates the captured launch.
cpd_status batch_apply_plan(cpd_batch* b, int e_items, int proj_kb) {
  const int n = b->n;
  plan_batch(b->pairs.data(), n, b->grid, e_items, proj_kb);
  size_t n_tickets = 0;
  for (int i = 0; i < n; ++i) n_tickets += (size_t)batch_tickets(b->pairs[i]);
  STATUS_TRY(b->tickets.ensure(n_tickets * sizeof(unsigned int)));
  b->n_tickets = n_tickets;
  const int np = batch_phases();
  STATUS_TRY(b->done.ensure((size_t)np * n * sizeof(unsigned int)));
  for (int i = 0, off = 0; i < n; ++i) {
    STATUS_TRY(batch_size_pair(b->ctx[i], b->pairs[i]));
    const int nt = batch_tickets(b->pairs[i]);
    b->pairs[i] = batch_pointers(b->ctx[i], b->pairs[i]);
    b->pairs[i].tix = b->tickets.as<unsigned int>() + off;
    b->pairs[i].done = b->done.as<unsigned int>() + (size_t)np * i;
    off += nt;
  }
  std::vector<BatchItem> items;
  batch_items(b->pairs.data(), n, items, b->phase_off_host);
  b->n_items = (int)items.size();
  STATUS_TRY(b->pairs_dev.ensure(sizeof(BatchPair) * (size_t)n));
  STATUS_TRY(b->items.ensure(sizeof(BatchItem) * items.size()));
  STATUS_TRY(b->phase_off.ensure(sizeof(int) * b->phase_off_host.size()));
  CUDA_TRY(cudaMemsetAsync(b->tickets.p, 0, n_tickets * sizeof(unsigned int), b->stream));
  CUDA_TRY(cudaMemcpyAsync(b->pairs_dev.p, b->pairs.data(), sizeof(BatchPair) * (size_t)n, cudaMemcpyHostToDevice,
                           b->stream));
  CUDA_TRY(cudaMemcpyAsync(b->items.p, items.data(), sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice,
                           b->stream));
  CUDA_TRY(cudaMemcpyAsync(b->phase_off.p, b->phase_off_host.data(), sizeof(int) * b->phase_off_host.size(),
                           cudaMemcpyHostToDevice, b->stream));
  CUDA_TRY(cudaStreamSynchronize(b->stream));      // the host vectors above are reused
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
  b->graph_iters = -1;
  b->tune_e = e_items;
  b->tune_p = proj_kb;
  return CPD_OK;
}

cpd_status batch_capture(cpd_batch* b, int n_iter, int extra) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
  b->graph_iters = -1;
  CUDA_TRY(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed));
  cudaError_t le = launch_batch(b->pairs_dev.as<BatchPair>(), b->n, b->items.as<BatchItem>(), b->phase_off.as<int>(),
                                b->ctl.as<BatchCtl>(), b->done.as<unsigned int>(), b->grid, n_iter, b->wait_s, extra,
                                b->cap);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(b->cap, &g);
  if (le != cudaSuccess || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return fail(CPD_ECUDA, std::string("capture of the batched launch: ") +
                               cudaGetErrorString(le != cudaSuccess ? le : e));
  }
  e = cudaGraphInstantiate(&b->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(CPD_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  b->graph_iters = n_iter;
  b->graph_extra = extra;
  return CPD_OK;
}

}  // namespace

extern "C" {

cpd_status cpd_batch_create(int32_t n_pairs, const void* const* X, const int64_t* M, const void* const* Y,
                            const int64_t* N, const cpd_params* p, double barrier_timeout_s, void* stream,
                            cpd_batch** out) {
  g_err.clear();
  STATUS_TRY(validate_params(p));
  if (!out) return fail(CPD_EINVAL, "out is NULL");
  if (n_pairs < 1 || n_pairs > kMaxBatch) return fail(CPD_EINVAL, "n_pairs must be in [1, 65536]");
  if (!X || !M || !Y || !N) return fail(CPD_EINVAL, "X, M, Y and N are required");
  if (p->precision != CPD_FP32 && p->precision != CPD_MIXED)
    return fail(CPD_EINVAL, "batched registrations run in CPD_FP32 or CPD_MIXED (FP16 basis)");
  if (p->flags & CPD_FLAG_SPECTRAL_TRIM) return fail(CPD_EINVAL, "batched registrations take no spectral trim");
  if (barrier_timeout_s == 0.0) barrier_timeout_s = 5.0;
  if (!(barrier_timeout_s > 0.0 && barrier_timeout_s <= 60.0))
    return fail(CPD_EINVAL, "barrier_timeout_s must be in (0, 60] (0 selects 5 s)");
  for (int i = 0; i < n_pairs; ++i) {
    if (!X[i] || !Y[i]) return fail(CPD_EINVAL, "pair " + std::to_string(i) + ": X or Y is NULL");
    if (M[i] < 1 || M[i] > kMaxM) return fail(CPD_EINVAL, "pair " + std::to_string(i) + ": M must be in [1, 46340]");
    if (N[i] < 1 || N[i] > kMaxN) return fail(CPD_EINVAL, "pair " + std::to_string(i) + ": N must be in [1, 2^30]");
  }
  if (fault_enabled("alloc")) return fail(CPD_ENOMEM, "injected allocation failure (CPD_FAULT=alloc)");

  cpd_batch* b = new (std::nothrow) cpd_batch();
  if (!b) return fail(CPD_ENOMEM, "host allocation failed");
  auto bail = [&](cpd_status s) {
    const std::string keep = g_err;
    if (b->stream) cudaStreamSynchronize(b->stream);
    delete b;
    g_err = keep;
    return s;
  };
  b->n = n_pairs;
  b->wait_s = barrier_timeout_s;
  b->stream = (cudaStream_t)stream;
  if (cudaGetDevice(&b->dev) != cudaSuccess) return bail(fail(CPD_ECUDA, "no CUDA device"));
  if (cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->dev) != cudaSuccess)
    return bail(fail(CPD_ECUDA, "cannot query the SM count"));
  int coop = 0;
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, b->dev);
  if (!coop) return bail(fail(CPD_ECUDA, "the device does not support cooperative launches"));
  if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess)
    return bail(fail(CPD_ECUDA, "cannot create the capture stream"));
  b->grid = batch_resident_blocks(b->sms);
  if (b->grid < 1) return bail(fail(CPD_ECUDA, "the persistent kernel cannot be made resident"));

  // Setup of every pair (Eq. 11, Eq. 16, Eq. 19): several host threads, each
  // on its own stream, so the eigensolves of small pairs overlap.
  b->ctx.assign((size_t)n_pairs, nullptr);
  std::vector<cpd_status> st((size_t)n_pairs, CPD_OK);
  std::vector<std::string> msg((size_t)n_pairs);
  std::atomic<int> next{0};
  std::atomic<bool> stop{false};
  const int nthreads = std::min(n_pairs, 8);
  auto worker = [&]() {
    cudaSetDevice(b->dev);
    cudaStream_t ws = nullptr;
    if (cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking) != cudaSuccess) {
      stop = true;
      return;
    }
    for (int i; !stop && (i = next.fetch_add(1)) < n_pairs;) {
      cpd_params pi = *p;
      pi.K = (p->K == 0 || p->K > M[i]) ? 0 : p->K;
      cpd_ctx* c = nullptr;
      st[i] = cpd_setup(X[i], M[i], &pi, ws, &c);
      if (st[i] != CPD_OK) {
        msg[i] = cpd_last_error();
        stop = true;
        break;
      }
      cudaStreamSynchronize(ws);
      c->stream = b->stream;
      b->ctx[i] = c;
    }
    cudaStreamSynchronize(ws);
    cudaStreamDestroy(ws);
  };
  std::vector<std::thread> pool;
  for (int t = 0; t < nthreads; ++t) pool.emplace_back(worker);
  for (auto& t : pool) t.join();
  for (int i = 0; i < n_pairs; ++i)
    if (st[i] != CPD_OK) return bail(fail(st[i], "pair " + std::to_string(i) + ": " + msg[i]));
  for (int i = 0; i < n_pairs; ++i)
    if (!b->ctx[i]) return bail(fail(CPD_ECUDA, "pair setup did not run (stream creation failed)"));

  // Work-item plan of the persistent kernel and the per-pair buffers it implies.
  b->pairs.assign((size_t)n_pairs, BatchPair{});
  for (int i = 0; i < n_pairs; ++i) {
    b->pairs[i].M = (int)M[i];
    b->pairs[i].N = (int)N[i];
    b->pairs[i].K = (int)b->ctx[i]->K;
  }
  cpd_status s;
  for (int i = 0; i < n_pairs; ++i)
    if ((s = batch_load_scene(b->ctx[i], N[i], Y[i])) != CPD_OK) return bail(s);
  if ((s = b->ctl.ensure(sizeof(BatchCtl))) != CPD_OK) return bail(s);
  if ((s = b->states.ensure(sizeof(DevState) * (size_t)n_pairs)) != CPD_OK) return bail(s);
  if ((s = batch_apply_plan(b, kBatchDefaultItems, kBatchDefaultProjKB)) != CPD_OK) return bail(s);
  for (int i = 0; i < n_pairs; ++i)
    if ((s = start_registration(b->ctx[i])) != CPD_OK) return bail(s);
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return bail(fail(CPD_ECUDA, "batch setup failed"));
  *out = b;
  return CPD_OK;
}

cpd_status cpd_batch_iterate(cpd_batch* b, int32_t n_iter) {
  g_err.clear();
  if (!b) return fail(CPD_EINVAL, "batch is NULL");
  if (n_iter < 0 || n_iter > (1 << 20)) return fail(CPD_EINVAL, "n_iter must be in [0, 2^20]");
  if (n_iter == 0) return CPD_OK;
  DeviceGuard guard(b->dev);
  const int extra = fault_enabled("barrier") ? 1 : 0;
  if (!b->graph || b->graph_iters != n_iter || b->graph_extra != extra) STATUS_TRY(batch_capture(b, n_iter, extra));
  CUDA_TRY(cudaGraphLaunch(b->graph, b->stream));
  BatchCtl& h = b->last;
  CUDA_TRY(cudaMemcpyAsync(&h, b->ctl.p, sizeof(BatchCtl), cudaMemcpyDeviceToHost, b->stream));
  CUDA_TRY(cudaStreamSynchronize(b->stream));
  b->last_iters = n_iter;
  if (h.status != 0)
    return fail((cpd_status)h.status, "a wait of the batched kernel for a pair's previous phase timed out (" +
                                          std::to_string(b->wait_s) + " s); the pairs' state is undefined until "
                                          "cpd_batch_reset" + (extra ? " (injected: CPD_FAULT=barrier)" : ""));
  return CPD_OK;
}

cpd_status cpd_batch_state(cpd_batch* b, double* sigma2, int32_t* iters, int32_t* device_status) {
  g_err.clear();
  if (!b) return fail(CPD_EINVAL, "batch is NULL");
  DeviceGuard guard(b->dev);
  std::vector<DevState> h((size_t)b->n);
  launch_batch_states(b->pairs_dev.as<BatchPair>(), b->n, b->states.as<DevState>(), b->stream);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemcpyAsync(h.data(), b->states.p, sizeof(DevState) * h.size(), cudaMemcpyDeviceToHost, b->stream));
  CUDA_TRY(cudaStreamSynchronize(b->stream));
  for (int i = 0; i < b->n; ++i) {
    if (sigma2) sigma2[i] = h[i].sigma2;
    if (iters) iters[i] = h[i].iter;
    if (device_status) device_status[i] = h[i].status;
  }
  return CPD_OK;
}

cpd_status cpd_batch_get_T(cpd_batch* b, int32_t i, void* T_out) {
  g_err.clear();
  if (!b || !T_out) return fail(CPD_EINVAL, "batch and T_out are required");
  if (i < 0 || i >= b->n) return fail(CPD_EINVAL, "pair index out of range");
  DeviceGuard guard(b->dev);
  cpd_ctx* c = b->ctx[i];
  return download_model(c, c->T4.p, T_out);
}

cpd_status cpd_batch_info(const cpd_batch* b, int32_t i, int64_t* M, int64_t* N, int64_t* K) {
  if (!b) return fail(CPD_EINVAL, "batch is NULL");
  if (i < 0 || i >= b->n) return fail(CPD_EINVAL, "pair index out of range");
  if (M) *M = b->ctx[i]->M;
  if (N) *N = b->ctx[i]->N;
  if (K) *K = b->ctx[i]->K;
  return CPD_OK;
}

cpd_status cpd_batch_launch_shape(const cpd_batch* b, int32_t* n_pairs, int32_t* grid, int32_t* n_items) {
  if (!b) return fail(CPD_EINVAL, "batch is NULL");
  if (n_pairs) *n_pairs = b->n;
  if (grid) *grid = b->grid;
  if (n_items) *n_items = b->n_items;
  return CPD_OK;
}

cpd_status cpd_batch_phase_ms(const cpd_batch* b, float* phase_ms) {
  if (!b || !phase_ms) return fail(CPD_EINVAL, "batch and phase_ms are required");
  if (b->last_iters < 1) return fail(CPD_ESTATE, "no batched call has completed yet");
  const int np = batch_phases();
  for (int ph = 0; ph < np; ++ph) {
    const double busy = (double)b->last.busy_ns[ph], wait = (double)b->last.wait_ns[ph];
    phase_ms[ph] = (float)(busy / (double)b->grid / 1e6 / b->last_iters);
    phase_ms[np + ph] = busy + wait > 0 ? (float)(busy / (busy + wait)) : 0.f;
  }
  return CPD_OK;
}

cpd_status cpd_batch_autotune(cpd_batch* b, int32_t n_iter, int32_t* e_items_out, int32_t* proj_kb_out,
                              float* ms_out) {
  g_err.clear();
  if (!b) return fail(CPD_EINVAL, "batch is NULL");
  if (n_iter < 1 || n_iter > 64) return fail(CPD_EINVAL, "n_iter must be in [1, 64]");
  DeviceGuard guard(b->dev);
  static const int cand[][2] = {{2, 256}, {2, 512}, {4, 256}, {4, 512}, {8, 256}, {8, 512}, {16, 256}, {16, 512}};
  const int nc = (int)(sizeof(cand) / sizeof(cand[0]));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CUDA_TRY(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(CPD_ECUDA, "cudaEventCreate failed");
  }
  cpd_status st = CPD_OK;
  float best = INFINITY;
  int bi = -1;
  for (int c = 0; c < nc && st == CPD_OK; ++c) {
    if ((st = batch_apply_plan(b, cand[c][0], cand[c][1])) != CPD_OK) break;
    if ((st = cpd_batch_reset(b)) != CPD_OK) break;
    if ((st = cpd_batch_iterate(b, n_iter)) != CPD_OK) break;       // capture + warm-up
    if ((st = cpd_batch_reset(b)) != CPD_OK) break;
    cudaEventRecord(e0, b->stream);
    if ((st = cpd_batch_iterate(b, n_iter)) != CPD_OK) break;
    cudaEventRecord(e1, b->stream);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms_out) ms_out[c] = ms;
    if (ms < best) { best = ms; bi = c; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != CPD_OK) return st;
  STATUS_TRY(batch_apply_plan(b, cand[bi][0], cand[bi][1]));
  STATUS_TRY(cpd_batch_reset(b));
  if (e_items_out) *e_items_out = cand[bi][0];
  if (proj_kb_out) *proj_kb_out = cand[bi][1];
  return CPD_OK;
}

cpd_status cpd_batch_reset(cpd_batch* b) {
  g_err.clear();
  if (!b) return fail(CPD_EINVAL, "batch is NULL");
  DeviceGuard guard(b->dev);
  for (cpd_ctx* c : b->ctx) STATUS_TRY(start_registration(c));
  // a launch that ended early (a barrier timeout) may have left tickets set
  CUDA_TRY(cudaMemsetAsync(b->tickets.p, 0, b->n_tickets * sizeof(unsigned int), b->stream));
  CUDA_TRY(cudaStreamSynchronize(b->stream));
  return CPD_OK;
}

void cpd_batch_destroy(cpd_batch* b) {
  if (!b) return;
  DeviceGuard guard(b->dev);
  cudaStreamSynchronize(b->stream);
  delete b;
}

}  // extern "C"
