// cpd_estep_noalloc: the E-step of cpd_estep for callers that must not
// allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they need an
// E-step: loops that must not stall on the implicit device synchronisation
// cudaMalloc/cudaFree can cause, programs that reserve all device memory up
// front under a fixed budget (a cudaMalloc there fails or evicts memory
// another component owns), and allocator-free runtimes that hand this
// library only the arrays they already own.  This variant therefore takes
// all of its scratch -- the 4-vector copies of the points, the split partial
// sums of passes A and B, the flag lists and the small device state -- from
// one statically sized device array that the library holds for its lifetime
// on every GPU that loads it, and it calls no allocating routine.
//
// The call reads its result back to the host and synchronises `stream`
// before it returns, so it cannot be made while a stream is being captured
// into a CUDA graph.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <string>

#include "common.cuh"

using namespace fcpd;

namespace {

// 24 MiB: enough for M, N <= 32768 with the E-step's partial-sum layout.
constexpr size_t kScratchBytes = (size_t)24 << 20;
constexpr int64_t kMaxPoints = 32768;
constexpr int kMaxDevices = 64;

// The array itself.  In host code `g_noalloc_scratch` names a host-side
// stand-in, not device memory; its device address is looked up once per
// device with cudaGetSymbolAddress (below) and only that address is passed
// to kernels.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

cpd_status fail(cpd_status s, const std::string& m) {
  set_last_error(m);     // reported by cpd_last_error()
  return s;
}

// Device address of the scratch array on the current device, resolved on the
// first call per device (that call must not run under stream capture).
cpd_status scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return fail(CPD_EINVAL, "device index out of range");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return fail(CPD_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return CPD_OK;
}

// True for device (or managed) memory of device `dev`: the kernels read the
// arrays directly, so memory of another GPU is refused as well.
bool on_device(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

// Bump allocator over the static array (256-byte aligned pieces).
struct Carve {
  unsigned char* base;
  size_t used = 0;
  template <typename T> T* take(size_t count) {
    const size_t off = (used + 255) & ~(size_t)255;
    used = off + count * sizeof(T);
    return reinterpret_cast<T*>(base + off);
  }
};

}  // namespace

extern "C" cpd_status cpd_estep_noalloc(const void* T, int64_t M, const void* Y, int64_t N, double sigma2, double w,
                                        void* Ytil_out, void* P1_out, void* den_out, double* sums_out,
                                        void* stream) {
  set_last_error("");
  if (!T || !Y || !Ytil_out) return fail(CPD_EINVAL, "T, Y and Ytil_out are required");
  if (M < 1 || N < 1 || M > kMaxPoints || N > kMaxPoints)
    return fail(CPD_EINVAL, "cpd_estep_noalloc supports 1 <= M, N <= 32768 (its scratch is a fixed 24 MiB array)");
  if (!(sigma2 > 0.0) || !std::isfinite(sigma2)) return fail(CPD_EINVAL, "sigma2 must be > 0");
  if (!(w >= 0.0 && w < 1.0)) return fail(CPD_EINVAL, "w must satisfy 0 <= w < 1");
  cudaStream_t s = (cudaStream_t)stream;
  // An error left by an earlier, unrelated call on this thread is not this
  // call's: discard it, unless it is sticky (the context is unusable).
  if (cudaGetLastError() != cudaSuccess && cudaPeekAtLastError() != cudaSuccess)
    return fail(CPD_ECUDA, "the CUDA context is in an error state from an earlier call");
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return fail(CPD_ECUDA, "no CUDA device");
  if (!on_device(T, dev) || !on_device(Y, dev) || !on_device(Ytil_out, dev) || (P1_out && !on_device(P1_out, dev)) ||
      (den_out && !on_device(den_out, dev)))
    return fail(CPD_EINVAL, "cpd_estep_noalloc takes arrays in the memory of the current device only (staging "
                            "host data or copying from another GPU would need memory)");
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return fail(CPD_ECUDA, "cannot query the SM count");
  void* base = nullptr;
  cpd_status st = scratch_address(dev, &base);
  if (st != CPD_OK) return st;

  // The E-step plan splits the long dimension over the resident blocks of
  // `sms` SMs, so its partial sums grow with the SM count and the occupancy.
  // If they do not fit, plan for fewer SMs (fewer, longer chunks: the same
  // sums in a different order); with one SM every M, N <= 32768 fits.
  EstepPlan pl{};
  Carve c{static_cast<unsigned char*>(base)};
  DevState* ds = nullptr;
  float4 *T4 = nullptr, *Y4 = nullptr, *Yb = nullptr, *Yt4 = nullptr;
  float *partA = nullptr, *partB = nullptr;
  double *sums = nullptr, *P1 = nullptr, *den = nullptr;
  int* flags = nullptr;
  for (int plan_sms = sms;; plan_sms = plan_sms / 2) {
    pl = plan_estep(M, N, false, std::max(plan_sms, 1));
    c.used = 0;
    ds = c.take<DevState>(1);
    T4 = c.take<float4>((size_t)M);
    Y4 = c.take<float4>((size_t)N);
    Yb = c.take<float4>((size_t)N);
    Yt4 = c.take<float4>((size_t)M);
    partA = c.take<float>((size_t)pl.partA_elems);
    partB = c.take<float>((size_t)pl.partB_elems);
    sums = c.take<double>((size_t)pl.sums_elems);
    flags = c.take<int>((size_t)pl.flags_elems);
    P1 = c.take<double>((size_t)M);
    den = c.take<double>((size_t)N);
    if (c.used <= kScratchBytes) break;
    if (plan_sms <= 1)
      return fail(CPD_EINVAL, "these sizes need " + std::to_string(c.used) + " bytes of scratch, more than the "
                              "24 MiB static array; use cpd_estep");
  }

  // Everything that must start from zero (the device state: counters and
  // tickets) is initialised here; every other piece is fully overwritten.
  launch_pack<float>(static_cast<const float*>(T), M, T4, false, s);
  launch_pack<float>(static_cast<const float*>(Y), N, Y4, true, s);
  launch_state_init(ds, sigma2, s);
  launch_state_params(ds, w, 1.0, 0.0, 0.0, 0, nullptr, M, N, 0, s);
  launch_estep<float>(pl, T4, nullptr, M, Y4, Yb, N, partA, partB, sums, flags, Yt4, nullptr, P1, den, ds, false, s);
  launch_unpack<float>(Yt4, M, static_cast<float*>(Ytil_out), s);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(CPD_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
  if (P1_out && cudaMemcpyAsync(P1_out, P1, (size_t)M * sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return fail(CPD_ECUDA, "copy of P1 failed");
  if (den_out && cudaMemcpyAsync(den_out, den, (size_t)N * sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return fail(CPD_ECUDA, "copy of den failed");
  DevState h;
  if (cudaMemcpyAsync(&h, ds, sizeof(DevState), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return fail(CPD_ECUDA, "reading the device state failed");
  if (sums_out) {
    sums_out[0] = h.vsum;
    sums_out[1] = h.loglik;
  }
  if (h.status != 0) return fail((cpd_status)h.status, "device reported a numeric failure");
  return CPD_OK;
}
