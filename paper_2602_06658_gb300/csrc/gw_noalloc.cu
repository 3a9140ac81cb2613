// gw_sinkhorn_softmin_noalloc: the softmin for callers that cannot allocate
// device memory.
//
// Some callers can't call cudaMalloc, or hand this library a workspace:
// runtimes that reserve all device memory up front and forbid allocation
// afterwards, host code that runs where an allocation's implicit device
// synchronisation is not allowed, and plug-in hosts that expose no allocator
// to their plug-ins.  For them this file keeps the softmin's scratch (the
// per-split running (max, sum) pairs) in one file-scope __device__ array of
// kStaticScratchBytes.  Every GPU that loads the library holds that array
// until the process exits.
#include <math.h>

#include <mutex>

#include "gw_internal.cuh"

namespace gw {
namespace {

// 2 MiB: the partials of every shape up to n ~ 131k source points when the
// column range is split, and of any shape that does not split.
constexpr size_t kStaticScratchBytes = size_t(2) << 20;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 256;
std::mutex g_scratch_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the static array on the current device.  In host code
// the symbol g_static_scratch is only a host-side stand-in, not a device
// address, so it is looked up once per device with that device current and
// cached.
int static_scratch(void** out) {
  int dev = -1;
  GW_CUDA_TRY(cudaGetDevice(&dev));
  GW_REQUIRE(dev >= 0 && dev < kMaxDevices, GW_EUNSUPPORTED, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (g_scratch_ptr[dev] == nullptr) {
    void* p = nullptr;
    GW_CUDA_TRY(cudaGetSymbolAddress(&p, g_static_scratch));
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return GW_OK;
}

}  // namespace
}  // namespace gw

extern "C" int gw_sinkhorn_softmin_noalloc(const float* A, const float* B, const float* sA,
                                           const float* sB, const float* h, const float* logw,
                                           float eps, int64_t n, int64_t m, int K, int prec,
                                           const float* avg_with, float* out,
                                           gw_stream_t stream) {
  using namespace gw;
  set_error("");
  GW_REQUIRE(eps > 0.0f && isfinite(eps), GW_EINVAL, "eps must be finite and > 0 (got %g)",
             static_cast<double>(eps));
  GW_REQUIRE(n >= 0 && m >= 1, GW_EINVAL, "need n >= 0 and m >= 1");
  GW_REQUIRE(K >= 1, GW_EINVAL, "need K >= 1 (got %d)", K);
  GW_REQUIRE(K <= GW_MAX_FEATURES, GW_EUNSUPPORTED, "K must be <= %d (got %d)", GW_MAX_FEATURES, K);
  GW_REQUIRE(n < (int64_t(1) << 40) && m < (int64_t(1) << 40), GW_EINVAL, "n, m too large");
  GW_REQUIRE(prec == GW_PREC_FP32, GW_EUNSUPPORTED, "precision %d is not available here", prec);
  if (n == 0) return GW_OK;
  GW_REQUIRE(A && B && sA && sB && h && logw && out, GW_EINVAL, "null input or output pointer");
  const size_t need = softmin_ws_bytes(n, m, K, prec);
  GW_REQUIRE(need <= kStaticScratchBytes, GW_ENOMEM,
             "n=%lld, m=%lld needs %zu bytes of scratch; the static scratch array holds %zu",
             static_cast<long long>(n), static_cast<long long>(m), need, kStaticScratchBytes);
  void* scratch = nullptr;
  GW_TRY(static_scratch(&scratch));
  // The kernels write every partial they later read, so nothing in the
  // array has to start at zero.
  Carver c(scratch, kStaticScratchBytes);
  SoftminTask T{};
  T.A = A;
  T.B = B;
  T.sA = sA;
  T.sB = sB;
  T.h = h;
  T.logw = logw;
  T.avg_with = avg_with;
  T.est = nullptr;
  T.out = out;
  T.n = n;
  T.m = m;
  T.K = K;
  T.eps = eps;
  return launch_softmin(&T, 1, prec, c, reinterpret_cast<cudaStream_t>(stream));
}
