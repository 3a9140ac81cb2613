// Throughput probe of the special-function unit's base-2 exponential, the
// unit that bounds the softmin epilogue (one ex2.approx per cell).  Each
// thread runs 8 independent chains x <- 2^-x (x stays in [0.5, 1), so no
// chain under- or overflows) entirely in registers; the result is written
// so that nothing is optimised away.  A measurement aid for the roofline,
// not part of the method.
#include "gw_internal.cuh"

namespace gw {
namespace {

constexpr int kProbeChains = 8;

__global__ void __launch_bounds__(512) probe_ex2_kernel(int iters, float* out) {
  float x[kProbeChains];
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) x[k] = 0.5f + 0.05f * k + 1e-6f * (threadIdx.x & 31);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
#pragma unroll
      for (int k = 0; k < kProbeChains; ++k) x[k] = ex2(-x[k]);
    }
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) s += x[k];
  out[static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace gw

extern "C" int gw_probe_ex2(int blocks, int iters, float* out, unsigned long long* h_ops,
                            gw_stream_t stream) {
  gw::set_error("");
  GW_REQUIRE(blocks >= 1 && blocks <= 65536 && iters >= 1 && iters <= (1 << 24), GW_EINVAL,
             "probe: blocks in [1, 65536], iters in [1, 2^24]");
  GW_REQUIRE(out != nullptr && h_ops != nullptr, GW_EINVAL, "probe: out and h_ops must not be NULL");
  gw::probe_ex2_kernel<<<blocks, 512, 0, reinterpret_cast<cudaStream_t>(stream)>>>(iters, out);
  GW_LAUNCH_CHECK();
  *h_ops = static_cast<unsigned long long>(blocks) * 512ull * static_cast<unsigned long long>(iters) *
           4ull * gw::kProbeChains;
  return GW_OK;
}
