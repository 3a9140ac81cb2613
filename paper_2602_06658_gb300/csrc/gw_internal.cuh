// Internal helpers shared by the libgw translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include <nvtx3/nvToolsExt.h>

#include "gw.h"

namespace gw {

// Tracing: a named NVTX range on the host thread for the scope's lifetime
// (an outer step of a solve, a lift, a server request).  The ranges mark
// where the host enqueues the work (inside a stream capture: where the graph
// is built); profilers correlate them with the kernels they launch.  Without
// a profiler attached the calls do nothing.
struct NvtxRange {
  explicit NvtxRange(const char* msg) { nvtxRangePushA(msg); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;
constexpr float kNegBig = -1.0e30f;   // "minus infinity" that keeps exp2(x - m) finite
constexpr int kSmCount = 152;         // GB300

// ---------------------------------------------------------------- errors
void set_error(const char* fmt, ...);
const char* last_error();

#define GW_REQUIRE(cond, code, ...)      \
  do {                                   \
    if (!(cond)) {                       \
      ::gw::set_error(__VA_ARGS__);      \
      return (code);                     \
    }                                    \
  } while (0)

#define GW_CUDA_TRY(call)                                                      \
  do {                                                                         \
    cudaError_t e_ = (call);                                                   \
    if (e_ != cudaSuccess) {                                                   \
      ::gw::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                      __FILE__, __LINE__);                                     \
      return GW_ECUDA;                                                         \
    }                                                                          \
  } while (0)

// Every kernel launch site calls GW_LAUNCH_CHECK() once, which also counts
// the launch (gw_kernel_launches()).
void count_launch();
#define GW_LAUNCH_CHECK()          \
  do {                             \
    ::gw::count_launch();          \
    GW_CUDA_TRY(cudaGetLastError()); \
  } while (0)

#define GW_TRY(expr)          \
  do {                        \
    int rc_ = (expr);         \
    if (rc_ != GW_OK) return rc_; \
  } while (0)

// ------------------------------------------------------------ workspace
// Bump allocator over the caller's workspace.  With base == nullptr it only
// measures, so gw_workspace_size() and the entry points share one layout.
struct Carver {
  char* base;
  size_t cap;
  size_t off = 0;
  bool overflow = false;
  Carver(void* b, size_t c) : base(static_cast<char*>(b)), cap(c) {}
  template <class T>
  T* take(size_t count) {
    size_t o = (off + 255) & ~size_t(255);
    off = o + count * sizeof(T);
    if (off > cap) overflow = true;
    return base ? reinterpret_cast<T*>(base + o) : nullptr;
  }
  size_t used() const { return (off + 255) & ~size_t(255); }
};

inline int check_ws(const Carver& c, void* ws) {
  GW_REQUIRE(reinterpret_cast<uintptr_t>(ws) % 256 == 0, GW_ENOMEM,
             "workspace must be 256-byte aligned");
  GW_REQUIRE(!c.overflow, GW_ENOMEM, "workspace too small: need %zu bytes, have %zu", c.used(),
             c.cap);
  return GW_OK;
}

// --------------------------------------------------------- bounded waits
namespace tc {
// Limit of the pipeline waits of one launch (nanoseconds of %globaltimer)
// and the device counter a CTA increments when one of its waits gave up
// (null: not counted).
struct WaitCtl {
  uint64_t limit_ns;
  unsigned int* gave_up;
};
}  // namespace tc
// The current limit (gw_set_wait_limit_ns) and this device's give-up counter.
tc::WaitCtl wait_ctl();

// ------------------------------------------------------------ device math
__device__ __forceinline__ float ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

inline int ceil_div(int64_t a, int64_t b) { return static_cast<int>((a + b - 1) / b); }

// ------------------------------------------------------------ softmin plan
// One softmin task: out_i = -eps LSE_j[logw_j + (h_j + 16<A_i,B_j> + 4 sA_i sB_j)/eps].
struct SoftminTask {
  const float* A;
  const float* B;
  const float* sA;
  const float* sB;
  const float* h;
  const float* logw;
  const float* avg_with;
  const float* est; // previous potential of the output side (shift estimate) or null
  float* out;
  float* pm;        // partial maxima  [splits][n] (base 2), used when splits > 1
  float* ps;        // partial sums    [splits][n]
  int64_t n, m;
  int K;
  int splits;       // column splits
  int cols_per_split;
  float eps;
  // tensor-core form: the 16-bit operands already in the workspace (same
  // carve position, same A, B, sA, sB, eps and precision) are still valid
  // apart from the bias and shift columns, which are refreshed
  int reuse_ops;
};

// Shape decisions of the softmin kernels (identical for sizing and launch).
struct SoftminShape {
  int rows_per_block;
  int row_blocks;
  int splits;
  int cols_per_split;
};
SoftminShape softmin_shape(int64_t n, int64_t m, int K, int prec);
size_t softmin_ws_bytes(int64_t n, int64_t m, int K, int prec);

// Tensor-core form (gw_softmin_tc.cu): support test, workspace and launch
// (fills splits / pm / ps of the tasks; the caller merges the partials).
bool softmin_tc_supported(int K, int prec);
size_t softmin_tc_ws_bytes(int64_t n, int64_t m, int K, int prec);
int launch_softmin_tc(SoftminTask* tasks, int ntasks, int prec, Carver& ws, cudaStream_t st);

// Launch one or two softmin tasks (two = the row and column half-steps of a
// symmetric Sinkhorn iteration in a single launch).  Partials come from the
// carver.  Host-side only; the tasks must already be validated.
int launch_softmin(SoftminTask* tasks, int ntasks, int prec, Carver& ws, cudaStream_t st);

// ------------------------------------------------------------ plan kernels
struct PlanArgs {
  const float* X;  // n x D
  const float* Y;  // m x E
  const float* s;
  const float* t;
  const float* a;
  const float* b;
  const float* f;
  const float* g;
  const double* Gamma_t;  // D x E
  float eps;
  int64_t n, m;
  int D, E;
};

// V = Gamma Y (m x D, float32) from a float64 Gamma.
int launch_gamma_y(const double* Gamma, const float* Y, int64_t m, int D, int E, float* V,
                   cudaStream_t st);

size_t cross_cov_ws_bytes(int64_t n, int64_t m, int D, int E, int prec);
// Gamma_out (D x E), stats[8], W (m x (D+2), float64; carved if W == nullptr)
int run_cross_cov(const PlanArgs& p, int prec, double* Gamma_out, double* stats, double* W,
                  Carver& ws, cudaStream_t st);

// Adjoint (gw_grad.cu)
size_t grad_ws_bytes(int64_t n, int64_t m, int D, int E, int dx_dim, int prec);
int run_grad(const gw_problem& p, const float* f, const float* g, const double* Gamma_t,
             const double* Gamma_pi, float eps, int prec, const float* x, int dx_dim, int kind,
             float param, const float* basis, const float* eigvals, float* dX, float* dx,
             void* ws, size_t ws_bytes, cudaStream_t st);

size_t moments_ws_bytes(int64_t n, int64_t m, int D, int E);
// C(alpha, beta) into *C (device)
int run_moments(const float* X, const float* a, int64_t n, int D, const float* Y, const float* b,
                int64_t m, int E, double* C, Carver& ws, cudaStream_t st);

size_t energy_ws_bytes(int64_t n, int64_t m, int D, int E, int prec);
// Full energy record.  C (device scalar) and log b are precomputed when
// C_pre / logb_pre are non-null.
int run_energy(const PlanArgs& p, int prec, const double* C_pre, const float* logb_pre,
               double* energy, double* Gamma_out, Carver& ws, cudaStream_t st);

// Persistent batched solver (gw_batch.cu); arguments as gw_solve_batch.
size_t batch_ws_bytes();
// Problems of up to n_max + m_max points at feature width D fit one CTA.
bool batch_fits(int64_t n_max, int64_t m_max, int D);
int run_solve_batch(int nprob, const int64_t* xo, const int64_t* yo, int64_t n_max, int64_t m_max,
                    int D, int E, const float* X, const float* Y, const float* s, const float* t,
                    const float* a, const float* b, const float* eps0, const float* eps1,
                    int n_outer, int n_inner, int symmetric, float* f, float* g, double* Gamma,
                    double* Gamma_plan, double* energy, double* history, void* ws,
                    size_t ws_bytes, cudaStream_t st);

// Kernel PCA / centering lift (gw_lift.cu); synchronous.
size_t lift_ws_bytes(int64_t n, int D);
// Its N x N block product Z = C P on the tensor cores (gw_lift_tc.cu):
// prepare once per point set (coordinate table and cost scale), then one
// matvec per block; Zp receives `splits` partials [splits][n][RP].
struct LiftTcBufs {
  float* xt;
  uint16_t *Ph, *Pl;
  unsigned *qmax, *r2;
  float *uinv, *scal;
  int splits;
};
LiftTcBufs carve_lift_tc(Carver& c, int64_t n, int RP);
int lift_tc_prepare(const float* x, int64_t n, int d, int kind, float param, int RP,
                    LiftTcBufs& B, cudaStream_t st);
int lift_tc_matvec(const float* P, int64_t n, int d, int kind, float param, int RP,
                   LiftTcBufs& B, float* Zp, cudaStream_t st);
int run_lift(const float* x, int64_t n, int d, const float* w, int kind, float param, int D,
             int n_iter, uint64_t seed, float* X, float* sqn, float* basis, float* eigvals,
             void* ws, size_t ws_bytes, cudaStream_t st);

// Stop rule of the Sinkhorn loop: Err of the last measured plan from two
// consecutive iterates (gw_plan.cu); `part` holds kMargBlocks doubles.
constexpr int kMargBlocks = 152;
int run_marginal_error(const float* f0, const float* f1, const float* a, int64_t n,
                       const float* g0, const float* g1, const float* b, int64_t m, float eps,
                       bool symmetric, double* part, double* out, cudaStream_t st);
// rec[GW_EN_NINNER], rec[GW_EN_STOPERR] (err may be null: -1); with
// gave_up0 (the device's give-up counter as the call began) the status
// becomes GW_ETIMEOUT when the counter moved since
int launch_record_extra(double* rec, int n_inner, const double* err, const unsigned* gave_up0,
                        cudaStream_t st);

// Plan-weighted column sums on the tensor cores (gw_plan_tc.cu): Wp partials
// [splits][m][D + 2] of W_j = sum_i pi_ij [X_i, s_i, 1]; *flag_out is set on
// the device when the FP32 kernel has to recompute them.
bool plan_tc_supported(int D, int prec);
size_t plan_tc_ws_bytes(int64_t n, int64_t m, int D, int prec);
// Ep_out (or null): the KL partials [splits][m][2] of the energy
// (A_j = sum_i pi_ij log2(pi_ij / b_j), B_j = sum_i pi_ij log a_i).
int run_plan_tc(const PlanArgs& p, int prec, const float* V, float** Wp_out, float** Ep_out,
                int* splits_out, int* rows_per_split_out, int** flag_out, Carver& ws,
                cudaStream_t st);

// Color / UV transfer (gw_transfer.cu)
size_t transfer_ws_bytes(int64_t n, int64_t m, int D, int k);
int run_transfer(const gw_problem& p, const float* f, const float* g, const double* Gamma_t,
                 float eps, const float* U, int k, float* out, float* mass, Carver& ws,
                 cudaStream_t st);

// Dense FP32-accuracy product on the tensor cores (gw_gemm_tc.cu):
// out[r][s] = scale sum_k A[s][k] Bt[r][k] + coef u[r] v[s] (out R x S
// row-major; A logical S x K stored row-major, or K x S when a_trans; Bt
// logical R x K, or K x R when b_trans; u, v may be null).
size_t gemm_tc_ws_bytes(int64_t S, int64_t R, int64_t K);
int gemm_tc_f16x3(const float* A, bool a_trans, const float* Bt, bool b_trans, int64_t S,
                  int64_t R, int64_t K, float scale, const float* u, const float* v, float coef,
                  float* out, Carver& ws, cudaStream_t st);

// Kernel-GW exact mode (gw_kernelgw.cu)
size_t kernel_gw_ws_bytes(int64_t n, int64_t m);
int run_kernel_gw(const float* CX, const float* CY, const float* a, const float* b, int64_t n,
                  int64_t m, const gw_options& o, float* pi_out, float* f_out, float* g_out,
                  double* energy, double* history, void* ws, size_t ws_bytes, cudaStream_t st);

// SGW divergence (gw_sgw.cu)
size_t sgw_ws_bytes(int64_t n, int64_t m, int D, int E, int prec, bool grad, int dx_dim);
int run_sgw(const gw_problem& p, const gw_options& o, double* out, double* records, float* dX,
            const float* x, int dx_dim, int kind, float param, const float* basis,
            const float* eigvals, float* dx, void* ws, size_t ws_bytes, cudaStream_t st);

// K-Means coarsening and Multiscale-GW (gw_multiscale.cu)
size_t coarsen_ws_bytes(int64_t n, int64_t k, int D);
int run_coarsen(const float* X, const float* a, int64_t n, int D, const int64_t* init_idx,
                int64_t k, int n_iter, float* Xc, float* ac, float* sc, int* assign_out,
                int64_t* k_out, Carver& ws, cudaStream_t st);
size_t multiscale_ws_bytes(int64_t n, int64_t m, int D, int E, int64_t kx, int64_t ky, int prec);
int run_multiscale(const gw_problem& p, const gw_options& oc, const gw_options& of,
                   const int64_t* init_x, int64_t kx, const int64_t* init_y, int64_t ky,
                   int km_iter, gw_result& r, double* coarse_energy, void* ws, size_t ws_bytes,
                   cudaStream_t st);

// logw_i = log(w_i)
int launch_log(const float* w, int64_t n, float* logw, cudaStream_t st);

}  // namespace gw
