// C-ABI entry points of libgw: validation, workspace layout and the CNT-GW
// solver loop (Algorithm 1 with Algorithm 3 as the inner Sinkhorn solver).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <mutex>
#include <vector>

#include "gw_internal.cuh"

namespace gw {

namespace {
thread_local char g_err[512] = {0};
}

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

const char* last_error() { return g_err; }

namespace {
std::atomic<unsigned long long> g_launches{0};
}

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

// ------------------------------------------------------------ bounded waits
// Every CTA of the tensor-core kernels whose pipeline wait gave up adds 1
// here (one counter per device).
__device__ unsigned int g_wait_gave_up = 0;

namespace {
std::atomic<unsigned long long> g_wait_limit_ns{2000000000ull};   // 2 s
constexpr int kMaxDevices = 64;
std::mutex g_gave_up_mu;
unsigned int* g_gave_up_ptr[kMaxDevices] = {nullptr};
}  // namespace

// The device address of this device's counter, looked up once per device
// (null when the lookup fails: the kernels then count nothing).
static unsigned int* gave_up_counter() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(g_gave_up_mu);
  if (g_gave_up_ptr[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_wait_gave_up) == cudaSuccess) {
      g_gave_up_ptr[dev] = static_cast<unsigned int*>(p);
    } else {
      cudaGetLastError();
    }
  }
  return g_gave_up_ptr[dev];
}

tc::WaitCtl wait_ctl() { return tc::WaitCtl{g_wait_limit_ns.load(), gave_up_counter()}; }

namespace {

bool prec_ok(int prec) { return prec >= GW_PREC_FP32 && prec <= GW_PREC_FP8; }

int check_eps(float eps) {
  GW_REQUIRE(eps > 0.0f && isfinite(eps), GW_EINVAL, "eps must be finite and > 0 (got %g)",
             static_cast<double>(eps));
  return GW_OK;
}

int check_dims(int64_t n, int64_t m, int D, int E) {
  GW_REQUIRE(n >= 0 && m >= 1, GW_EINVAL, "need n >= 0 and m >= 1 (got n=%lld m=%lld)",
             static_cast<long long>(n), static_cast<long long>(m));
  GW_REQUIRE(D >= 1 && E >= 1, GW_EINVAL, "need D, E >= 1 (got %d, %d)", D, E);
  GW_REQUIRE(D <= GW_MAX_FEATURES && E <= GW_MAX_FEATURES, GW_EUNSUPPORTED,
             "D, E must be <= %d (got %d, %d)", GW_MAX_FEATURES, D, E);
  GW_REQUIRE(n < (int64_t(1) << 40) && m < (int64_t(1) << 40), GW_EINVAL, "n, m too large");
  return GW_OK;
}

int check_prec(int prec) {
  GW_REQUIRE(prec >= GW_PREC_FP32 && prec <= GW_PREC_FP8, GW_EINVAL, "unknown precision %d",
             prec);
  GW_REQUIRE(prec_ok(prec), GW_EUNSUPPORTED, "precision %d is not supported", prec);
  return GW_OK;
}

#define NONNULL(p) GW_REQUIRE((p) != nullptr, GW_EINVAL, "%s must not be NULL", #p)

size_t solve_fixed_bytes(int64_t n, int64_t m, int D, int E) {
  Carver c(nullptr, ~size_t(0));
  c.take<float>(n);                 // log a
  c.take<float>(m);                 // log b
  c.take<float>(n);                 // f ping
  c.take<float>(n);                 // f pong
  c.take<float>(m);                 // g ping
  c.take<float>(m);                 // g pong
  c.take<float>(static_cast<size_t>(m) * D);  // V
  c.take<double>(static_cast<size_t>(D) * E); // Gamma cur
  c.take<double>(static_cast<size_t>(D) * E); // Gamma next
  c.take<double>(4);                // C
  c.take<double>(GW_EN_LEN);        // scratch energy record
  c.take<double>(kMargBlocks);      // stop-rule partials
  c.take<double>(2);                // stop-rule Err
  c.take<unsigned>(1);              // give-up counter as the call began
  return c.used();
}

size_t iteration_ws_bytes(int64_t n, int64_t m, int K, int prec);

size_t solve_ws_bytes(int64_t n, int64_t m, int D, int E, int prec) {
  const size_t inner = iteration_ws_bytes(n, m, D, prec);
  size_t step = energy_ws_bytes(n, m, D, E, prec);
  const size_t mom = moments_ws_bytes(n, m, D, E);
  if (mom > step) step = mom;
  return solve_fixed_bytes(n, m, D, E) + (inner > step ? inner : step) + 256;
}

size_t iteration_ws_bytes(int64_t n, int64_t m, int K, int prec) {
  return softmin_ws_bytes(n, m, K, prec) + softmin_ws_bytes(m, n, K, prec) + 512;
}

// One iteration (both half-steps), shared by gw_solve and gw_sinkhorn_iteration.
int launch_iteration(const float* X, const float* V, const float* s, const float* t,
                     const float* loga, const float* logb, const float* f, const float* g,
                     float* f_out, float* g_out, float eps, int64_t n, int64_t m, int K, int prec,
                     bool symmetric, bool reuse, char* ws, size_t ws_bytes, cudaStream_t st) {
  Carver sub(ws, ws_bytes);
  SoftminTask row{}, col{};
  row.A = X;
  row.B = V;
  row.sA = s;
  row.sB = t;
  row.h = g;
  row.logw = logb;
  row.est = f;      // the row log-sum-exp is close to -f / eps
  row.n = n;
  row.m = m;
  row.K = K;
  row.eps = eps;
  col.A = V;
  col.B = X;
  col.sA = t;
  col.sB = s;
  col.logw = loga;
  col.est = g;
  col.n = m;
  col.m = n;
  col.K = K;
  col.eps = eps;
  // within an outer step only the potentials change: the tensor-core form
  // keeps its 16-bit operands and refreshes the bias columns
  row.reuse_ops = col.reuse_ops = reuse ? 1 : 0;
  if (symmetric) {
    // Algorithm 3: both halves read iterate n, then average.
    row.avg_with = f;
    row.out = f_out;
    col.h = f;
    col.avg_with = g;
    col.out = g_out;
    SoftminTask both[2] = {row, col};
    return launch_softmin(both, 2, prec, sub, st);
  }
  // Algorithm 2: f from g^n, then g from f^{n+1}.
  row.avg_with = nullptr;
  row.out = f_out;
  GW_TRY(launch_softmin(&row, 1, prec, sub, st));
  // the column task keeps its own operands beside the row task's
  const size_t off = (softmin_ws_bytes(n, m, K, prec) + 255) & ~size_t(255);
  Carver sub2(ws + off, ws_bytes - off);
  col.h = f_out;
  col.avg_with = nullptr;
  col.out = g_out;
  return launch_softmin(&col, 1, prec, sub2, st);
}

struct SolveBufs {
  float *loga, *logb, *f[2], *g[2], *V;
  double *G[2], *C, *en, *mpart, *merr;
  unsigned* gave_up0;
};

// read one device double (the stream is drained first)
int read_back(const double* d, double* h, cudaStream_t st) {
  GW_CUDA_TRY(cudaMemcpyAsync(h, d, sizeof(double), cudaMemcpyDeviceToHost, st));
  GW_CUDA_TRY(cudaStreamSynchronize(st));
  return GW_OK;
}

int enqueue_solve(const gw_problem& p, const gw_options& o, const gw_result& r, void* ws,
                  size_t ws_bytes, cudaStream_t st, bool replay = false) {
  Carver c(ws, ws_bytes);
  SolveBufs B;
  B.loga = c.take<float>(p.n);
  B.logb = c.take<float>(p.m);
  B.f[0] = c.take<float>(p.n);
  B.f[1] = c.take<float>(p.n);
  B.g[0] = c.take<float>(p.m);
  B.g[1] = c.take<float>(p.m);
  B.V = c.take<float>(static_cast<size_t>(p.m) * p.D);
  B.G[0] = c.take<double>(static_cast<size_t>(p.D) * p.E);
  B.G[1] = c.take<double>(static_cast<size_t>(p.D) * p.E);
  B.C = c.take<double>(4);
  B.en = c.take<double>(GW_EN_LEN);
  B.mpart = c.take<double>(kMargBlocks);
  B.merr = c.take<double>(2);
  B.gave_up0 = c.take<unsigned>(1);
  GW_TRY(check_ws(c, ws));
  const size_t mark = c.used();
  char* base = static_cast<char*>(ws);

  const size_t DE = static_cast<size_t>(p.D) * p.E;
  // the records report GW_ETIMEOUT when the give-up counter moves during the call
  const unsigned* counter = wait_ctl().gave_up;
  if (counter) {
    GW_CUDA_TRY(cudaMemcpyAsync(B.gave_up0, counter, sizeof(unsigned), cudaMemcpyDeviceToDevice, st));
  } else {
    B.gave_up0 = nullptr;
  }
  GW_TRY(launch_log(p.a, p.n, B.loga, st));
  GW_TRY(launch_log(p.b, p.m, B.logb, st));
  if (o.f0) {
    GW_CUDA_TRY(cudaMemcpyAsync(B.f[0], o.f0, sizeof(float) * p.n, cudaMemcpyDeviceToDevice, st));
  } else {
    GW_CUDA_TRY(cudaMemsetAsync(B.f[0], 0, sizeof(float) * p.n, st));
  }
  if (o.g0) {
    GW_CUDA_TRY(cudaMemcpyAsync(B.g[0], o.g0, sizeof(float) * p.m, cudaMemcpyDeviceToDevice, st));
  } else {
    GW_CUDA_TRY(cudaMemsetAsync(B.g[0], 0, sizeof(float) * p.m, st));
  }
  if (o.Gamma0) {
    GW_CUDA_TRY(cudaMemcpyAsync(B.G[0], o.Gamma0, sizeof(double) * DE, cudaMemcpyDeviceToDevice, st));
  } else {
    GW_CUDA_TRY(cudaMemsetAsync(B.G[0], 0, sizeof(double) * DE, st));
  }
  {
    Carver sub(base + mark, ws_bytes - mark);
    GW_TRY(run_moments(p.X, p.a, p.n, p.D, p.Y, p.b, p.m, p.E, B.C, sub, st));
  }

  const bool stop_rule = o.stop_tol > 0.0f;
  const int cap = o.n_inner_max > o.n_inner ? o.n_inner_max : o.n_inner;
  int n_cur = o.n_inner;   // Algorithm 6: the count of the coming outer step
  double E_prev = 0.0;
  int fc = 0, gc = 0, Gc = 0;
  for (int t = 0; t < o.n_outer; ++t) {
    // position in the eps schedule (a resumed solve continues its schedule)
    const int T_all = o.outer_total > 0 ? o.outer_total : o.n_outer;
    const int t_all = (o.outer_total > 0 ? o.outer_offset : 0) + t;
    float eps = o.eps;
    if (o.eps_final > 0.0f && o.eps_final != o.eps && T_all > 1) {
      eps = static_cast<float>(static_cast<double>(o.eps) *
                               pow(static_cast<double>(o.eps_final) / o.eps,
                                   static_cast<double>(t_all) / (T_all - 1)));
    }
    char label[64];
    snprintf(label, sizeof(label), "gw outer step %d (eps %.3g)", t, static_cast<double>(eps));
    NvtxRange range(label);
    // Zbar_j <- Gamma_t Y_j (Algorithm 1)
    GW_TRY(launch_gamma_y(B.G[Gc], p.Y, p.m, p.D, p.E, B.V, st));
    int n_run = n_cur;
    bool checked = false;
    auto iterate = [&](bool reuse) -> int {
      GW_TRY(launch_iteration(p.X, B.V, p.s, p.t, B.loga, B.logb, B.f[fc], B.g[gc], B.f[fc ^ 1],
                              B.g[gc ^ 1], eps, p.n, p.m, p.D, o.prec, o.symmetric != 0, reuse,
                              base + mark, ws_bytes - mark, st));
      fc ^= 1;
      gc ^= 1;
      return GW_OK;
    };
    int it0 = 0;
    if (replay && !stop_rule && n_cur >= 3) {
      // the first iteration prepares the outer step's operands; the others
      // differ only in which potential buffers they read and write, so an
      // even number of them (f, g back in the buffers they started in) is
      // captured once and replayed
      GW_TRY(iterate(false));
      const int left = n_cur - 1;
      const int body = left >= 20 ? 10 : 2;
      cudaGraph_t graph = nullptr;
      GW_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
      int rc = GW_OK;
      for (int k = 0; k < body && rc == GW_OK; ++k) rc = iterate(true);
      const cudaError_t ec = cudaStreamEndCapture(st, &graph);
      if (rc != GW_OK || ec != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        if (rc != GW_OK) return rc;
        set_error("iteration graph capture failed: %s", cudaGetErrorString(ec));
        return GW_ECUDA;
      }
      cudaGraphExec_t exec = nullptr;
      const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      GW_REQUIRE(ei == cudaSuccess, GW_ECUDA, "iteration graph instantiate failed: %s",
                 cudaGetErrorString(ei));
      cudaError_t el = cudaSuccess;
      for (int k = 0; k < left / body && el == cudaSuccess; ++k) el = cudaGraphLaunch(exec, st);
      cudaGraphExecDestroy(exec);
      GW_REQUIRE(el == cudaSuccess, GW_ECUDA, "iteration graph launch failed: %s",
                 cudaGetErrorString(el));
      it0 = 1 + (left / body) * body;
    }
    for (int it = it0; it < n_cur; ++it) {
      GW_TRY(iterate(it > 0));
      if (stop_rule && (it + 1) % o.stop_every == 0) {
        // hybrid stop: Err of the plan this iteration measured
        GW_TRY(run_marginal_error(B.f[fc ^ 1], B.f[fc], p.a, p.n, B.g[gc ^ 1], B.g[gc], p.b, p.m,
                                  eps, o.symmetric != 0, B.mpart, B.merr, st));
        checked = true;
        double err = 0.0;
        GW_TRY(read_back(B.merr, &err, st));
        if (err < static_cast<double>(o.stop_tol)) {
          n_run = it + 1;
          break;
        }
      }
    }
    // Xtilde and Gamma_{t+1} of Algorithm 1, plus the energy record
    PlanArgs pa;
    pa.X = p.X;
    pa.Y = p.Y;
    pa.s = p.s;
    pa.t = p.t;
    pa.a = p.a;
    pa.b = p.b;
    pa.f = B.f[fc];
    pa.g = B.g[gc];
    pa.Gamma_t = B.G[Gc];
    pa.eps = eps;
    pa.n = p.n;
    pa.m = p.m;
    pa.D = p.D;
    pa.E = p.E;
    Carver sub(base + mark, ws_bytes - mark);
    const bool last = t == o.n_outer - 1;
    if (o.record || last || o.adaptive) {
      double* rec = (o.record && r.history) ? r.history + static_cast<size_t>(t) * GW_EN_LEN : B.en;
      GW_TRY(run_energy(pa, o.prec, B.C, B.logb, rec, B.G[Gc ^ 1], sub, st));
      GW_TRY(launch_record_extra(rec, n_run, checked ? B.merr : nullptr, B.gave_up0, st));
      if (o.adaptive) {
        // Algorithm 6: an energy increase means Sinkhorn was not converged
        double E = 0.0;
        GW_TRY(read_back(rec + GW_EN_E, &E, st));
        if (t > 0 && E > E_prev + static_cast<double>(o.adapt_rtol) * fabs(E_prev))
          n_cur = 2 * n_cur < cap ? 2 * n_cur : cap;
        E_prev = E;
      }
      if (last) {
        GW_CUDA_TRY(cudaMemcpyAsync(r.energy, rec, sizeof(double) * GW_EN_LEN,
                                    cudaMemcpyDeviceToDevice, st));
      }
    } else {
      GW_TRY(run_cross_cov(pa, o.prec, B.G[Gc ^ 1], nullptr, nullptr, sub, st));
    }
    Gc ^= 1;
  }
  GW_CUDA_TRY(cudaMemcpyAsync(r.Gamma, B.G[Gc], sizeof(double) * DE, cudaMemcpyDeviceToDevice, st));
  if (r.Gamma_plan) {
    GW_CUDA_TRY(cudaMemcpyAsync(r.Gamma_plan, B.G[Gc ^ 1], sizeof(double) * DE,
                                cudaMemcpyDeviceToDevice, st));
  }
  GW_CUDA_TRY(cudaMemcpyAsync(r.f, B.f[fc], sizeof(float) * p.n, cudaMemcpyDeviceToDevice, st));
  GW_CUDA_TRY(cudaMemcpyAsync(r.g, B.g[gc], sizeof(float) * p.m, cudaMemcpyDeviceToDevice, st));
  return GW_OK;
}

}  // namespace

}  // namespace gw

using namespace gw;

extern "C" {

const char* gw_last_error(void) { return gw::last_error(); }

int gw_version(void) { return 100; }

unsigned long long gw_kernel_launches(int reset) {
  return reset ? g_launches.exchange(0) : g_launches.load();
}

int gw_set_wait_limit_ns(unsigned long long ns) {
  gw::set_error("");
  GW_REQUIRE(ns >= 1 && ns <= 600000000000ull, GW_EINVAL,
             "wait limit must be in [1 ns, 600 s] (got %llu)", ns);
  g_wait_limit_ns.store(ns);
  return GW_OK;
}

unsigned long long gw_wait_limit_ns(void) { return g_wait_limit_ns.load(); }

int gw_wait_status(int reset) {
  gw::set_error("");
  unsigned int* p = gave_up_counter();
  GW_REQUIRE(p != nullptr, GW_ECUDA, "the give-up counter of this device is not reachable");
  GW_CUDA_TRY(cudaDeviceSynchronize());
  unsigned int v = 0;
  GW_CUDA_TRY(cudaMemcpy(&v, p, sizeof(v), cudaMemcpyDeviceToHost));
  if (reset) GW_CUDA_TRY(cudaMemset(p, 0, sizeof(unsigned int)));
  if (v != 0) {
    gw::set_error("%u CTA(s) gave up a bounded wait", v);
    return GW_ETIMEOUT;
  }
  return GW_OK;
}

size_t gw_workspace_size(int op, int64_t n, int64_t m, int D, int E, int prec) {
  if (n < 0 || m < 1 || D < 1 || E < 1 || D > GW_MAX_FEATURES || E > GW_MAX_FEATURES) return 0;
  switch (op) {
    case GW_OP_SOFTMIN: return softmin_ws_bytes(n, m, D, prec) + 256;
    case GW_OP_CROSS_COV: return cross_cov_ws_bytes(n, m, D, E, prec) + 256;
    case GW_OP_ENERGY: return energy_ws_bytes(n, m, D, E, prec) + 256;
    case GW_OP_SOLVE: return solve_ws_bytes(n, m, D, E, prec);
    case GW_OP_LIFT: return lift_ws_bytes(n, D) + 256;   /* (n points, D features) */
    case GW_OP_GRAD: return grad_ws_bytes(n, m, D, E, 4, prec) + 256;
    case GW_OP_COARSEN: return n >= 1 ? coarsen_ws_bytes(n, m, D) + 256 : 0;   /* (n points, m = k) */
    case GW_OP_ITERATION: return iteration_ws_bytes(n, m, D, prec);
    default: return 0;
  }
}

int gw_sinkhorn_softmin(const float* A, const float* B, const float* sA, const float* sB,
                        const float* h, const float* logw, float eps, int64_t n, int64_t m,
                        int K, int prec, const float* avg_with, float* out, void* ws,
                        size_t ws_bytes, gw_stream_t stream) {
  gw::set_error("");
  GW_TRY(check_eps(eps));
  GW_TRY(check_dims(n, m, K, 1));
  GW_TRY(check_prec(prec));
  if (n == 0) return GW_OK;
  NONNULL(A);
  NONNULL(B);
  NONNULL(sA);
  NONNULL(sB);
  NONNULL(h);
  NONNULL(logw);
  NONNULL(out);
  Carver c(ws, ws_bytes);
  SoftminTask T{};
  T.A = A;
  T.B = B;
  T.sA = sA;
  T.sB = sB;
  T.h = h;
  T.logw = logw;
  T.avg_with = avg_with;
  T.est = avg_with;   // the previous potential doubles as the shift estimate
  T.out = out;
  T.n = n;
  T.m = m;
  T.K = K;
  T.eps = eps;
  GW_REQUIRE(ws_bytes == 0 || reinterpret_cast<uintptr_t>(ws) % 256 == 0, GW_ENOMEM,
             "workspace must be 256-byte aligned");
  return launch_softmin(&T, 1, prec, c, reinterpret_cast<cudaStream_t>(stream));
}

static int check_plan_args(const float* X, const float* Y, const float* s, const float* t,
                           const float* a, const float* b, const float* f, const float* g,
                           const double* Gamma_t, float eps, int64_t n, int64_t m, int D, int E,
                           int prec) {
  GW_TRY(check_eps(eps));
  GW_TRY(check_dims(n, m, D, E));
  GW_REQUIRE(n >= 1, GW_EINVAL, "n must be >= 1");
  GW_TRY(check_prec(prec));
  NONNULL(X);
  NONNULL(Y);
  NONNULL(s);
  NONNULL(t);
  NONNULL(a);
  NONNULL(b);
  NONNULL(f);
  NONNULL(g);
  NONNULL(Gamma_t);
  return GW_OK;
}

int gw_cross_cov(const float* X, const float* Y, const float* s, const float* t,
                 const float* a, const float* b, const float* f, const float* g,
                 const double* Gamma_t, float eps, int64_t n, int64_t m, int D, int E,
                 int prec, double* Gamma_out, double* stats, double* W_opt, void* ws,
                 size_t ws_bytes, gw_stream_t stream) {
  gw::set_error("");
  GW_TRY(check_plan_args(X, Y, s, t, a, b, f, g, Gamma_t, eps, n, m, D, E, prec));
  NONNULL(Gamma_out);
  NONNULL(stats);
  Carver c(ws, ws_bytes);
  GW_REQUIRE(reinterpret_cast<uintptr_t>(ws) % 256 == 0, GW_ENOMEM,
             "workspace must be 256-byte aligned");
  PlanArgs pa{X, Y, s, t, a, b, f, g, Gamma_t, eps, n, m, D, E};
  return run_cross_cov(pa, prec, Gamma_out, stats, W_opt, c,
                       reinterpret_cast<cudaStream_t>(stream));
}

int gw_energy(const float* X, const float* Y, const float* s, const float* t, const float* a,
              const float* b, const float* f, const float* g, const double* Gamma_t, float eps,
              int64_t n, int64_t m, int D, int E, int prec, double* energy, double* Gamma_out,
              void* ws, size_t ws_bytes, gw_stream_t stream) {
  gw::set_error("");
  GW_TRY(check_plan_args(X, Y, s, t, a, b, f, g, Gamma_t, eps, n, m, D, E, prec));
  NONNULL(energy);
  Carver c(ws, ws_bytes);
  GW_REQUIRE(reinterpret_cast<uintptr_t>(ws) % 256 == 0, GW_ENOMEM,
             "workspace must be 256-byte aligned");
  PlanArgs pa{X, Y, s, t, a, b, f, g, Gamma_t, eps, n, m, D, E};
  return run_energy(pa, prec, nullptr, nullptr, energy, Gamma_out, c,
                    reinterpret_cast<cudaStream_t>(stream));
}

int gw_solve(const gw_problem* p, const gw_options* o, gw_result* r, void* ws, size_t ws_bytes,
             gw_stream_t stream) {
  gw::set_error("");
  NONNULL(p);
  NONNULL(o);
  NONNULL(r);
  GW_TRY(check_dims(p->n, p->m, p->D, p->E));
  GW_REQUIRE(p->n >= 1, GW_EINVAL, "n must be >= 1");
  GW_TRY(check_eps(o->eps));
  GW_REQUIRE(o->eps_final <= 0.0f || isfinite(o->eps_final), GW_EINVAL, "eps_final not finite");
  GW_REQUIRE(o->n_outer >= 1 && o->n_inner >= 1, GW_EINVAL, "n_outer, n_inner must be >= 1");
  GW_REQUIRE(o->n_outer <= 100000 && o->n_inner <= 1000000, GW_EINVAL, "iteration counts too large");
  GW_TRY(check_prec(o->prec));
  // the FP8 softmin needs plan sums on the same rounded features (tensor-core plan, D + 3 <= 80)
  GW_REQUIRE(o->prec != GW_PREC_FP8 || plan_tc_supported(p->D, o->prec), GW_EUNSUPPORTED,
             "GW_PREC_FP8 solves need D + 3 <= 80 (D = %d); the FP8 softmin alone takes D <= 128",
             p->D);
  NONNULL(p->X);
  NONNULL(p->Y);
  NONNULL(p->s);
  NONNULL(p->t);
  NONNULL(p->a);
  NONNULL(p->b);
  NONNULL(r->Gamma);
  NONNULL(r->f);
  NONNULL(r->g);
  NONNULL(r->energy);
  GW_REQUIRE(!o->record || r->history != nullptr, GW_EINVAL, "record = 1 needs result.history");
  GW_REQUIRE(o->n_inner_max <= 1000000, GW_EINVAL, "n_inner_max too large");
  GW_REQUIRE(o->adapt_rtol >= 0.0f && isfinite(o->adapt_rtol), GW_EINVAL, "adapt_rtol must be >= 0");
  GW_REQUIRE(!(o->stop_tol > 0.0f) || (isfinite(o->stop_tol) && o->stop_every >= 1), GW_EINVAL,
             "stop_tol > 0 needs a finite tolerance and stop_every >= 1");
  GW_REQUIRE(o->outer_total <= 0 ||
                 (o->outer_offset >= 0 && o->outer_offset + o->n_outer <= o->outer_total),
             GW_EINVAL, "outer_offset %d + n_outer %d must lie within outer_total %d",
             o->outer_offset, o->n_outer, o->outer_total);
  const size_t need = solve_ws_bytes(p->n, p->m, p->D, p->E, o->prec);
  GW_REQUIRE(ws != nullptr && ws_bytes >= need, GW_ENOMEM,
             "workspace too small: need %zu bytes, have %zu", need, ws_bytes);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  (void)wait_ctl();   // looks the counter up outside any capture
  NvtxRange range("gw_solve");
  const bool host_driven = o->adaptive || o->stop_tol > 0.0f;
  if (!o->use_graph || st == nullptr || host_driven) return enqueue_solve(*p, *o, *r, ws, ws_bytes, st);
  if (o->use_graph == 2) return enqueue_solve(*p, *o, *r, ws, ws_bytes, st, true);

  cudaGraph_t graph = nullptr;
  GW_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  const int rc = enqueue_solve(*p, *o, *r, ws, ws_bytes, st);
  const cudaError_t ec = cudaStreamEndCapture(st, &graph);
  if (rc != GW_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (ec != cudaSuccess) {
    gw::set_error("graph capture failed: %s", cudaGetErrorString(ec));
    if (graph) cudaGraphDestroy(graph);
    return GW_ECUDA;
  }
  cudaGraphExec_t exec = nullptr;
  cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess) {
    gw::set_error("graph instantiate failed: %s", cudaGetErrorString(ei));
    return GW_ECUDA;
  }
  cudaError_t el = cudaGraphLaunch(exec, st);
  cudaGraphExecDestroy(exec);
  if (el != cudaSuccess) {
    gw::set_error("graph launch failed: %s", cudaGetErrorString(el));
    return GW_ECUDA;
  }
  return GW_OK;
}

int gw_lift(const float* x, int64_t n, int d, const float* w, int kind, float param, int D,
            int n_iter, uint64_t seed, float* X, float* sqn, float* basis_opt,
            float* eigvals_opt, void* ws, size_t ws_bytes, gw_stream_t stream) {
  gw::set_error("");
  NONNULL(x);
  NONNULL(X);
  NONNULL(sqn);
  GW_REQUIRE(n >= 2, GW_EINVAL, "gw_lift needs n >= 2 points (got %lld)", static_cast<long long>(n));
  GW_REQUIRE(d >= 1 && d <= 4, GW_EUNSUPPORTED, "gw_lift takes points of dimension 1..4 (got %d)", d);
  GW_REQUIRE(D >= 1 && D <= GW_MAX_FEATURES, GW_EUNSUPPORTED, "D must be in [1, %d]", GW_MAX_FEATURES);
  GW_REQUIRE(kind == GW_PEN_SQEUCLID || kind == GW_PEN_POWER || kind == GW_PEN_GAUSS, GW_EINVAL,
             "unknown penalty %d", kind);
  GW_REQUIRE(kind != GW_PEN_POWER || (param > 0.0f && param <= 2.0f), GW_EINVAL,
             "power penalty needs 0 < p <= 2 (got %g)", static_cast<double>(param));
  GW_REQUIRE(kind != GW_PEN_GAUSS || param > 0.0f, GW_EINVAL, "gaussian penalty needs sigma > 0");
  GW_REQUIRE(n_iter >= 0 && n_iter <= 10000, GW_EINVAL, "n_iter out of range");
  return run_lift(x, n, d, w, kind, param, D, n_iter, seed, X, sqn, basis_opt, eigvals_opt, ws,
                  ws_bytes, reinterpret_cast<cudaStream_t>(stream));
}

int gw_grad_x(const gw_problem* p, const float* f, const float* g, const double* Gamma_t,
              const double* Gamma_pi, float eps, int prec, const float* x, int dx_dim, int kind,
              float param, const float* basis, const float* eigvals, float* dX, float* dx,
              void* ws, size_t ws_bytes, gw_stream_t stream) {
  gw::set_error("");
  NONNULL(p);
  GW_TRY(check_dims(p->n, p->m, p->D, p->E));
  GW_REQUIRE(p->n >= 1, GW_EINVAL, "n must be >= 1");
  GW_TRY(check_eps(eps));
  GW_TRY(check_prec(prec));
  NONNULL(p->X);
  NONNULL(p->Y);
  NONNULL(p->s);
  NONNULL(p->t);
  NONNULL(p->a);
  NONNULL(p->b);
  NONNULL(f);
  NONNULL(g);
  NONNULL(Gamma_t);
  NONNULL(dX);
  if (x != nullptr) {
    GW_REQUIRE(dx_dim >= 1 && dx_dim <= 4, GW_EUNSUPPORTED, "points of dimension 1..4 (got %d)", dx_dim);
    NONNULL(dx);
    NONNULL(basis);
    NONNULL(eigvals);
    GW_REQUIRE(kind == GW_PEN_SQEUCLID || kind == GW_PEN_POWER || kind == GW_PEN_GAUSS, GW_EINVAL,
               "unknown penalty %d", kind);
  } else {
    dx_dim = 0;
  }
  const size_t need = grad_ws_bytes(p->n, p->m, p->D, p->E, dx_dim, prec);
  GW_REQUIRE(ws != nullptr && ws_bytes >= need, GW_ENOMEM,
             "workspace too small: need %zu bytes, have %zu", need, ws_bytes);
  return run_grad(*p, f, g, Gamma_t, Gamma_pi, eps, prec, x, dx_dim, kind, param, basis, eigvals,
                  dX, dx, ws, ws_bytes, reinterpret_cast<cudaStream_t>(stream));
}

int gw_sinkhorn_iteration(const float* X, const float* V, const float* s, const float* t,
                          const float* loga, const float* logb, const float* f, const float* g,
                          float* f_out, float* g_out, float eps, int64_t n, int64_t m, int K,
                          int prec, int symmetric, int reuse, void* ws, size_t ws_bytes,
                          gw_stream_t stream) {
  gw::set_error("");
  GW_TRY(check_eps(eps));
  GW_TRY(check_dims(n, m, K, 1));
  GW_TRY(check_prec(prec));
  GW_REQUIRE(n >= 1, GW_EINVAL, "n must be >= 1");
  NONNULL(X);
  NONNULL(V);
  NONNULL(s);
  NONNULL(t);
  NONNULL(loga);
  NONNULL(logb);
  NONNULL(f);
  NONNULL(g);
  NONNULL(f_out);
  NONNULL(g_out);
  GW_REQUIRE(f_out != f && g_out != g, GW_EINVAL, "f_out / g_out must not alias f / g");
  const size_t need = iteration_ws_bytes(n, m, K, prec);
  GW_REQUIRE(ws != nullptr && ws_bytes >= need && reinterpret_cast<uintptr_t>(ws) % 256 == 0,
             GW_ENOMEM, "workspace too small or unaligned: need %zu bytes, have %zu", need, ws_bytes);
  return launch_iteration(X, V, s, t, loga, logb, f, g, f_out, g_out, eps, n, m, K, prec,
                          symmetric != 0, reuse != 0, static_cast<char*>(ws), ws_bytes,
                          reinterpret_cast<cudaStream_t>(stream));
}

int gw_coarsen(const float* X, const float* a, int64_t n, int D, const int64_t* init_idx,
               int64_t k, int n_iter, float* Xc, float* ac, float* sc, int* assign,
               int64_t* h_k_out, void* ws, size_t ws_bytes, gw_stream_t stream) {
  gw::set_error("");
  NONNULL(X);
  NONNULL(init_idx);
  NONNULL(Xc);
  NONNULL(ac);
  NONNULL(sc);
  NONNULL(h_k_out);
  GW_REQUIRE(n >= 1 && k >= 1 && k <= n, GW_EINVAL, "need 1 <= k <= n");
  GW_REQUIRE(D >= 1 && D <= GW_MAX_FEATURES, GW_EUNSUPPORTED, "D must be in [1, %d]", GW_MAX_FEATURES);
  GW_REQUIRE(n_iter >= 0 && n_iter <= 10000, GW_EINVAL, "n_iter out of range");
  Carver c(ws, ws_bytes);
  GW_REQUIRE(reinterpret_cast<uintptr_t>(ws) % 256 == 0, GW_ENOMEM, "workspace must be 256-byte aligned");
  return run_coarsen(X, a, n, D, init_idx, k, n_iter, Xc, ac, sc, assign, h_k_out, c,
                     reinterpret_cast<cudaStream_t>(stream));
}

size_t gw_transfer_workspace_size(int64_t n, int64_t m, int D, int k) {
  if (n < 1 || m < 1 || D < 1 || D > GW_MAX_FEATURES || k < 1 || k > 16) return 0;
  return transfer_ws_bytes(n, m, D, k);
}

int gw_transfer(const gw_problem* p, const float* f, const float* g, const double* Gamma_t,
                float eps, const float* U, int k, float* out, float* mass, void* ws,
                size_t ws_bytes, gw_stream_t stream) {
  gw::set_error("");
  NONNULL(p);
  GW_TRY(check_dims(p->n, p->m, p->D, p->E));
  GW_REQUIRE(p->n >= 1, GW_EINVAL, "n must be >= 1");
  GW_TRY(check_eps(eps));
  GW_REQUIRE(k >= 1 && k <= 16, GW_EUNSUPPORTED, "k must be in [1, 16] (got %d)", k);
  NONNULL(p->X);
  NONNULL(p->Y);
  NONNULL(p->s);
  NONNULL(p->t);
  NONNULL(p->a);
  NONNULL(p->b);
  NONNULL(f);
  NONNULL(g);
  NONNULL(Gamma_t);
  NONNULL(U);
  NONNULL(out);
  GW_REQUIRE(reinterpret_cast<uintptr_t>(ws) % 256 == 0, GW_ENOMEM, "workspace must be 256-byte aligned");
  Carver c(ws, ws_bytes);
  return run_transfer(*p, f, g, Gamma_t, eps, U, k, out, mass, c,
                      reinterpret_cast<cudaStream_t>(stream));
}

size_t gw_kernel_gw_workspace_size(int64_t n, int64_t m) {
  if (n < 1 || m < 1) return 0;
  return kernel_gw_ws_bytes(n, m);
}

int gw_kernel_gw(const float* CX, const float* CY, const float* a, const float* b, int64_t n,
                 int64_t m, const gw_options* o, float* pi, float* f, float* g, double* energy,
                 double* history, void* ws, size_t ws_bytes, gw_stream_t stream) {
  gw::set_error("");
  NONNULL(CX);
  NONNULL(CY);
  NONNULL(a);
  NONNULL(b);
  NONNULL(o);
  NONNULL(pi);
  NONNULL(f);
  NONNULL(g);
  NONNULL(energy);
  GW_REQUIRE(n >= 1 && m >= 1, GW_EINVAL, "n, m must be >= 1");
  GW_TRY(check_eps(o->eps));
  GW_REQUIRE(o->eps_final <= 0.0f || isfinite(o->eps_final), GW_EINVAL, "eps_final not finite");
  GW_REQUIRE(o->n_outer >= 1 && o->n_inner >= 1, GW_EINVAL, "n_outer, n_inner must be >= 1");
  GW_REQUIRE(!o->record || history != nullptr, GW_EINVAL, "record = 1 needs history");
  const size_t need = kernel_gw_ws_bytes(n, m);
  GW_REQUIRE(ws != nullptr && ws_bytes >= need, GW_ENOMEM,
             "workspace too small: need %zu bytes, have %zu", need, ws_bytes);
  return run_kernel_gw(CX, CY, a, b, n, m, *o, pi, f, g, energy, history, ws, ws_bytes,
                       reinterpret_cast<cudaStream_t>(stream));
}

size_t gw_sgw_workspace_size(int64_t n, int64_t m, int D, int E, int prec, int want_grad,
                             int dx_dim) {
  if (n < 1 || m < 1 || D < 1 || E < 1 || D > GW_MAX_FEATURES || E > GW_MAX_FEATURES) return 0;
  return sgw_ws_bytes(n, m, D, E, prec, want_grad != 0, want_grad ? dx_dim : 0);
}

int gw_sgw(const gw_problem* p, const gw_options* o, double* sgw, double* records, float* dX,
           const float* x, int dx_dim, int kind, float param, const float* basis,
           const float* eigvals, float* dx, void* ws, size_t ws_bytes, gw_stream_t stream) {
  gw::set_error("");
  NONNULL(p);
  NONNULL(o);
  NONNULL(sgw);
  GW_TRY(check_dims(p->n, p->m, p->D, p->E));
  GW_REQUIRE(p->n >= 1 && p->m >= 1, GW_EINVAL, "n, m must be >= 1");
  if (dX != nullptr && x != nullptr) {
    GW_REQUIRE(dx_dim >= 1 && dx_dim <= 4, GW_EUNSUPPORTED, "points of dimension 1..4 (got %d)", dx_dim);
    NONNULL(dx);
    NONNULL(basis);
    NONNULL(eigvals);
    GW_REQUIRE(kind == GW_PEN_SQEUCLID || kind == GW_PEN_POWER || kind == GW_PEN_GAUSS, GW_EINVAL,
               "unknown penalty %d", kind);
  }
  const int dxd = (dX != nullptr && x != nullptr) ? dx_dim : 0;
  const size_t need = sgw_ws_bytes(p->n, p->m, p->D, p->E, o->prec, dX != nullptr, dxd);
  GW_REQUIRE(ws != nullptr && ws_bytes >= need, GW_ENOMEM,
             "workspace too small: need %zu bytes, have %zu", need, ws_bytes);
  return run_sgw(*p, *o, sgw, records, dX, dxd ? x : nullptr, dxd, kind, param, basis, eigvals,
                 dx, ws, ws_bytes, reinterpret_cast<cudaStream_t>(stream));
}

size_t gw_solve_batch_workspace_size(void) { return batch_ws_bytes(); }

int gw_solve_batch(int nprob, const int64_t* xo, const int64_t* yo, int64_t n_max, int64_t m_max,
                   int D, int E, const float* X, const float* Y, const float* s, const float* t,
                   const float* a, const float* b, const float* eps0, const float* eps1,
                   int n_outer, int n_inner, int symmetric, float* f, float* g, double* Gamma,
                   double* Gamma_plan, double* energy, double* history, void* ws,
                   size_t ws_bytes, gw_stream_t stream) {
  gw::set_error("");
  GW_REQUIRE(nprob >= 1, GW_EINVAL, "nprob must be >= 1 (got %d)", nprob);
  NONNULL(xo);
  NONNULL(yo);
  NONNULL(X);
  NONNULL(Y);
  NONNULL(s);
  NONNULL(t);
  NONNULL(a);
  NONNULL(b);
  NONNULL(eps0);
  NONNULL(f);
  NONNULL(g);
  NONNULL(Gamma);
  NONNULL(Gamma_plan);
  NONNULL(energy);
  GW_REQUIRE(D >= 1 && D <= 4 && E >= 1 && E <= 4, GW_EUNSUPPORTED,
             "the batched solver takes feature widths 1..4 (got D=%d, E=%d)", D, E);
  GW_REQUIRE(n_max >= 1 && m_max >= 1 && n_max <= (1 << 20) && m_max <= (1 << 20), GW_EINVAL,
             "n_max, m_max must be in 1..2^20");
  GW_REQUIRE(n_outer >= 1 && n_inner >= 1, GW_EINVAL, "n_outer, n_inner must be >= 1");
  GW_REQUIRE(n_outer <= 100000 && n_inner <= 1000000, GW_EINVAL, "iteration counts too large");
  return run_solve_batch(nprob, xo, yo, n_max, m_max, D, E, X, Y, s, t, a, b, eps0, eps1, n_outer,
                         n_inner, symmetric != 0 ? 1 : 0, f, g, Gamma, Gamma_plan, energy, history,
                         ws, ws_bytes, reinterpret_cast<cudaStream_t>(stream));
}

size_t gw_multiscale_workspace_size(int64_t n, int64_t m, int D, int E, int64_t kx, int64_t ky,
                                    int prec) {
  if (n < 1 || m < 1 || kx < 1 || ky < 1 || D < 1 || E < 1) return 0;
  return multiscale_ws_bytes(n, m, D, E, kx, ky, prec);
}

int gw_multiscale(const gw_problem* p, const gw_options* coarse, const gw_options* fine,
                  const int64_t* init_x, int64_t kx, const int64_t* init_y, int64_t ky,
                  int km_iter, gw_result* r, double* coarse_energy, void* ws, size_t ws_bytes,
                  gw_stream_t stream) {
  gw::set_error("");
  NONNULL(p);
  NONNULL(coarse);
  NONNULL(fine);
  NONNULL(r);
  NONNULL(init_x);
  NONNULL(init_y);
  GW_TRY(check_dims(p->n, p->m, p->D, p->E));
  GW_REQUIRE(kx >= 1 && kx <= p->n && ky >= 1 && ky <= p->m, GW_EINVAL, "need 1 <= kx <= n, 1 <= ky <= m");
  GW_TRY(check_eps(coarse->eps));
  GW_TRY(check_eps(fine->eps));
  GW_TRY(check_prec(coarse->prec));
  GW_TRY(check_prec(fine->prec));
  GW_REQUIRE(coarse->n_outer >= 1 && coarse->n_inner >= 1 && fine->n_outer >= 1 && fine->n_inner >= 1,
             GW_EINVAL, "iteration counts must be >= 1");
  GW_REQUIRE(!fine->record || r->history != nullptr, GW_EINVAL, "record = 1 needs result.history");
  const size_t need = multiscale_ws_bytes(p->n, p->m, p->D, p->E, kx, ky,
                                          fine->prec > coarse->prec ? fine->prec : coarse->prec);
  GW_REQUIRE(ws != nullptr && ws_bytes >= need, GW_ENOMEM,
             "workspace too small: need %zu bytes, have %zu", need, ws_bytes);
  return run_multiscale(*p, *coarse, *fine, init_x, kx, init_y, ky, km_iter, *r, coarse_energy, ws,
                        ws_bytes, reinterpret_cast<cudaStream_t>(stream));
}

}  // extern "C"
