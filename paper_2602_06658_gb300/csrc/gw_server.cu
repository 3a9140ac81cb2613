// Continuous-batching request server for CNT-GW solves.
//
// Requests (two point clouds, a penalty, eps and iteration counts) arrive
// at any time.  A scheduler thread admits a pending request as soon as a
// worker slot is free and its device memory fits in the caller's pool (a
// first-fit allocator over one caller-provided device buffer: the server
// allocates no device memory).  Each admitted request is driven by its own
// worker thread on its own CUDA stream: copy in, lift (Kernel PCA or
// centering), the solve captured as one CUDA graph, copy the energy record
// out.  With time slicing (gw_server_set_slice) a request runs a few outer
// steps per admission and, when others wait, is checkpointed to host memory
// and queued again; it resumes from that state later.  Admitted requests therefore overlap on the device, and requests that
// arrive while others run join as soon as a slot and memory free up.
// Kernels are deterministic and each request owns its memory, so a result
// does not depend on what else is running.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "gw_internal.cuh"

namespace gw {
namespace {

constexpr double kSmallCells = 8.0e6;   // N*M below which requests run the FP32 kernels


double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over [0, cap) in 256-byte units.
class Pool {
 public:
  Pool(char* base, size_t cap) : base_(base), cap_(cap) { free_[0] = cap; }
  char* alloc(size_t bytes) {
    bytes = (bytes + 255) & ~size_t(255);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        const size_t off = it->first, len = it->second;
        free_.erase(it);
        if (len > bytes) free_[off + bytes] = len - bytes;
        used_[off] = bytes;
        return base_ + off;
      }
    }
    return nullptr;
  }
  void release(char* p) {
    const size_t off = static_cast<size_t>(p - base_);
    auto u = used_.find(off);
    if (u == used_.end()) return;
    size_t len = u->second;
    used_.erase(u);
    size_t start = off;
    auto nx = free_.lower_bound(off);
    if (nx != free_.end() && nx->first == off + len) {
      len += nx->second;
      free_.erase(nx);
    }
    auto pv = free_.lower_bound(off);
    if (pv != free_.begin()) {
      --pv;
      if (pv->first + pv->second == off) {
        start = pv->first;
        len += pv->second;
        free_.erase(pv);
      }
    }
    free_[start] = len;
  }
  size_t capacity() const { return cap_; }

 private:
  char* base_;
  size_t cap_;
  std::map<size_t, size_t> free_;
  std::map<size_t, size_t> used_;
};

struct Job {
  gw_request req;
  std::vector<float> x, y;
  double t_submit = 0.0, t_admit = 0.0;
  size_t bytes = 0;
  char* mem = nullptr;   // device memory from the pool while admitted
  // checkpoint of a preempted request (host copies): lifted features and
  // the solver state after outer_done outer steps
  int outer_done = 0;
  int preempted = 0;
  int stop_code = 0;     // GW_ECANCELED / GW_ETIMEOUT once asked to stop
  std::vector<float> X, Y, s, t, f, g;
  std::vector<double> G;
};

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Below ~8e6 cells an iteration of the tensor-core forms is bound by its
// ~10 small launches (operand refresh, two passes, merges); the FP32 kernels
// are faster there and at least as accurate.  The one rule for the
// precision a request runs in (sizing and solve).
bool small_request(const gw_request& r) {
  return static_cast<double>(r.n) * static_cast<double>(r.m) < kSmallCells;
}
int run_prec(const gw_request& r) { return small_request(r) ? GW_PREC_FP32 : r.prec; }

// Device bytes a request needs (inputs, features, state, the larger of the
// lift and solve workspaces, the solve's sized for the precision it runs in).
size_t request_bytes(const gw_request& r) {
  const int D = r.kind == GW_PEN_SQEUCLID ? r.d : r.D;
  size_t b = 0;
  b += align256(sizeof(float) * r.n * r.d) + align256(sizeof(float) * r.m * r.d);   // x, y
  b += align256(sizeof(float) * r.n) * 2 + align256(sizeof(float) * r.m) * 2;       // a, s / b, t
  b += align256(sizeof(float) * r.n * D) + align256(sizeof(float) * r.m * D);       // X, Y
  b += align256(sizeof(float) * r.n) + align256(sizeof(float) * r.m);               // f, g
  b += 2 * align256(sizeof(double) * D * D) + align256(sizeof(double) * GW_EN_LEN);  // Gamma x2, energy
  size_t ws = gw_workspace_size(GW_OP_SOLVE, r.n, r.m, D, D, run_prec(r));
  if (r.kind != GW_PEN_SQEUCLID) {
    ws = std::max(ws, gw_workspace_size(GW_OP_LIFT, r.n, r.n, D, r.d, GW_PREC_FP32));
    ws = std::max(ws, gw_workspace_size(GW_OP_LIFT, r.m, r.m, D, r.d, GW_PREC_FP32));
  }
  return b + align256(ws) + 4096;
}

__global__ void fill_kernel(float* p, int64_t n, float v) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

// ------------------------------------------------------------ batch lane
// Small squared-penalty requests (the lift is a centering, D = d <= 4) go to
// the persistent batched solver: the requests waiting when the lane is free
// are solved in one gw_solve_batch launch, one CTA per request, on the lane's
// own stream and thread (no worker slot).  One SM solves such a request in
// about 0.1 s at 20 x 50 iterations; the lane keeps them off the slots the
// large requests queue for.  A request's path depends on the request alone,
// and the batched solver's result does not depend on the batch, so a result
// is the same alone and in the mix.
constexpr double kBatchCells = 1.5e6;     // n m at most
constexpr int kBatchMax = 2 * kSmCount;   // requests per launch

bool batchable(const gw_request& r) {
  return r.kind == GW_PEN_SQEUCLID && r.d <= 4 &&
         static_cast<double>(r.n) * static_cast<double>(r.m) <= kBatchCells &&
         batch_fits(r.n, r.m, r.d);
}

struct BatchJob {
  std::vector<Job*> members;
  int d = 0, n_outer = 0, n_inner = 0;
  int64_t n_max = 0, m_max = 0;
  size_t bytes = 0;
  char* mem = nullptr;
};

// Device layout of a batch (carved in this order; nullptr base: sizing).
struct BatchBufs {
  float *x, *y, *X, *Y, *s, *t, *a, *b, *f, *g, *eps0, *eps1;
  int64_t *xo, *yo;
  double *G, *Gp, *en;
  char* ws;
};

BatchBufs carve_batch(Carver& c, int64_t SN, int64_t SM, int Q, int d) {
  BatchBufs B;
  B.x = c.take<float>(static_cast<size_t>(SN) * d);
  B.y = c.take<float>(static_cast<size_t>(SM) * d);
  B.X = c.take<float>(static_cast<size_t>(SN) * d);
  B.Y = c.take<float>(static_cast<size_t>(SM) * d);
  B.s = c.take<float>(SN);
  B.t = c.take<float>(SM);
  B.a = c.take<float>(SN);
  B.b = c.take<float>(SM);
  B.f = c.take<float>(SN);
  B.g = c.take<float>(SM);
  B.eps0 = c.take<float>(Q);
  B.eps1 = c.take<float>(Q);
  B.xo = c.take<int64_t>(Q + 1);
  B.yo = c.take<int64_t>(Q + 1);
  B.G = c.take<double>(static_cast<size_t>(Q) * d * d);
  B.Gp = c.take<double>(static_cast<size_t>(Q) * d * d);
  B.en = c.take<double>(static_cast<size_t>(Q) * GW_EN_LEN);
  B.ws = c.take<char>(batch_ws_bytes());
  return B;
}

// Centering of each problem's cloud (the lift of the squared penalty with
// uniform weights): X_i = x_i - mean, s_i = ||X_i||^2, a_i = 1 / n; one block
// per problem, the mean summed in FP64 in a fixed order.
__global__ void batch_center_kernel(const float* x, const int64_t* off, int d, float* X,
                                    float* sq, float* w) {
  __shared__ double red[256][4];
  __shared__ double mean[4];
  const int q = blockIdx.x;
  const int64_t i0 = off[q], i1 = off[q + 1];
  const int64_t n = i1 - i0;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x)
    for (int k = 0; k < d; ++k) acc[k] += static_cast<double>(x[i * d + k]);
  for (int k = 0; k < 4; ++k) red[threadIdx.x][k] = acc[k];
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (static_cast<int>(threadIdx.x) < h)
      for (int k = 0; k < 4; ++k) red[threadIdx.x][k] += red[threadIdx.x + h][k];
    __syncthreads();
  }
  if (threadIdx.x < 4) mean[threadIdx.x] = n > 0 ? red[0][threadIdx.x] / static_cast<double>(n) : 0.0;
  __syncthreads();
  for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    float s = 0.0f;
    for (int k = 0; k < d; ++k) {
      const float v = static_cast<float>(static_cast<double>(x[i * d + k]) - mean[k]);
      X[i * d + k] = v;
      s = fmaf(v, v, s);
    }
    sq[i] = s;
    w[i] = 1.0f / static_cast<float>(n);
  }
}

}  // namespace
}  // namespace gw

struct gw_server {
  int device = 0;
  int max_active = 1;
  gw::Pool* pool = nullptr;
  std::mutex mu;
  std::condition_variable cv_sched, cv_done;
  std::deque<gw::Job*> pending;
  std::vector<gw_response> done;
  int active = 0;
  int inflight = 0;   // submitted and not yet reported
  int slice = 0;      // outer steps per admission (0: all)
  double deadline = 0.0;                 // seconds after submission (0: none)
  std::vector<gw::Job*> running;         // admitted (ready or on a worker)
  bool stop = false;
  bool batching = true;                  // small squared requests through gw_solve_batch
  bool batch_busy = false;               // a batch is formed and not yet answered
  std::deque<gw::BatchJob*> batch_ready;
  std::condition_variable cv_batch;
  std::thread batch_thread;
  std::thread scheduler;
  std::vector<std::thread> workers;
  std::deque<gw::Job*> ready;   // admitted, waiting for a worker
  std::condition_variable cv_work;
};

namespace gw {
namespace {

// Drive one admitted request on stream st.  Returns false when the request
// was checkpointed and queued again (time slicing), true when it finished
// (its response is then posted).
bool run_job(gw_server* S, Job* J, cudaStream_t st, char* mem) {
  const gw_request& r = J->req;
  gw_response out;
  memset(&out, 0, sizeof(out));
  out.id = r.id;
  out.t_submit = J->t_submit;
  out.t_admit = J->t_admit;
  const int D = r.kind == GW_PEN_SQEUCLID ? r.d : r.D;
  char label[64];
  snprintf(label, sizeof(label), "gw request %llu", static_cast<unsigned long long>(r.id));
  NvtxRange range(label);
  char* p = mem;
  auto take = [&](size_t bytes) {
    char* q = p;
    p += align256(bytes);
    return q;
  };
  float* dx = reinterpret_cast<float*>(take(sizeof(float) * r.n * r.d));
  float* dy = reinterpret_cast<float*>(take(sizeof(float) * r.m * r.d));
  float* a = reinterpret_cast<float*>(take(sizeof(float) * r.n));
  float* s = reinterpret_cast<float*>(take(sizeof(float) * r.n));
  float* b = reinterpret_cast<float*>(take(sizeof(float) * r.m));
  float* t = reinterpret_cast<float*>(take(sizeof(float) * r.m));
  float* X = reinterpret_cast<float*>(take(sizeof(float) * r.n * D));
  float* Y = reinterpret_cast<float*>(take(sizeof(float) * r.m * D));
  float* f = reinterpret_cast<float*>(take(sizeof(float) * r.n));
  float* g = reinterpret_cast<float*>(take(sizeof(float) * r.m));
  double* G = reinterpret_cast<double*>(take(sizeof(double) * D * D));
  double* Gp = reinterpret_cast<double*>(take(sizeof(double) * D * D));
  double* en = reinterpret_cast<double*>(take(sizeof(double) * GW_EN_LEN));
  char* ws = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(p) + 255) & ~uintptr_t(255));
  const size_t ws_bytes = J->bytes - static_cast<size_t>(ws - mem);
  int slice = 0;
  double deadline = 0.0;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    slice = S->slice;
    deadline = S->deadline;
  }
  // the host watchdog: cancelled, or past its deadline?
  auto stop_code = [&]() {
    std::lock_guard<std::mutex> lk(S->mu);
    if (J->stop_code == 0 && deadline > 0.0 && now_s() > J->t_submit + deadline)
      J->stop_code = GW_ETIMEOUT;
    return J->stop_code;
  };
  const bool resumed = J->outer_done > 0;
  int rc = GW_OK;
  bool requeue = false;
  auto h2d = [&](void* dst, const void* src, size_t bytes) {
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st) == cudaSuccess;
  };
  auto d2h = [&](void* dst, const void* src, size_t bytes) {
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, st) == cudaSuccess;
  };
  do {
    if ((rc = stop_code()) != GW_OK) break;
    fill_kernel<<<ceil_div(r.n, 256), 256, 0, st>>>(a, r.n, 1.0f / static_cast<float>(r.n));
    fill_kernel<<<ceil_div(r.m, 256), 256, 0, st>>>(b, r.m, 1.0f / static_cast<float>(r.m));
    count_launch();
    count_launch();
    if (cudaGetLastError() != cudaSuccess) {
      rc = GW_ECUDA;
      break;
    }
    gw_stream_t gs = reinterpret_cast<gw_stream_t>(st);
    if (!resumed) {
      if (!h2d(dx, J->x.data(), sizeof(float) * r.n * r.d) ||
          !h2d(dy, J->y.data(), sizeof(float) * r.m * r.d)) {
        rc = GW_ECUDA;
        break;
      }
      rc = gw_lift(dx, r.n, r.d, a, r.kind, r.param, D, 0, r.id, X, s, nullptr, nullptr, ws, ws_bytes, gs);
      if (rc != GW_OK) break;
      rc = gw_lift(dy, r.m, r.d, b, r.kind, r.param, D, 0, r.id + 1, Y, t, nullptr, nullptr, ws, ws_bytes, gs);
      if (rc != GW_OK) break;
    } else {
      // resume from the checkpoint: features and the state after outer_done steps
      if (!h2d(X, J->X.data(), sizeof(float) * r.n * D) || !h2d(Y, J->Y.data(), sizeof(float) * r.m * D) ||
          !h2d(s, J->s.data(), sizeof(float) * r.n) || !h2d(t, J->t.data(), sizeof(float) * r.m) ||
          !h2d(f, J->f.data(), sizeof(float) * r.n) || !h2d(g, J->g.data(), sizeof(float) * r.m) ||
          !h2d(G, J->G.data(), sizeof(double) * D * D)) {
        rc = GW_ECUDA;
        break;
      }
    }
    gw_problem P{X, Y, s, t, a, b, r.n, r.m, D, D};
    while (J->outer_done < r.n_outer) {
      gw_options O{};
      O.eps = r.eps;
      O.eps_final = r.eps_final;
      const int left = r.n_outer - J->outer_done;
      O.n_outer = (slice > 0 && slice < left) ? slice : left;
      O.outer_offset = J->outer_done;
      O.outer_total = r.n_outer;
      O.n_inner = r.n_inner;
      O.symmetric = 1;
      O.prec = run_prec(r);
      O.record = 0;
      // per outer step, the Sinkhorn iterations replay from one captured
      // graph: the host enqueues O(n_outer) work per request
      O.use_graph = 2;
      // every slice after the first starts from the state the previous left
      if (J->outer_done > 0) {
        O.Gamma0 = G;
        O.f0 = f;
        O.g0 = g;
      }
      gw_result R{G, Gp, f, g, en, nullptr};
      rc = gw_solve(&P, &O, &R, ws, ws_bytes, gs);
      if (rc != GW_OK) break;
      J->outer_done += O.n_outer;
      if (J->outer_done >= r.n_outer) break;
      // a slice boundary: wait for the slice (the heartbeat the watchdog
      // follows), then honour a cancel or a passed deadline
      if (cudaStreamSynchronize(st) != cudaSuccess) {
        rc = GW_ECUDA;
        break;
      }
      if ((rc = stop_code()) != GW_OK) break;
      bool waiting = false;
      {
        // a request waits for a slot (batchable ones wait for the lane instead)
        std::lock_guard<std::mutex> lk(S->mu);
        for (const Job* P : S->pending)
          if (!(S->batching && batchable(P->req))) {
            waiting = true;
            break;
          }
      }
      if (waiting) {
        // checkpoint: the features and the state to host memory, then requeue
        J->X.resize(static_cast<size_t>(r.n) * D);
        J->Y.resize(static_cast<size_t>(r.m) * D);
        J->s.resize(r.n);
        J->t.resize(r.m);
        J->f.resize(r.n);
        J->g.resize(r.m);
        J->G.resize(static_cast<size_t>(D) * D);
        if (!d2h(J->X.data(), X, sizeof(float) * r.n * D) || !d2h(J->Y.data(), Y, sizeof(float) * r.m * D) ||
            !d2h(J->s.data(), s, sizeof(float) * r.n) || !d2h(J->t.data(), t, sizeof(float) * r.m) ||
            !d2h(J->f.data(), f, sizeof(float) * r.n) || !d2h(J->g.data(), g, sizeof(float) * r.m) ||
            !d2h(J->G.data(), G, sizeof(double) * D * D) || cudaStreamSynchronize(st) != cudaSuccess) {
          rc = GW_ECUDA;
          break;
        }
        requeue = true;
        break;
      }
    }
    if (rc != GW_OK || requeue) break;
    if (cudaMemcpyAsync(out.energy, en, sizeof(double) * GW_EN_LEN, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      rc = GW_ECUDA;
      break;
    }
    const double es = out.energy[GW_EN_STATUS];
    if (es != 0.0) rc = es == static_cast<double>(GW_ETIMEOUT) ? GW_ETIMEOUT : GW_ENONFINITE;
  } while (false);
  if (rc != GW_OK) cudaStreamSynchronize(st);
  std::lock_guard<std::mutex> lk(S->mu);
  S->pool->release(mem);
  S->active -= 1;
  S->running.erase(std::remove(S->running.begin(), S->running.end(), J), S->running.end());
  if (requeue && rc == GW_OK && J->stop_code != 0) {
    requeue = false;      // asked to stop during the checkpoint
    rc = J->stop_code;
  }
  // cancelled while its last slice (or, without slicing, its whole solve) ran:
  // the answer is the cancellation (the record it carries is complete)
  if (!requeue && rc == GW_OK && J->stop_code == GW_ECANCELED) rc = GW_ECANCELED;
  if (requeue && rc == GW_OK) {
    J->preempted += 1;
    J->mem = nullptr;
    S->pending.push_back(J);
    S->cv_sched.notify_all();
    return false;
  }
  out.status = rc;
  out.preempted = J->preempted;
  out.t_done = now_s();
  S->done.push_back(out);
  S->cv_sched.notify_all();
  S->cv_done.notify_all();
  return true;
}

void worker_loop(gw_server* S) {
  cudaSetDevice(S->device);
  cudaStream_t st;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  while (true) {
    Job* J = nullptr;
    char* mem = nullptr;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_work.wait(lk, [&] { return S->stop || !S->ready.empty(); });
      if (S->ready.empty()) break;
      J = S->ready.front();
      S->ready.pop_front();
      mem = J->mem;
    }
    if (run_job(S, J, st, mem)) delete J;
  }
  cudaStreamDestroy(st);
}

// Solve one batch on stream st and post its responses.
void run_batch(gw_server* S, BatchJob* BJ, cudaStream_t st) {
  const int Q = static_cast<int>(BJ->members.size());
  const int d = BJ->d;
  std::vector<int64_t> xo(Q + 1, 0), yo(Q + 1, 0);
  for (int q = 0; q < Q; ++q) {
    xo[q + 1] = xo[q] + BJ->members[q]->req.n;
    yo[q + 1] = yo[q] + BJ->members[q]->req.m;
  }
  const int64_t SN = xo[Q], SM = yo[Q];
  Carver c(BJ->mem, BJ->bytes);
  BatchBufs B = carve_batch(c, SN, SM, Q, d);
  std::vector<float> hx(static_cast<size_t>(SN) * d), hy(static_cast<size_t>(SM) * d);
  std::vector<float> e0(Q), e1(Q);
  for (int q = 0; q < Q; ++q) {
    const Job* J = BJ->members[q];
    std::copy(J->x.begin(), J->x.end(), hx.begin() + xo[q] * d);
    std::copy(J->y.begin(), J->y.end(), hy.begin() + yo[q] * d);
    e0[q] = J->req.eps;
    e1[q] = J->req.eps_final > 0.0f ? J->req.eps_final : J->req.eps;
  }
  std::vector<double> en(static_cast<size_t>(Q) * GW_EN_LEN, 0.0);
  int rc = GW_OK;
  do {
    if (c.overflow) {
      rc = GW_ENOMEM;
      break;
    }
    auto h2d = [&](void* dst, const void* src, size_t bytes) {
      return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st) == cudaSuccess;
    };
    if (!h2d(B.x, hx.data(), hx.size() * sizeof(float)) ||
        !h2d(B.y, hy.data(), hy.size() * sizeof(float)) ||
        !h2d(B.xo, xo.data(), xo.size() * sizeof(int64_t)) ||
        !h2d(B.yo, yo.data(), yo.size() * sizeof(int64_t)) ||
        !h2d(B.eps0, e0.data(), e0.size() * sizeof(float)) ||
        !h2d(B.eps1, e1.data(), e1.size() * sizeof(float))) {
      rc = GW_ECUDA;
      break;
    }
    batch_center_kernel<<<Q, 256, 0, st>>>(B.x, B.xo, d, B.X, B.s, B.a);
    batch_center_kernel<<<Q, 256, 0, st>>>(B.y, B.yo, d, B.Y, B.t, B.b);
    count_launch();
    count_launch();
    if (cudaGetLastError() != cudaSuccess) {
      rc = GW_ECUDA;
      break;
    }
    rc = run_solve_batch(Q, B.xo, B.yo, BJ->n_max, BJ->m_max, d, d, B.X, B.Y, B.s, B.t, B.a, B.b,
                         B.eps0, B.eps1, BJ->n_outer, BJ->n_inner, 1, B.f, B.g, B.G, B.Gp, B.en,
                         nullptr, B.ws, batch_ws_bytes(), st);
    if (rc != GW_OK) break;
    if (cudaMemcpyAsync(en.data(), B.en, en.size() * sizeof(double), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      rc = GW_ECUDA;
  } while (false);
  if (rc != GW_OK) cudaStreamSynchronize(st);
  std::lock_guard<std::mutex> lk(S->mu);
  S->pool->release(BJ->mem);
  const double t_done = now_s();
  for (int q = 0; q < Q; ++q) {
    Job* J = BJ->members[q];
    gw_response out;
    memset(&out, 0, sizeof(out));
    out.id = J->req.id;
    out.t_submit = J->t_submit;
    out.t_admit = J->t_admit;
    out.t_done = t_done;
    int st_q = rc;
    if (rc == GW_OK) {
      memcpy(out.energy, en.data() + static_cast<size_t>(q) * GW_EN_LEN, sizeof(out.energy));
      const double es = out.energy[GW_EN_STATUS];
      if (es != 0.0)
        st_q = es == static_cast<double>(GW_EINVAL)     ? GW_EINVAL
               : es == static_cast<double>(GW_ETIMEOUT) ? GW_ETIMEOUT
                                                        : GW_ENONFINITE;
    }
    // asked to stop while the batch ran: its answer is the stop
    if (J->stop_code != 0) st_q = J->stop_code;
    out.status = st_q;
    S->done.push_back(out);
    S->running.erase(std::remove(S->running.begin(), S->running.end(), J), S->running.end());
    delete J;
  }
  S->batch_busy = false;
  S->cv_sched.notify_all();
  S->cv_done.notify_all();
}

void batch_loop(gw_server* S) {
  cudaSetDevice(S->device);
  cudaStream_t st;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  while (true) {
    BatchJob* BJ = nullptr;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_batch.wait(lk, [&] { return S->stop || !S->batch_ready.empty(); });
      if (S->batch_ready.empty()) break;
      BJ = S->batch_ready.front();
      S->batch_ready.pop_front();
    }
    run_batch(S, BJ, st);
    delete BJ;
  }
  cudaStreamDestroy(st);
}

// With the lane free, gather the waiting batchable requests that share the
// first one's (d, n_outer, n_inner), in arrival order, while the batch's
// largest clouds still fit one CTA; reserve their memory and hand the batch
// to the lane.  Called with S->mu held.
bool form_batch(gw_server* S) {
  if (!S->batching || S->batch_busy) return false;
  BatchJob* BJ = nullptr;
  for (Job* J : S->pending) {
    if (!batchable(J->req)) continue;
    if (BJ == nullptr) {
      BJ = new BatchJob();
      BJ->d = J->req.d;
      BJ->n_outer = J->req.n_outer;
      BJ->n_inner = J->req.n_inner;
    } else if (J->req.d != BJ->d || J->req.n_outer != BJ->n_outer ||
               J->req.n_inner != BJ->n_inner) {
      continue;
    }
    const int64_t nm = std::max<int64_t>(BJ->n_max, J->req.n);
    const int64_t mm = std::max<int64_t>(BJ->m_max, J->req.m);
    if (!batch_fits(nm, mm, BJ->d)) continue;
    BJ->n_max = nm;
    BJ->m_max = mm;
    BJ->members.push_back(J);
    if (static_cast<int>(BJ->members.size()) >= kBatchMax) break;
  }
  if (BJ == nullptr) return false;
  int64_t SN = 0, SM = 0;
  for (Job* J : BJ->members) {
    SN += J->req.n;
    SM += J->req.m;
  }
  Carver c(nullptr, ~size_t(0));
  carve_batch(c, SN, SM, static_cast<int>(BJ->members.size()), BJ->d);
  BJ->bytes = c.used() + 256;
  BJ->mem = S->pool->alloc(BJ->bytes);
  if (BJ->mem == nullptr) {
    delete BJ;
    return false;
  }
  const double t = now_s();
  for (Job* J : BJ->members) {
    S->pending.erase(std::find(S->pending.begin(), S->pending.end(), J));
    S->running.push_back(J);
    J->t_admit = t;
  }
  S->batch_busy = true;
  S->batch_ready.push_back(BJ);
  S->cv_batch.notify_one();
  return true;
}

void scheduler_loop(gw_server* S) {
  std::unique_lock<std::mutex> lk(S->mu);
  while (!S->stop) {
    // admit in arrival order while a slot and memory are free
    bool admitted = false;
    Job* expired = nullptr;
    if (S->deadline > 0.0) {
      const double now = now_s();
      for (Job* J : S->pending)
        if (now > J->t_submit + S->deadline) {
          expired = J;
          break;
        }
    }
    if (expired != nullptr) {
      // past its deadline before it could run: answered without running
      Job* J = expired;
      S->pending.erase(std::find(S->pending.begin(), S->pending.end(), J));
      gw_response out;
      memset(&out, 0, sizeof(out));
      out.id = J->req.id;
      out.status = GW_ETIMEOUT;
      out.t_submit = J->t_submit;
      out.t_admit = J->t_admit;
      out.t_done = now_s();
      out.preempted = J->preempted;
      S->done.push_back(out);
      S->cv_done.notify_all();
      delete J;
      continue;
    }
    if (form_batch(S)) continue;
    // the first waiting request of the slot path (batchable ones wait for the lane)
    Job* J = nullptr;
    for (Job* P : S->pending)
      if (!(S->batching && batchable(P->req))) {
        J = P;
        break;
      }
    if (J != nullptr && S->active < S->max_active) {
      char* mem = S->pool->alloc(J->bytes);
      if (mem) {
        S->pending.erase(std::find(S->pending.begin(), S->pending.end(), J));
        S->running.push_back(J);
        if (J->preempted == 0) J->t_admit = now_s();
        J->mem = mem;
        S->active += 1;
        S->ready.push_back(J);
        S->cv_work.notify_one();
        admitted = true;
      }
    }
    if (!admitted) {
      // with a deadline, look again at least every 10 ms
      if (S->deadline > 0.0) S->cv_sched.wait_for(lk, std::chrono::milliseconds(10));
      else S->cv_sched.wait(lk);
    }
  }
}

}  // namespace
}  // namespace gw

using namespace gw;

extern "C" {

gw_server* gw_server_create(void* pool, size_t pool_bytes, int max_active, int device) {
  set_error("");
  if (pool == nullptr || pool_bytes < 4096 || max_active < 1 || max_active > 256) {
    set_error("gw_server_create: need a device pool and 1 <= max_active <= 256");
    return nullptr;
  }
  if (reinterpret_cast<uintptr_t>(pool) % 256 != 0) {
    set_error("gw_server_create: the pool must be 256-byte aligned");
    return nullptr;
  }
  gw_server* S = new gw_server();
  S->device = device;
  S->max_active = max_active;
  S->pool = new Pool(static_cast<char*>(pool), pool_bytes);
  for (int k = 0; k < max_active; ++k) S->workers.emplace_back(worker_loop, S);
  S->batch_thread = std::thread(batch_loop, S);
  S->scheduler = std::thread(scheduler_loop, S);
  return S;
}

int gw_server_submit(gw_server* S, const gw_request* r, const float* h_x, const float* h_y) {
  set_error("");
  GW_REQUIRE(S && r && h_x && h_y, GW_EINVAL, "gw_server_submit: null argument");
  GW_REQUIRE(r->n >= 2 && r->m >= 2 && r->d >= 1 && r->d <= 4, GW_EINVAL, "bad request sizes");
  GW_REQUIRE(r->eps > 0.0f && r->n_outer >= 1 && r->n_inner >= 1, GW_EINVAL, "bad request options");
  const int D = r->kind == GW_PEN_SQEUCLID ? r->d : r->D;
  GW_REQUIRE(D >= 1 && D <= GW_MAX_FEATURES, GW_EUNSUPPORTED, "bad feature dimension %d", D);
  Job* J = new Job();
  J->req = *r;
  J->x.assign(h_x, h_x + r->n * r->d);
  J->y.assign(h_y, h_y + r->m * r->d);
  J->bytes = request_bytes(*r);
  J->t_submit = now_s();
  std::lock_guard<std::mutex> lk(S->mu);
  if (J->bytes > S->pool->capacity()) {
    const size_t need = J->bytes;
    delete J;
    set_error("request needs %zu bytes of device memory, the pool holds %zu", need,
              S->pool->capacity());
    return GW_ENOMEM;
  }
  S->pending.push_back(J);
  S->inflight += 1;
  S->cv_sched.notify_all();
  return GW_OK;
}

int gw_server_poll(gw_server* S, gw_response* out, int max_out, int wait_ms) {
  if (!S || !out || max_out < 1) return 0;
  std::unique_lock<std::mutex> lk(S->mu);
  if (S->done.empty() && wait_ms != 0) {
    if (wait_ms < 0) {
      S->cv_done.wait(lk, [&] { return !S->done.empty() || S->inflight == 0; });
    } else {
      S->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return !S->done.empty(); });
    }
  }
  const int k = std::min<int>(max_out, static_cast<int>(S->done.size()));
  for (int i = 0; i < k; ++i) out[i] = S->done[i];
  S->done.erase(S->done.begin(), S->done.begin() + k);
  S->inflight -= k;
  return k;
}

int gw_server_set_slice(gw_server* S, int outer_steps) {
  set_error("");
  GW_REQUIRE(S != nullptr && outer_steps >= 0, GW_EINVAL,
             "gw_server_set_slice: need a server and outer_steps >= 0");
  std::lock_guard<std::mutex> lk(S->mu);
  S->slice = outer_steps;
  return GW_OK;
}

int gw_server_cancel(gw_server* S, uint64_t id) {
  set_error("");
  GW_REQUIRE(S != nullptr, GW_EINVAL, "gw_server_cancel: null server");
  std::lock_guard<std::mutex> lk(S->mu);
  for (auto it = S->pending.begin(); it != S->pending.end(); ++it) {
    if ((*it)->req.id != id) continue;
    Job* J = *it;
    S->pending.erase(it);
    gw_response out;
    memset(&out, 0, sizeof(out));
    out.id = id;
    out.status = GW_ECANCELED;
    out.t_submit = J->t_submit;
    out.t_admit = J->t_admit;
    out.t_done = now_s();
    out.preempted = J->preempted;
    S->done.push_back(out);
    S->cv_done.notify_all();
    S->cv_sched.notify_all();
    delete J;
    return GW_OK;
  }
  for (Job* J : S->running) {
    if (J->req.id != id) continue;
    if (J->stop_code == 0) J->stop_code = GW_ECANCELED;
    return GW_OK;
  }
  set_error("gw_server_cancel: no request %llu in flight", static_cast<unsigned long long>(id));
  return GW_EINVAL;
}

int gw_server_set_batching(gw_server* S, int on) {
  set_error("");
  GW_REQUIRE(S != nullptr, GW_EINVAL, "gw_server_set_batching: null server");
  std::lock_guard<std::mutex> lk(S->mu);
  S->batching = on != 0;
  S->cv_sched.notify_all();
  return GW_OK;
}

int gw_server_set_deadline(gw_server* S, double seconds) {
  set_error("");
  GW_REQUIRE(S != nullptr && isfinite(seconds), GW_EINVAL, "gw_server_set_deadline: bad argument");
  std::lock_guard<std::mutex> lk(S->mu);
  S->deadline = seconds > 0.0 ? seconds : 0.0;
  S->cv_sched.notify_all();
  return GW_OK;
}

size_t gw_server_request_bytes(const gw_request* r) {
  if (!r || r->n < 2 || r->m < 2 || r->d < 1 || r->d > 4) return 0;
  return request_bytes(*r);
}

int gw_server_stats(gw_server* S, int* pending, int* active) {
  if (!S) return GW_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  if (pending) *pending = static_cast<int>(S->pending.size());
  if (active) *active = S->active;
  return GW_OK;
}

void gw_server_destroy(gw_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    S->cv_sched.notify_all();
    S->cv_work.notify_all();
    S->cv_batch.notify_all();
  }
  S->scheduler.join();
  for (auto& w : S->workers) w.join();
  S->batch_thread.join();
  for (Job* J : S->pending) delete J;
  for (Job* J : S->ready) delete J;
  for (BatchJob* B : S->batch_ready) {
    for (Job* J : B->members) delete J;
    delete B;
  }
  delete S->pool;
  delete S;
}

}  // extern "C"
