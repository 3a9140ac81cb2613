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
        std::lock_guard<std::mutex> lk(S->mu);
        waiting = !S->pending.empty();
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

void scheduler_loop(gw_server* S) {
  std::unique_lock<std::mutex> lk(S->mu);
  while (!S->stop) {
    // admit in arrival order while a slot and memory are free
    bool admitted = false;
    if (!S->pending.empty() && S->deadline > 0.0 &&
        now_s() > S->pending.front()->t_submit + S->deadline) {
      // past its deadline before it could run: answered without running
      Job* J = S->pending.front();
      S->pending.pop_front();
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
    if (!S->pending.empty() && S->active < S->max_active) {
      Job* J = S->pending.front();
      char* mem = S->pool->alloc(J->bytes);
      if (mem) {
        S->pending.pop_front();
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
  }
  S->scheduler.join();
  for (auto& w : S->workers) w.join();
  for (Job* J : S->pending) delete J;
  for (Job* J : S->ready) delete J;
  delete S->pool;
  delete S;
}

}  // extern "C"
