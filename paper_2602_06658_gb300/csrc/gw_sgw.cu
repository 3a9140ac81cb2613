// Sinkhorn GW divergence (Section 4.1):
//   SGW_eps(alpha, beta) = GW_eps(alpha, beta) - (GW_eps(alpha, alpha) + GW_eps(beta, beta)) / 2,
// three CNT-GW solves with the same options, and its gradient with respect
// to the source features (and points) with every plan at its optimum
// (envelope theorem, Appendix B.6).  GW_eps(alpha, alpha) depends on X through
// both of its sides; the target side is the source side of the transposed
// problem (potentials exchanged, Gamma transposed).
#include <math.h>

#include "gw_internal.cuh"

namespace gw {

namespace {

struct SgwBufs {
  double *G[3], *Gp[3], *en[3];
  float *f[3], *g[3];
  double *GT, *GpT;
  float *dA, *dB, *xa, *xb;
};

SgwBufs carve_sgw(Carver& c, int64_t n, int64_t m, int D, int E, bool grad, int dx_dim) {
  SgwBufs B{};
  const int64_t rows[3] = {n, n, m};
  const int64_t cols[3] = {m, n, m};
  const int dl[3] = {D, D, E};
  const int dr[3] = {E, D, E};
  for (int k = 0; k < 3; ++k) {
    B.G[k] = c.take<double>(static_cast<size_t>(dl[k]) * dr[k]);
    B.Gp[k] = c.take<double>(static_cast<size_t>(dl[k]) * dr[k]);
    B.en[k] = c.take<double>(GW_EN_LEN);
    B.f[k] = c.take<float>(static_cast<size_t>(rows[k]));
    B.g[k] = c.take<float>(static_cast<size_t>(cols[k]));
  }
  if (grad) {
    B.GT = c.take<double>(static_cast<size_t>(D) * D);
    B.GpT = c.take<double>(static_cast<size_t>(D) * D);
    B.dA = c.take<float>(static_cast<size_t>(n) * D);
    B.dB = c.take<float>(static_cast<size_t>(n) * D);
    if (dx_dim > 0) {
      B.xa = c.take<float>(static_cast<size_t>(n) * dx_dim);
      B.xb = c.take<float>(static_cast<size_t>(n) * dx_dim);
    }
  }
  return B;
}

// out = [SGW, GW(a,b), GW(a,a), GW(b,b)]
__global__ void sgw_value_kernel(const double* eab, const double* eaa, const double* ebb,
                                 double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    out[0] = eab[GW_EN_E] - 0.5 * (eaa[GW_EN_E] + ebb[GW_EN_E]);
    out[1] = eab[GW_EN_E];
    out[2] = eaa[GW_EN_E];
    out[3] = ebb[GW_EN_E];
  }
}

__global__ void transpose_kernel(const double* G, int D, double* GT) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < D * D) GT[(q % D) * D + q / D] = G[q];
}

// A <- A - (B + C) / 2
__global__ void sgw_combine_kernel(float* A, const float* B, const float* C, int64_t count) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < count) A[i] = A[i] - 0.5f * (B[i] + C[i]);
}

float last_eps(const gw_options& o) {
  if (o.eps_final > 0.0f && o.eps_final != o.eps && o.n_outer > 1) {
    // the solver's schedule at t = n_outer - 1
    return static_cast<float>(static_cast<double>(o.eps) *
                              pow(static_cast<double>(o.eps_final) / o.eps, 1.0));
  }
  return o.eps;
}

}  // namespace

size_t sgw_ws_bytes(int64_t n, int64_t m, int D, int E, int prec, bool grad, int dx_dim) {
  Carver c(nullptr, ~size_t(0));
  carve_sgw(c, n, m, D, E, grad, dx_dim);
  size_t scratch = gw_workspace_size(GW_OP_SOLVE, n, m, D, E, prec);
  const size_t s_aa = gw_workspace_size(GW_OP_SOLVE, n, n, D, D, prec);
  const size_t s_bb = gw_workspace_size(GW_OP_SOLVE, m, m, E, E, prec);
  if (s_aa > scratch) scratch = s_aa;
  if (s_bb > scratch) scratch = s_bb;
  if (grad) {
    const size_t g_ab = grad_ws_bytes(n, m, D, E, dx_dim, prec);
    const size_t g_aa = grad_ws_bytes(n, n, D, D, dx_dim, prec);
    if (g_ab > scratch) scratch = g_ab;
    if (g_aa > scratch) scratch = g_aa;
  }
  return c.used() + scratch;
}

int run_sgw(const gw_problem& p, const gw_options& o, double* out, double* records, float* dX,
            const float* x, int dx_dim, int kind, float param, const float* basis,
            const float* eigvals, float* dx, void* ws, size_t ws_bytes, cudaStream_t st) {
  Carver c(ws, ws_bytes);
  const SgwBufs B = carve_sgw(c, p.n, p.m, p.D, p.E, dX != nullptr, x ? dx_dim : 0);
  GW_TRY(check_ws(c, ws));
  char* base = static_cast<char*>(ws) + c.used();
  const size_t rest = ws_bytes - c.used();
  const gw_problem P[3] = {p,
                           {p.X, p.X, p.s, p.s, p.a, p.a, p.n, p.n, p.D, p.D},
                           {p.Y, p.Y, p.t, p.t, p.b, p.b, p.m, p.m, p.E, p.E}};
  for (int k = 0; k < 3; ++k) {
    gw_options ok = o;
    ok.record = 0;
    if (k > 0) {   // a caller's start only fits the alpha-beta problem
      ok.Gamma0 = nullptr;
      ok.f0 = nullptr;
      ok.g0 = nullptr;
    }
    gw_result R{B.G[k], B.Gp[k], B.f[k], B.g[k], B.en[k], nullptr};
    GW_TRY(gw_solve(&P[k], &ok, &R, base, rest, reinterpret_cast<gw_stream_t>(st)));
  }
  sgw_value_kernel<<<1, 32, 0, st>>>(B.en[0], B.en[1], B.en[2], out);
  GW_LAUNCH_CHECK();
  if (records) {
    for (int k = 0; k < 3; ++k)
      GW_CUDA_TRY(cudaMemcpyAsync(records + k * GW_EN_LEN, B.en[k], sizeof(double) * GW_EN_LEN,
                                  cudaMemcpyDeviceToDevice, st));
  }
  if (!dX) return GW_OK;
  const float eT = last_eps(o);
  const int dxd = x ? dx_dim : 0;
  // alpha-beta, then the two sides of alpha-alpha
  GW_TRY(run_grad(P[0], B.f[0], B.g[0], B.Gp[0], B.G[0], eT, o.prec, x, dxd, kind, param, basis,
                  eigvals, dX, dx, base, rest, st));
  GW_TRY(run_grad(P[1], B.f[1], B.g[1], B.Gp[1], B.G[1], eT, o.prec, x, dxd, kind, param, basis,
                  eigvals, B.dA, B.xa, base, rest, st));
  const int DD = p.D * p.D;
  transpose_kernel<<<ceil_div(DD, 256), 256, 0, st>>>(B.G[1], p.D, B.GT);
  GW_LAUNCH_CHECK();
  transpose_kernel<<<ceil_div(DD, 256), 256, 0, st>>>(B.Gp[1], p.D, B.GpT);
  GW_LAUNCH_CHECK();
  GW_TRY(run_grad(P[1], B.g[1], B.f[1], B.GpT, B.GT, eT, o.prec, x, dxd, kind, param, basis,
                  eigvals, B.dB, B.xb, base, rest, st));
  const int64_t nD = p.n * p.D;
  sgw_combine_kernel<<<ceil_div(nD, 256), 256, 0, st>>>(dX, B.dA, B.dB, nD);
  GW_LAUNCH_CHECK();
  if (x && dx) {
    const int64_t nd = p.n * dxd;
    sgw_combine_kernel<<<ceil_div(nd, 256), 256, 0, st>>>(dx, B.xa, B.xb, nd);
    GW_LAUNCH_CHECK();
  }
  return GW_OK;
}

}  // namespace gw
