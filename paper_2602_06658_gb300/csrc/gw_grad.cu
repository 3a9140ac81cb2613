// Gradient of the EGW energy with respect to the source points through the
// converged plan (Appendix B.6, envelope theorem; Algorithms 9-13).
//
// With pi held at the plan encoded by (f, g) on c_{Gamma_t} and Gamma_pi =
// sum_ij pi_ij X_i Y_j^T, the Lemma (Appendix C.1) gives, per feature row,
//   dX_i = 8 a_i [(s_i + m2_X) X_i + 2 Sigma_X X_i - mu3_X] - 8 a_i m2_Y X_i
//          - 16 Gamma_pi w_i - 8 q_i X_i,
//   w_i = sum_j pi_ij Y_j,  q_i = sum_j pi_ij t_j,  mu3_X = sum_k a_k s_k X_k,
// then the adjoint of the centering X = x - sum a x:
//   dX_i <- dX_i - a_i sum_k dX_k.
// For lifted features (Algorithm 12) the features of a moving point come
// from Kernel-Proj (Algorithm 13) frozen at the training points, and
//   dx_i = sum_d dX_id grad_x Pi_d(x_i)
//        = 1/2 [ -sum_k P_ik grad_1 c(x_i, x_k) + (sum_k P_ik) sum_l a_l grad_1 c(x_i, x_l) ],
//   P_ik = sum_d dX_id V_kd / sqrt(Lambda_d),
// one N x N matrix-free pass.
#include <math.h>

#include "gw_internal.cuh"

namespace gw {

namespace {

constexpr int kRed = 148;
constexpr int kVjpThreads = 128;
constexpr int kVjpTile = 32;

// U_i[e] = sum_d X_i[d] Gamma[d][e]  (n x E)
// Gt[e][d] = Gamma[d][e]
__global__ void transpose_de_kernel(const double* Gamma, int D, int E, double* Gt) {
  for (int q = threadIdx.x; q < D * E; q += blockDim.x) Gt[(q % E) * D + q / E] = Gamma[q];
}

// partial [m2, Sigma (D x D), mu3 (D)] of a-weighted centered features:
// rows staged 32 at a time in shared memory with their norms s_i; each
// thread accumulates its Sigma entries, thread d < D the component mu3_d,
// thread 0 also m2 (fixed order: deterministic)
__global__ void __launch_bounds__(256)
    grad_moments_kernel(const float* X, const float* a, int64_t n, int D, double* part) {
  __shared__ double Xs[32][129];
  __shared__ double ws[32], ss[32];
  const int L = 1 + D * D + D;
  const int per = (D * D + 255) / 256;
  double acc[64];
  for (int q = 0; q < per; ++q) acc[q] = 0.0;
  double m2 = 0.0, mu3 = 0.0;
  const int tid = threadIdx.x;
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t i0 = blockIdx.x * chunk;
  const int64_t i1 = i0 + chunk < n ? i0 + chunk : n;
  for (int64_t ib = i0; ib < i1; ib += 32) {
    const int cnt = static_cast<int>(i1 - ib < 32 ? i1 - ib : 32);
    __syncthreads();
    for (int idx = tid; idx < cnt * D; idx += 256) Xs[idx / D][idx % D] = X[(ib + idx / D) * D + idx % D];
    if (tid < cnt) ws[tid] = a[ib + tid];
    __syncthreads();
    if (tid < cnt) {
      double s = 0.0;
      for (int d = 0; d < D; ++d) s = fma(Xs[tid][d], Xs[tid][d], s);
      ss[tid] = s;
    }
    __syncthreads();
    for (int q = 0; q < per; ++q) {
      const int e = tid + q * 256;
      if (e < D * D) {
        const int d0 = e / D, d1 = e % D;
        for (int r = 0; r < cnt; ++r) acc[q] = fma(ws[r] * Xs[r][d0], Xs[r][d1], acc[q]);
      }
    }
    if (tid < D)
      for (int r = 0; r < cnt; ++r) mu3 = fma(ws[r] * ss[r], Xs[r][tid], mu3);
    if (tid == 0)
      for (int r = 0; r < cnt; ++r) m2 = fma(ws[r], ss[r], m2);
  }
  double* out = part + static_cast<int64_t>(blockIdx.x) * L;
  for (int q = 0; q < per; ++q) {
    const int e = tid + q * 256;
    if (e < D * D) out[1 + e] = acc[q];
  }
  if (tid < D) out[1 + D * D + tid] = mu3;
  if (tid == 0) out[0] = m2;
}

__global__ void sum_partials_kernel(const double* part, int blocks, int L, double* out) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < L; e += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < blocks; ++b) s += part[static_cast<int64_t>(b) * L + e];
    out[e] = s;
  }
}

// m2_Y = sum b t
__global__ void weighted_dot_kernel(const float* w, const float* v, int64_t n, double* out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += static_cast<double>(w[i]) * v[i];
  red[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < static_cast<int>(blockDim.x); ++k) t += red[k];
    *out = t;
  }
}

// dX_i from the closed form; mom = [m2_X, Sigma_X, mu3_X], Wr_i = [w_i (E), q_i, r_i]
__global__ void grad_rows_kernel(const float* X, const float* s, const float* a, const double* mom,
                                 const double* m2y, const double* Gpi, const double* Wr, int64_t n,
                                 int D, int E, float* dX) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double m2x = mom[0];
  const double* Sig = mom + 1;
  const double* mu3 = mom + 1 + D * D;
  const double ai = a[i];
  const double si = s[i];
  const double* wi = Wr + i * (E + 2);
  const double qi = wi[E];
  for (int d = 0; d < D; ++d) {
    double sx = 0.0;
    for (int k = 0; k < D; ++k) sx = fma(Sig[d * D + k], static_cast<double>(X[i * D + k]), sx);
    double gw = 0.0;
    for (int e = 0; e < E; ++e) gw = fma(Gpi[d * E + e], wi[e], gw);
    const double xd = X[i * D + d];
    const double v = 8.0 * ai * ((si + m2x) * xd + 2.0 * sx - mu3[d]) - 8.0 * ai * (*m2y) * xd -
                     16.0 * gw - 8.0 * qi * xd;
    dX[i * D + d] = static_cast<float>(v);
  }
}

// column sums of dX (partials per block), D <= 128
__global__ void colsum_rows_kernel(const float* M, int64_t n, int D, double* part) {
  const int d = threadIdx.x;
  if (d >= D) return;
  double s = 0.0;
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x) s += M[i * D + d];
  part[static_cast<int64_t>(blockIdx.x) * D + d] = s;
}

// dX_i <- dX_i - a_i sum_k dX_k
__global__ void center_adjoint_kernel(float* dX, const float* a, const double* cs, int64_t n, int D) {
  const int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= n * D) return;
  const int64_t i = q / D;
  dX[q] = static_cast<float>(static_cast<double>(dX[q]) - static_cast<double>(a[i]) * cs[q % D]);
}

__device__ __forceinline__ float grad1_coef(float d2, int kind, float param) {
  // grad_1 c(x, y) = coef * (x - y)
  if (kind == GW_PEN_SQEUCLID) return 2.0f;
  if (kind == GW_PEN_POWER) {
    if (!(d2 > 0.0f)) return 0.0f;
    if (param == 1.0f) return rsqrtf(d2);
    return param * exp2f((0.5f * param - 1.0f) * log2f(d2));
  }
  const float s2 = param * param;
  return (2.0f / s2) * expf(-d2 / (2.0f * s2));
}

// Kernel-Proj vector-Jacobian product, one source point per thread:
// out[split][i] = [sum_k P_ik grad(i,k) (dd), sum_k P_ik, sum_k a_k grad(i,k) (dd)]
template <int DP>
__global__ void __launch_bounds__(kVjpThreads)
    kproj_vjp_kernel(const float* x, int dd, const float* a, const float* V, const float* dX,
                     const float* inv_sqrt_lam, int64_t n, int D, int kind, float param,
                     int64_t cols_per_split, float* part) {
  __shared__ __align__(16) float Vs[kVjpTile][DP];
  __shared__ float xs[kVjpTile][4];
  __shared__ float as[kVjpTile];
  const int64_t i = static_cast<int64_t>(blockIdx.x) * kVjpThreads + threadIdx.x;
  const bool ok = i < n;
  float G[DP];
#pragma unroll
  for (int d = 0; d < DP; ++d) G[d] = (ok && d < D) ? dX[i * D + d] * inv_sqrt_lam[d] : 0.0f;
  float xi[4] = {0.f, 0.f, 0.f, 0.f};
  for (int c = 0; c < dd; ++c) xi[c] = ok ? x[i * dd + c] : 0.f;
  float S1[4] = {0.f, 0.f, 0.f, 0.f}, S2[4] = {0.f, 0.f, 0.f, 0.f}, S0 = 0.f;
  const int64_t k0 = static_cast<int64_t>(blockIdx.y) * cols_per_split;
  const int64_t k1 = k0 + cols_per_split < n ? k0 + cols_per_split : n;
  for (int64_t kb = k0; kb < k1; kb += kVjpTile) {
    __syncthreads();
    for (int idx = threadIdx.x; idx < kVjpTile * DP; idx += kVjpThreads) {
      const int kk = idx / DP, d = idx % DP;
      const int64_t k = kb + kk;
      Vs[kk][d] = (k < k1 && d < D) ? V[k * D + d] : 0.f;
    }
    if (threadIdx.x < kVjpTile) {
      const int64_t k = kb + threadIdx.x;
      for (int c = 0; c < 4; ++c) xs[threadIdx.x][c] = (k < k1 && c < dd) ? x[k * dd + c] : 0.f;
      as[threadIdx.x] = k < k1 ? a[k] : 0.f;
    }
    __syncthreads();
    const int cnt = static_cast<int>(k1 - kb < kVjpTile ? k1 - kb : kVjpTile);
    for (int kk = 0; kk < cnt; ++kk) {
      float P = 0.f;
#pragma unroll
      for (int d = 0; d < DP; ++d) P = fmaf(G[d], Vs[kk][d], P);
      float diff[4], d2 = 0.f;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        diff[c] = xi[c] - xs[kk][c];
        d2 = fmaf(diff[c], diff[c], d2);
      }
      const float coef = grad1_coef(d2, kind, param);
      S0 += P;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const float gr = coef * diff[c];
        S1[c] = fmaf(P, gr, S1[c]);
        S2[c] = fmaf(as[kk], gr, S2[c]);
      }
    }
  }
  if (!ok) return;
  float* out = part + (static_cast<int64_t>(blockIdx.y) * n + i) * 9;
  for (int c = 0; c < 4; ++c) {
    out[c] = S1[c];
    out[5 + c] = S2[c];
  }
  out[4] = S0;
}

// dx_i = 1/2 (-S1 + S0 S2), summed over splits in float64
__global__ void kproj_finish_kernel(const float* part, int splits, int64_t n, int dd, float* dx) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double S[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int s = 0; s < splits; ++s)
    for (int k = 0; k < 9; ++k) S[k] += part[(static_cast<int64_t>(s) * n + i) * 9 + k];
  for (int c = 0; c < dd; ++c) dx[i * dd + c] = static_cast<float>(0.5 * (-S[c] + S[4] * S[5 + c]));
}

__global__ void inv_sqrt_kernel(const float* lam, int D, float* out) {
  const int d = threadIdx.x;
  if (d < D) out[d] = lam[d] > 0.f ? rsqrtf(lam[d]) : 0.f;
}

int vjp_splits(int64_t n) {
  const int rb = ceil_div(n, kVjpThreads);
  int s = ceil_div(4 * kSmCount, rb);
  const int smax = ceil_div(n, 256);
  if (s > smax) s = smax;
  return s < 1 ? 1 : s;
}

struct GradBufs {
  double *Gpi, *stats, *U_unused, *Wr, *mpart, *mom, *m2y, *cpart, *cs;
  double* GtT;   // Gamma_t^T (E x D)
  double* Gsc;   // Gamma of the transposed plan (E x D, not used)
  float* vpart;
  float* isl;
};

}  // namespace

size_t grad_ws_bytes(int64_t n, int64_t m, int D, int E, int dx_dim, int prec) {
  Carver c(nullptr, ~size_t(0));
  c.take<double>(static_cast<size_t>(D) * E);          // Gamma_pi
  c.take<double>(8);
  c.take<double>(static_cast<size_t>(D) * E);          // Gamma_t^T
  c.take<double>(static_cast<size_t>(D) * E);          // Gamma of the transposed plan
  c.take<double>(static_cast<size_t>(n) * (E + 2));    // row sums
  c.take<double>(static_cast<size_t>(kRed) * (1 + D * D + D));
  c.take<double>(static_cast<size_t>(1 + D * D + D));
  c.take<double>(4);
  c.take<double>(static_cast<size_t>(kRed) * D);
  c.take<double>(static_cast<size_t>(D));
  c.take<float>(static_cast<size_t>(D));
  if (dx_dim > 0) c.take<float>(static_cast<size_t>(vjp_splits(n)) * n * 9);
  size_t scratch = cross_cov_ws_bytes(m, n, E, D, prec);
  const size_t cc = cross_cov_ws_bytes(n, m, D, E, prec);
  if (cc > scratch) scratch = cc;
  return c.used() + scratch + 512;
}

int run_grad(const gw_problem& p, const float* f, const float* g, const double* Gamma_t,
             const double* Gamma_pi, float eps, int prec, const float* x, int dx_dim, int kind,
             float param, const float* basis, const float* eigvals, float* dX, float* dx,
             void* ws, size_t ws_bytes, cudaStream_t st) {
  const int64_t n = p.n, m = p.m;
  const int D = p.D, E = p.E;
  Carver c(ws, ws_bytes);
  GradBufs B;
  B.Gpi = c.take<double>(static_cast<size_t>(D) * E);
  B.stats = c.take<double>(8);
  B.GtT = c.take<double>(static_cast<size_t>(D) * E);
  B.Gsc = c.take<double>(static_cast<size_t>(D) * E);
  B.Wr = c.take<double>(static_cast<size_t>(n) * (E + 2));
  B.mpart = c.take<double>(static_cast<size_t>(kRed) * (1 + D * D + D));
  B.mom = c.take<double>(static_cast<size_t>(1 + D * D + D));
  B.m2y = c.take<double>(4);
  B.cpart = c.take<double>(static_cast<size_t>(kRed) * D);
  B.cs = c.take<double>(static_cast<size_t>(D));
  B.isl = c.take<float>(static_cast<size_t>(D));
  B.vpart = dx_dim > 0 ? c.take<float>(static_cast<size_t>(vjp_splits(n)) * n * 9) : nullptr;
  GW_TRY(check_ws(c, ws));
  const size_t mark = c.used();
  char* base = static_cast<char*>(ws);

  // Gamma_pi of the plan (when not given)
  const double* Gpi = Gamma_pi;
  if (!Gpi) {
    Carver sub(base + mark, ws_bytes - mark);
    PlanArgs pa{p.X, p.Y, p.s, p.t, p.a, p.b, f, g, Gamma_t, eps, n, m, D, E};
    GW_TRY(run_cross_cov(pa, prec, B.Gpi, B.stats, nullptr, sub, st));
    Gpi = B.Gpi;
  }
  // row-direction plan sums [w_i, q_i, r_i] = sum_j pi_ij [Y_j, t_j, 1]: the
  // plan-weighted column sums of the transposed problem (Y as sources, X as
  // targets, Gamma_t^T: its cost c'_ji = c_ij, so its plan is pi^T), in the
  // request's precision (on the tensor cores for the 16-bit forms)
  transpose_de_kernel<<<1, 256, 0, st>>>(Gamma_t, D, E, B.GtT);
  GW_LAUNCH_CHECK();
  {
    Carver sub(base + mark, ws_bytes - mark);
    PlanArgs pt{p.Y, p.X, p.t, p.s, p.b, p.a, g, f, B.GtT, eps, m, n, E, D};
    GW_TRY(run_cross_cov(pt, prec, B.Gsc, nullptr, B.Wr, sub, st));
  }
  // moments of X and m2_Y
  const int L = 1 + D * D + D;
  grad_moments_kernel<<<kRed, 256, 0, st>>>(p.X, p.a, n, D, B.mpart);
  GW_LAUNCH_CHECK();
  sum_partials_kernel<<<ceil_div(L, 256), 256, 0, st>>>(B.mpart, kRed, L, B.mom);
  GW_LAUNCH_CHECK();
  weighted_dot_kernel<<<1, 256, 0, st>>>(p.b, p.t, m, B.m2y);
  GW_LAUNCH_CHECK();
  grad_rows_kernel<<<ceil_div(n, 128), 128, 0, st>>>(p.X, p.s, p.a, B.mom, B.m2y, Gpi, B.Wr, n, D,
                                                    E, dX);
  GW_LAUNCH_CHECK();
  colsum_rows_kernel<<<kRed, 128, 0, st>>>(dX, n, D, B.cpart);
  GW_LAUNCH_CHECK();
  sum_partials_kernel<<<1, 128, 0, st>>>(B.cpart, kRed, D, B.cs);
  GW_LAUNCH_CHECK();
  center_adjoint_kernel<<<ceil_div(n * D, 256), 256, 0, st>>>(dX, p.a, B.cs, n, D);
  GW_LAUNCH_CHECK();
  if (dx_dim == 0) return GW_OK;

  // Kernel-Proj chain for lifted features
  inv_sqrt_kernel<<<1, 128, 0, st>>>(eigvals, D, B.isl);
  GW_LAUNCH_CHECK();
  const int splits = vjp_splits(n);
  const int64_t cps = (static_cast<int64_t>(ceil_div(n, splits)) + kVjpTile - 1) / kVjpTile * kVjpTile;
  const int sp = ceil_div(n, cps);
  dim3 grid(ceil_div(n, kVjpThreads), sp);
  const int DP = D <= 16 ? 16 : (D <= 32 ? 32 : (D <= 64 ? 64 : 128));
  switch (DP) {
    case 16: kproj_vjp_kernel<16><<<grid, kVjpThreads, 0, st>>>(x, dx_dim, p.a, basis, dX, B.isl, n, D, kind, param, cps, B.vpart); break;
    case 32: kproj_vjp_kernel<32><<<grid, kVjpThreads, 0, st>>>(x, dx_dim, p.a, basis, dX, B.isl, n, D, kind, param, cps, B.vpart); break;
    case 64: kproj_vjp_kernel<64><<<grid, kVjpThreads, 0, st>>>(x, dx_dim, p.a, basis, dX, B.isl, n, D, kind, param, cps, B.vpart); break;
    default: kproj_vjp_kernel<128><<<grid, kVjpThreads, 0, st>>>(x, dx_dim, p.a, basis, dX, B.isl, n, D, kind, param, cps, B.vpart); break;
  }
  GW_LAUNCH_CHECK();
  kproj_finish_kernel<<<ceil_div(n, 256), 256, 0, st>>>(B.vpart, sp, n, dx_dim, dx);
  GW_LAUNCH_CHECK();
  return GW_OK;
}

}  // namespace gw
