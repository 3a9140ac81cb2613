// Kernel-GW (Algorithm 5, Appendix B.3): the exact kernelised scheme for
// small N, with dense N x M matrices.  From cost matrices C^X (N x N) and
// C^Y (M x M), Algorithm 4 gives the centered kernels K^X, K^Y; every outer
// step builds the dense cost C = -4 K^X_ii K^Y_jj - 16 K^X pi K^Y, runs
// Sinkhorn on it and forms the plan pi = a b^T exp((f + g - C)/eps).
//
// The two products K^X (pi K^Y) (O(N^2 M + N M^2) per step) run on the
// tensor cores at FP32 accuracy in this library's own split-f16 product
// (gw_gemm_tc.cu), the rank-one term -4 k l^T fused into the second one's
// epilogue.  Everything else (centering, softmins over the dense cost, plan,
// energy) runs in the kernels below.
//
// Energy of pi_{t+1} (Lemma, Appendix C.1, in kernel form): with
// k_i = K^X_ii, l_j = K^Y_jj and C_{t+1} the next step's cost,
//   T = sum pi k l,  ||Gamma||^2 = <pi, K^X pi K^Y> = -(4 T + <pi, C_{t+1}>) / 16,
//   eps KL = sum pi (f + g - C_t),  C(alpha, beta) from the kernel moments.
#include <math.h>

#include <mutex>

#include "gw_internal.cuh"

namespace gw {

namespace {

// ------------------------------------------------------------ Algorithm 4
// K0_ij = (C_i0 + C_0j - C_ij) / 2
__global__ void kg_base_kernel(const float* C, int64_t n, float* K) {
  const int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= n * n) return;
  const int64_t i = q / n, j = q % n;
  K[q] = 0.5f * (C[i * n] + C[j] - C[q]);
}

// rows[i] = sum_j a_j K_ij (one warp per row), in float64
__global__ void kg_rowsum_kernel(const float* K, const float* a, int64_t n, double* rows) {
  const int64_t i = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  double s = 0.0;
  for (int64_t j = lane; j < n; j += 32) s += static_cast<double>(a[j]) * K[i * n + j];
  s = warp_sum(s);
  if (lane == 0) rows[i] = s;
}

// cols[j] = sum_i a_i K_ij (one thread per column, coalesced over j)
__global__ void kg_colsum_kernel(const float* K, const float* a, int64_t n, double* cols) {
  const int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += static_cast<double>(a[i]) * K[i * n + j];
  cols[j] = s;
}

// tot = sum_i a_i rows_i (one block, fixed order)
__global__ void kg_total_kernel(const double* rows, const float* a, int64_t n, double* tot) {
  __shared__ double red[8];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += 256) s += static_cast<double>(a[i]) * rows[i];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int q = 0; q < 8; ++q) v += red[q];
    *tot = v;
  }
}

// K_ij = K0_ij - cols_j - rows_i + tot; diag_i = K_ii
__global__ void kg_center_kernel(float* K, int64_t n, const double* rows, const double* cols,
                                 const double* tot, float* diag) {
  const int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= n * n) return;
  const int64_t i = q / n, j = q % n;
  const float v = static_cast<float>(static_cast<double>(K[q]) - cols[j] - rows[i] + *tot);
  K[q] = v;
  if (i == j) diag[i] = v;
}

// per row: {a_i K_ii, a_i K_ii^2, a_i sum_k a_k K_ik^2}
__global__ void kg_moment_rows_kernel(const float* K, const float* a, int64_t n, double* part) {
  const int64_t i = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  double s = 0.0;
  for (int64_t k = lane; k < n; k += 32) {
    const double v = K[i * n + k];
    s += static_cast<double>(a[k]) * v * v;
  }
  s = warp_sum(s);
  if (lane == 0) {
    const double ai = a[i], kii = K[i * n + i];
    part[i * 3 + 0] = ai * kii;
    part[i * 3 + 1] = ai * kii * kii;
    part[i * 3 + 2] = ai * s;
  }
}

// out[0] = 2 m4 + 2 m2^2 + 4 ||Sigma||^2, out[1] = m2 (one block, fixed order)
__global__ void kg_moment_total_kernel(const double* part, int64_t n, double* out) {
  __shared__ double red[3][8];
  double v[3] = {0.0, 0.0, 0.0};
  for (int64_t i = threadIdx.x; i < n; i += 256)
    for (int c = 0; c < 3; ++c) v[c] += part[i * 3 + c];
  for (int c = 0; c < 3; ++c) {
    const double w = warp_sum(v[c]);
    if ((threadIdx.x & 31) == 0) red[c][threadIdx.x >> 5] = w;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double m2 = 0.0, m4 = 0.0, s2 = 0.0;
    for (int q = 0; q < 8; ++q) {
      m2 += red[0][q];
      m4 += red[1][q];
      s2 += red[2][q];
    }
    out[0] = 2.0 * m4 + 2.0 * m2 * m2 + 4.0 * s2;
    out[1] = m2;
  }
}

// ------------------------------------------------------------ dense cost and Sinkhorn
__global__ void kg_outer_kernel(const float* a, const float* b, int64_t n, int64_t m, float* P) {
  const int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q < n * m) P[q] = a[q / m] * b[q % m];
}

// out_i = -eps ln sum_j w_j exp((h_j - C_ij)/eps), one warp per row
// (averaged with avg_i when avg is not null: Algorithm 3)
__global__ void kg_row_softmin_kernel(const float* C, int64_t n, int64_t m, const float* h,
                                      const float* logw, float eps, const float* avg, float* out) {
  const int64_t i = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  const float sc = kLog2e / eps;
  float M = kNegBig, S = 0.0f;
  for (int64_t j = lane; j < m; j += 32) {
    const float z = (h[j] - C[i * m + j]) * sc + logw[j] * kLog2e;
    if (z > M) {
      S = S * ex2(M - z) + 1.0f;
      M = z;
    } else {
      S += ex2(z - M);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float M2 = __shfl_xor_sync(0xffffffffu, M, o);
    const float S2 = __shfl_xor_sync(0xffffffffu, S, o);
    const float Mn = fmaxf(M, M2);
    S = S * ex2(M - Mn) + S2 * ex2(M2 - Mn);
    M = Mn;
  }
  if (lane == 0) {
    float v = -eps * kLn2 * (M + log2f(S));
    if (avg) v = 0.5f * (avg[i] + v);
    out[i] = v;
  }
}

// column softmin partials: block = 32 columns x 8 warps over a slice of rows
__global__ void __launch_bounds__(256)
    kg_col_partial_kernel(const float* C, int64_t n, int64_t m, const float* h, const float* logw,
                          float eps, int rows_per_split, float* pm, float* ps) {
  __shared__ float sm[8][32], ss[8][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t j = static_cast<int64_t>(blockIdx.x) * 32 + lane;
  const int64_t i0 = static_cast<int64_t>(blockIdx.y) * rows_per_split;
  const int64_t i1 = i0 + rows_per_split < n ? i0 + rows_per_split : n;
  const float sc = kLog2e / eps;
  float M = kNegBig, S = 0.0f;
  if (j < m) {
    for (int64_t i = i0 + w; i < i1; i += 8) {
      const float z = (h[i] - C[i * m + j]) * sc + logw[i] * kLog2e;
      if (z > M) {
        S = S * ex2(M - z) + 1.0f;
        M = z;
      } else {
        S += ex2(z - M);
      }
    }
  }
  sm[w][lane] = M;
  ss[w][lane] = S;
  __syncthreads();
  if (w == 0 && j < m) {
    float Mt = kNegBig;
    for (int q = 0; q < 8; ++q) Mt = fmaxf(Mt, sm[q][lane]);
    float St = 0.0f;
    for (int q = 0; q < 8; ++q) St += ss[q][lane] * ex2(sm[q][lane] - Mt);
    pm[static_cast<int64_t>(blockIdx.y) * m + j] = Mt;
    ps[static_cast<int64_t>(blockIdx.y) * m + j] = St;
  }
}

__global__ void kg_col_combine_kernel(const float* pm, const float* ps, int splits, int64_t m,
                                      float eps, const float* avg, float* out) {
  const int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= m) return;
  float M = kNegBig;
  for (int s = 0; s < splits; ++s) M = fmaxf(M, pm[static_cast<int64_t>(s) * m + j]);
  float S = 0.0f;
  for (int s = 0; s < splits; ++s)
    S += ps[static_cast<int64_t>(s) * m + j] * ex2(pm[static_cast<int64_t>(s) * m + j] - M);
  float v = -eps * kLn2 * (M + log2f(S));
  if (avg) v = 0.5f * (avg[j] + v);
  out[j] = v;
}

// pi_ij = a_i b_j exp((f_i + g_j - C_ij) / eps)
__global__ void kg_plan_kernel(const float* C, const float* a, const float* b, const float* f,
                               const float* g, int64_t n, int64_t m, float eps, float* P) {
  const int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= n * m) return;
  const int64_t i = q / m, j = q % m;
  P[q] = a[i] * b[j] * ex2((f[i] + g[j] - C[q]) * (kLog2e / eps));
}

// ------------------------------------------------------------ energy record
// per row i: {sum_j pi C_next, sum_j pi k l, sum_j pi (f + g - C_cur), r_i, sum_j pi C_cur}
__global__ void kg_energy_rows_kernel(const float* P, const float* Ccur, const float* Cnext,
                                      const float* k, const float* l, const float* f,
                                      const float* g, int64_t n, int64_t m, double* rp) {
  const int64_t i = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  double s1 = 0.0, st = 0.0, kl = 0.0, r = 0.0, s0 = 0.0;
  const double fi = f[i], ki = k[i];
  for (int64_t j = lane; j < m; j += 32) {
    const double p = P[i * m + j];
    s1 += p * Cnext[i * m + j];
    s0 += p * Ccur[i * m + j];
    st += p * ki * l[j];
    kl += p * (fi + g[j] - static_cast<double>(Ccur[i * m + j]));
    r += p;
  }
  s1 = warp_sum(s1);
  st = warp_sum(st);
  kl = warp_sum(kl);
  r = warp_sum(r);
  s0 = warp_sum(s0);
  if (lane == 0) {
    rp[i * 5 + 0] = s1;
    rp[i * 5 + 1] = st;
    rp[i * 5 + 2] = kl;
    rp[i * 5 + 3] = r;
    rp[i * 5 + 4] = s0;
  }
}

__global__ void kg_colsum_plan_kernel(const float* P, int64_t n, int64_t m, double* c) {
  const int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= m) return;
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += P[i * m + j];
  c[j] = s;
}

// state[0] = ||Gamma_t||^2 of the previous plan (updated here)
__global__ void kg_energy_finalize_kernel(const double* rp, int64_t n, const double* cs, int64_t m,
                                          const float* a, const float* b, const double* MX,
                                          const double* MY, float eps, double* state,
                                          double* en) {
  __shared__ double red[7][8];
  double v[7] = {0, 0, 0, 0, 0, 0, 0};   // s1, T, KL, mass, s0, row L1, col L1
  double rmax = 0.0, cmax = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += 256) {
    v[0] += rp[i * 5 + 0];
    v[1] += rp[i * 5 + 1];
    v[2] += rp[i * 5 + 2];
    v[3] += rp[i * 5 + 3];
    v[4] += rp[i * 5 + 4];
    const double d = fabs(rp[i * 5 + 3] - static_cast<double>(a[i]));
    v[5] += d;
    rmax = fmax(rmax, d / a[i]);
  }
  for (int64_t j = threadIdx.x; j < m; j += 256) {
    const double d = fabs(cs[j] - static_cast<double>(b[j]));
    v[6] += d;
    cmax = fmax(cmax, d / b[j]);
  }
  for (int c = 0; c < 7; ++c) {
    const double w = warp_sum(v[c]);
    if ((threadIdx.x & 31) == 0) red[c][threadIdx.x >> 5] = w;
  }
  rmax = warp_max(rmax);
  cmax = warp_max(cmax);
  __shared__ double rx[2][8];
  if ((threadIdx.x & 31) == 0) {
    rx[0][threadIdx.x >> 5] = rmax;
    rx[1][threadIdx.x >> 5] = cmax;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double t[7] = {0, 0, 0, 0, 0, 0, 0};
  double r1 = 0.0, c1 = 0.0;
  for (int q = 0; q < 8; ++q) {
    for (int c = 0; c < 7; ++c) t[c] += red[c][q];
    r1 = fmax(r1, rx[0][q]);
    c1 = fmax(c1, rx[1][q]);
  }
  const double T = t[1];
  const double G2 = -(4.0 * T + t[0]) / 16.0;        // <pi, K^X pi K^Y>
  const double Gx = -(4.0 * T + t[4]) / 16.0;        // <pi_{t+1}, K^X pi_t K^Y>
  const double Cc = MX[0] + MY[0] - 4.0 * MX[1] * MY[1];
  const double L = Cc - 8.0 * G2 - 4.0 * T;
  const double epsKL = t[2];
  const double dG2 = G2 - 2.0 * Gx + state[0];
  state[0] = G2;
  en[GW_EN_E] = L + epsKL;
  en[GW_EN_L] = L;
  en[GW_EN_KL] = epsKL / eps;
  en[GW_EN_C] = Cc;
  en[GW_EN_GAMMA2] = G2;
  en[GW_EN_T] = T;
  en[GW_EN_ROW_L1] = t[5];
  en[GW_EN_COL_L1] = t[6];
  en[GW_EN_ROW_RELMAX] = r1;
  en[GW_EN_COL_RELMAX] = c1;
  en[GW_EN_MASS] = t[3];
  en[GW_EN_DGAMMA] = sqrt(fmax(dG2, 0.0));
  en[GW_EN_EPS] = eps;
  bool finite = true;
  for (int k = 0; k < GW_EN_STATUS; ++k) finite = finite && isfinite(en[k]);
  en[GW_EN_STATUS] = finite ? 0.0 : static_cast<double>(GW_ENONFINITE);
  en[GW_EN_NINNER] = 0.0;
  en[GW_EN_STOPERR] = -1.0;
}

__global__ void kg_set_ninner_kernel(double* en, double v) {
  if (threadIdx.x == 0 && blockIdx.x == 0) en[GW_EN_NINNER] = v;
}

struct KgBufs {
  float *KX, *KY, *k, *l, *loga, *logb, *P, *C[2], *T, *f[2], *g[2], *pm, *ps;
  double *rows, *cols, *tot, *mpart, *MX, *MY, *rp, *cs, *state, *en;
  char* gemm_ws;           // split operands of the tensor-core products
  size_t gemm_ws_bytes;
};

int col_splits(int64_t n, int64_t m) {
  const int64_t cb = (m + 31) / 32;
  int64_t s = (4 * kSmCount + cb - 1) / cb;
  const int64_t smax = (n + 63) / 64;
  if (s > smax) s = smax;
  if (s < 1) s = 1;
  return static_cast<int>(s);
}

KgBufs carve_kg(Carver& c, int64_t n, int64_t m) {
  KgBufs B;
  const size_t nm = static_cast<size_t>(n) * m;
  const int64_t nn = n > m ? n : m;
  B.KX = c.take<float>(static_cast<size_t>(n) * n);
  B.KY = c.take<float>(static_cast<size_t>(m) * m);
  B.k = c.take<float>(n);
  B.l = c.take<float>(m);
  B.loga = c.take<float>(n);
  B.logb = c.take<float>(m);
  B.P = c.take<float>(nm);
  B.C[0] = c.take<float>(nm);
  B.C[1] = c.take<float>(nm);
  B.T = c.take<float>(nm);
  B.f[0] = c.take<float>(n);
  B.f[1] = c.take<float>(n);
  B.g[0] = c.take<float>(m);
  B.g[1] = c.take<float>(m);
  const int S = col_splits(n, m);
  B.pm = c.take<float>(static_cast<size_t>(S) * m);
  B.ps = c.take<float>(static_cast<size_t>(S) * m);
  B.rows = c.take<double>(nn);
  B.cols = c.take<double>(nn);
  B.tot = c.take<double>(2);
  B.mpart = c.take<double>(static_cast<size_t>(nn) * 3);
  B.MX = c.take<double>(2);
  B.MY = c.take<double>(2);
  B.rp = c.take<double>(static_cast<size_t>(n) * 5);
  B.cs = c.take<double>(m);
  B.state = c.take<double>(2);
  B.en = c.take<double>(GW_EN_LEN);
  const size_t g1 = gemm_tc_ws_bytes(m, n, m), g2 = gemm_tc_ws_bytes(m, n, n);
  B.gemm_ws_bytes = g1 > g2 ? g1 : g2;
  B.gemm_ws = c.take<char>(B.gemm_ws_bytes);
  return B;
}

int kernel_from_cost_dev(const float* Cm, const float* w, int64_t n, float* K, float* diag,
                         double* MOM, const KgBufs& B, cudaStream_t st) {
  const int64_t nn = n * n;
  kg_base_kernel<<<ceil_div(nn, 256), 256, 0, st>>>(Cm, n, K);
  GW_LAUNCH_CHECK();
  kg_rowsum_kernel<<<ceil_div(n * 32, 256), 256, 0, st>>>(K, w, n, B.rows);
  GW_LAUNCH_CHECK();
  kg_colsum_kernel<<<ceil_div(n, 256), 256, 0, st>>>(K, w, n, B.cols);
  GW_LAUNCH_CHECK();
  kg_total_kernel<<<1, 256, 0, st>>>(B.rows, w, n, B.tot);
  GW_LAUNCH_CHECK();
  kg_center_kernel<<<ceil_div(nn, 256), 256, 0, st>>>(K, n, B.rows, B.cols, B.tot, diag);
  GW_LAUNCH_CHECK();
  kg_moment_rows_kernel<<<ceil_div(n * 32, 256), 256, 0, st>>>(K, w, n, B.mpart);
  GW_LAUNCH_CHECK();
  kg_moment_total_kernel<<<1, 256, 0, st>>>(B.mpart, n, MOM);
  GW_LAUNCH_CHECK();
  return GW_OK;
}

// C = -4 k l^T - 16 K^X P K^Y (n x m row-major): T = P K^Y, then
// C = -16 K^X T - 4 k l^T, both through gemm_tc_f16x3 (out[r][s] =
// scale sum_k A[s][k] Bt[r][k] + coef u[r] v[s]); the kernels are symmetric,
// so K^Y serves as its own transpose, and T is read transposed.
int dense_cost(const KgBufs& B, const float* P, float* C, int64_t n, int64_t m, cudaStream_t st) {
  Carver g(B.gemm_ws, B.gemm_ws_bytes);
  GW_TRY(gemm_tc_f16x3(B.KY, false, P, false, m, n, m, 1.0f, nullptr, nullptr, 0.0f, B.T, g, st));
  Carver g2(B.gemm_ws, B.gemm_ws_bytes);
  GW_TRY(gemm_tc_f16x3(B.T, true, B.KX, false, m, n, n, -16.0f, B.k, B.l, -4.0f, C, g2, st));
  return GW_OK;
}

}  // namespace

size_t kernel_gw_ws_bytes(int64_t n, int64_t m) {
  Carver c(nullptr, ~size_t(0));
  carve_kg(c, n, m);
  return c.used();
}

int run_kernel_gw(const float* CX, const float* CY, const float* a, const float* b, int64_t n,
                  int64_t m, const gw_options& o, float* pi_out, float* f_out, float* g_out,
                  double* energy, double* history, void* ws, size_t ws_bytes, cudaStream_t st) {
  Carver c(ws, ws_bytes);
  const KgBufs B = carve_kg(c, n, m);
  GW_TRY(check_ws(c, ws));
  GW_REQUIRE(n * m <= (int64_t(1) << 31) && n <= (int64_t(1) << 30) && m <= (int64_t(1) << 30),
             GW_EUNSUPPORTED, "Kernel-GW is the small-N exact mode (n m <= 2^31)");
  // Algorithm 4 on both sides (the kernels of Algorithm 5)
  GW_TRY(kernel_from_cost_dev(CX, a, n, B.KX, B.k, B.MX, B, st));
  GW_TRY(kernel_from_cost_dev(CY, b, m, B.KY, B.l, B.MY, B, st));
  GW_TRY(launch_log(a, n, B.loga, st));
  GW_TRY(launch_log(b, m, B.logb, st));
  if (o.f0) {
    GW_CUDA_TRY(cudaMemcpyAsync(B.f[0], o.f0, sizeof(float) * n, cudaMemcpyDeviceToDevice, st));
  } else {
    GW_CUDA_TRY(cudaMemsetAsync(B.f[0], 0, sizeof(float) * n, st));
  }
  if (o.g0) {
    GW_CUDA_TRY(cudaMemcpyAsync(B.g[0], o.g0, sizeof(float) * m, cudaMemcpyDeviceToDevice, st));
  } else {
    GW_CUDA_TRY(cudaMemsetAsync(B.g[0], 0, sizeof(float) * m, st));
  }
  GW_CUDA_TRY(cudaMemsetAsync(B.state, 0, sizeof(double) * 2, st));
  // pi^0 = a b^T, its cost C_0
  kg_outer_kernel<<<ceil_div(n * m, 256), 256, 0, st>>>(a, b, n, m, B.P);
  GW_LAUNCH_CHECK();
  int cc = 0, fc = 0, gc = 0;
  GW_TRY(dense_cost(B, B.P, B.C[cc], n, m, st));
  const int S = col_splits(n, m);
  const int rows_per_split = static_cast<int>((n + S - 1) / S);
  for (int t = 0; t < o.n_outer; ++t) {
    float eps = o.eps;
    if (o.eps_final > 0.0f && o.eps_final != o.eps && o.n_outer > 1) {
      eps = static_cast<float>(static_cast<double>(o.eps) *
                               pow(static_cast<double>(o.eps_final) / o.eps,
                                   static_cast<double>(t) / (o.n_outer - 1)));
    }
    const float* C = B.C[cc];
    for (int it = 0; it < o.n_inner; ++it) {
      if (o.symmetric) {
        kg_row_softmin_kernel<<<ceil_div(n * 32, 256), 256, 0, st>>>(C, n, m, B.g[gc], B.logb, eps,
                                                                     B.f[fc], B.f[fc ^ 1]);
        GW_LAUNCH_CHECK();
        kg_col_partial_kernel<<<dim3(static_cast<unsigned>(ceil_div(m, 32)), S), 256, 0, st>>>(
            C, n, m, B.f[fc], B.loga, eps, rows_per_split, B.pm, B.ps);
        GW_LAUNCH_CHECK();
        kg_col_combine_kernel<<<ceil_div(m, 256), 256, 0, st>>>(B.pm, B.ps, S, m, eps, B.g[gc],
                                                                B.g[gc ^ 1]);
        GW_LAUNCH_CHECK();
      } else {
        kg_row_softmin_kernel<<<ceil_div(n * 32, 256), 256, 0, st>>>(C, n, m, B.g[gc], B.logb, eps,
                                                                     nullptr, B.f[fc ^ 1]);
        GW_LAUNCH_CHECK();
        kg_col_partial_kernel<<<dim3(static_cast<unsigned>(ceil_div(m, 32)), S), 256, 0, st>>>(
            C, n, m, B.f[fc ^ 1], B.loga, eps, rows_per_split, B.pm, B.ps);
        GW_LAUNCH_CHECK();
        kg_col_combine_kernel<<<ceil_div(m, 256), 256, 0, st>>>(B.pm, B.ps, S, m, eps, nullptr,
                                                                B.g[gc ^ 1]);
        GW_LAUNCH_CHECK();
      }
      fc ^= 1;
      gc ^= 1;
    }
    // pi^{t+1} (Algorithm 5) and the cost it induces, C_{t+1}
    kg_plan_kernel<<<ceil_div(n * m, 256), 256, 0, st>>>(C, a, b, B.f[fc], B.g[gc], n, m, eps, B.P);
    GW_LAUNCH_CHECK();
    GW_TRY(dense_cost(B, B.P, B.C[cc ^ 1], n, m, st));
    const bool last = t == o.n_outer - 1;
    double* rec = (o.record && history) ? history + static_cast<size_t>(t) * GW_EN_LEN : B.en;
    kg_energy_rows_kernel<<<ceil_div(n * 32, 256), 256, 0, st>>>(B.P, C, B.C[cc ^ 1], B.k, B.l,
                                                                 B.f[fc], B.g[gc], n, m, B.rp);
    GW_LAUNCH_CHECK();
    kg_colsum_plan_kernel<<<ceil_div(m, 256), 256, 0, st>>>(B.P, n, m, B.cs);
    GW_LAUNCH_CHECK();
    kg_energy_finalize_kernel<<<1, 256, 0, st>>>(B.rp, n, B.cs, m, a, b, B.MX, B.MY, eps, B.state,
                                                 rec);
    GW_LAUNCH_CHECK();
    kg_set_ninner_kernel<<<1, 32, 0, st>>>(rec, static_cast<double>(o.n_inner));
    GW_LAUNCH_CHECK();
    if (last) {
      GW_CUDA_TRY(cudaMemcpyAsync(energy, rec, sizeof(double) * GW_EN_LEN, cudaMemcpyDeviceToDevice,
                                  st));
    }
    cc ^= 1;
  }
  GW_CUDA_TRY(cudaMemcpyAsync(pi_out, B.P, sizeof(float) * n * m, cudaMemcpyDeviceToDevice, st));
  GW_CUDA_TRY(cudaMemcpyAsync(f_out, B.f[fc], sizeof(float) * n, cudaMemcpyDeviceToDevice, st));
  GW_CUDA_TRY(cudaMemcpyAsync(g_out, B.g[gc], sizeof(float) * m, cudaMemcpyDeviceToDevice, st));
  return GW_OK;
}

}  // namespace gw
