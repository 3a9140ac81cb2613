// Color / UV transfer (Appendix E): the barycentric projection of source
// attributes U (n x k) through the plan encoded by (f, g) on c_{Gamma_t},
//   out_j = sum_i pi_ij U_i / b_j,   pi_ij = a_i b_j exp((f_i + g_j - c_ij) / eps),
// a plan-weighted column reduction like the cross-covariance: one thread per
// target column, source rows streamed through shared memory (the features for
// the exponent, the attributes for the sums), row splits reduced in a fixed
// order (deterministic).
#include "gw_internal.cuh"

namespace gw {

namespace {

constexpr int kTrThreads = 128;
constexpr int kTrRows = 32;

struct TransferArgs {
  const float *X, *s, *a, *f, *U;  // source side
  const float *V, *t, *b, *g;      // target side (V = Gamma_t Y)
  float eps;
  int64_t n, m;
  int D, k;
  int rows_per_split;
  float* part;                     // [splits][m][k + 1]
};

template <int DP, int KP>
__global__ void __launch_bounds__(kTrThreads) transfer_kernel(TransferArgs P) {
  __shared__ __align__(16) float Xs[kTrRows][DP];
  __shared__ float Us[kTrRows][KP];
  __shared__ float rb[kTrRows], us[kTrRows];
  const int tid = threadIdx.x;
  const int64_t j = static_cast<int64_t>(blockIdx.x) * kTrThreads + tid;
  const bool ok = j < P.m;
  const float alpha = 16.0f * kLog2e / P.eps;
  const float beta = 4.0f * kLog2e / P.eps;
  const float hs = kLog2e / P.eps;
  float v[DP];
#pragma unroll
  for (int q = 0; q < DP; ++q) v[q] = (ok && q < P.D) ? P.V[j * P.D + q] * alpha : 0.0f;
  const float tj = ok ? P.t[j] : 0.0f;
  const float cb = ok ? P.g[j] * hs + log2f(P.b[j]) : kNegBig;
  float acc[KP];
#pragma unroll
  for (int q = 0; q < KP; ++q) acc[q] = 0.0f;
  float mass = 0.0f;
  const int64_t r_begin = static_cast<int64_t>(blockIdx.y) * P.rows_per_split;
  const int64_t r_end = r_begin + P.rows_per_split < P.n ? r_begin + P.rows_per_split : P.n;
  for (int64_t r0 = r_begin; r0 < r_end; r0 += kTrRows) {
    __syncthreads();
    for (int idx = tid; idx < kTrRows * DP; idx += kTrThreads) {
      const int ii = idx / DP, q = idx % DP;
      const int64_t i = r0 + ii;
      Xs[ii][q] = (i < r_end && q < P.D) ? P.X[i * P.D + q] : 0.0f;
    }
    for (int idx = tid; idx < kTrRows * KP; idx += kTrThreads) {
      const int ii = idx / KP, q = idx % KP;
      const int64_t i = r0 + ii;
      Us[ii][q] = (i < r_end && q < P.k) ? P.U[i * P.k + q] : 0.0f;
    }
    if (tid < kTrRows) {
      const int64_t i = r0 + tid;
      rb[tid] = i < r_end ? P.f[i] * hs + log2f(P.a[i]) : kNegBig;
      us[tid] = i < r_end ? P.s[i] * beta : 0.0f;
    }
    __syncthreads();
    for (int ii = 0; ii < kTrRows; ++ii) {
      // base-2 exponent of pi_ij: log2 a_i + log2 b_j + (f_i + g_j - c_ij) log2(e) / eps
      float z = fmaf(us[ii], tj, rb[ii] + cb);
#pragma unroll
      for (int q = 0; q < DP; ++q) z = fmaf(v[q], Xs[ii][q], z);
      const float p = ex2(z);
      mass += p;
#pragma unroll
      for (int q = 0; q < KP; ++q) acc[q] = fmaf(p, Us[ii][q], acc[q]);
    }
  }
  if (!ok) return;
  float* out = P.part + (static_cast<int64_t>(blockIdx.y) * P.m + j) * (P.k + 1);
  for (int q = 0; q < P.k; ++q) out[q] = acc[q];
  out[P.k] = mass;
}

// out_j = sum_splits part / b_j (fixed split order); mass_j = column sum
__global__ void transfer_reduce_kernel(const float* part, int splits, int64_t m, int k,
                                       const float* b, float* out, float* mass) {
  const int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= m) return;
  const double inv_b = 1.0 / static_cast<double>(b[j]);
  for (int q = 0; q <= k; ++q) {
    double sacc = 0.0;
    for (int sp = 0; sp < splits; ++sp) sacc += part[(static_cast<int64_t>(sp) * m + j) * (k + 1) + q];
    if (q < k) out[j * k + q] = static_cast<float>(sacc * inv_b);
    else if (mass) mass[j] = static_cast<float>(sacc);
  }
}

int splits_for(int64_t n, int64_t m) {
  const int64_t cb = ceil_div(m, kTrThreads);
  int64_t sp = ceil_div(4 * kSmCount, cb);
  const int64_t smax = ceil_div(n, 4 * kTrRows);
  if (sp > smax) sp = smax;
  if (sp < 1) sp = 1;
  return static_cast<int>(sp);
}

template <int KP>
int launch_transfer_k(const TransferArgs& A, dim3 grid, cudaStream_t st) {
  switch (A.D <= 4 ? 4 : A.D <= 8 ? 8 : A.D <= 16 ? 16 : A.D <= 32 ? 32 : A.D <= 64 ? 64 : 128) {
    case 4: transfer_kernel<4, KP><<<grid, kTrThreads, 0, st>>>(A); break;
    case 8: transfer_kernel<8, KP><<<grid, kTrThreads, 0, st>>>(A); break;
    case 16: transfer_kernel<16, KP><<<grid, kTrThreads, 0, st>>>(A); break;
    case 32: transfer_kernel<32, KP><<<grid, kTrThreads, 0, st>>>(A); break;
    case 64: transfer_kernel<64, KP><<<grid, kTrThreads, 0, st>>>(A); break;
    default: transfer_kernel<128, KP><<<grid, kTrThreads, 0, st>>>(A); break;
  }
  GW_LAUNCH_CHECK();
  return GW_OK;
}

}  // namespace

size_t transfer_ws_bytes(int64_t n, int64_t m, int D, int k) {
  Carver c(nullptr, ~size_t(0));
  c.take<float>(static_cast<size_t>(m) * D);
  c.take<float>(static_cast<size_t>(splits_for(n, m)) * m * (k + 1));
  return c.used();
}

int run_transfer(const gw_problem& p, const float* f, const float* g, const double* Gamma_t,
                 float eps, const float* U, int k, float* out, float* mass, Carver& ws,
                 cudaStream_t st) {
  const int sp = splits_for(p.n, p.m);
  float* V = ws.take<float>(static_cast<size_t>(p.m) * p.D);
  float* part = ws.take<float>(static_cast<size_t>(sp) * p.m * (k + 1));
  GW_REQUIRE(!ws.overflow, GW_ENOMEM, "workspace too small for the transfer");
  GW_TRY(launch_gamma_y(Gamma_t, p.Y, p.m, p.D, p.E, V, st));
  TransferArgs A;
  A.X = p.X;
  A.s = p.s;
  A.a = p.a;
  A.f = f;
  A.U = U;
  A.V = V;
  A.t = p.t;
  A.b = p.b;
  A.g = g;
  A.eps = eps;
  A.n = p.n;
  A.m = p.m;
  A.D = p.D;
  A.k = k;
  A.rows_per_split = static_cast<int>(ceil_div(p.n, sp));
  A.part = part;
  const dim3 grid(static_cast<unsigned>(ceil_div(p.m, kTrThreads)), sp);
  if (k <= 4) {
    GW_TRY(launch_transfer_k<4>(A, grid, st));
  } else if (k <= 8) {
    GW_TRY(launch_transfer_k<8>(A, grid, st));
  } else {
    GW_TRY(launch_transfer_k<16>(A, grid, st));
  }
  transfer_reduce_kernel<<<ceil_div(p.m, 256), 256, 0, st>>>(part, sp, p.m, k, p.b, out, mass);
  GW_LAUNCH_CHECK();
  return GW_OK;
}

}  // namespace gw
