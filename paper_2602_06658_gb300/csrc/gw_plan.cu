// Plan-weighted reductions of CNT-GW (the Xtilde and Gamma_{t+1} steps of
// Algorithm 1, Theorem 3.3), the moments behind C(alpha, beta) (Lemma, Appendix C.1),
// the marginals and the energy record, FP32 CUDA-core form.
//
// The plan pi_ij = a_i b_j exp((f_i + g_j - C_ij)/eps) is rebuilt tile by tile
// from the potentials and never stored.  All cross-CTA sums go through fixed
// per-block partial buffers reduced in a fixed order (no atomics), so results
// are bitwise reproducible run to run.
#include <math.h>

#include "gw_internal.cuh"

namespace gw {

namespace {

constexpr int kThreads = 128;
constexpr int kBR = 32;          // rows per shared-memory tile
constexpr int kRedBlocks = 148;  // blocks of the second-stage reductions
constexpr int kStats = 8;

int dpad(int D) {
  if (D <= 4) return 4;
  if (D <= 8) return 8;
  if (D <= 16) return 16;
  if (D <= 32) return 32;
  if (D <= 64) return 64;
  return 128;
}

__device__ __forceinline__ uint64_t pk2(float lo, float hi) {
  uint64_t p;
  asm("mov.b64 %0, {%1, %2};" : "=l"(p) : "f"(lo), "f"(hi));
  return p;
}
__device__ __forceinline__ void upk2(uint64_t p, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(p));
}
__device__ __forceinline__ uint64_t fm2(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

struct ColSumArgs {
  const float* X;  // n x D
  const float* s;
  const float* a;
  const float* f;
  const float* V;  // m x D  (V_j = Gamma_t Y_j)
  const float* t;
  const float* b;
  const float* g;
  float eps;
  int64_t n, m;
  int D;
  int rows_per_split;
  float* Wp;       // [splits][m][D+2]
  float* Ep;       // [splits][m][2]: A_j, B_j of the KL term (or null)
  const int* cond; // run only when *cond != 0 (null: always)
};

// W_j = sum_i pi_ij [X_i, s_i, 1] over one row split, one column per thread;
// with P.Ep also the KL partials A_j = sum_i pi_ij log2(pi_ij / b_j) and
// B_j = sum_i pi_ij log a_i (KL(pi | a x b) = sum_j ln2 A_j - B_j).
template <int DP>
__global__ void __launch_bounds__(kThreads) plan_colsum_kernel(ColSumArgs P) {
  __shared__ __align__(16) float Xs[kBR][DP];
  __shared__ float rb[kBR];
  __shared__ float us[kBR];
  __shared__ float ss[kBR];
  __shared__ float la[kBR];
  if (P.cond != nullptr && *P.cond == 0) return;   // the tensor-core pass succeeded

  const int tid = threadIdx.x;
  const int64_t j = static_cast<int64_t>(blockIdx.x) * kThreads + tid;
  const bool colok = j < P.m;
  const float inv_eps = 1.0f / P.eps;
  const float alpha = 16.0f * kLog2e * inv_eps;
  const float beta = 4.0f * kLog2e * inv_eps;
  const float hs = kLog2e * inv_eps;

  float v[DP];
#pragma unroll
  for (int k = 0; k < DP; ++k) v[k] = (colok && k < P.D) ? P.V[j * P.D + k] * alpha : 0.0f;
  const float tj = colok ? P.t[j] : 0.0f;
  const float cb = colok ? P.g[j] * hs + log2f(P.b[j]) : kNegBig;

  uint64_t acc2[DP / 2];
#pragma unroll
  for (int k = 0; k < DP / 2; ++k) acc2[k] = pk2(0.0f, 0.0f);
  float acc_s = 0.0f, acc_1 = 0.0f, acc_z = 0.0f, acc_la = 0.0f;
  const bool ent = P.Ep != nullptr;

  const int64_t r_begin = static_cast<int64_t>(blockIdx.y) * P.rows_per_split;
  const int64_t r_end = r_begin + P.rows_per_split < P.n ? r_begin + P.rows_per_split : P.n;
  for (int64_t r0 = r_begin; r0 < r_end; r0 += kBR) {
    __syncthreads();
    for (int idx = tid; idx < kBR * DP; idx += kThreads) {
      const int ii = idx / DP, k = idx % DP;
      const int64_t i = r0 + ii;
      Xs[ii][k] = (i < r_end && k < P.D) ? P.X[i * P.D + k] : 0.0f;
    }
    if (tid < kBR) {
      const int64_t i = r0 + tid;
      if (i < r_end) {
        rb[tid] = P.f[i] * hs + log2f(P.a[i]);
        us[tid] = P.s[i] * beta;
        ss[tid] = P.s[i];
        la[tid] = P.a[i] > 0.0f ? logf(P.a[i]) : 0.0f;   // zero weight: p = 0
      } else {
        rb[tid] = kNegBig;
        us[tid] = 0.0f;
        ss[tid] = 0.0f;
        la[tid] = 0.0f;
      }
    }
    __syncthreads();
    // packed FP32x2 arithmetic: the dot product and the accumulation both
    // run as fma.rn.f32x2 on feature pairs
#pragma unroll 2
    for (int ii = 0; ii < kBR; ++ii) {
      const float4* xr = reinterpret_cast<const float4*>(&Xs[ii][0]);
      uint64_t z2 = pk2(fmaf(us[ii], tj, rb[ii] + cb), 0.0f);
#pragma unroll
      for (int k4 = 0; k4 < DP / 4; ++k4) {
        const float4 xv = xr[k4];
        z2 = fm2(pk2(v[4 * k4 + 0], v[4 * k4 + 1]), pk2(xv.x, xv.y), z2);
        z2 = fm2(pk2(v[4 * k4 + 2], v[4 * k4 + 3]), pk2(xv.z, xv.w), z2);
      }
      float z0, z1;
      upk2(z2, z0, z1);
      const float z = z0 + z1;   // log2 pi_ij
      const float p = ex2(fminf(z, 126.0f));
      if (ent) {
        acc_z = fmaf(p, fmaxf(z, -1000.0f), acc_z);   // z = -inf (zero weight) has p = 0
        acc_la = fmaf(p, la[ii], acc_la);
      }
      const uint64_t pp = pk2(p, p);
#pragma unroll
      for (int k4 = 0; k4 < DP / 4; ++k4) {
        const float4 xv = xr[k4];
        acc2[2 * k4 + 0] = fm2(pp, pk2(xv.x, xv.y), acc2[2 * k4 + 0]);
        acc2[2 * k4 + 1] = fm2(pp, pk2(xv.z, xv.w), acc2[2 * k4 + 1]);
      }
      acc_s = fmaf(p, ss[ii], acc_s);
      acc_1 += p;
    }
  }
  if (!colok) return;
  float* out = P.Wp + (static_cast<int64_t>(blockIdx.y) * P.m + j) * (P.D + 2);
#pragma unroll
  for (int k = 0; k < DP / 2; ++k) {
    float lo, hi;
    upk2(acc2[k], lo, hi);
    if (2 * k < P.D) out[2 * k] = lo;
    if (2 * k + 1 < P.D) out[2 * k + 1] = hi;
  }
  out[P.D] = acc_s;
  out[P.D + 1] = acc_1;
  if (ent) {
    // sum_i pi_ij (log2 pi_ij - log2 b_j) = acc_z - log2(b_j) acc_1
    float* e2 = P.Ep + (static_cast<int64_t>(blockIdx.y) * P.m + j) * 2;
    e2[0] = acc_z - (P.b[j] > 0.0f ? log2f(P.b[j]) : 0.0f) * acc_1;
    e2[1] = acc_la;
  }
}

// KL partials: per block of kRedBlocks, sum over its targets j (splits added
// in order, FP64) of ln2 A_j - B_j.
__global__ void __launch_bounds__(256)
    kl_partial_kernel(const float* Ep, int splits, int64_t m, double* Kp) {
  double v = 0.0;
  for (int64_t j = static_cast<int64_t>(blockIdx.x) * 256 + threadIdx.x; j < m;
       j += static_cast<int64_t>(gridDim.x) * 256) {
    double A = 0.0, B = 0.0;
    for (int s = 0; s < splits; ++s) {
      A += static_cast<double>(Ep[(static_cast<int64_t>(s) * m + j) * 2 + 0]);
      B += static_cast<double>(Ep[(static_cast<int64_t>(s) * m + j) * 2 + 1]);
    }
    v += 0.6931471805599453 * A - B;
  }
  __shared__ double red[8];
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < 8; ++q) t += red[q];
    Kp[blockIdx.x] = t;
  }
}

// W[j][k] = sum over row splits (float64, fixed order).
__global__ void reduce_splits_kernel(const float* Wp, int splits, int64_t count, double* W) {
  const int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= count) return;
  double acc = 0.0;
  for (int s = 0; s < splits; ++s) acc += static_cast<double>(Wp[s * count + q]);
  W[q] = acc;
}

// Per-block partials of Gamma = sum_j W_j[0:D] Y_j^T and the column stats.
// Gp[block][D*E + kStats]:  stats = {T, sum g colsum, mass, col L1, col relmax}
__global__ void __launch_bounds__(256)
    gamma_partial_kernel(const double* W, const float* Y, const float* t, const float* b,
                         const float* g, int64_t m, int D, int E, double* Gp) {
  extern __shared__ double sh[];
  const int W2 = D + 2;
  double* Wsh = sh;                 // [32][D+2]
  double* Ysh = sh + 32 * W2;       // [32][E]
  const int tid = threadIdx.x;
  const int DE = D * E;
  const int64_t chunk = (m + gridDim.x - 1) / gridDim.x;
  const int64_t j0 = blockIdx.x * chunk;
  const int64_t j1 = j0 + chunk < m ? j0 + chunk : m;

  double acc[64];  // up to 256*64 = 16384 = 128*128 entries
  const int per = (DE + 255) / 256;
  for (int q = 0; q < per; ++q) acc[q] = 0.0;
  double T = 0.0, gc = 0.0, mass = 0.0, l1 = 0.0, rmax = 0.0;

  for (int64_t jb = j0; jb < j1; jb += 32) {
    __syncthreads();
    const int cnt = static_cast<int>(j1 - jb < 32 ? j1 - jb : 32);
    for (int idx = tid; idx < cnt * W2; idx += 256) Wsh[idx] = W[jb * W2 + idx];
    for (int idx = tid; idx < cnt * E; idx += 256) Ysh[idx] = static_cast<double>(Y[jb * E + idx]);
    __syncthreads();
    for (int jj = 0; jj < cnt; ++jj) {
      for (int q = 0; q < per; ++q) {
        const int e_idx = tid + q * 256;
        if (e_idx < DE) {
          const int d = e_idx / E, e = e_idx % E;
          acc[q] = fma(Wsh[jj * W2 + d], Ysh[jj * E + e], acc[q]);
        }
      }
    }
    if (tid < cnt) {
      const int64_t j = jb + tid;
      const double col = Wsh[tid * W2 + D + 1];
      const double bj = static_cast<double>(b[j]);
      T += Wsh[tid * W2 + D] * static_cast<double>(t[j]);
      gc += static_cast<double>(g[j]) * col;
      mass += col;
      l1 += fabs(col - bj);
      rmax = fmax(rmax, fabs(col - bj) / bj);
    }
  }
  double* out = Gp + static_cast<int64_t>(blockIdx.x) * (DE + kStats);
  for (int q = 0; q < per; ++q) {
    const int e_idx = tid + q * 256;
    if (e_idx < DE) out[e_idx] = acc[q];
  }
  // block reduction of the stats (fixed order)
  __shared__ double red[5][8];
  T = warp_sum(T);
  gc = warp_sum(gc);
  mass = warp_sum(mass);
  l1 = warp_sum(l1);
  rmax = warp_max(rmax);
  const int w = tid >> 5, l = tid & 31;
  if (l == 0) {
    red[0][w] = T;
    red[1][w] = gc;
    red[2][w] = mass;
    red[3][w] = l1;
    red[4][w] = rmax;
  }
  __syncthreads();
  if (tid == 0) {
    double v[5] = {0, 0, 0, 0, 0};
    for (int q = 0; q < 8; ++q) {
      for (int k = 0; k < 4; ++k) v[k] += red[k][q];
      v[4] = fmax(v[4], red[4][q]);
    }
    for (int k = 0; k < 5; ++k) out[DE + k] = v[k];
    for (int k = 5; k < kStats; ++k) out[DE + k] = 0.0;
  }
}

// Weighted moments of centered features: partial [m2, m4, Sigma (DxD)].
__global__ void __launch_bounds__(256)
    moments_partial_kernel(const float* X, const float* a, int64_t n, int D, double* Mp) {
  extern __shared__ double sh[];
  double* Xsh = sh;              // [32][D]
  double* ash = sh + 32 * D;     // [32]
  const int tid = threadIdx.x;
  const int DD = D * D;
  const int per = (DD + 255) / 256;
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t i0 = blockIdx.x * chunk;
  const int64_t i1 = i0 + chunk < n ? i0 + chunk : n;
  double acc[64];
  for (int q = 0; q < per; ++q) acc[q] = 0.0;
  double m2 = 0.0, m4 = 0.0;
  for (int64_t ib = i0; ib < i1; ib += 32) {
    __syncthreads();
    const int cnt = static_cast<int>(i1 - ib < 32 ? i1 - ib : 32);
    for (int idx = tid; idx < cnt * D; idx += 256) Xsh[idx] = static_cast<double>(X[ib * D + idx]);
    if (tid < cnt) ash[tid] = static_cast<double>(a[ib + tid]);
    __syncthreads();
    for (int ii = 0; ii < cnt; ++ii) {
      for (int q = 0; q < per; ++q) {
        const int e_idx = tid + q * 256;
        if (e_idx < DD) {
          const int d = e_idx / D, e = e_idx % D;
          acc[q] = fma(ash[ii] * Xsh[ii * D + d], Xsh[ii * D + e], acc[q]);
        }
      }
    }
    if (tid < cnt) {
      double sq = 0.0;
      for (int k = 0; k < D; ++k) sq = fma(Xsh[tid * D + k], Xsh[tid * D + k], sq);
      m2 += ash[tid] * sq;
      m4 += ash[tid] * sq * sq;
    }
  }
  double* out = Mp + static_cast<int64_t>(blockIdx.x) * (DD + 2);
  for (int q = 0; q < per; ++q) {
    const int e_idx = tid + q * 256;
    if (e_idx < DD) out[2 + e_idx] = acc[q];
  }
  __shared__ double red[2][8];
  m2 = warp_sum(m2);
  m4 = warp_sum(m4);
  if ((tid & 31) == 0) {
    red[0][tid >> 5] = m2;
    red[1][tid >> 5] = m4;
  }
  __syncthreads();
  if (tid == 0) {
    double v0 = 0.0, v1 = 0.0;
    for (int q = 0; q < 8; ++q) {
      v0 += red[0][q];
      v1 += red[1][q];
    }
    out[0] = v0;
    out[1] = v1;
  }
}

// Row marginal r_i = a_i exp((f_i - S_b(g)_i)/eps): partial {sum f r, L1, relmax}.
__global__ void __launch_bounds__(256)
    row_stats_kernel(const float* a, const float* f, const float* fhat, float eps, int64_t n,
                     double* Rp) {
  const int tid = threadIdx.x;
  double fr = 0.0, l1 = 0.0, rmax = 0.0;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * 256 + tid; i < n;
       i += static_cast<int64_t>(gridDim.x) * 256) {
    const double ai = a[i];
    const double r = ai * exp((static_cast<double>(f[i]) - static_cast<double>(fhat[i])) / eps);
    fr += static_cast<double>(f[i]) * r;
    l1 += fabs(r - ai);
    rmax = fmax(rmax, fabs(r - ai) / ai);
  }
  __shared__ double red[3][8];
  fr = warp_sum(fr);
  l1 = warp_sum(l1);
  rmax = warp_max(rmax);
  if ((tid & 31) == 0) {
    red[0][tid >> 5] = fr;
    red[1][tid >> 5] = l1;
    red[2][tid >> 5] = rmax;
  }
  __syncthreads();
  if (tid == 0) {
    double v0 = 0, v1 = 0, v2 = 0;
    for (int q = 0; q < 8; ++q) {
      v0 += red[0][q];
      v1 += red[1][q];
      v2 = fmax(v2, red[2][q]);
    }
    Rp[blockIdx.x * 4 + 0] = v0;
    Rp[blockIdx.x * 4 + 1] = v1;
    Rp[blockIdx.x * 4 + 2] = v2;
    Rp[blockIdx.x * 4 + 3] = 0.0;
  }
}

// Marginal error of the stop rule from consecutive potentials (no extra
// softmin): for one side with weights w, sum_i w_i |exp(k (p0_i - p1_i) / eps) - 1|.
// Algorithm 3 (k = 2): p1 = (p0 + S)/2, so the sums of the plan (f^n, g^n)
// are w exp(2 (p0 - p1) / eps).  Algorithm 2 (k = 1, columns only): the
// columns of (f^{n+1}, g^n) are b exp((g^n - g^{n+1}) / eps).  Fixed grid,
// fixed-order sums: deterministic.
__global__ void __launch_bounds__(256)
    marg_err_partial_kernel(const float* f0, const float* f1, const float* a, int64_t n,
                            const float* g0, const float* g1, const float* b, int64_t m,
                            double kf, double kg, double* part) {
  const int tid = threadIdx.x;
  double acc = 0.0;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * 256;
  if (kf != 0.0) {
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * 256 + tid; i < n; i += stride)
      acc += static_cast<double>(a[i]) *
             fabs(expm1(kf * (static_cast<double>(f0[i]) - static_cast<double>(f1[i]))));
  }
  for (int64_t j = static_cast<int64_t>(blockIdx.x) * 256 + tid; j < m; j += stride)
    acc += static_cast<double>(b[j]) *
           fabs(expm1(kg * (static_cast<double>(g0[j]) - static_cast<double>(g1[j]))));
  __shared__ double red[8];
  acc = warp_sum(acc);
  if ((tid & 31) == 0) red[tid >> 5] = acc;
  __syncthreads();
  if (tid == 0) {
    double v = 0.0;
    for (int q = 0; q < 8; ++q) v += red[q];
    part[blockIdx.x] = v;
  }
}

__global__ void marg_err_final_kernel(const double* part, int nb, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double v = 0.0;
    for (int q = 0; q < nb; ++q) v += part[q];
    *out = v;
  }
}

// rec[GW_EN_NINNER] = iterations run, rec[GW_EN_STOPERR] = *err (or -1)
__global__ void record_extra_kernel(double* rec, double n_inner, const double* err,
                                    const unsigned* gave_up, const unsigned* gave_up0) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    rec[GW_EN_NINNER] = n_inner;
    rec[GW_EN_STOPERR] = err ? *err : -1.0;
    // a bounded wait gave up since the call began: its rows were written as
    // NaN, and the record says why
    if (gave_up != nullptr && gave_up0 != nullptr && *gave_up != *gave_up0)
      rec[GW_EN_STATUS] = static_cast<double>(GW_ETIMEOUT);
  }
}

struct FinalizeArgs {
  const double* Gp;
  int gblocks;
  int D, E;
  const double* Gamma_t;  // D x E or null
  double* Gamma_out;      // D x E or null
  double* stats_out;      // kStats or null
  const double* Rp;       // row stats partials or null (no energy)
  int rblocks;
  const double* Kp;       // KL partials (kl_partial_kernel)
  int kblocks;
  const double* MpX;      // moments partials or null (use C_pre)
  const double* MpY;
  int mblocks;
  const double* C_pre;
  double* C_out;          // where C is stored when computed (or null)
  double* energy;         // GW_EN_LEN or null
  float eps;
};

__device__ double block_sum256(double v, double* red) {
  v = warp_sum(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  for (int q = 0; q < 8; ++q) s += red[q];
  return s;
}

__device__ double moments_C_part(const double* Mp, int mblocks, int D, double* red,
                                 double* m2_out) {
  // returns 2 m4 + 2 m2^2 + 4 ||Sigma||^2 and sets *m2_out
  const int DD = D * D;
  double sig2 = 0.0;
  for (int e_idx = threadIdx.x; e_idx < DD; e_idx += 256) {
    double v = 0.0;
    for (int b = 0; b < mblocks; ++b) v += Mp[static_cast<int64_t>(b) * (DD + 2) + 2 + e_idx];
    sig2 += v * v;
  }
  sig2 = block_sum256(sig2, red);
  double m2 = 0.0, m4 = 0.0;
  for (int b = 0; b < mblocks; ++b) {
    m2 += Mp[static_cast<int64_t>(b) * (DD + 2) + 0];
    m4 += Mp[static_cast<int64_t>(b) * (DD + 2) + 1];
  }
  *m2_out = m2;
  return 2.0 * m4 + 2.0 * m2 * m2 + 4.0 * sig2;
}

__global__ void __launch_bounds__(256) finalize_kernel(FinalizeArgs F) {
  __shared__ double red[8];
  const int DE = F.D * F.E;
  double g2 = 0.0, gdot = 0.0, dg2 = 0.0;
  for (int e_idx = threadIdx.x; e_idx < DE; e_idx += 256) {
    double v = 0.0;
    for (int b = 0; b < F.gblocks; ++b) v += F.Gp[static_cast<int64_t>(b) * (DE + kStats) + e_idx];
    if (F.Gamma_out) F.Gamma_out[e_idx] = v;
    g2 += v * v;
    if (F.Gamma_t) {
      const double gt = F.Gamma_t[e_idx];
      gdot += gt * v;
      dg2 += (v - gt) * (v - gt);
    } else {
      dg2 += v * v;
    }
  }
  g2 = block_sum256(g2, red);
  gdot = block_sum256(gdot, red);
  dg2 = block_sum256(dg2, red);

  double st[kStats] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int b = 0; b < F.gblocks; ++b) {
    const double* p = F.Gp + static_cast<int64_t>(b) * (DE + kStats) + DE;
    for (int k = 0; k < 4; ++k) st[k] += p[k];
    st[4] = fmax(st[4], p[4]);
  }
  if (F.stats_out && threadIdx.x < kStats) F.stats_out[threadIdx.x] = st[threadIdx.x];

  double C = 0.0;
  if (F.energy) {
    if (F.C_pre) {
      C = *F.C_pre;
    } else {
      double m2x = 0.0, m2y = 0.0;
      const double cx = moments_C_part(F.MpX, F.mblocks, F.D, red, &m2x);
      const double cy = moments_C_part(F.MpY, F.mblocks, F.E, red, &m2y);
      C = cx + cy - 4.0 * m2x * m2y;
    }
  }
  if (threadIdx.x != 0 || !F.energy) {
    if (threadIdx.x == 0 && F.C_out && !F.energy) *F.C_out = C;
    return;
  }
  double fr = 0.0, rl1 = 0.0, rmax = 0.0;
  for (int b = 0; b < F.rblocks; ++b) {
    fr += F.Rp[b * 4 + 0];
    rl1 += F.Rp[b * 4 + 1];
    rmax = fmax(rmax, F.Rp[b * 4 + 2]);
  }
  const double T = st[0];
  const double eps = F.eps;
  // KL as the plan's own sum of pi log(pi / (a b)) (partials of the plan
  // pass).  Through the potentials it would be (sum f r + sum g c + 16
  // <Gamma_t, Gamma_{t+1}> + 4 T) / eps, whose terms are ~|f| / eps each and
  // cancel: at small eps the FP32 rounding of the row sums r behind it moved
  // KL by ~0.3%.
  (void)fr;
  (void)gdot;
  double KL = 0.0;
  for (int b = 0; b < F.kblocks; ++b) KL += F.Kp[b];
  const double epsKL = eps * KL;
  const double L = C - 8.0 * g2 - 4.0 * T;
  double* en = F.energy;
  en[GW_EN_E] = L + epsKL;
  en[GW_EN_L] = L;
  en[GW_EN_KL] = KL;
  en[GW_EN_C] = C;
  en[GW_EN_GAMMA2] = g2;
  en[GW_EN_T] = T;
  en[GW_EN_ROW_L1] = rl1;
  en[GW_EN_COL_L1] = st[3];
  en[GW_EN_ROW_RELMAX] = rmax;
  en[GW_EN_COL_RELMAX] = st[4];
  en[GW_EN_MASS] = st[2];
  en[GW_EN_DGAMMA] = sqrt(dg2);
  en[GW_EN_EPS] = eps;
  bool finite = true;
  for (int k = 0; k < GW_EN_STATUS; ++k) finite = finite && isfinite(en[k]);
  en[GW_EN_STATUS] = finite ? 0.0 : static_cast<double>(GW_ENONFINITE);
  en[14] = 0.0;
  en[15] = 0.0;
  if (F.C_out) *F.C_out = C;
}

// V[j][d] = sum_e Gamma[d][e] Y[j][e]
__global__ void gamma_y_kernel(const double* Gamma, const float* Y, int64_t m, int D, int E,
                               float* V) {
  const int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= m * D) return;
  const int64_t j = q / D;
  const int d = static_cast<int>(q % D);
  double acc = 0.0;
  for (int e = 0; e < E; ++e) acc = fma(Gamma[d * E + e], static_cast<double>(Y[j * E + e]), acc);
  V[q] = static_cast<float>(acc);
}

__global__ void __launch_bounds__(256)
    moments_C_kernel(const double* MpX, const double* MpY, int mblocks, int D, int E, double* C) {
  __shared__ double red[8];
  double m2x = 0.0, m2y = 0.0;
  const double cx = moments_C_part(MpX, mblocks, D, red, &m2x);
  const double cy = moments_C_part(MpY, mblocks, E, red, &m2y);
  if (threadIdx.x == 0) *C = cx + cy - 4.0 * m2x * m2y;
}

__global__ void log_kernel(const float* w, int64_t n, float* logw) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) logw[i] = logf(w[i]);
}

int colsum_row_splits(int64_t n, int64_t m) {
  const int cblocks = ceil_div(m, kThreads);
  int splits = ceil_div(4 * kSmCount, cblocks);
  const int max_splits = ceil_div(n, 256);
  if (splits > max_splits) splits = max_splits;
  if (splits < 1) splits = 1;
  return splits;
}

struct CrossCovLayout {
  float* V;
  float* Wp;
  float* Ep;       // KL partials (energy only)
  double* W;
  double* Gp;
  double* Kp;      // [kRedBlocks] (energy only)
  int splits;      // row splits of the partials actually written
  int rows_per_split;
};

CrossCovLayout carve_cross_cov(Carver& c, int64_t n, int64_t m, int D, int E, bool need_W) {
  CrossCovLayout L;
  L.splits = colsum_row_splits(n, m);
  L.rows_per_split = ceil_div(n, L.splits);
  L.rows_per_split = ((L.rows_per_split + kBR - 1) / kBR) * kBR;
  L.splits = ceil_div(n, L.rows_per_split);
  L.V = c.take<float>(static_cast<size_t>(m) * D);
  L.Wp = c.take<float>(static_cast<size_t>(L.splits) * m * (D + 2));
  L.W = need_W ? c.take<double>(static_cast<size_t>(m) * (D + 2)) : nullptr;
  L.Gp = c.take<double>(static_cast<size_t>(kRedBlocks) * (D * E + kStats));
  L.Ep = c.take<float>(static_cast<size_t>(L.splits) * m * 2);
  L.Kp = c.take<double>(static_cast<size_t>(kRedBlocks));
  return L;
}

}  // namespace

int launch_gamma_y(const double* Gamma, const float* Y, int64_t m, int D, int E, float* V,
                   cudaStream_t st) {
  const int64_t total = m * D;
  if (total == 0) return GW_OK;
  gamma_y_kernel<<<ceil_div(total, 256), 256, 0, st>>>(Gamma, Y, m, D, E, V);
  GW_LAUNCH_CHECK();
  return GW_OK;
}

size_t cross_cov_ws_bytes(int64_t n, int64_t m, int D, int E, int prec) {
  Carver c(nullptr, ~size_t(0));
  carve_cross_cov(c, n, m, D, E, true);
  return c.used() + (plan_tc_supported(D, prec) ? plan_tc_ws_bytes(n, m, D, prec) : 0);
}

static void launch_colsum(const ColSumArgs& A, dim3 grid, cudaStream_t st) {
  switch (dpad(A.D)) {
    case 4: plan_colsum_kernel<4><<<grid, kThreads, 0, st>>>(A); break;
    case 8: plan_colsum_kernel<8><<<grid, kThreads, 0, st>>>(A); break;
    case 16: plan_colsum_kernel<16><<<grid, kThreads, 0, st>>>(A); break;
    case 32: plan_colsum_kernel<32><<<grid, kThreads, 0, st>>>(A); break;
    case 64: plan_colsum_kernel<64><<<grid, kThreads, 0, st>>>(A); break;
    default: plan_colsum_kernel<128><<<grid, kThreads, 0, st>>>(A); break;
  }
}

// Enqueue everything up to the Gamma partials; the caller finalizes.
static int cross_cov_stage(const PlanArgs& p, int prec, double* W_user, Carver& ws,
                           cudaStream_t st, CrossCovLayout* out, bool want_kl = false) {
  GW_REQUIRE(prec >= GW_PREC_FP32 && prec <= GW_PREC_FP8, GW_EUNSUPPORTED, "precision %d", prec);
  // FP8 plan sums must see the softmin's rounded features: only the tensor-core form does
  GW_REQUIRE(prec != GW_PREC_FP8 || plan_tc_supported(p.D, prec), GW_EUNSUPPORTED,
             "GW_PREC_FP8 plan sums need D + 3 <= 80 (D = %d)", p.D);
  CrossCovLayout L = carve_cross_cov(ws, p.n, p.m, p.D, p.E, W_user == nullptr);
  GW_REQUIRE(!ws.overflow, GW_ENOMEM, "workspace too small for cross-covariance");
  if (W_user) L.W = W_user;
  GW_TRY(launch_gamma_y(p.Gamma_t, p.Y, p.m, p.D, p.E, L.V, st));
  ColSumArgs A;
  A.X = p.X;
  A.s = p.s;
  A.a = p.a;
  A.f = p.f;
  A.V = L.V;
  A.t = p.t;
  A.b = p.b;
  A.g = p.g;
  A.eps = p.eps;
  A.n = p.n;
  A.m = p.m;
  A.D = p.D;
  A.cond = nullptr;
  A.Ep = nullptr;
  const int64_t count = p.m * (p.D + 2);
  if (plan_tc_supported(p.D, prec)) {
    // both contractions on the tensor cores; the FP32 kernel recomputes the
    // same partials only when that pass flagged a value it could not hold
    float* Wp = nullptr;
    int splits = 0, rps = 0;
    int* flag = nullptr;
    float* Ep = nullptr;
    GW_TRY(run_plan_tc(p, prec, L.V, &Wp, want_kl ? &Ep : nullptr, &splits, &rps, &flag, ws, st));
    A.rows_per_split = rps;
    A.Wp = Wp;
    A.Ep = Ep;
    A.cond = flag;
    launch_colsum(A, dim3(ceil_div(p.m, kThreads), splits), st);
    GW_LAUNCH_CHECK();
    reduce_splits_kernel<<<ceil_div(count, 256), 256, 0, st>>>(Wp, splits, count, L.W);
    GW_LAUNCH_CHECK();
    L.Ep = Ep;
    L.splits = splits;
  } else {
    A.rows_per_split = L.rows_per_split;
    A.Wp = L.Wp;
    A.Ep = want_kl ? L.Ep : nullptr;
    launch_colsum(A, dim3(ceil_div(p.m, kThreads), L.splits), st);
    GW_LAUNCH_CHECK();
    reduce_splits_kernel<<<ceil_div(count, 256), 256, 0, st>>>(L.Wp, L.splits, count, L.W);
    GW_LAUNCH_CHECK();
  }
  if (want_kl) {
    kl_partial_kernel<<<kRedBlocks, 256, 0, st>>>(L.Ep, L.splits, p.m, L.Kp);
    GW_LAUNCH_CHECK();
  }
  const size_t shbytes = sizeof(double) * 32 * (p.D + 2 + p.E);
  gamma_partial_kernel<<<kRedBlocks, 256, shbytes, st>>>(L.W, p.Y, p.t, p.b, p.g, p.m, p.D, p.E,
                                                         L.Gp);
  GW_LAUNCH_CHECK();
  *out = L;
  return GW_OK;
}

int run_cross_cov(const PlanArgs& p, int prec, double* Gamma_out, double* stats, double* W,
                  Carver& ws, cudaStream_t st) {
  CrossCovLayout L;
  GW_TRY(cross_cov_stage(p, prec, W, ws, st, &L));
  FinalizeArgs F{};
  F.Gp = L.Gp;
  F.gblocks = kRedBlocks;
  F.D = p.D;
  F.E = p.E;
  F.Gamma_t = p.Gamma_t;
  F.Gamma_out = Gamma_out;
  F.stats_out = stats;
  F.eps = p.eps;
  finalize_kernel<<<1, 256, 0, st>>>(F);
  GW_LAUNCH_CHECK();
  return GW_OK;
}

size_t moments_ws_bytes(int64_t n, int64_t m, int D, int E) {
  (void)n;
  (void)m;
  Carver c(nullptr, ~size_t(0));
  c.take<double>(static_cast<size_t>(kRedBlocks) * (D * D + 2));
  c.take<double>(static_cast<size_t>(kRedBlocks) * (E * E + 2));
  return c.used();
}

static int moments_stage(const float* X, const float* a, int64_t n, int D, const float* Y,
                         const float* b, int64_t m, int E, Carver& ws, cudaStream_t st,
                         double** MpX, double** MpY) {
  *MpX = ws.take<double>(static_cast<size_t>(kRedBlocks) * (D * D + 2));
  *MpY = ws.take<double>(static_cast<size_t>(kRedBlocks) * (E * E + 2));
  GW_REQUIRE(!ws.overflow, GW_ENOMEM, "workspace too small for moments");
  moments_partial_kernel<<<kRedBlocks, 256, sizeof(double) * 32 * (D + 1), st>>>(X, a, n, D, *MpX);
  GW_LAUNCH_CHECK();
  moments_partial_kernel<<<kRedBlocks, 256, sizeof(double) * 32 * (E + 1), st>>>(Y, b, m, E, *MpY);
  GW_LAUNCH_CHECK();
  return GW_OK;
}

int run_moments(const float* X, const float* a, int64_t n, int D, const float* Y, const float* b,
                int64_t m, int E, double* C, Carver& ws, cudaStream_t st) {
  double *MpX, *MpY;
  GW_TRY(moments_stage(X, a, n, D, Y, b, m, E, ws, st, &MpX, &MpY));
  moments_C_kernel<<<1, 256, 0, st>>>(MpX, MpY, kRedBlocks, D, E, C);
  GW_LAUNCH_CHECK();
  return GW_OK;
}

int launch_log(const float* w, int64_t n, float* logw, cudaStream_t st) {
  if (n == 0) return GW_OK;
  log_kernel<<<ceil_div(n, 256), 256, 0, st>>>(w, n, logw);
  GW_LAUNCH_CHECK();
  return GW_OK;
}

size_t energy_ws_bytes(int64_t n, int64_t m, int D, int E, int prec) {
  Carver c(nullptr, ~size_t(0));
  carve_cross_cov(c, n, m, D, E, true);
  c.take<double>(static_cast<size_t>(kRedBlocks) * (D * D + 2));
  c.take<double>(static_cast<size_t>(kRedBlocks) * (E * E + 2));
  c.take<float>(static_cast<size_t>(n));        // fhat
  c.take<float>(static_cast<size_t>(m));        // log b
  c.take<double>(static_cast<size_t>(kRedBlocks) * 4);
  return c.used() + softmin_ws_bytes(n, m, D, prec) + 256 +
         (plan_tc_supported(D, prec) ? plan_tc_ws_bytes(n, m, D, prec) : 0);
}

int run_marginal_error(const float* f0, const float* f1, const float* a, int64_t n,
                       const float* g0, const float* g1, const float* b, int64_t m, float eps,
                       bool symmetric, double* part, double* out, cudaStream_t st) {
  const double inv = 1.0 / static_cast<double>(eps);
  marg_err_partial_kernel<<<kMargBlocks, 256, 0, st>>>(f0, f1, a, n, g0, g1, b, m,
                                                       symmetric ? 2.0 * inv : 0.0,
                                                       symmetric ? 2.0 * inv : inv, part);
  GW_LAUNCH_CHECK();
  marg_err_final_kernel<<<1, 32, 0, st>>>(part, kMargBlocks, out);
  GW_LAUNCH_CHECK();
  return GW_OK;
}

int launch_record_extra(double* rec, int n_inner, const double* err, const unsigned* gave_up0,
                        cudaStream_t st) {
  record_extra_kernel<<<1, 32, 0, st>>>(rec, static_cast<double>(n_inner), err,
                                        gave_up0 ? wait_ctl().gave_up : nullptr, gave_up0);
  GW_LAUNCH_CHECK();
  return GW_OK;
}

int run_energy(const PlanArgs& p, int prec, const double* C_pre, const float* logb_pre,
               double* energy, double* Gamma_out, Carver& ws, cudaStream_t st) {
  CrossCovLayout L;
  GW_TRY(cross_cov_stage(p, prec, nullptr, ws, st, &L, true));
  double *MpX = nullptr, *MpY = nullptr;
  if (!C_pre) GW_TRY(moments_stage(p.X, p.a, p.n, p.D, p.Y, p.b, p.m, p.E, ws, st, &MpX, &MpY));
  float* fhat = ws.take<float>(static_cast<size_t>(p.n));
  float* logb = logb_pre ? nullptr : ws.take<float>(static_cast<size_t>(p.m));
  double* Rp = ws.take<double>(static_cast<size_t>(kRedBlocks) * 4);
  GW_REQUIRE(!ws.overflow, GW_ENOMEM, "workspace too small for energy");
  if (!logb_pre) GW_TRY(launch_log(p.b, p.m, logb, st));
  // raw row softmin with the final g on c_{Gamma_t}: fhat = S_b(g)
  // (L.V holds Gamma_t Y from the cross-covariance stage)
  SoftminTask T{};
  T.A = p.X;
  T.B = L.V;
  T.sA = p.s;
  T.sB = p.t;
  T.h = p.g;
  T.logw = logb_pre ? logb_pre : logb;
  T.avg_with = nullptr;
  T.est = p.f;   // at convergence S_b(g) is close to f
  T.out = fhat;
  T.n = p.n;
  T.m = p.m;
  T.K = p.D;
  T.eps = p.eps;
  GW_TRY(launch_softmin(&T, 1, prec, ws, st));
  row_stats_kernel<<<kRedBlocks, 256, 0, st>>>(p.a, p.f, fhat, p.eps, p.n, Rp);
  GW_LAUNCH_CHECK();
  FinalizeArgs F{};
  F.Gp = L.Gp;
  F.gblocks = kRedBlocks;
  F.D = p.D;
  F.E = p.E;
  F.Gamma_t = p.Gamma_t;
  F.Gamma_out = Gamma_out;
  F.stats_out = nullptr;
  F.Rp = Rp;
  F.rblocks = kRedBlocks;
  F.Kp = L.Kp;
  F.kblocks = kRedBlocks;
  F.MpX = MpX;
  F.MpY = MpY;
  F.mblocks = kRedBlocks;
  F.C_pre = C_pre;
  F.energy = energy;
  F.eps = p.eps;
  finalize_kernel<<<1, 256, 0, st>>>(F);
  GW_LAUNCH_CHECK();
  return GW_OK;
}

}  // namespace gw
