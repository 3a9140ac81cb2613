// Persistent batched solver: many small CNT-GW problems in one launch.
//
// Each CTA takes problems from a device work queue and runs Algorithm 1 for
// one problem at a time entirely in shared memory: the moments constant C of
// the Lemma (App. C.1), then per outer step Zbar = Gamma_t Y, n_inner Sinkhorn
// iterations on the bilinear cost (Algorithm 3, or Algorithm 2), the plan-
// weighted sums W_j = sum_i pi_ij [X_i, s_i, 1] that give Gamma_{t+1} and T,
// and the energy record.  The arithmetic is that of the FP32 path of
// gw_solve (the same base-2 exponent, FP64 cross-covariance and energy),
// except that each softmin sum is taken against the current potential as a
// known shift, with the exact online max/sum of gw_solve (chunks of 8
// columns) only where that sum leaves a safe range; a problem never depends
// on the others, and
// every reduction runs in a fixed order inside its CTA, so a result is
// bitwise the same alone and in any batch.
//
// Shared memory of one problem (n, m padded to multiples of 8; padding
// entries carry a bias of -1e30 and zero features, so they add nothing):
//   rows:    rp0[i] = (bias_i, s_i, X_i0, X_i1), rp1[i] = (X_i2, X_i3) when D > 2,
//            f, f_next, log a
//   columns: cp0[j] = (bias_j, t_j, V_j0, V_j1), cp1[j] = (V_j2, V_j3) when D > 2,
//            g, g_next, log b
// with bias the base-2 potential term of the other half-step (h log2(e) / eps
// + log2(e) log w) and V = Gamma_t Y.
#include <math.h>

#include <mutex>

#include "gw_internal.cuh"

namespace gw {

namespace {

constexpr int kBt = 512;                 // threads per CTA
constexpr int kBw = kBt / 32;            // warps per CTA
constexpr int kBChunk = 8;               // columns per online-max update
constexpr int kBRed = 16 + 6;            // doubles reduced at once (D E <= 16, + stats)

struct BatchArgs {
  int nprob;
  const int64_t* xo;
  const int64_t* yo;
  int64_t n_max, m_max, n_pad, m_pad;
  int D, E;
  const float *X, *Y, *s, *t, *a, *b, *eps0, *eps1;
  int n_outer, n_inner, symmetric;
  float *f, *g;
  double *Gamma, *Gamma_plan, *energy, *history;
  int* queue;
};

__host__ __device__ __forceinline__ int64_t pad8(int64_t v) { return (v + 7) / 8 * 8; }

// floats of shared memory per row (or column) entry
int batch_floats_per_entry(int D) { return (D > 2 ? 8 : 4) + 3; }

size_t batch_smem_bytes(int64_t n_max, int64_t m_max, int D) {
  const int64_t pts = pad8(n_max) + pad8(m_max);
  return static_cast<size_t>(pts) * batch_floats_per_entry(D) * sizeof(float) +
         sizeof(double) * (kBw * kBRed + 2 * 16 + 32);
}

// Sum (or max, for the entries flagged in `is_max`) of cnt per-thread values
// over the CTA, in a fixed order: warps by shuffles, then warp 0 over the
// warps.  Every thread gets the results in out[0..cnt).
__device__ void block_reduce(double* v, int cnt, unsigned is_max, double* red, double* out) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  for (int k = 0; k < cnt; ++k) {
    double x = v[k];
    const bool mx = (is_max >> k) & 1u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double y = __shfl_xor_sync(0xffffffffu, x, o);
      x = mx ? fmax(x, y) : x + y;
    }
    if (l == 0) red[w * kBRed + k] = x;
  }
  __syncthreads();
  if (threadIdx.x < cnt) {
    const int k = threadIdx.x;
    const bool mx = (is_max >> k) & 1u;
    double acc = red[k];
    for (int q = 1; q < kBw; ++q) acc = mx ? fmax(acc, red[q * kBRed + k]) : acc + red[q * kBRed + k];
    out[k] = acc;
  }
  __syncthreads();
}

__device__ __forceinline__ uint64_t b_pack2(float lo, float hi) {
  uint64_t p;
  asm("mov.b64 %0, {%1, %2};" : "=l"(p) : "f"(lo), "f"(hi));
  return p;
}
__device__ __forceinline__ void b_unpack2(uint64_t p, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(p));
}
__device__ __forceinline__ uint64_t b_add2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

// Exponent of one cell in base 2, minus `shift`, as a chain of FMAs that
// starts from the other side's bias:
//   bias_l - shift + beta sq_k sq_l + alpha <F_k, F_l>.
template <int DP>
__device__ __forceinline__ float cell(const float (&a)[DP], float u, float nshift, float4 o,
                                      float4 o2) {
  float z = fmaf(u, o.y, o.x + nshift);
  z = fmaf(a[0], o.z, z);
  z = fmaf(a[1], o.w, z);
  if constexpr (DP == 4) {
    z = fmaf(a[2], o2.x, z);
    z = fmaf(a[3], o2.y, z);
  }
  return z;
}

// Exact base-2 log-sum-exp of one own entry with a running max (updated per
// chunk of 8), for the entries whose shifted sum left the safe range.
template <int DP>
__device__ float lse2_exact(const float (&a)[DP], float u, const float4* oth0, const float4* oth1,
                            int n_oth_pad) {
  float M = kNegBig, S = 0.0f;
  for (int l0 = 0; l0 < n_oth_pad; l0 += kBChunk) {
    float z[kBChunk];
#pragma unroll
    for (int c = 0; c < kBChunk; ++c)
      z[c] = cell<DP>(a, u, 0.0f, oth0[l0 + c], DP == 4 ? oth1[l0 + c] : make_float4(0, 0, 0, 0));
    float cm = z[0];
#pragma unroll
    for (int c = 1; c < kBChunk; ++c) cm = fmaxf(cm, z[c]);
    if (cm > M) {
      S *= ex2(M - cm);
      M = cm;
    }
    float tsum = 0.0f;
#pragma unroll
    for (int c = 0; c < kBChunk; ++c) tsum += ex2(z[c] - M);
    S += tsum;
  }
  return M + log2f(S);
}

// One log-sum-exp half-step for the entries of one side ("own": rows for the
// row softmin, columns for the column one) against the packed entries of
// the other side:
//   out_k = -eps ln2 LSE2_l [bias_l + beta sq_k sq_l + alpha <F_k, F_l>],
// averaged with avg_k when avg is not null (Algorithm 3).  Two own entries
// per thread share every broadcast load of the other side.  The sum runs
// against a known shift instead of a running max: the own side's current
// potential est_k, whose softmin is close to est_k, gives LSE2 ~ -est_k hs,
// so sum_l 2^(z_kl + est_k hs) stays near 1 and needs neither a max nor a
// subtraction per cell (the two entries' terms are added as one FP32x2
// pair).  An entry whose sum lands outside [2^-20, 2^100] (the estimate far
// off: overflow, or most of the mass below the FP32 range) is redone exactly.
template <int DP>
__device__ void lse_side(const float4* own0, const float4* own1, int n_own, const float4* oth0,
                         const float4* oth1, int n_oth_pad, float alpha, float beta, float eps,
                         float hs, const float* est, const float* avg, float* out) {
  for (int k0 = threadIdx.x; k0 < n_own; k0 += 2 * kBt) {
    const int k1 = k0 + kBt;
    const bool has1 = k1 < n_own;
    const float4 p0 = own0[k0];
    const float4 p1 = has1 ? own0[k1] : make_float4(0.f, 0.f, 0.f, 0.f);
    float a0[DP], a1[DP];
    a0[0] = p0.z * alpha;
    a0[1] = p0.w * alpha;
    a1[0] = p1.z * alpha;
    a1[1] = p1.w * alpha;
    if constexpr (DP == 4) {
      const float4 q0 = own1[k0];
      const float4 q1 = has1 ? own1[k1] : make_float4(0.f, 0.f, 0.f, 0.f);
      a0[2] = q0.x * alpha;
      a0[3] = q0.y * alpha;
      a1[2] = q1.x * alpha;
      a1[3] = q1.y * alpha;
    }
    const float u0 = p0.y * beta, u1 = p1.y * beta;
    const float ns0 = est[k0] * hs, ns1 = has1 ? est[k1] * hs : 0.0f;   // -shift
    uint64_t S01 = b_pack2(0.0f, 0.0f);
    for (int l0 = 0; l0 < n_oth_pad; l0 += kBChunk) {
#pragma unroll
      for (int c = 0; c < kBChunk; ++c) {
        const float4 o = oth0[l0 + c];
        const float4 o2 = DP == 4 ? oth1[l0 + c] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float z0 = cell<DP>(a0, u0, ns0, o, o2);
        const float z1 = cell<DP>(a1, u1, ns1, o, o2);
        S01 = b_add2(S01, b_pack2(ex2(z0), ex2(z1)));
      }
    }
    float S0, S1;
    b_unpack2(S01, S0, S1);
    float l0v = S0 >= 9.5367431640625e-07f && S0 <= 1.2676506e30f ? log2f(S0) - ns0
                                                                 : lse2_exact<DP>(a0, u0, oth0, oth1, n_oth_pad);
    float v0 = -eps * kLn2 * l0v;
    if (avg) v0 = 0.5f * (avg[k0] + v0);
    out[k0] = v0;
    if (has1) {
      float l1v = S1 >= 9.5367431640625e-07f && S1 <= 1.2676506e30f ? log2f(S1) - ns1
                                                                   : lse2_exact<DP>(a1, u1, oth0, oth1, n_oth_pad);
      float v1 = -eps * kLn2 * l1v;
      if (avg) v1 = 0.5f * (avg[k1] + v1);
      out[k1] = v1;
    }
  }
}

// Algorithm 1 for problem q (sources x0 .. x0 + n, targets y0 .. y0 + m).
template <int DP>
__device__ void solve_one(const BatchArgs& A, int q, int64_t x0, int64_t y0, int n, int m,
                          unsigned char* bsm) {
  const int tid = threadIdx.x;
  const int D = A.D, E = A.E, DE = D * E;
  const int64_t NP = A.n_pad, MP = A.m_pad;
  float4* rp0 = reinterpret_cast<float4*>(bsm);
  float4* rp1 = rp0 + NP;
  float4* cp0 = rp1 + (DP == 4 ? NP : 0);
  float4* cp1 = cp0 + MP;
  float* fbuf = reinterpret_cast<float*>(cp1 + (DP == 4 ? MP : 0));   // [2][NP]
  float* la = fbuf + 2 * NP;
  float* gbuf = la + NP;                                               // [2][MP]
  float* lb = gbuf + 2 * MP;
  double* red = reinterpret_cast<double*>(lb + MP);
  double* Gt = red + kBw * kBRed;
  double* Gn = Gt + 16;
  double* rr = Gn + 16;                                                // [32] reduction results
  const int npad = static_cast<int>(pad8(n)), mpad = static_cast<int>(pad8(m));

  // ---- load the problem; f = g = 0, Gamma = 0
  for (int i = tid; i < npad; i += kBt) {
    float x[4] = {0.f, 0.f, 0.f, 0.f};
    float si = 0.f;
    if (i < n) {
      for (int k = 0; k < D; ++k) x[k] = A.X[(x0 + i) * D + k];
      si = A.s[x0 + i];
      la[i] = logf(A.a[x0 + i]);
    } else {
      la[i] = 0.f;
    }
    rp0[i] = make_float4(kNegBig, si, x[0], x[1]);
    if constexpr (DP == 4) rp1[i] = make_float4(x[2], x[3], 0.f, 0.f);
    fbuf[i] = 0.f;
    fbuf[NP + i] = 0.f;
  }
  for (int j = tid; j < mpad; j += kBt) {
    cp0[j] = make_float4(kNegBig, j < m ? A.t[y0 + j] : 0.f, 0.f, 0.f);
    if constexpr (DP == 4) cp1[j] = make_float4(0.f, 0.f, 0.f, 0.f);
    lb[j] = j < m ? logf(A.b[y0 + j]) : 0.f;
    gbuf[j] = 0.f;
    gbuf[MP + j] = 0.f;
  }
  if (tid < 16) Gt[tid] = 0.0;

  // ---- C(alpha, beta) of the Lemma from the weighted moments (FP64):
  // 2 m4 + 2 m2^2 + 4 ||Sigma||^2 per side, minus 4 m2_X m2_Y
  double C = 0.0, m2x = 0.0;
  for (int side = 0; side < 2; ++side) {
    const int K = side == 0 ? D : E;
    const int cnt = side == 0 ? n : m;
    double v[kBRed];
    for (int k = 0; k < kBRed; ++k) v[k] = 0.0;
    for (int i = tid; i < cnt; i += kBt) {
      double xv[4] = {0.0, 0.0, 0.0, 0.0};
      double w, sq = 0.0;
      if (side == 0) {
        w = A.a[x0 + i];
        for (int k = 0; k < K; ++k) xv[k] = A.X[(x0 + i) * D + k];
      } else {
        w = A.b[y0 + i];
        for (int k = 0; k < K; ++k) xv[k] = A.Y[(y0 + i) * E + k];
      }
      for (int k = 0; k < K; ++k) sq = fma(xv[k], xv[k], sq);
      v[0] += w * sq;
      v[1] += w * sq * sq;
      for (int d = 0; d < K; ++d)
        for (int e = 0; e < K; ++e) v[2 + d * K + e] = fma(w * xv[d], xv[e], v[2 + d * K + e]);
    }
    block_reduce(v, 2 + K * K, 0u, red, rr);
    double sig2 = 0.0;
    for (int k = 0; k < K * K; ++k) sig2 += rr[2 + k] * rr[2 + k];
    C += 2.0 * rr[1] + 2.0 * rr[0] * rr[0] + 4.0 * sig2;
    if (side == 0) m2x = rr[0];
    else C -= 4.0 * m2x * rr[0];
    __syncthreads();
  }

  int fc = 0, gc = 0;
  for (int t = 0; t < A.n_outer; ++t) {
    float eps = A.eps0[q];
    if (A.eps1 != nullptr && A.eps1[q] != eps && A.n_outer > 1) {
      const double e0 = eps, e1 = A.eps1[q];
      eps = static_cast<float>(e0 * pow(e1 / e0, static_cast<double>(t) / (A.n_outer - 1)));
    }
    const float inv_eps = 1.0f / eps;
    const float alpha = 16.0f * kLog2e * inv_eps;   // scale of <X_i, V_j>
    const float beta = 4.0f * kLog2e * inv_eps;     // scale of s_i t_j
    const float hs = kLog2e * inv_eps;              // scale of a potential

    // Zbar_j = Gamma_t Y_j (Algorithm 1), in FP64, stored as FP32
    for (int j = tid; j < m; j += kBt) {
      float v[4] = {0.f, 0.f, 0.f, 0.f};
      for (int d = 0; d < D; ++d) {
        double acc = 0.0;
        for (int e = 0; e < E; ++e) acc = fma(Gt[d * E + e], static_cast<double>(A.Y[(y0 + j) * E + e]), acc);
        v[d] = static_cast<float>(acc);
      }
      float4 c = cp0[j];
      c.z = v[0];
      c.w = v[1];
      cp0[j] = c;
      if constexpr (DP == 4) cp1[j] = make_float4(v[2], v[3], 0.f, 0.f);
    }

    for (int it = 0; it < A.n_inner; ++it) {
      float* f = fbuf + fc * NP;
      float* g = gbuf + gc * MP;
      if (A.symmetric) {
        // Algorithm 3: both half-steps read iterate n, then average
        for (int i = tid; i < n; i += kBt) rp0[i].x = f[i] * hs + la[i] * kLog2e;
        for (int j = tid; j < m; j += kBt) cp0[j].x = g[j] * hs + lb[j] * kLog2e;
        __syncthreads();
        lse_side<DP>(rp0, rp1, n, cp0, cp1, mpad, alpha, beta, eps, hs, f, f, fbuf + (fc ^ 1) * NP);
        lse_side<DP>(cp0, cp1, m, rp0, rp1, npad, alpha, beta, eps, hs, g, g, gbuf + (gc ^ 1) * MP);
        __syncthreads();
        fc ^= 1;
        gc ^= 1;
      } else {
        // Algorithm 2: f from g^n, then g from f^{n+1}
        for (int j = tid; j < m; j += kBt) cp0[j].x = g[j] * hs + lb[j] * kLog2e;
        __syncthreads();
        lse_side<DP>(rp0, rp1, n, cp0, cp1, mpad, alpha, beta, eps, hs, f, nullptr, fbuf + (fc ^ 1) * NP);
        __syncthreads();
        fc ^= 1;
        f = fbuf + fc * NP;
        for (int i = tid; i < n; i += kBt) rp0[i].x = f[i] * hs + la[i] * kLog2e;
        __syncthreads();
        lse_side<DP>(cp0, cp1, m, rp0, rp1, npad, alpha, beta, eps, hs, g, nullptr, gbuf + (gc ^ 1) * MP);
        __syncthreads();
        gc ^= 1;
      }
    }
    const float* f = fbuf + fc * NP;
    const float* g = gbuf + gc * MP;

    // ---- W_j = sum_i pi_ij [X_i, s_i, 1] with pi_ij = 2^(rb_i + cb_j + beta s_i t_j
    // + alpha <X_i, V_j>), rb = f log2(e) / eps + log2 a; then Gamma_{t+1} = sum_j
    // W_j[0:D] Y_j^T, T = sum_j W_j[D] t_j and the column statistics (FP64)
    for (int i = tid; i < n; i += kBt) rp0[i].x = f[i] * hs + log2f(A.a[x0 + i]);
    __syncthreads();
    double v[kBRed];
    for (int k = 0; k < kBRed; ++k) v[k] = 0.0;
    for (int j = tid; j < m; j += kBt) {
      const float4 c = cp0[j];
      const float tj = c.y;
      const float cb = g[j] * hs + log2f(A.b[y0 + j]);
      float vv[DP];
      vv[0] = c.z * alpha;
      vv[1] = c.w * alpha;
      if constexpr (DP == 4) {
        const float4 c2 = cp1[j];
        vv[2] = c2.x * alpha;
        vv[3] = c2.y * alpha;
      }
      float W[DP + 2];
      for (int k = 0; k < DP + 2; ++k) W[k] = 0.0f;
      float Wz = 0.0f, Wla = 0.0f;   // sum_i pi_ij log2 pi_ij, sum_i pi_ij log a_i
      for (int i = 0; i < n; ++i) {
        const float4 r = rp0[i];
        float z = fmaf(r.y * beta, tj, r.x + cb);
        z = fmaf(vv[0], r.z, z);
        z = fmaf(vv[1], r.w, z);
        float r2x = 0.f, r2y = 0.f;
        if constexpr (DP == 4) {
          const float4 r2 = rp1[i];
          r2x = r2.x;
          r2y = r2.y;
          z = fmaf(vv[2], r2x, z);
          z = fmaf(vv[3], r2y, z);
        }
        const float p = ex2(fminf(z, 126.0f));
        W[0] = fmaf(p, r.z, W[0]);
        W[1] = fmaf(p, r.w, W[1]);
        if constexpr (DP == 4) {
          W[2] = fmaf(p, r2x, W[2]);
          W[3] = fmaf(p, r2y, W[3]);
        }
        W[DP] = fmaf(p, r.y, W[DP]);
        W[DP + 1] += p;
        Wz = fmaf(p, fmaxf(z, -1000.0f), Wz);          // p = 0 where z = -inf
        Wla = fmaf(p, fmaxf(la[i], -1.0e30f), Wla);
      }
      const double col = W[DP + 1];
      const double bj = A.b[y0 + j];
      // KL(pi | a x b) over this column: sum_i pi_ij log(pi_ij / (a_i b_j))
      v[DE + 5] += 0.6931471805599453 * (static_cast<double>(Wz) - log2(bj) * col) -
                   static_cast<double>(Wla);
      for (int d = 0; d < D; ++d)
        for (int e = 0; e < E; ++e)
          v[d * E + e] = fma(static_cast<double>(W[d]), static_cast<double>(A.Y[(y0 + j) * E + e]),
                             v[d * E + e]);
      v[DE + 0] += static_cast<double>(W[DP]) * static_cast<double>(tj);
      v[DE + 1] += static_cast<double>(g[j]) * col;
      v[DE + 2] += col;
      v[DE + 3] += fabs(col - bj);
      v[DE + 4] = fmax(v[DE + 4], fabs(col - bj) / bj);
    }
    block_reduce(v, DE + 6, 1u << (DE + 4), red, rr);
    if (tid < DE) Gn[tid] = rr[tid];
    const double T = rr[DE], mass = rr[DE + 2], cl1 = rr[DE + 3], crmax = rr[DE + 4],
                 KLd = rr[DE + 5];
    __syncthreads();

    const bool last = t == A.n_outer - 1;
    if (last || A.history != nullptr) {
      // energy record (Lemma, App. C.1): fhat = S_b(g) on c_{Gamma_t}, row
      // marginal r_i = a_i exp((f_i - fhat_i) / eps)
      for (int j = tid; j < m; j += kBt) cp0[j].x = g[j] * hs + lb[j] * kLog2e;
      __syncthreads();
      float* fhat = fbuf + (fc ^ 1) * NP;
      lse_side<DP>(rp0, rp1, n, cp0, cp1, mpad, alpha, beta, eps, hs, f, nullptr, fhat);
      __syncthreads();
      double w3[kBRed];
      for (int k = 0; k < kBRed; ++k) w3[k] = 0.0;
      for (int i = tid; i < n; i += kBt) {
        const double ai = A.a[x0 + i];
        const double r = ai * exp((static_cast<double>(f[i]) - static_cast<double>(fhat[i])) /
                                  static_cast<double>(eps));
        w3[1] += fabs(r - ai);
        w3[2] = fmax(w3[2], fabs(r - ai) / ai);
      }
      block_reduce(w3, 3, 4u, red, rr);
      if (tid == 0) {
        double g2 = 0.0, dg2 = 0.0;
        for (int k = 0; k < DE; ++k) {
          g2 += Gn[k] * Gn[k];
          dg2 += (Gn[k] - Gt[k]) * (Gn[k] - Gt[k]);
        }
        // KL summed over the plan's own entries (the potential form, f r +
        // g c + 16 <Gamma_t, Gamma_{t+1}> + 4 T over eps, cancels terms of
        // size |f| / eps)
        const double L = C - 8.0 * g2 - 4.0 * T;
        double en[GW_EN_LEN];
        en[GW_EN_E] = L + static_cast<double>(eps) * KLd;
        en[GW_EN_L] = L;
        en[GW_EN_KL] = KLd;
        en[GW_EN_C] = C;
        en[GW_EN_GAMMA2] = g2;
        en[GW_EN_T] = T;
        en[GW_EN_ROW_L1] = rr[1];
        en[GW_EN_COL_L1] = cl1;
        en[GW_EN_ROW_RELMAX] = rr[2];
        en[GW_EN_COL_RELMAX] = crmax;
        en[GW_EN_MASS] = mass;
        en[GW_EN_DGAMMA] = sqrt(dg2);
        en[GW_EN_EPS] = eps;
        bool finite = true;
        for (int k = 0; k < GW_EN_STATUS; ++k) finite = finite && isfinite(en[k]);
        en[GW_EN_STATUS] = finite ? 0.0 : static_cast<double>(GW_ENONFINITE);
        en[GW_EN_NINNER] = A.n_inner;
        en[GW_EN_STOPERR] = -1.0;
        if (A.history)
          for (int k = 0; k < GW_EN_LEN; ++k)
            A.history[(static_cast<int64_t>(q) * A.n_outer + t) * GW_EN_LEN + k] = en[k];
        if (last)
          for (int k = 0; k < GW_EN_LEN; ++k) A.energy[static_cast<int64_t>(q) * GW_EN_LEN + k] = en[k];
      }
    }
    if (last && tid < DE) {
      A.Gamma_plan[static_cast<int64_t>(q) * DE + tid] = Gt[tid];
      A.Gamma[static_cast<int64_t>(q) * DE + tid] = Gn[tid];
    }
    __syncthreads();
    if (tid < DE) Gt[tid] = Gn[tid];
    __syncthreads();
  }
  const float* f = fbuf + fc * NP;
  const float* g = gbuf + gc * MP;
  for (int i = tid; i < n; i += kBt) A.f[x0 + i] = f[i];
  for (int j = tid; j < m; j += kBt) A.g[y0 + j] = g[j];
  __syncthreads();
}

template <int DP>
__global__ void __launch_bounds__(kBt, 2) batch_solve_kernel(BatchArgs A) {
  extern __shared__ __align__(16) unsigned char bsm[];
  __shared__ int qsh;
  for (;;) {
    if (threadIdx.x == 0) qsh = atomicAdd(A.queue, 1);
    __syncthreads();
    const int q = qsh;
    __syncthreads();
    if (q >= A.nprob) break;
    const int64_t x0 = A.xo[q], y0 = A.yo[q];
    const int64_t n = A.xo[q + 1] - x0, m = A.yo[q + 1] - y0;
    const float e0 = A.eps0[q];
    const float e1 = A.eps1 != nullptr ? A.eps1[q] : e0;
    const bool eps_ok = e0 > 0.0f && isfinite(e0) && e1 > 0.0f && isfinite(e1);
    if (n < 1 || m < 1 || n > A.n_max || m > A.m_max || x0 < 0 || y0 < 0 || !eps_ok) {
      // the whole record, so that a caller that did not clear it reads no
      // stale terms: NaN everywhere, the status GW_EINVAL
      if (threadIdx.x < GW_EN_LEN) {
        double v = __longlong_as_double(0x7ff8000000000000ll);
        if (threadIdx.x == GW_EN_STATUS) v = static_cast<double>(GW_EINVAL);
        if (threadIdx.x == GW_EN_NINNER) v = 0.0;
        if (threadIdx.x == GW_EN_STOPERR) v = -1.0;
        A.energy[static_cast<int64_t>(q) * GW_EN_LEN + threadIdx.x] = v;
      }
      continue;
    }
    solve_one<DP>(A, q, x0, y0, static_cast<int>(n), static_cast<int>(m), bsm);
  }
}

}  // namespace

size_t batch_ws_bytes() { return 256; }

bool batch_fits(int64_t n_max, int64_t m_max, int D) {
  return D >= 1 && D <= 4 && n_max >= 1 && m_max >= 1 &&
         batch_smem_bytes(n_max, m_max, D) <= 227 * 1024 - 64;
}

int run_solve_batch(int nprob, const int64_t* xo, const int64_t* yo, int64_t n_max, int64_t m_max,
                    int D, int E, const float* X, const float* Y, const float* s, const float* t,
                    const float* a, const float* b, const float* eps0, const float* eps1,
                    int n_outer, int n_inner, int symmetric, float* f, float* g, double* Gamma,
                    double* Gamma_plan, double* energy, double* history, void* ws,
                    size_t ws_bytes, cudaStream_t st) {
  GW_REQUIRE(ws_bytes >= batch_ws_bytes() && ws != nullptr, GW_ENOMEM,
             "workspace too small: need %zu bytes", batch_ws_bytes());
  GW_REQUIRE(reinterpret_cast<uintptr_t>(ws) % 256 == 0, GW_ENOMEM,
             "workspace must be 256-byte aligned");
  const size_t smem = batch_smem_bytes(n_max, m_max, D);
  GW_REQUIRE(smem <= 227 * 1024 - 64, GW_EUNSUPPORTED,
             "problems of up to %lld + %lld points at D = %d need %zu bytes of shared memory "
             "(at most %d per CTA); use gw_solve for them",
             static_cast<long long>(n_max), static_cast<long long>(m_max), D, smem, 227 * 1024 - 64);
  BatchArgs A;
  A.nprob = nprob;
  A.xo = xo;
  A.yo = yo;
  A.n_max = n_max;
  A.m_max = m_max;
  A.n_pad = pad8(n_max);
  A.m_pad = pad8(m_max);
  A.D = D;
  A.E = E;
  A.X = X;
  A.Y = Y;
  A.s = s;
  A.t = t;
  A.a = a;
  A.b = b;
  A.eps0 = eps0;
  A.eps1 = eps1;
  A.n_outer = n_outer;
  A.n_inner = n_inner;
  A.symmetric = symmetric;
  A.f = f;
  A.g = g;
  A.Gamma = Gamma;
  A.Gamma_plan = Gamma_plan;
  A.energy = energy;
  A.history = history;
  A.queue = static_cast<int*>(ws);
  GW_CUDA_TRY(cudaMemsetAsync(ws, 0, sizeof(int), st));
  auto kern = D > 2 ? batch_solve_kernel<4> : batch_solve_kernel<2>;
  // the limit is raised once, to the largest size this entry accepts
  // (per-call settings would race between host threads)
  static std::once_flag once[2];
  static cudaError_t attr_rc[2] = {cudaSuccess, cudaSuccess};
  const int which = D > 2 ? 1 : 0;
  std::call_once(once[which], [&] {
    attr_rc[which] = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          227 * 1024 - 64);
  });
  GW_CUDA_TRY(attr_rc[which]);
  int per_sm = 0;
  GW_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBt, smem));
  if (per_sm < 1) per_sm = 1;
  int grid = per_sm * kSmCount;
  if (grid > nprob) grid = nprob;
  kern<<<grid, kBt, smem, st>>>(A);
  GW_LAUNCH_CHECK();
  return GW_OK;
}

}  // namespace gw
