// Embeddings feeding Algorithm 1 (Section 5 "CNT Embeddings"; Appendix B.2).
//
// Squared-Euclidean cost: X = x - sum_i w_i x_i.
// Other CNT costs: Kernel PCA of the kernel of Prop. 2.3 centered as in
// Algorithm 4.  With u_i = c(x_i, x_1), the kernel is K = (u 1^T + 1 u^T - C)/2
// and the weighted double centering (I - 1 w^T) . (I - w 1^T) removes the
// rank-one u terms, so
//     K~ = -1/2 (I - 1 w^T) C (I - w 1^T).
// Its D largest eigenpairs come from block subspace iteration: Q <- K~ Q
// (matrix-free: C is never stored, each product is one N x N tiled pass on
// the tensor cores, gw_lift_tc.cu),
// re-orthonormalised by Cholesky QR, and a final Rayleigh-Ritz step.  The
// small r x r Cholesky, triangular inverse and eigen-problem (cyclic Jacobi)
// run on the device too, one block each in float64, so a lift makes no host
// round trip at all: it is asynchronous on its stream.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "gw_internal.cuh"

namespace gw {

namespace {

constexpr int kGramBlocks = 148;

struct CostParams {
  int kind;
  float param;
};

// Column sums weighted by w (or plain) of an n x RP matrix: partials per block.
__global__ void colsum_partial_kernel(const float* Q, const float* w, double wu, int64_t n,
                                      int RP, double* part) {
  // blockDim = (RP <= 128, 4): column r, row group y; the rows are strided
  // over blocks and groups, two in flight per thread (the loads' latency,
  // not the adds, bounds this); the groups' sums merge in a fixed order.
  // Weight w_i, or wu.
  __shared__ double red[4][128];
  const int r = threadIdx.x, y = threadIdx.y;
  const int64_t step = static_cast<int64_t>(gridDim.x) * 4;
  double a0 = 0.0, a1 = 0.0;
  int64_t i = static_cast<int64_t>(blockIdx.x) * 4 + y;
  for (; i + step < n; i += 2 * step) {
    const int64_t i1 = i + step;
    const double w0 = w ? static_cast<double>(w[i]) : wu;
    const double w1 = w ? static_cast<double>(w[i1]) : wu;
    a0 += w0 * static_cast<double>(Q[i * RP + r]);
    a1 += w1 * static_cast<double>(Q[i1 * RP + r]);
  }
  if (i < n) a0 += (w ? static_cast<double>(w[i]) : wu) * static_cast<double>(Q[i * RP + r]);
  red[y][r] = a0 + a1;
  __syncthreads();
  if (y == 0)
    part[static_cast<int64_t>(blockIdx.x) * RP + r] = (red[0][r] + red[1][r]) + (red[2][r] + red[3][r]);
}

// Sum of cnt values at p[0], p[stride], ... in a fixed order, as four
// interleaved chains (FP64 adds are long-latency here) combined at the end.
__device__ __forceinline__ double strided_sum4(const double* p, int cnt, int64_t stride) {
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  int b = 0;
  for (; b + 4 <= cnt; b += 4) {
    a0 += p[(b + 0) * stride];
    a1 += p[(b + 1) * stride];
    a2 += p[(b + 2) * stride];
    a3 += p[(b + 3) * stride];
  }
  for (; b < cnt; ++b) a0 += p[b * stride];
  return (a0 + a1) + (a2 + a3);
}

__global__ void colsum_final_kernel(const double* part, int blocks, int RP, double* out) {
  const int r = threadIdx.x;
  if (r >= RP) return;
  out[r] = strided_sum4(part + r, blocks, RP);
}

// P = Q - w (1^T Q)
__global__ void center_right_kernel(const float* Q, const float* w, float wu, const double* cs,
                                    int64_t n, int RP, float* P) {
  const int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= n * RP) return;
  const int64_t i = q / RP;
  const int r = static_cast<int>(q % RP);
  const float wi = w ? w[i] : wu;
  P[q] = Q[q] - wi * static_cast<float>(cs[r]);
}

// Z = -1/2 (Zraw - 1 (w^T Zraw)), Zraw = sum over splits of Zp
__global__ void reduce_splits_f32_kernel(const float* Zp, int splits, int64_t count, float* Z) {
  const int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= count) return;
  float acc = 0.f;
  for (int s = 0; s < splits; ++s) acc += Zp[s * count + q];
  Z[q] = acc;
}

__global__ void center_left_kernel(float* Z, const double* wz, int64_t n, int RP) {
  const int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= n * RP) return;
  const int r = static_cast<int>(q % RP);
  Z[q] = -0.5f * (Z[q] - static_cast<float>(wz[r]));
}

// Gram partials: part[b][r1][r2] = sum_{i in block b} U_i[r1] Z_i[r2]
// (when sym, U == Z and only r1 <= r2 is computed)
__global__ void gram_partial_kernel(const float* U, const float* Z, int64_t n, int RP, bool sym,
                                    double* part) {
  // the chunk's rows as float64, converted once on load (each is used by
  // every entry of the Gram; conversions run on the slow FP64 pipe too)
  extern __shared__ double shd[];
  double* Us = shd;             // [32][RP]
  double* Zs = shd + 32 * RP;   // [32][RP]
  const int RR = RP * RP;
  const int per = (RR + blockDim.x - 1) / blockDim.x;
  double acc[64];
  for (int q = 0; q < per; ++q) acc[q] = 0.0;
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t i0 = blockIdx.x * chunk;
  const int64_t i1 = i0 + chunk < n ? i0 + chunk : n;
  for (int64_t ib = i0; ib < i1; ib += 32) {
    __syncthreads();
    const int cnt = static_cast<int>(i1 - ib < 32 ? i1 - ib : 32);
    for (int idx = threadIdx.x; idx < cnt * RP; idx += blockDim.x) {
      Us[idx] = static_cast<double>(U[ib * RP + idx]);
      Zs[idx] = static_cast<double>(Z[ib * RP + idx]);
    }
    __syncthreads();
    for (int q = 0; q < per; ++q) {
      const int e = threadIdx.x + q * blockDim.x;
      if (e >= RR) break;
      const int r1 = e / RP, r2 = e % RP;
      if (sym && r1 > r2) continue;
      double a = 0.0;
      for (int ii = 0; ii < cnt; ++ii) a = fma(Us[ii * RP + r1], Zs[ii * RP + r2], a);
      acc[q] += a;
    }
  }
  for (int q = 0; q < per; ++q) {
    const int e = threadIdx.x + q * blockDim.x;
    if (e < RR) part[static_cast<int64_t>(blockIdx.x) * RR + e] = acc[q];
  }
}

__global__ void gram_final_kernel(const double* part, int blocks, int RP, bool sym, double* G) {
  const int RR = RP * RP;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= RR) return;
  const int r1 = e / RP, r2 = e % RP;
  const int src = (sym && r1 > r2) ? r2 * RP + r1 : e;   // the mirrored entry
  G[e] = strided_sum4(part + src, blocks, RR);
}

// A float64 matrix entry stored as two floats: hi = fl(v), lo = fl(v - hi).
__device__ __forceinline__ void store_split(float* M, int64_t lo_off, int64_t e, double v) {
  const float hi = static_cast<float>(v);
  M[e] = hi;
  M[lo_off + e] = static_cast<float>(v - static_cast<double>(hi));
}

// Out_i[c] = sum_r In_i[r] M[r][c]  (M: RP x cols as hi + lo float pairs, the
// lo block lo_off entries after the hi block), cols <= RP.  FP64 runs at 1/64
// of the FP32 rate on GB300, so the sum is double-float on the FP32 lanes: each product
// In_ir (M_hi + M_lo) is exact to ~2^-48 by Dekker's TwoProduct (one FMA for
// the error of In_ir M_hi) and accumulated by Knuth's TwoSum, the rounding
// errors collected in a second float; the result (~44 bits) is rounded to
// FP32 once, as the float64 form did.
__global__ void right_mult_kernel(const float* In, int64_t n, int RP, const float* M,
                                  int64_t lo_off, int cols, int out_stride, float* Out) {
  const int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= n * cols) return;
  const int64_t i = q / cols;
  const int c = static_cast<int>(q % cols);
  float sh = 0.0f, sl = 0.0f;
  for (int r = 0; r < RP; ++r) {
    const float a = In[i * RP + r];
    const float mh = M[r * cols + c], ml = M[lo_off + r * cols + c];
    const float ph = __fmul_rn(a, mh);
    const float pl = __fadd_rn(__fmaf_rn(a, mh, -ph), __fmul_rn(a, ml));
    const float sn = __fadd_rn(sh, ph);
    const float v = __fsub_rn(sn, sh);
    const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(sn, v)), __fsub_rn(ph, v));
    sh = sn;
    sl = __fadd_rn(sl, __fadd_rn(err, pl));
  }
  Out[i * out_stride + c] = __fadd_rn(sh, sl);
}

// Deterministic start block: uniform(-1, 1) from a counter hash (splitmix64).
__global__ void random_block_kernel(float* Q, int64_t count, uint64_t seed) {
  const int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= count) return;
  uint64_t z = seed + 0x9E3779B97F4A7C15ull * static_cast<uint64_t>(q + 1);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  Q[q] = static_cast<float>(static_cast<double>(z >> 11) * (2.0 / 9007199254740992.0) - 1.0);
}

// Sign convention: the entry of largest magnitude of each eigenvector is positive.
// Per block of rows (in order) and column c < D: the largest |V_ic| and the
// first row that holds it.  blockDim.x >= D.
__global__ void sign_partial_kernel(const float* V, int64_t n, int D, double* best,
                                    double* where) {
  const int c = threadIdx.x;
  if (c >= D) return;
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t i0 = blockIdx.x * chunk;
  const int64_t i1 = i0 + chunk < n ? i0 + chunk : n;
  float b = -1.f;
  int64_t at = i0;
  for (int64_t i = i0; i < i1; ++i) {
    const float v = fabsf(V[i * D + c]);
    if (v > b) {
      b = v;
      at = i;
    }
  }
  best[static_cast<int64_t>(blockIdx.x) * D + c] = b;
  where[static_cast<int64_t>(blockIdx.x) * D + c] = static_cast<double>(at);
}

// flip[c] = 1 when the first entry of largest magnitude of column c is negative
__global__ void sign_final_kernel(const float* V, int D, int blocks, const double* best,
                                  const double* where, double* flip) {
  const int c = threadIdx.x;
  if (c >= D) return;
  double b = -1.0, at = 0.0;
  for (int k = 0; k < blocks; ++k) {
    const double v = best[static_cast<int64_t>(k) * D + c];
    if (v > b) {
      b = v;
      at = where[static_cast<int64_t>(k) * D + c];
    }
  }
  flip[c] = V[static_cast<int64_t>(at) * D + c] < 0.f ? 1.0 : 0.0;
}

// Sign convention applied: V_c <- -V_c where flipped; X = V diag(sqrt(lam)),
// sqn = ||X_i||^2 (one warp per row)
__global__ void sign_apply_kernel(float* V, int64_t n, int D, const double* flip, float* X,
                                  float* sqn, const float* sqrt_lam) {
  const int64_t i = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  float s = 0.f;
  for (int c = lane; c < D; c += 32) {
    float v = V[i * D + c];
    if (flip[c] != 0.0) v = -v;
    V[i * D + c] = v;
    const float xv = v * sqrt_lam[c];
    X[i * D + c] = xv;
    s = fmaf(xv, xv, s);
  }
  s = warp_sum(s);
  if (lane == 0) sqn[i] = s;
}

// Squared lift: X = x - sum w x; sqn = ||X||^2.  The weighted mean comes from
// per-block partials over row chunks (kGramBlocks blocks, blockDim.x = d)
// summed in a fixed order (colsum_partial / colsum_final), then
// every row is centered in parallel.
__global__ void center_apply_kernel(const float* x, const double* mean, int64_t n, int d,
                                    float* X, float* sqn) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float s = 0.f;
  for (int c = 0; c < d; ++c) {
    const float v = static_cast<float>(static_cast<double>(x[i * d + c]) - mean[c]);
    X[i * d + c] = v;
    s = fmaf(v, v, s);
  }
  sqn[i] = s;
}

// ---- the small dense steps on the device (one block each, float64) ----
// Cholesky QR step: G (RP x RP Gram, global) -> M = R^{-1} with G + delta I =
// R^T R (upper R), delta = 1e-13 tr(G) / RP keeping the factorisation defined
// when a direction vanishes.  A trace that is not positive and finite, or a
// pivot that is not positive, sets *status = 1 and leaves M = I (the result is
// then discarded by the caller).  Dynamic shared memory: RP x RP doubles.
__global__ void __launch_bounds__(256) chol_inv_kernel(const double* G, int RP, float* M,
                                                       int* status) {
  // R: the factor in the upper triangle; below the diagonal, M's entries
  // M_kc (k < c) at R[c][k] once the inverse is formed
  extern __shared__ double R[];   // [RP][RP]
  __shared__ double red[8];
  __shared__ double rd[128];      // diagonal of R, then its reciprocals
  __shared__ double md[128];      // diagonal of M
  __shared__ double ivd[128];     // 1 / pivot, formed once by the lane that updates it
  __shared__ int bad;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int nw = static_cast<int>(blockDim.x >> 5);
  const int RR = RP * RP;
  double tr = 0.0;
  for (int e = tid; e < RR; e += blockDim.x) R[e] = G[e];
  for (int i = tid; i < RP; i += blockDim.x) tr += G[i * RP + i];
  tr = warp_sum(tr);
  if (lane == 0) red[wid] = tr;
  if (tid == 0) bad = 0;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int q = 0; q < nw; ++q) t += red[q];
    red[0] = t;
    if (!(t > 0.0) || !isfinite(t)) bad = 1;
  }
  __syncthreads();
  const double shift = 1e-13 * red[0] / RP;
  for (int i = tid; i < RP; i += blockDim.x) R[i * RP + i] += shift;
  if (tid == 0) ivd[0] = 1.0 / (G[0] + shift);
  __syncthreads();
  // right-looking, one barrier per pivot: the trailing update takes row j
  // unscaled (R_jr R_jc = a_jr a_jc / d_j); the rows are scaled afterwards.
  // FP64 division is slow on GB300, so 1 / d_{j+1} is formed once, by the
  // lane that writes d_{j+1}.  Every thread reads the same pivot, so all
  // leave the loop together.
  bool fail = bad != 0;
  for (int j = 0; j < RP && !fail; ++j) {
    const double d = R[j * RP + j];
    if (!(d > 0.0)) {
      fail = true;
      break;
    }
    const double inv = ivd[j];
    for (int r = j + 1 + wid; r < RP; r += nw) {
      const double f = R[j * RP + r] * inv;
      for (int c = r + lane; c < RP; c += 32) {
        const double v = R[r * RP + c] - f * R[j * RP + c];
        R[r * RP + c] = v;
        if (c == j + 1) ivd[c] = 1.0 / v;   // the next pivot
      }
    }
    __syncthreads();
  }
  if (fail) {
    for (int e = tid; e < RR; e += blockDim.x) store_split(M, RR, e, (e / RP == e % RP) ? 1.0 : 0.0);
    if (tid == 0) *status = 1;
    return;
  }
  for (int i = tid; i < RP; i += blockDim.x) {
    const double q = sqrt(R[i * RP + i]);
    R[i * RP + i] = q;
    rd[i] = 1.0 / q;
  }
  __syncthreads();
  for (int e = tid; e < RR; e += blockDim.x) {
    const int r = e / RP, c = e - r * RP;
    if (c > r) R[e] *= rd[r];
  }
  __syncthreads();
  // M = R^{-1}: column c by back substitution (one thread per column), its
  // entries kept in shared memory (row c below the diagonal, and md[c])
  for (int c = tid; c < RP; c += blockDim.x) {
    for (int i = c; i >= 0; --i) {
      double acc = (i == c) ? 1.0 : 0.0;
      for (int k = i + 1; k <= c; ++k) acc -= R[i * RP + k] * (k == c ? md[c] : R[c * RP + k]);
      const double v = acc * rd[i];
      if (i == c) md[c] = v;
      else R[c * RP + i] = v;
    }
  }
  __syncthreads();
  for (int e = tid; e < RR; e += blockDim.x) {
    const int r = e / RP, c = e - r * RP;
    store_split(M, RR, e, r < c ? R[c * RP + r] : (r == c ? md[r] : 0.0));
  }
}

// Rayleigh-Ritz on the device: T (RP x RP, global) is symmetrised and
// diagonalised by cyclic Jacobi rotations in the round-robin order (RP / 2
// disjoint pairs per step, rotated at once); U (global, RP x RP) accumulates
// the vectors.  Then the D largest eigenvalues (ties: lower index) give
// Msel (RP x D, their vectors), lam and sqrt(max(lam, 0)).  Sweeps stop when
// the off-diagonal mass is below 1e-30 of the total (at most 100).
// Dynamic shared memory: RP x RP doubles.
__global__ void __launch_bounds__(256) ritz_eig_kernel(const double* T, int RP, int D, double* U,
                                                       float* Msel, float* lam, float* sl) {
  extern __shared__ double A[];   // [RP][RP]
  __shared__ double cs[64][2];
  __shared__ double red[2][8];
  __shared__ int done;
  const int tid = threadIdx.x;
  const int RR = RP * RP;
  const int half = RP / 2;
  for (int e = tid; e < RR; e += blockDim.x) {
    const int r = e / RP, c = e % RP;
    A[e] = 0.5 * (T[r * RP + c] + T[c * RP + r]);
    U[e] = r == c ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int e = tid; e < RR; e += blockDim.x) {
      const double v = A[e] * A[e];
      tot += v;
      if (e / RP != e % RP) off += v;
    }
    off = warp_sum(off);
    tot = warp_sum(tot);
    if ((tid & 31) == 0) {
      red[0][tid >> 5] = off;
      red[1][tid >> 5] = tot;
    }
    __syncthreads();
    if (tid == 0) {
      double o = 0.0, t = 0.0;
      for (int q = 0; q < static_cast<int>(blockDim.x >> 5); ++q) {
        o += red[0][q];
        t += red[1][q];
      }
      done = (o <= 1e-30 * t) ? 1 : 0;
    }
    __syncthreads();
    if (done) break;
    for (int step = 0; step < RP - 1; ++step) {
      // pair i: positions i and RP-1-i of the arrangement [0, 1 + (k - 1 + step) mod (RP - 1)]
      if (tid < half) {
        const int i = tid;
        const int p0 = i == 0 ? 0 : 1 + (i - 1 + step) % (RP - 1);
        const int q0 = 1 + (RP - 2 - i + step) % (RP - 1);
        const int p = p0 < q0 ? p0 : q0, q = p0 < q0 ? q0 : p0;
        const double apq = A[p * RP + q];
        double c = 1.0, sn = 0.0;
        if (fabs(apq) >= 1e-300) {
          const double theta = (A[q * RP + q] - A[p * RP + p]) / (2.0 * apq);
          const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
          c = 1.0 / sqrt(t * t + 1.0);
          sn = t * c;
        }
        cs[i][0] = c;
        cs[i][1] = sn;
      }
      __syncthreads();
      // rows p, q of every pair: A <- J^T A
      for (int w = tid; w < half * RP; w += blockDim.x) {
        const int i = w / RP, k = w % RP;
        const int p0 = i == 0 ? 0 : 1 + (i - 1 + step) % (RP - 1);
        const int q0 = 1 + (RP - 2 - i + step) % (RP - 1);
        const int p = p0 < q0 ? p0 : q0, q = p0 < q0 ? q0 : p0;
        const double c = cs[i][0], sn = cs[i][1];
        const double apk = A[p * RP + k], aqk = A[q * RP + k];
        A[p * RP + k] = c * apk - sn * aqk;
        A[q * RP + k] = sn * apk + c * aqk;
      }
      __syncthreads();
      // columns p, q: A <- A J, U <- U J
      for (int w = tid; w < half * RP; w += blockDim.x) {
        const int i = w / RP, k = w % RP;
        const int p0 = i == 0 ? 0 : 1 + (i - 1 + step) % (RP - 1);
        const int q0 = 1 + (RP - 2 - i + step) % (RP - 1);
        const int p = p0 < q0 ? p0 : q0, q = p0 < q0 ? q0 : p0;
        const double c = cs[i][0], sn = cs[i][1];
        const double akp = A[k * RP + p], akq = A[k * RP + q];
        A[k * RP + p] = c * akp - sn * akq;
        A[k * RP + q] = sn * akp + c * akq;
        const double ukp = U[k * RP + p], ukq = U[k * RP + q];
        U[k * RP + p] = c * ukp - sn * ukq;
        U[k * RP + q] = sn * ukp + c * ukq;
      }
      __syncthreads();
    }
  }
  // the D largest eigenvalues, in decreasing order
  for (int k = tid; k < RP; k += blockDim.x) {
    const double lk = A[k * RP + k];
    int rank = 0;
    for (int j = 0; j < RP; ++j) {
      const double lj = A[j * RP + j];
      rank += (lj > lk || (lj == lk && j < k)) ? 1 : 0;
    }
    if (rank < D) {
      lam[rank] = static_cast<float>(lk);
      sl[rank] = static_cast<float>(sqrt(lk > 0.0 ? lk : 0.0));
      for (int r = 0; r < RP; ++r) store_split(Msel, RR, r * D + rank, U[r * RP + k]);
    }
  }
}

// A lift whose Cholesky step failed (*status != 0) fills its outputs with NaN.
__global__ void lift_poison_kernel(const int* status, int64_t n, int D, float* X, float* sqn,
                                   float* basis) {
  if (*status == 0) return;
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float nan = __int_as_float(0x7fc00000);
  sqn[i] = nan;
  for (int c = 0; c < D; ++c) {
    X[i * D + c] = nan;
    if (basis) basis[i * D + c] = nan;
  }
}

int rpad(int D) {
  const int want = D + 8;
  const int opts[] = {16, 32, 48, 64, 80, 96, 128};
  for (int o : opts)
    if (o >= want) return o;
  return 128;
}

struct LiftBufs {
  float *Q, *P, *Z, *Zp, *V, *sl, *lam;
  double *cs_part, *cs, *g_part, *G;
  float* M;   // R^-1 (or the Ritz vectors) as hi + lo float pairs
  int* status;
  int splits, RP;
  LiftTcBufs tc;
};

LiftBufs carve_lift(Carver& c, int64_t n, int D) {
  LiftBufs B;
  B.RP = rpad(D);
  B.tc = carve_lift_tc(c, n, B.RP);
  B.splits = B.tc.splits;
  const size_t nr = static_cast<size_t>(n) * B.RP;
  B.Q = c.take<float>(nr);
  B.P = c.take<float>(nr);
  B.Z = c.take<float>(nr);
  B.Zp = B.splits > 1 ? c.take<float>(nr * B.splits) : nullptr;
  B.V = c.take<float>(static_cast<size_t>(n) * D);
  B.sl = c.take<float>(static_cast<size_t>(D));
  B.lam = c.take<float>(static_cast<size_t>(D));
  B.cs_part = c.take<double>(static_cast<size_t>(kGramBlocks) * B.RP);
  B.cs = c.take<double>(B.RP);
  B.g_part = c.take<double>(static_cast<size_t>(kGramBlocks) * B.RP * B.RP);
  B.G = c.take<double>(static_cast<size_t>(B.RP) * B.RP);
  B.M = c.take<float>(static_cast<size_t>(2) * B.RP * B.RP);   // hi, then lo
  B.status = c.take<int>(4);
  return B;
}

int weighted_colsum(const float* Q, const float* w, double wu, int64_t n, int RP, LiftBufs& B,
                    cudaStream_t st) {
  colsum_partial_kernel<<<kGramBlocks, dim3(RP, 4), 0, st>>>(Q, w, wu, n, RP, B.cs_part);
  GW_LAUNCH_CHECK();
  colsum_final_kernel<<<1, 128, 0, st>>>(B.cs_part, kGramBlocks, RP, B.cs);
  GW_LAUNCH_CHECK();
  return GW_OK;
}

// Z = K~ Q = -1/2 (I - 1 w^T) C (I - w 1^T) Q
int apply_kernel(int64_t n, int d, const float* w, CostParams cp, LiftBufs& B, cudaStream_t st) {
  const int RP = B.RP;
  const int64_t nr = n * RP;
  const float wu = 1.0f / static_cast<float>(n);
  GW_TRY(weighted_colsum(B.Q, nullptr, 1.0, n, RP, B, st));            // 1^T Q
  center_right_kernel<<<ceil_div(nr, 256), 256, 0, st>>>(B.Q, w, wu, B.cs, n, RP, B.P);
  GW_LAUNCH_CHECK();
  const int splits = B.splits;
  GW_TRY(lift_tc_matvec(B.P, n, d, cp.kind, cp.param, RP, B.tc, splits > 1 ? B.Zp : B.Z, st));
  if (splits > 1) {
    reduce_splits_f32_kernel<<<ceil_div(nr, 256), 256, 0, st>>>(B.Zp, splits, nr, B.Z);
    GW_LAUNCH_CHECK();
  }
  GW_TRY(weighted_colsum(B.Z, w, 1.0 / static_cast<double>(n), n, RP, B, st));   // w^T Z
  center_left_kernel<<<ceil_div(nr, 256), 256, 0, st>>>(B.Z, B.cs, n, RP);
  GW_LAUNCH_CHECK();
  return GW_OK;
}

// G = U^T Z on the device (float64, fixed-order partials)
int gram(const float* U, const float* Z, int64_t n, int RP, LiftBufs& B, cudaStream_t st) {
  const size_t shb = sizeof(double) * 2 * 32 * RP;
  const bool sym = U == Z;
  gram_partial_kernel<<<kGramBlocks, 256, shb, st>>>(U, Z, n, RP, sym, B.g_part);
  GW_LAUNCH_CHECK();
  gram_final_kernel<<<ceil_div(RP * RP, 256), 256, 0, st>>>(B.g_part, kGramBlocks, RP, sym, B.G);
  GW_LAUNCH_CHECK();
  return GW_OK;
}

// the dense r x r kernels take up to 128 x 128 doubles of shared memory
int small_kernel_attrs() {
  static std::once_flag once;
  static cudaError_t rc = cudaSuccess;
  std::call_once(once, [] {
    rc = cudaFuncSetAttribute(chol_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              128 * 128 * 8);
    if (rc == cudaSuccess)   // the Gram's row chunks: 2 x 32 x 128 doubles at most
      rc = cudaFuncSetAttribute(gram_partial_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                2 * 32 * 128 * 8);
    if (rc == cudaSuccess)
      rc = cudaFuncSetAttribute(ritz_eig_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                128 * 128 * 8);
  });
  GW_CUDA_TRY(rc);
  return GW_OK;
}

// Q <- Z R^{-1} with Z^T Z = R^T R (Cholesky QR), all on the device
int orthonormalize(int64_t n, LiftBufs& B, cudaStream_t st) {
  const int RP = B.RP;
  GW_TRY(gram(B.Z, B.Z, n, RP, B, st));
  chol_inv_kernel<<<1, 256, sizeof(double) * RP * RP, st>>>(B.G, RP, B.M, B.status);
  GW_LAUNCH_CHECK();
  right_mult_kernel<<<ceil_div(n * RP, 256), 256, 0, st>>>(B.Z, n, RP, B.M,
                                                            static_cast<int64_t>(RP) * RP, RP, RP,
                                                            B.Q);
  GW_LAUNCH_CHECK();
  return GW_OK;
}

}  // namespace

size_t lift_ws_bytes(int64_t n, int D) {
  Carver c(nullptr, ~size_t(0));
  carve_lift(c, n, D);
  return c.used();
}

int run_lift(const float* x, int64_t n, int d, const float* w, int kind, float param, int D,
             int n_iter, uint64_t seed, float* X, float* sqn, float* basis, float* eigvals,
             void* ws, size_t ws_bytes, cudaStream_t st) {
  if (kind == GW_PEN_SQEUCLID && D == d && basis == nullptr && eigvals == nullptr) {
    Carver c(ws, ws_bytes);
    double* part = c.take<double>(static_cast<size_t>(kGramBlocks) * d);
    double* mean = c.take<double>(static_cast<size_t>(d));
    GW_TRY(check_ws(c, ws));
    colsum_partial_kernel<<<kGramBlocks, dim3(d, 4), 0, st>>>(x, w, 1.0 / static_cast<double>(n), n, d,
                                                       part);
    GW_LAUNCH_CHECK();
    colsum_final_kernel<<<1, 128, 0, st>>>(part, kGramBlocks, d, mean);
    GW_LAUNCH_CHECK();
    center_apply_kernel<<<ceil_div(n, 256), 256, 0, st>>>(x, mean, n, d, X, sqn);
    GW_LAUNCH_CHECK();
    return GW_OK;
  }
  NvtxRange range("gw_lift (Kernel PCA)");
  Carver c(ws, ws_bytes);
  LiftBufs B = carve_lift(c, n, D);
  GW_TRY(check_ws(c, ws));
  const int RP = B.RP;
  GW_REQUIRE(n > RP, GW_EINVAL, "Kernel PCA with D=%d needs more than %d points (n=%lld)", D, RP,
             static_cast<long long>(n));
  CostParams cp{kind, param};
  GW_TRY(small_kernel_attrs());
  GW_CUDA_TRY(cudaMemsetAsync(B.status, 0, sizeof(int) * 4, st));
  GW_TRY(lift_tc_prepare(x, n, d, kind, param, RP, B.tc, st));
  const int iters = n_iter > 0 ? n_iter : 40;
  random_block_kernel<<<ceil_div(n * RP, 256), 256, 0, st>>>(B.Q, n * RP, seed);
  GW_LAUNCH_CHECK();
  for (int it = 0; it < iters; ++it) {
    GW_TRY(apply_kernel(n, d, w, cp, B, st));
    GW_TRY(orthonormalize(n, B, st));
  }
  // Rayleigh-Ritz: T = Q^T K~ Q, eigenpairs of T, V = Q U_{1:D} (device)
  GW_TRY(apply_kernel(n, d, w, cp, B, st));
  GW_TRY(gram(B.Q, B.Z, n, RP, B, st));
  ritz_eig_kernel<<<1, 256, sizeof(double) * RP * RP, st>>>(B.G, RP, D, B.g_part, B.M, B.lam,
                                                             B.sl);
  GW_LAUNCH_CHECK();
  right_mult_kernel<<<ceil_div(n * D, 256), 256, 0, st>>>(B.Q, n, RP, B.M,
                                                           static_cast<int64_t>(RP) * RP, D, D,
                                                           B.V);
  GW_LAUNCH_CHECK();
  sign_partial_kernel<<<kGramBlocks, 128, 0, st>>>(B.V, n, D, B.g_part, B.g_part + kGramBlocks * D);
  GW_LAUNCH_CHECK();
  sign_final_kernel<<<1, 128, 0, st>>>(B.V, D, kGramBlocks, B.g_part, B.g_part + kGramBlocks * D,
                                       B.cs);
  GW_LAUNCH_CHECK();
  sign_apply_kernel<<<ceil_div(n * 32, 256), 256, 0, st>>>(B.V, n, D, B.cs, X, sqn, B.sl);
  GW_LAUNCH_CHECK();
  if (basis) {
    GW_CUDA_TRY(cudaMemcpyAsync(basis, B.V, sizeof(float) * n * D, cudaMemcpyDeviceToDevice, st));
  }
  if (eigvals) {
    GW_CUDA_TRY(cudaMemcpyAsync(eigvals, B.lam, sizeof(float) * D, cudaMemcpyDeviceToDevice, st));
  }
  // a failed Cholesky step (degenerate block) leaves NaN features, which a
  // solve on them reports as GW_ENONFINITE; nothing is read back
  lift_poison_kernel<<<ceil_div(n, 256), 256, 0, st>>>(B.status, n, D, X, sqn, basis);
  GW_LAUNCH_CHECK();
  return GW_OK;
}

}  // namespace gw
