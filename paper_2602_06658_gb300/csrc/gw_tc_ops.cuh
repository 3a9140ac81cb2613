// Operand preparation shared by the tensor-core kernels (the softmin and the
// plan-weighted reduction): the 16-bit operand matrices whose product is the
// whole base-2 exponent of the plan on c_Gamma (layout and splits described in
// gw_softmin_tc.cu), their scales, the per-iteration refresh of the potential
// columns, tensor-map encoding and a bounded mbarrier drain.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <math.h>

#include <mutex>

#include "gw_internal.cuh"
#include "gw_tc.cuh"

namespace gw {

namespace {

constexpr float kBiasConst = 32768.0f;       // A-side multiplier of the bias columns
constexpr float kHalfMax = 65504.0f;
constexpr float kShiftBias = 30.0f;          // fast-pass shift sits this far below the estimate

struct TcOperandShape {
  int K;        // feature dimension
  int mult;     // 1 or 3 products in the dot
  int Ks;       // mult == 3: dims taken as three products (the rest as one)
  int KP;       // padded operand width
  int col_u;    // first rank-one column
  int col_w;    // first column-bias column
  int col_e;    // first row-estimate column
  int col_k;    // mask column (-inf for padded and zero-weight target columns)
  int used;     // non-zero columns
  int k8;       // GW_PREC_FP8: leading MMA K-steps of E4M3 features (32 dims each,
                // two to a 16-bit column); 0 in the 16-bit modes
};

TcOperandShape tc_shape(int K, int prec) {
  TcOperandShape s;
  s.K = K;
  s.mult = (prec == GW_PREC_BF16 || prec == GW_PREC_FP8) ? 1 : 3;
  s.Ks = K;
  s.k8 = prec == GW_PREC_FP8 ? (K + 31) / 32 : 0;
  // FP8: the dims as bytes, 32 per K-step of 16 columns
  s.col_u = s.k8 > 0 ? 16 * s.k8 : s.mult * K;
  s.col_w = s.col_u + 3;
  s.col_e = s.col_w + 3;
  s.col_k = s.col_e + 3;
  s.used = s.col_k + 1;
  s.KP = ((s.used + 63) / 64) * 64;
  return s;
}

// Split layout of a fixed width KP for the split precisions: the Ks dims of
// largest product bound as three products, the other K - Ks as one product
// (the most dims KP holds beside the 10 bias, shift and mask columns).
TcOperandShape tc_shape_split(int K, int prec, int KP) {
  TcOperandShape s = tc_shape(K, prec);
  int ks = (KP - 10 - K) / 2;
  if (ks > K) ks = K;
  if (ks < 0) ks = 0;
  s.Ks = ks;
  s.col_u = 3 * ks + (K - ks);
  s.col_w = s.col_u + 3;
  s.col_e = s.col_w + 3;
  s.col_k = s.col_e + 3;
  s.used = s.col_k + 1;
  s.KP = KP;
  return s;
}

// The split layout of shape s (its KP kept) with ks dims as three products.
__host__ __device__ inline TcOperandShape shape_ks(TcOperandShape s, int ks) {
  if (ks > s.K) ks = s.K;
  if (ks < 0) ks = 0;
  s.Ks = ks;
  s.col_u = 3 * ks + (s.K - ks);
  s.col_w = s.col_u + 3;
  s.col_e = s.col_w + 3;
  s.col_k = s.col_e + 3;
  s.used = s.col_k + 1;
  return s;
}

// Relative error of a single 16-bit product X_k V_k (both operands rounded
// once): 2^-10 in f16, 2^-7 in bf16.  A dim may run as one product when its
// bound P_k = max|X_k| max|V_k| is at most TERM_REL / single_rel times the
// largest P: its error then stays below TERM_REL times the largest term, the
// bound the split products keep (2^-20 for F16X3, 2^-15 for BF16X3).
__host__ __device__ inline float split_threshold(int prec) {
  return prec == GW_PREC_F16X3 ? 9.765625e-04f /* 2^-10 */ : 3.90625e-03f /* 2^-8 */;
}

bool tc_is_bf16(int prec) { return prec != GW_PREC_F16X3; }

int max_splits(int col_tiles) { return col_tiles < 64 ? col_tiles : 64; }

template <class T>
__device__ __forceinline__ T to16(float x);
template <>
__device__ __forceinline__ __half to16<__half>(float x) {
  return __float2half_rn(x);
}
template <>
__device__ __forceinline__ __nv_bfloat16 to16<__nv_bfloat16>(float x) {
  return __float2bfloat16_rn(x);
}
__device__ __forceinline__ float from16(__half x) { return __half2float(x); }
__device__ __forceinline__ float from16(__nv_bfloat16 x) { return __bfloat162float(x); }

// Part `part` (0, 1, 2) of a three-way 16-bit split of x (hi + mid + lo).
template <class T>
__device__ __forceinline__ float split3(float x, int part) {
  const float x0 = from16(to16<T>(x));
  const float r1 = x - x0;
  const float x1 = from16(to16<T>(r1));
  return part == 0 ? x0 : (part == 1 ? x1 : r1 - x1);
}

// Largest magnitudes that set the operand scales -> mx[0..5] (non-negative
// floats compare as unsigned ints): |A|, |B|, |sA|, |sB|, the finite column
// biases |w_j| and the row shifts |e_i| (when an estimate is given).
__global__ void tc_absmax_kernel(const float* A, int64_t nA, const float* B, int64_t nB,
                                 const float* sA, int64_t n, const float* sB, int64_t m,
                                 const float* h, const float* logw, const float* est,
                                 float inv_eps, unsigned* mx, float shift_bias = kShiftBias) {
  float v[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  const int64_t t0 = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  for (int64_t i = t0; i < nA; i += stride) v[0] = fmaxf(v[0], fabsf(A[i]));
  for (int64_t i = t0; i < nB; i += stride) v[1] = fmaxf(v[1], fabsf(B[i]));
  for (int64_t i = t0; i < n; i += stride) v[2] = fmaxf(v[2], fabsf(sA[i]));
  for (int64_t i = t0; i < m; i += stride) {
    v[3] = fmaxf(v[3], fabsf(sB[i]));
    const float w = (h[i] * inv_eps + logw[i]) * kLog2e;
    if (isfinite(w)) v[4] = fmaxf(v[4], fabsf(w));
  }
  if (est)
    for (int64_t i = t0; i < n; i += stride)
      v[5] = fmaxf(v[5], fabsf(est[i] * inv_eps * kLog2e + shift_bias));
#pragma unroll
  for (int k = 0; k < 6; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] = fmaxf(v[k], __shfl_xor_sync(0xffffffffu, v[k], o));
    if ((threadIdx.x & 31) == 0) atomicMax(&mx[k], __float_as_uint(v[k]));
  }
}

// Power-of-two scale that brings max |x| / c to at most 2^14 (so a three-way
// 16-bit split keeps all three parts normal), within [2^-14, 2^15].
__device__ __forceinline__ float pow2_scale(float mxv) {
  float c = 6.103515625e-05f;   // 2^-14
  while (c < 32768.0f && mxv > 16384.0f * c) c *= 2.0f;
  return c;
}

// Scale pair (sa, sb) with sa * sb = prod that balances max|x sa| and max|y sb|.
__device__ __forceinline__ void balance(float prod, float mxa, float mxb, float* sa, float* sb) {
  if (!(mxa > 0.f) || !(mxb > 0.f)) {
    *sa = 1.0f;
    *sb = prod;
    return;
  }
  const float r = sqrtf(prod * mxb / mxa);
  *sa = r;
  *sb = prod / r;
}

// Largest e4m3 magnitude, and the power-of-two scale 2^e that brings a
// group's max |x| to at most 448 (the largest such e; e in [-40, 40] so the
// bias columns times the scale stay far inside BF16 range; 1 for an all-zero
// or non-finite group).  m = f 2^E with f in [0.5, 1): f 2^9 <= 448 iff
// f <= 0.875.
constexpr float kE4M3Max = 448.0f;
__device__ __forceinline__ float e4m3_group_scale(float m) {
  if (!(m > 0.0f) || !isfinite(m)) return 1.0f;
  int E = 0;
  const float f = frexpf(m, &E);
  int e = (f <= 0.875f ? 9 : 8) - E;
  e = e < -40 ? -40 : (e > 40 ? 40 : e);
  return ldexpf(1.0f, e);
}

// FP8 (GW_PREC_FP8) operand scales: one power of two per group of
// kFp8Group rows of a feature matrix, fs[g] = e4m3_group_scale(max |X_ik|
// over the group's rows); groups past the last row up to ngroups get 1.  The
// e4m3 features e4m3(X_ik fs[i / kFp8Group]) depend on the matrix alone, not
// on the side of the product it takes, so the row and column softmins and
// the plan sums all multiply the same rounded features.  One warp per group.
constexpr int kFp8Group = 128;
__global__ void fp8_scale_kernel(const float* X, int64_t rows, int K, int64_t ngroups, float* fs) {
  const int64_t g = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (g >= ngroups) return;
  const int64_t r0 = g * kFp8Group;
  const int64_t r1 = r0 + kFp8Group < rows ? r0 + kFp8Group : rows;
  float v = 0.0f;
  for (int64_t q = r0 * K + lane; q < r1 * K; q += 32) v = fmaxf(v, fabsf(X[q]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if (lane == 0) fs[g] = r0 < rows ? e4m3_group_scale(v) : 1.0f;
}

// FP8: the accumulator holds z / kappa with kappa = alpha / (fs_row fs_col)
// (the features unscaled by alpha, the other columns divided by it); this
// multiplies the tile back into base-2 exponent units.
template <int N>
__device__ __forceinline__ void unscale(uint32_t (&r)[N], float kap) {
  const uint64_t k2 = tc::pack2(kap, kap);
#pragma unroll
  for (int k = 0; k < N; k += 2) {
    float a, b;
    tc::unpack2(tc::mul2(tc::pack2(__uint_as_float(r[k]), __uint_as_float(r[k + 1])), k2), a, b);
    r[k] = __float_as_uint(a);
    r[k + 1] = __float_as_uint(b);
  }
}

__device__ __forceinline__ uint32_t e4m3_bits(float x) {
  return static_cast<uint32_t>(__nv_cvt_float_to_fp8(x, __NV_SATFINITE, __NV_E4M3));
}

// Operand rows.  role 0 = A side (row operand), role 1 = B side (column
// operand, bias columns included).  Rows >= rows_valid are padding: zeros,
// and for the B side a bias of -65504 * kBiasConst so they add nothing.
// With `lay` (the device's layout decision, tc_layout_kernel) and lay[0] set,
// the rows take the split layout shp_a (dims in the order lay[2..]) padded to
// rows_pad_a; otherwise shp padded to rows_pad.
template <class T>
__global__ void tc_prep_kernel(const float* X, const float* sq, const float* h, const float* logw,
                               const float* est, int64_t rows_valid, int64_t rows_pad_f,
                               TcOperandShape shp_f, int role, float alpha, float beta,
                               float inv_eps, const unsigned* mx, T* op,
                               float shift_bias = kShiftBias, const int* lay = nullptr,
                               TcOperandShape shp_a = TcOperandShape{}, int64_t rows_pad_a = 0,
                               const float* fs = nullptr) {
  const bool ad = lay != nullptr && lay[0] != 0;
  const TcOperandShape shp = ad ? shape_ks(shp_a, lay[1]) : shp_f;
  const int64_t rows_pad = ad ? rows_pad_a : rows_pad_f;
  const int* perm = ad ? lay + 2 : nullptr;
  const int64_t r = static_cast<int64_t>(blockIdx.x) * blockDim.y + threadIdx.y;
  if (r >= rows_pad) return;
  const float mA = __uint_as_float(mx[0]), mB = __uint_as_float(mx[1]);
  const float msA = __uint_as_float(mx[2]), msB = __uint_as_float(mx[3]);
  // FP8 (fs given): the features are not scaled by alpha; the rank-one, bias
  // and shift columns are in units of alpha (beta / alpha = 1/4 exactly), and
  // the epilogue multiplies by alpha / (fs_row fs_col).  wa = 1 otherwise.
  const bool f8 = fs != nullptr;
  const float wa = f8 ? alpha : 1.0f;
  const float cw = pow2_scale(__uint_as_float(mx[4]) / wa);
  const float ce = pow2_scale(__uint_as_float(mx[5]) / wa);
  float sa, sb, ua, ub;
  balance(alpha, mA, mB, &sa, &sb);
  balance(f8 ? 0.25f : beta, msA, msB, &ua, &ub);
  const float sc = role == 0 ? sa : sb;
  const float us = role == 0 ? ua : ub;
  T* row = op + r * shp.KP;
  const bool valid = r < rows_valid;
  const int K = shp.K;
  // FP8: the row group's power-of-two scale multiplies every column
  const float fr = f8 ? fs[r / kFp8Group] : 1.0f;
  for (int k = threadIdx.x; k < shp.KP; k += blockDim.x) {
    float v = 0.0f;
    if (f8 && k < shp.col_u) {
      // two E4M3 dims per 16-bit column, the lower index in the low byte
      uint32_t bits = 0;
      if (valid) {
        const int d0 = 2 * k, d1 = 2 * k + 1;
        const float x0 = d0 < K ? X[r * K + d0] * fr : 0.0f;
        const float x1 = d1 < K ? X[r * K + d1] * fr : 0.0f;
        bits = e4m3_bits(x0) | (e4m3_bits(x1) << 8);
      }
      reinterpret_cast<uint16_t*>(row)[k] = static_cast<uint16_t>(bits);
      continue;
    }
    if (valid) {
      if (k < shp.col_u) {
        // three-product dims: slots [0, Ks) as parts 0, 1, 2; one-product
        // dims after them (mult 1: every dim once)
        const int Ks = shp.mult == 3 ? shp.Ks : 0;
        int part = 0, slot = k;
        if (k < 3 * Ks) {
          part = k / Ks;
          slot = k % Ks;
        } else {
          slot = Ks + (k - 3 * Ks);
        }
        const int kk = perm ? perm[slot] : slot;
        const float x = X[r * K + kk] * sc;
        const float hi = from16(to16<T>(x));
        // A side [hi, hi, lo], B side [hi, lo, hi]: hi*hi + hi*lo + lo*hi
        const bool lo = k < 3 * Ks && ((role == 0 && part == 2) || (role == 1 && part == 1));
        v = lo ? x - hi : hi;
      } else if (k < shp.col_w) {
        const int part = k - shp.col_u;
        const float x = sq[r] * us;
        const float hi = from16(to16<T>(x));
        if (role == 0) v = part < 2 ? hi : x - hi;   // [hi, hi, lo]
        else v = part == 1 ? x - hi : hi;            // [hi, lo, hi]
      } else if (k < shp.col_e) {
        // column bias w_j = (h_j/eps + logw_j) log2(e) as c_w * split(w_j / c_w)
        if (role == 0) {
          v = cw;
        } else {
          const float w = (h[r] * inv_eps + logw[r]) * kLog2e;
          v = isfinite(w) ? split3<T>(w / wa / cw, k - shp.col_w) : 0.0f;
        }
      } else if (k < shp.col_k) {
        // row shift e_i = -est_i log2(e) / eps - kShiftBias as -c_e * split(-e_i / c_e)
        if (role == 1) {
          v = ce;
        } else if (est) {
          v = split3<T>((est[r] * inv_eps * kLog2e + shift_bias) / wa / ce, k - shp.col_e);
        }
      } else if (k == shp.col_k) {
        // mask: zero-weight target columns never contribute
        if (role == 0) v = kBiasConst;
        else v = isfinite(logw[r]) ? 0.0f : -kHalfMax;
      }
    } else if (role == 1 && k == shp.col_k) {
      v = -kHalfMax;   // padding columns never contribute
    }
    row[k] = to16<T>(v * fr);
  }
}

// Per-iteration refresh of up to two tasks in two launches.  The first writes
// each block's largest |w_j| (finite) and |e_i| per task to part[task][block][2]
// and zeroes the tasks' recompute flags; the second reduces those partials in
// every block (a max, so the order does not matter: the same scales as one
// grid-wide maximum) and rewrites the bias and shift columns of both sides of
// both tasks.  Operands come out identical to tc_bias_absmax + tc_refresh.
struct RefreshTask {
  const float* h;       // column potentials (B side)
  const float* logw;    // column log-weights
  const float* est;     // row shift estimate (A side) or null
  int64_t n, m;         // A rows, B rows
  float inv_eps;
  int* flags;
  int nflags;
  void* opA;
  void* opB;
  const float* fsA;     // FP8: per-group scales of the A side, or null
  const float* fsB;     // FP8: per-group scales of the B side
  float wa;             // FP8: alpha (the bias and shift columns in its units); else 1
};

__global__ void tc_refresh_max_kernel(RefreshTask t0, RefreshTask t1, int ntasks, float* part) {
  __shared__ float red[2][8];
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  const int64_t i0 = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  for (int q = 0; q < ntasks; ++q) {
    const RefreshTask& T = q == 0 ? t0 : t1;
    float vw = 0.f, ve = 0.f;
    for (int64_t i = i0; i < T.m; i += stride) {
      const float w = (T.h[i] * T.inv_eps + T.logw[i]) * kLog2e;
      if (isfinite(w)) vw = fmaxf(vw, fabsf(w));
    }
    if (T.est)
      for (int64_t i = i0; i < T.n; i += stride)
        ve = fmaxf(ve, fabsf(T.est[i] * T.inv_eps * kLog2e + kShiftBias));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      vw = fmaxf(vw, __shfl_xor_sync(0xffffffffu, vw, o));
      ve = fmaxf(ve, __shfl_xor_sync(0xffffffffu, ve, o));
    }
    if ((threadIdx.x & 31) == 0) {
      red[0][threadIdx.x >> 5] = vw;
      red[1][threadIdx.x >> 5] = ve;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      float a = 0.f, b = 0.f;
      for (int k = 0; k < static_cast<int>(blockDim.x >> 5); ++k) {
        a = fmaxf(a, red[0][k]);
        b = fmaxf(b, red[1][k]);
      }
      part[(static_cast<int64_t>(q) * gridDim.x + blockIdx.x) * 2 + 0] = a;
      part[(static_cast<int64_t>(q) * gridDim.x + blockIdx.x) * 2 + 1] = b;
    }
    __syncthreads();
    if (blockIdx.x == 0)
      for (int k = threadIdx.x; k < T.nflags; k += blockDim.x) T.flags[k] = 0;
  }
}

template <class T>
__global__ void tc_refresh_multi_kernel(RefreshTask t0, RefreshTask t1, int ntasks,
                                        TcOperandShape shp_f, const float* part, int nparts,
                                        const int* lay = nullptr,
                                        TcOperandShape shp_a = TcOperandShape{}) {
  const TcOperandShape shp = (lay != nullptr && lay[0] != 0) ? shape_ks(shp_a, lay[1]) : shp_f;
  __shared__ float cw[2], ce[2];
  if (threadIdx.x < 32) {
    for (int q = 0; q < ntasks; ++q) {
      float a = 0.f, b = 0.f;
      for (int k = threadIdx.x; k < nparts; k += 32) {
        a = fmaxf(a, part[(static_cast<int64_t>(q) * nparts + k) * 2 + 0]);
        b = fmaxf(b, part[(static_cast<int64_t>(q) * nparts + k) * 2 + 1]);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        a = fmaxf(a, __shfl_xor_sync(0xffffffffu, a, o));
        b = fmaxf(b, __shfl_xor_sync(0xffffffffu, b, o));
      }
      if (threadIdx.x == 0) {
        const float wa = (q == 0 ? t0 : t1).wa;
        cw[q] = pow2_scale(a / wa);
        ce[q] = pow2_scale(b / wa);
      }
    }
  }
  __syncthreads();
  // rows: task 0 A, task 0 B, task 1 A, task 1 B
  int64_t r = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  for (int q = 0; q < ntasks; ++q) {
    const RefreshTask& K = q == 0 ? t0 : t1;
    if (r < K.n) {
      T* row = static_cast<T*>(K.opA) + r * shp.KP;
      const float e = K.est ? (K.est[r] * K.inv_eps * kLog2e + kShiftBias) / K.wa / ce[q] : 0.0f;
      const float fr = K.fsA ? K.fsA[r / kFp8Group] : 1.0f;
      for (int k = 0; k < 3; ++k) {
        row[shp.col_w + k] = to16<T>(cw[q] * fr);
        row[shp.col_e + k] = to16<T>((K.est ? split3<T>(e, k) : 0.0f) * fr);
      }
      return;
    }
    r -= K.n;
    if (r < K.m) {
      T* row = static_cast<T*>(K.opB) + r * shp.KP;
      const float w = (K.h[r] * K.inv_eps + K.logw[r]) * kLog2e;
      const bool fin = isfinite(w);
      const float fr = K.fsB ? K.fsB[r / kFp8Group] : 1.0f;
      for (int k = 0; k < 3; ++k) {
        row[shp.col_w + k] = to16<T>((fin ? split3<T>(w / K.wa / cw[q], k) : 0.0f) * fr);
        row[shp.col_e + k] = to16<T>(ce[q] * fr);
      }
      return;
    }
    r -= K.m;
  }
}

__device__ __forceinline__ bool mbar_drain(uint64_t* bar, uint32_t parity) {
  const uint64_t t0 = tc::globaltimer();
  while (!tc::mbar_try_wait(bar, parity)) {
    if (tc::globaltimer() - t0 > tc::kWaitLimitNs) return false;
  }
  return true;
}
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

int make_map(CUtensorMap* map, void* ptr, int64_t rows, int KP, bool bf16, int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  GW_REQUIRE(enc != nullptr, GW_ECUDA, "cuTensorMapEncodeTiled is not available");
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(KP), static_cast<cuuint64_t>(rows)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(KP) * 2};
  cuuint32_t box[2] = {64, static_cast<cuuint32_t>(box_rows)};
  cuuint32_t es[2] = {1, 1};
  CUresult r = enc(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2,
                   ptr, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  GW_REQUIRE(r == CUDA_SUCCESS, GW_ECUDA, "cuTensorMapEncodeTiled failed (%d)", static_cast<int>(r));
  return GW_OK;
}

}  // namespace

}  // namespace gw
