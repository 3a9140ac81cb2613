// Softmin on the bilinear cost with the cost tile on the 5th-generation
// tensor cores (tcgen05), sm_103a.
//
//   out_i = -eps * LSE_j [ logw_j + (h_j + 16 <A_i, B_j> + 4 sA_i sB_j) / eps ]
//
// The whole exponent z_ij (base 2) is one matrix product of two 16-bit
// operand matrices built from A and B (the discrete Sinkhorn operator,
// Eq. sinkhorn_operators, on c_Gamma):
//   columns [0, mult*K)        the scaled dot product alpha <A_i, B_j>, with
//                              alpha = 16 log2(e) / eps, as one product
//                              (mult = 1) or as a two-way split
//                              hi*hi + hi*lo + lo*hi (mult = 3);
//   3 columns                  beta sA_i sB_j (beta = 4 log2(e) / eps) as a
//                              two-way split product;
//   3 columns                  the column bias w_j = (h_j/eps + logw_j) log2(e),
//                              a three-way split times a power-of-two constant;
//   3 columns                  minus a per-row shift estimate e_i (three-way split),
//                              when an estimate is given;
//   zero padding to KP (a multiple of 64).
// With an estimate (the previous potential of the output side, which the
// row's log-sum-exp equals at convergence) the epilogue only sums exp2 of
// what the MMA wrote: no subtraction, no max.  A row whose sum over- or
// underflows marks its CTA, and a second launch recomputes exactly those
// CTAs with the safe epilogue (running shift, a chunk redone against its
// own maximum when a value jumps above the shift).
//
// CTA layout (one CTA per SM): 256 rows as two M = 128 accumulators, column
// tiles of BN = 128 streamed by TMA through a ring of S stages (128-byte
// swizzle), double-buffered in TMEM (2 buffers x 2 halves x 128 columns =
// all 512 columns).  Warp 0 issues TMA, warp 1 issues tcgen05.mma, warps 2-9
// each own 32 rows (one TMEM lane quarter of one half).  Every wait is
// bounded in time; on a timeout the CTA drains its copies and MMAs, frees
// TMEM and writes NaN rows.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>
#include <string.h>

#include <mutex>

#include "gw_internal.cuh"
#include "gw_tc.cuh"
#include "gw_tc_ops.cuh"

namespace gw {

namespace {

constexpr int kBM = 256;       // rows per CTA (two M = 128 halves)
// columns per tile: 128, or 64 for the widest operands (KP = 256) so that the
// ring still fits in shared memory
__host__ __device__ constexpr int tile_cols(int KP) { return KP >= 256 ? 64 : 128; }
constexpr int kEpiWarps = 16;  // 4 per scheduler: 2 per (half, lane quarter), one per column half
constexpr int kThreadsTc = 64 + 32 * kEpiWarps;
constexpr float kRunInit = -1.0e9f;          // running max start (below every real exponent)
constexpr float kSumLo = 8.673617e-19f;      // 2^-60: a total below this underflowed
constexpr float kSumHi = 1.3292280e36f;      // 2^120: a sum above this (or inf/NaN) overflowed

struct TcTask {
  tc::WaitCtl wc;         // pipeline wait limit and the give-up counter
  const int* gate;        // layout decision (device); the launch runs only when
  int gate_on;            // *gate == gate_on (gate null: always); gate_on = 1 is the
  int K;                  // split layout, whose K-steps follow its dim count gate[1]
  int64_t n, m;           // real rows / columns
  int ksteps;             // MMA K-steps of 16 that hold non-zero operand columns
  const float* est;       // per-row shift estimate (fast pass), or null
  int* flags;             // per-CTA "recompute" flags shared by the two passes
  int row_tiles;          // ceil(n / 256)
  int col_tiles;          // m_pad / 128
  int splits;
  int tiles_per_split;
  int blocks;
  float eps;
  const float* avg_with;
  float* out;
  float* pm;
  float* ps;
  int k8;                 // FP8: leading K-steps of E4M3 features (kind::f8f6f4)
  const float* fsA;       // FP8: power-of-two scale of each 128-row group of A
  const float* fsB;       // FP8: the same per 128-row group of B (one per tile)
  float alpha8;           // FP8: 16 log2(e) / eps, applied in the epilogue
};

template <int KP, int S, int BN>
struct TcSmem {
  static constexpr int KB = KP / 64;
  static constexpr int kABytes = 2 * KB * 16384;          // 256 rows
  static constexpr int kBBlock = BN * 128;                // one 64-wide K-block of a B tile
  static constexpr int kStageBytes = KB * kBBlock;
  static constexpr int kBarOff = kABytes + S * kStageBytes;
  // + barriers and the row-merge buffers (3 x 256 words) + alignment slack;
  // at least 120 KB so that one CTA owns the SM (it allocates all 512 TMEM
  // columns)
  static constexpr int kTail = 256 + 3 * 1024 + 1024;
  static constexpr int kBytes = kBarOff + kTail > 122880 ? kBarOff + kTail : 122880;
};


// Sum of exp2(v_k - shift) over 32 values, with the shift and the sum as
// packed FP32x2 adds.
__device__ __forceinline__ float exp2_sum32(const float (&v)[32], float shift) {
  const uint64_t neg = tc::pack2(-shift, -shift);
  uint64_t acc0 = tc::pack2(0.f, 0.f), acc1 = acc0;
#pragma unroll
  for (int k = 0; k < 32; k += 4) {
    float d0, d1, d2, d3;
    tc::unpack2(tc::add2(tc::pack2(v[k], v[k + 1]), neg), d0, d1);
    tc::unpack2(tc::add2(tc::pack2(v[k + 2], v[k + 3]), neg), d2, d3);
    acc0 = tc::add2(acc0, tc::pack2(ex2(d0), ex2(d1)));
    acc1 = tc::add2(acc1, tc::pack2(ex2(d2), ex2(d3)));
  }
  float s0, s1;
  tc::unpack2(tc::add2(acc0, acc1), s0, s1);
  return s0 + s1;
}

// Fold 32 base-2 exponents into the running (shift, sum): lse = shift +
// log2(sum) holds for any shift, so the common path exponentiates against
// the current shift with no max in the dependency chain.  Only when a value
// lies more than ~43 above the shift (the partial sum reaches 2^48, or is
// inf/NaN after an overflow) is the chunk redone against its own maximum,
// which then becomes the shift.  The shift only ever takes values of real
// exponents, so nothing that matters underflows.
__device__ __forceinline__ void lse_chunk(const uint32_t (&r)[32], float& shift, float& sum) {
  float v[32];
#pragma unroll
  for (int k = 0; k < 32; ++k) v[k] = __uint_as_float(r[k]);
  float acc = exp2_sum32(v, shift);
  if (!(acc < 281474976710656.0f)) {   // 2^48
    float a[11];
#pragma unroll
    for (int k = 0; k < 10; ++k) a[k] = tc::max3(v[3 * k], v[3 * k + 1], v[3 * k + 2]);
    a[10] = fmaxf(v[30], v[31]);
    const float b0 = tc::max3(a[0], a[1], a[2]);
    const float b1 = tc::max3(a[3], a[4], a[5]);
    const float b2 = tc::max3(a[6], a[7], a[8]);
    const float b3 = tc::max3(a[9], a[10], shift);
    const float mnew = fmaxf(tc::max3(b0, b1, b2), b3);
    sum *= ex2(shift - mnew);
    shift = mnew;
    acc = exp2_sum32(v, shift);
  }
  sum += acc;
}

// Fast pass: the 32 values are already shifted; just sum their exp2.
__device__ __forceinline__ float exp2_sum32_noshift(const float (&v)[32]) {
  uint64_t acc0 = tc::pack2(0.f, 0.f), acc1 = acc0, acc2 = acc0, acc3 = acc0;
#pragma unroll
  for (int k = 0; k < 32; k += 8) {
    acc0 = tc::add2(acc0, tc::pack2(ex2(v[k]), ex2(v[k + 1])));
    acc1 = tc::add2(acc1, tc::pack2(ex2(v[k + 2]), ex2(v[k + 3])));
    acc2 = tc::add2(acc2, tc::pack2(ex2(v[k + 4]), ex2(v[k + 5])));
    acc3 = tc::add2(acc3, tc::pack2(ex2(v[k + 6]), ex2(v[k + 7])));
  }
  float s0, s1;
  tc::unpack2(tc::add2(tc::add2(acc0, acc1), tc::add2(acc2, acc3)), s0, s1);
  return s0 + s1;
}

template <bool FAST>
__device__ __forceinline__ void chunk(const uint32_t (&r)[32], float& shift, float& sum) {
  if (FAST) {
    float v[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) v[k] = __uint_as_float(r[k]);
    sum += exp2_sum32_noshift(v);
  } else {
    lse_chunk(r, shift, sum);
  }
}

template <int KP, int S, int BN, bool BF16, bool FAST, bool F8>
__global__ void __launch_bounds__(kThreadsTc, 1)
    softmin_tc_kernel(const __grid_constant__ CUtensorMap mA0, const __grid_constant__ CUtensorMap mB0,
                      const __grid_constant__ CUtensorMap mA1, const __grid_constant__ CUtensorMap mB1,
                      TcTask t0, TcTask t1) {
  using L = TcSmem<KP, S, BN>;
  constexpr int KB = L::KB;
  constexpr int kTmemCols = 4 * BN;   // 2 buffers x 2 halves
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* As = smem;
  unsigned char* Bs = smem + L::kABytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::kBarOff);
  uint64_t* full = bars;                // [S]
  uint64_t* empty = bars + S;           // [S]
  uint64_t* tfull = bars + 2 * S;       // [2]
  uint64_t* tempty = bars + 2 * S + 2;  // [2]
  uint64_t* afull = bars + 2 * S + 4;
  uint64_t* drain = bars + 2 * S + 5;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  __shared__ int consumed;

  const bool second = static_cast<int>(blockIdx.x) >= t0.blocks;
  const TcTask& T = second ? t1 : t0;
  const CUtensorMap* mA = second ? &mA1 : &mA0;
  const CUtensorMap* mB = second ? &mB1 : &mB0;
  const int bid = second ? blockIdx.x - t0.blocks : blockIdx.x;
  const int rt = bid / T.splits;
  const int sp = bid % T.splits;
  const int row0 = rt * kBM;
  const int tile0 = sp * T.tiles_per_split;
  const int ntiles = min(T.tiles_per_split, T.col_tiles - tile0);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // the operands are in the other layout: that launch does the work
  if (T.gate != nullptr && *T.gate != T.gate_on) return;
  // the split layout holds 2 gate[1] + K + 10 non-zero operand columns
  const int nks_run =
      (T.gate != nullptr && T.gate_on == 1) ? (2 * T.gate[1] + T.K + 10 + 15) / 16 : T.ksteps;
  // the safe pass only recomputes the row tiles the fast pass marked
  if (!FAST && T.flags != nullptr && T.flags[rt] == 0) return;

  if (threadIdx.x == 0) {
    abort_flag = 0;
    consumed = 0;
    for (int s = 0; s < S; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&tfull[b], 1);
      tc::mbar_init(&tempty[b], kEpiWarps);
    }
    tc::mbar_init(afull, 1);
    tc::mbar_init(drain, 1);
    tc::fence_mbar_init();
  }
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base, kTmemCols);
    tc::tmem_relinquish();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tbase = tmem_base;
  volatile int* ab = &abort_flag;
  const uint64_t lim = T.wc.limit_ns;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------------------------------------------------- producer
      tc::prefetch_tmap(mA);
      tc::prefetch_tmap(mB);
      tc::mbar_arrive_expect_tx(afull, L::kABytes);
      for (int h = 0; h < 2; ++h)
        for (int kb = 0; kb < KB; ++kb)
          tc::tma_load_2d(As + (h * KB + kb) * 16384, mA, kb * 64, row0 + h * 128, afull);
      int issued = 0;
      for (int t = 0; t < ntiles; ++t) {
        const int s = t % S;
        if (!tc::mbar_wait(&empty[s], ((t / S) & 1) ^ 1, ab, lim)) break;
        tc::mbar_arrive_expect_tx(&full[s], L::kStageBytes);
        for (int kb = 0; kb < KB; ++kb)
          tc::tma_load_2d(Bs + s * L::kStageBytes + kb * L::kBBlock, mB, kb * 64, (tile0 + t) * BN,
                          &full[s]);
        issued = t + 1;
      }
      if (*ab) {
        // wind down: wait for the copies still in flight before leaving
        mbar_drain(afull, 0);
        const int done = *reinterpret_cast<volatile int*>(&consumed);
        for (int t = done; t < issued; ++t) mbar_drain(&full[t % S], (t / S) & 1);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ------------------------------------------------------- MMA issuer
      const uint32_t idesc = tc::f16_idesc(128, BN, BF16);
      constexpr uint32_t idesc8 = tc::f16_idesc(128, BN, false);   // E4M3 x E4M3
      const int k8 = F8 ? T.k8 : 0;
      bool ok = tc::mbar_wait(afull, 0, ab, lim);
      for (int t = 0; ok && t < ntiles; ++t) {
        const int s = t % S, b = t & 1;
        if (!tc::mbar_wait(&tempty[b], ((t >> 1) & 1) ^ 1, ab, lim)) break;
        if (!tc::mbar_wait(&full[s], (t / S) & 1, ab, lim)) break;
        tc::tc_fence_after();
        const unsigned char* Bst = Bs + s * L::kStageBytes;
        const int nks = nks_run;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
#pragma unroll
          for (int ks = 0; ks < KP / 16; ++ks) {
            if (ks >= nks) break;   // the rest of the operand row is zero padding
            const uint32_t aaddr = tc::smem_u32(As + (h * KB + ks / 4) * 16384 + (ks % 4) * 32);
            const uint32_t baddr = tc::smem_u32(Bst + (ks / 4) * L::kBBlock + (ks % 4) * 32);
            if (F8 && ks < k8)
              tc::mma_f8(tbase + (b * 2 + h) * BN, tc::sw128_desc(aaddr), tc::sw128_desc(baddr),
                         idesc8, ks > 0 ? 1u : 0u);
            else
              tc::mma_f16(tbase + (b * 2 + h) * BN, tc::sw128_desc(aaddr), tc::sw128_desc(baddr),
                          idesc, ks > 0 ? 1u : 0u);
          }
        }
        tc::mma_commit(&empty[s]);
        tc::mma_commit(&tfull[b]);
        *reinterpret_cast<volatile int*>(&consumed) = t + 1;
      }
      // every MMA issued above has finished before TMEM is freed
      tc::mma_commit(drain);
      mbar_drain(drain, 0);
    }
  } else {
    // ------------------------------------------------------------ epilogue
    // warp -> (half h, lane quarter q = warp % 4, column half ch): each row's
    // 128 columns per tile are shared by two warps, merged at the end
    const int e = warp - 2;
    const int g = e >> 2;
    const int h = g & 1;
    const int ch = g >> 1;
    const int q = warp & 3;
    const int64_t row = static_cast<int64_t>(row0) + h * 128 + q * 32 + lane;
    // fast pass: the MMA already subtracted the shift e_i, the sum starts at 0
    float mrun = FAST ? 0.0f : kRunInit, srun = 0.0f;
    bool ok = true;
    // FP8: alpha / fsA of this half's row group (the scales cover n_pad rows)
    static_assert(!F8 || BN == kFp8Group, "FP8 column tiles are the scale groups");
    const float a_over = F8 ? T.alpha8 / T.fsA[(row0 >> 7) + h] : 1.0f;
    for (int t = 0; t < ntiles; ++t) {
      const int b = t & 1;
      // one lane waits, the warp follows: tcgen05.ld needs a converged warp
      int got = 0;
      if (lane == 0) got = tc::mbar_wait(&tfull[b], (t >> 1) & 1, ab, lim) ? 1 : 0;
      got = __shfl_sync(0xffffffffu, got, 0);
      if (!got) {
        ok = false;
        break;
      }
      tc::tc_fence_after();
      const uint32_t tcol =
          tbase + (static_cast<uint32_t>(q * 32) << 16) + (b * 2 + h) * BN + ch * (BN / 2);
      uint32_t ra[32];
      if constexpr (BN == 128) {
        // the warp's 64 columns in one TMEM load, reduced as two chunks of 32
        uint32_t r64[64];
        tc::tmem_ld64_issue(tcol, r64);
        tc::tmem_ld_wait(r64);
        if constexpr (F8) unscale(r64, a_over / T.fsB[tile0 + t]);
        chunk<FAST>(*reinterpret_cast<const uint32_t(*)[32]>(&r64[0]), mrun, srun);
        chunk<FAST>(*reinterpret_cast<const uint32_t(*)[32]>(&r64[32]), mrun, srun);
      } else {
        tc::tmem_ld32_issue(tcol, ra);
        tc::tmem_ld_wait(ra);
        if constexpr (F8) unscale(ra, a_over / T.fsB[tile0 + t]);
        chunk<FAST>(ra, mrun, srun);
      }
      tc::tc_fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&tempty[b]);
    }
    // merge the two column halves of each row (named barrier of the epilogue
    // warps only); the ch = 0 warp writes the row
    {
      float* xm = reinterpret_cast<float*>(bars + 2 * S + 8);   // [256] shifts
      float* xs = xm + 256;                                     // [256] sums
      int* xo = reinterpret_cast<int*>(xs + 256);               // [256] ok
      const int slot = h * 128 + q * 32 + lane;
      if (ch == 1) {
        xm[slot] = mrun;
        xs[slot] = srun;
        xo[slot] = ok ? 1 : 0;
      }
      asm volatile("bar.sync 1, %0;" ::"r"(32 * kEpiWarps) : "memory");
      if (ch == 1) goto epilogue_done;
      const float m2 = xm[slot], s2 = xs[slot];
      ok = ok && xo[slot] != 0;
      if (FAST) {
        srun += s2;   // both halves sum against the same shift
      } else {
        const float M = fmaxf(mrun, m2);
        srun = srun * ex2(mrun - M) + s2 * ex2(m2 - M);
        mrun = M;
      }
    }
    if (row < T.n) {
      // z' = z - shift_i came out of the MMA when an estimate was folded in
      const float shift_i = T.est ? -T.est[row] * (kLog2e / T.eps) - kShiftBias : 0.0f;
      const int64_t po = static_cast<int64_t>(sp) * T.n + row;
      if (!ok || *ab) {
        const float nan = __int_as_float(0x7fc00000);   // a wait gave up
        if (T.splits == 1) T.out[row] = nan;
        else T.pm[po] = T.ps[po] = nan;
      } else if (FAST) {
        // a split may hold none of the row's mass (its sum underflows
        // harmlessly); only overflow, or a total out of range, needs the
        // safe pass, which then recomputes the whole row tile
        if (T.splits == 1) {
          if (srun > kSumLo && srun < kSumHi) {
            float v = -T.eps * kLn2 * (shift_i + log2f(srun));
            if (T.avg_with) v = 0.5f * (T.avg_with[row] + v);
            T.out[row] = v;
          } else {
            T.flags[rt] = 1;
          }
        } else if (srun < kSumHi) {
          T.pm[po] = shift_i;
          T.ps[po] = srun;
        } else {
          T.flags[rt] = 1;
        }
      } else if (T.splits == 1) {
        float v = -T.eps * kLn2 * (shift_i + mrun + log2f(srun));
        if (T.avg_with) v = 0.5f * (T.avg_with[row] + v);
        T.out[row] = v;
      } else {
        T.pm[po] = shift_i + mrun;
        T.ps[po] = srun;
      }
    }
  epilogue_done:;
  }
  tc::tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0) tc::note_gave_up(T.wc, ab);
  if (warp == 0) {
    __syncwarp();
    tc::tc_fence_after();
    tc::tmem_dealloc(tbase, kTmemCols);
  }
}

// Per-dim maxima of |A_ik| -> out[k] (block: 128 x 2 threads, k = x).
__global__ void tc_dimmax_kernel(const float* A, int64_t n, int K, unsigned* out) {
  const int k = threadIdx.x;
  if (k >= K) return;
  float v = 0.0f;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.y + threadIdx.y; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.y)
    v = fmaxf(v, fabsf(A[i * K + k]));
  atomicMax(&out[k], __float_as_uint(v));
}

// Layout decision of the split precisions (one block of 128 threads):
// P_k = max|A_k| max|B_k| bounds every product of dim k; the dims are ordered
// by P_k (largest first, ties by index) into lay[2 .. 2 + K), lay[1] = the
// count of dims with P_k above tau max P (those run as three products, the
// others as one, within the split products' error bound), and lay[0] = 1
// (the split layout) when that count fits the layout (at most ks_max).
__global__ void tc_layout_kernel(const unsigned* mxA, const unsigned* mxB, int K, float tau,
                                 int ks_max, int* lay) {
  __shared__ float P[128];
  const int k = threadIdx.x;
  float pk = -1.0f;
  if (k < K) {
    pk = __uint_as_float(mxA[k]) * __uint_as_float(mxB[k]);
    if (!(pk == pk)) pk = -1.0f;   // NaN sorts last
  }
  P[k] = pk;
  __syncthreads();
  float pmax = 0.0f;
  for (int j = 0; j < K; ++j) pmax = fmaxf(pmax, P[j]);
  const int big = __syncthreads_count(k < K && pk > tau * pmax);
  if (k < K) {
    int rank = 0;
    for (int j = 0; j < K; ++j) rank += (P[j] > pk || (P[j] == pk && j < k)) ? 1 : 0;
    lay[2 + rank] = k;
  }
  if (k == 0) {
    lay[0] = big <= ks_max ? 1 : 0;
    lay[1] = big;
  }
}

// Merge split partials.  mode 0: every row; mode 1 (after the fast pass):
// rows of unflagged tiles whose total is in range are written, the others
// flag their tile; mode 2 (after the safe pass): rows of flagged tiles only.
__global__ void tc_combine_kernel(TcTask t0, TcTask t1, int64_t n0, int mode) {
  const int64_t gi = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const bool second = gi >= n0;
  const TcTask& T = second ? t1 : t0;
  const int64_t i = second ? gi - n0 : gi;
  if (i >= T.n || T.splits == 1) return;
  const int rt = static_cast<int>(i / kBM);
  if (mode == 1 && T.flags[rt] != 0) return;
  if (mode == 2 && T.flags[rt] == 0) return;
  float M = kNegBig;
  for (int s = 0; s < T.splits; ++s) M = fmaxf(M, T.pm[static_cast<int64_t>(s) * T.n + i]);
  float S = 0.0f;
  for (int s = 0; s < T.splits; ++s) {
    const int64_t o = static_cast<int64_t>(s) * T.n + i;
    S += T.ps[o] * ex2(T.pm[o] - M);
  }
  if (mode == 1 && !(S > kSumLo && S < kSumHi)) {
    T.flags[rt] = 1;
    return;
  }
  float v = -T.eps * kLn2 * (M + log2f(S));
  if (T.avg_with) v = 0.5f * (T.avg_with[i] + v);
  T.out[i] = v;
}

int run_combine(const TcTask& a, const TcTask& b, int mode, cudaStream_t st) {
  if (a.splits == 1 && (b.blocks == 0 || b.splits == 1)) return GW_OK;
  const int64_t nn = a.n + (b.blocks ? b.n : 0);
  tc_combine_kernel<<<ceil_div(nn, 256), 256, 0, st>>>(a, b, a.n, mode);
  GW_LAUNCH_CHECK();
  return GW_OK;
}

// ------------------------------------------------------------ host side
int tc_splits(int row_tiles, int col_tiles, int other_blocks) {
  // Pick the column split that fills whole waves of 152 CTAs best.
  int best = 1;
  double best_eff = 0.0;
  const int smax = max_splits(col_tiles);
  for (int s = 1; s <= smax; ++s) {
    const int blocks = row_tiles * s + other_blocks * s;
    const int waves = (blocks + kSmCount - 1) / kSmCount;
    const double eff = static_cast<double>(blocks) / (static_cast<double>(waves) * kSmCount);
    const double tiles = static_cast<double>(col_tiles) / s;
    if (tiles < 4.0 && s > 1) break;   // keep >= 4 tiles per CTA to amortise set-up
    if (eff > best_eff + 1e-3) {
      best_eff = eff;
      best = s;
    }
    if (eff > 0.97) break;
  }
  return best;
}

template <int KP, int S, bool BF16, bool FAST, bool F8 = false>
int launch_tc_kernel(const CUtensorMap* maps, const TcTask& a, const TcTask& b, cudaStream_t st) {
  constexpr int BN = tile_cols(KP);
  using L = TcSmem<KP, S, BN>;
  auto kern = softmin_tc_kernel<KP, S, BN, BF16, FAST, F8>;
  static std::once_flag once;   // the attribute is the same for every call
  static cudaError_t attr_rc = cudaSuccess;
  std::call_once(once, [&] {
    attr_rc = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L::kBytes);
  });
  GW_CUDA_TRY(attr_rc);
  kern<<<a.blocks + b.blocks, kThreadsTc, L::kBytes, st>>>(maps[0], maps[1], maps[2], maps[3], a, b);
  GW_LAUNCH_CHECK();
  return GW_OK;
}

template <bool BF16, bool FAST>
int dispatch_tc(int KP, const CUtensorMap* maps, const TcTask& a, const TcTask& b, cudaStream_t st) {
  switch (KP) {
    case 64: return launch_tc_kernel<64, 4, BF16, FAST>(maps, a, b, st);
    case 128: return launch_tc_kernel<128, 3, BF16, FAST>(maps, a, b, st);
    case 192: return launch_tc_kernel<192, 2, BF16, FAST>(maps, a, b, st);
    case 256: return launch_tc_kernel<256, 2, BF16, FAST>(maps, a, b, st);
    default: break;
  }
  set_error("tensor-core softmin: operand width %d (K too large for this precision)", KP);
  return GW_EUNSUPPORTED;
}

// FP8 operands (E4M3 features, BF16 bias columns): KP 64 or 128 only
template <bool FAST>
int dispatch_tc_f8(int KP, const CUtensorMap* maps, const TcTask& a, const TcTask& b,
                   cudaStream_t st) {
  switch (KP) {
    case 64: return launch_tc_kernel<64, 4, true, FAST, true>(maps, a, b, st);
    case 128: return launch_tc_kernel<128, 3, true, FAST, true>(maps, a, b, st);
    default: break;
  }
  set_error("tensor-core softmin (FP8): operand width %d (K too large)", KP);
  return GW_EUNSUPPORTED;
}

int run_tc(bool bf16, bool fast, int KP, const CUtensorMap* maps, const TcTask& a, const TcTask& b,
           cudaStream_t st) {
  if (a.k8 > 0) return fast ? dispatch_tc_f8<true>(KP, maps, a, b, st)
                            : dispatch_tc_f8<false>(KP, maps, a, b, st);
  if (bf16) return fast ? dispatch_tc<true, true>(KP, maps, a, b, st)
                        : dispatch_tc<true, false>(KP, maps, a, b, st);
  return fast ? dispatch_tc<false, true>(KP, maps, a, b, st)
              : dispatch_tc<false, false>(KP, maps, a, b, st);
}

}  // namespace

bool softmin_tc_supported(int K, int prec) {
  if (prec == GW_PREC_FP8) return tc_shape(K, prec).KP <= 128;
  if (prec != GW_PREC_BF16 && prec != GW_PREC_BF16X3 && prec != GW_PREC_F16X3) return false;
  return tc_shape(K, prec).KP <= 256;
}

// The narrow split layout is tried for the split precisions when the full
// layout needs 192 or more operand columns (K >= 40): it holds the dims of
// largest product bound as three products and the rest as one, in 128 columns.
constexpr int kNarrowKP = 128;
// (measured: on K = 32 lifted features the split layout in the full 128
// columns, 5 instead of 7 K-steps, made the fused iteration slower, 3.43 ms
// against 3.22 ms at N = M = 100k: the kernel is bound by its epilogue there)
bool narrow_enabled(const TcOperandShape& f) { return f.mult == 3 && f.KP >= 192; }
// width of the split layout: 128 columns when the full one needs more,
// else the full width (then every dim count fits and one launch does)
int narrow_kp(const TcOperandShape& f) { return f.KP > kNarrowKP ? kNarrowKP : f.KP; }

size_t softmin_tc_ws_bytes(int64_t n, int64_t m, int K, int prec) {
  const TcOperandShape shp = tc_shape(K, prec);
  const int64_t n_pad = ((n + kBM - 1) / kBM) * kBM;
  const int bn = tile_cols(shp.KP);
  const int64_t m_pad = ((m + bn - 1) / bn) * bn;
  Carver c(nullptr, ~size_t(0));
  c.take<uint16_t>(static_cast<size_t>(n_pad) * shp.KP);
  c.take<uint16_t>(static_cast<size_t>(m_pad) * shp.KP);
  c.take<unsigned>(8);
  // partials for the largest split count any launch may pick
  const int s = max_splits(static_cast<int>(m_pad / bn));
  c.take<float>(static_cast<size_t>(s) * n);
  c.take<float>(static_cast<size_t>(s) * n);
  c.take<int>(static_cast<size_t>(n_pad / kBM));       // recompute flags per row tile
  if (narrow_enabled(shp)) {
    c.take<unsigned>(256);                             // per-dim maxima of A and B
    c.take<int>(2 + 128);                              // layout decision
  }
  c.take<float>(static_cast<size_t>(2 * 2 * kSmCount));  // per-block maxima of the refresh
  if (shp.k8 > 0) {
    c.take<float>(static_cast<size_t>(n_pad / kFp8Group));   // FP8 group scales of A
    c.take<float>(static_cast<size_t>(m_pad / kFp8Group));   // and of B
  }
  return c.used();
}

// Prepare operands for one or two tasks and launch the tensor-core kernel.
// Fills tasks[q].splits / pm / ps so the caller can merge split partials.
// The split precisions take the device's layout decision (tc_layout_kernel,
// made from the first task's maxima when the operands are prepared): the dims
// of large product bound as three products, the rest as one, in the split
// layout (tc_shape_split; the MMA runs only its non-zero K-steps).  Where the
// full layout is wider than 128 columns (K >= 40) it stays as the fallback
// for spectra too flat for 128 columns: both kernels are launched and the
// device's decision lets exactly one run, the other returns at once; both use
// the same column splits, so their partials merge alike.
int launch_softmin_tc(SoftminTask* tasks, int ntasks, int prec, Carver& ws, cudaStream_t st) {
  GW_REQUIRE(softmin_tc_supported(tasks[0].K, prec), GW_EUNSUPPORTED,
             "tensor-core softmin does not support K=%d with precision %d", tasks[0].K, prec);
  const bool bf16 = tc_is_bf16(prec);
  CUtensorMap maps[4], maps_a[4];
  TcTask tt[2], ta[2];
  memset(tt, 0, sizeof(tt));
  memset(ta, 0, sizeof(ta));
  const TcOperandShape shp = tc_shape(tasks[0].K, prec);
  const bool narrow = narrow_enabled(shp);
  const TcOperandShape shp_a = narrow ? tc_shape_split(tasks[0].K, prec, narrow_kp(shp)) : shp;
  const int kp_a = shp_a.KP;
  // the split layout in the full width needs no second launch
  const bool two_launches = narrow && kp_a != shp.KP;
  const int bn_f = tile_cols(shp.KP), bn_a = tile_cols(kp_a);
  int row_tiles[2] = {0, 0}, col_tiles[2] = {0, 0};
  for (int q = 0; q < ntasks; ++q) {
    row_tiles[q] = ceil_div(tasks[q].n, kBM);
    col_tiles[q] = ceil_div(tasks[q].m, bn_f);
  }
  // the fast pass needs an estimate for every task (not aliased to the output)
  bool all_est = true;
  for (int q = 0; q < ntasks; ++q)
    all_est = all_est && tasks[q].est != nullptr && tasks[q].est != tasks[q].out;
  // one split count for the launch, chosen from both tasks' tiles
  const int splits = tc_splits(row_tiles[0], col_tiles[0], ntasks == 2 ? row_tiles[1] : 0);
  RefreshTask refresh[2];
  memset(refresh, 0, sizeof(refresh));
  int* lay = nullptr;
  for (int q = 0; q < ntasks; ++q) {
    SoftminTask& T = tasks[q];
    const int64_t n_pad = static_cast<int64_t>(row_tiles[q]) * kBM;
    const int64_t m_pad = static_cast<int64_t>(col_tiles[q]) * bn_f;
    const int col_tiles_a = ceil_div(T.m, bn_a);
    const int64_t m_pad_a = static_cast<int64_t>(col_tiles_a) * bn_a;
    uint16_t* opA = ws.take<uint16_t>(static_cast<size_t>(n_pad) * shp.KP);
    uint16_t* opB = ws.take<uint16_t>(static_cast<size_t>(m_pad) * shp.KP);
    unsigned* mx = ws.take<unsigned>(8);
    int s = splits < col_tiles[q] ? splits : col_tiles[q];
    int tps = ceil_div(col_tiles[q], s);
    // the narrow layout's tiles are bn_a / bn_f full tiles wide: an even
    // count of full tiles per split gives both layouts the same splits
    if (narrow && bn_a != bn_f && (tps % 2) != 0) tps += 1;
    s = ceil_div(col_tiles[q], tps);
    T.splits = s;
    T.cols_per_split = tps * bn_f;
    T.pm = T.ps = nullptr;
    if (s > 1) {
      T.pm = ws.take<float>(static_cast<size_t>(s) * T.n);
      T.ps = ws.take<float>(static_cast<size_t>(s) * T.n);
    }
    const bool use_est = all_est;
    int* flags = ws.take<int>(static_cast<size_t>(row_tiles[q]));
    unsigned* mxd = nullptr;
    if (narrow && q == 0) {
      mxd = ws.take<unsigned>(256);
      lay = ws.take<int>(2 + 128);
    }
    float* fsA = nullptr;
    float* fsB = nullptr;
    if (shp.k8 > 0) {
      fsA = ws.take<float>(static_cast<size_t>(n_pad / kFp8Group));
      fsB = ws.take<float>(static_cast<size_t>(m_pad / kFp8Group));
    }
    GW_REQUIRE(!ws.overflow, GW_ENOMEM, "workspace too small for the tensor-core softmin");
    const int tps_a = narrow ? tps * bn_f / bn_a : tps;
    GW_REQUIRE(!narrow || ceil_div(col_tiles_a, tps_a) == s, GW_ECUDA,
               "internal: split layouts disagree (%d tiles, %d per split)", col_tiles_a, tps_a);
    const float inv_eps = 1.0f / T.eps;
    if (T.reuse_ops) {
      // main, rank-one and mask columns are unchanged: the bias and shift
      // columns of every task are refreshed after this loop, in two launches
      refresh[q] = RefreshTask{T.h, T.logw, use_est ? T.est : nullptr, T.n, T.m, inv_eps, flags,
                               row_tiles[q], opA, opB, fsA, fsB,
                               shp.k8 > 0 ? 16.0f * kLog2e * inv_eps : 1.0f};
    } else {
      GW_CUDA_TRY(cudaMemsetAsync(flags, 0, sizeof(int) * row_tiles[q], st));
      GW_CUDA_TRY(cudaMemsetAsync(mx, 0, 8 * sizeof(unsigned), st));
      tc_absmax_kernel<<<2 * kSmCount, 256, 0, st>>>(T.A, T.n * T.K, T.B, T.m * T.K, T.sA, T.n,
                                                     T.sB, T.m, T.h, T.logw,
                                                     use_est ? T.est : nullptr, inv_eps, mx);
      GW_LAUNCH_CHECK();
      if (mxd != nullptr) {
        // the layout decision, from this task's per-dim maxima (the other
        // task's are the same products with the roles exchanged)
        GW_CUDA_TRY(cudaMemsetAsync(mxd, 0, 256 * sizeof(unsigned), st));
        tc_dimmax_kernel<<<kSmCount, dim3(128, 2), 0, st>>>(T.A, T.n, T.K, mxd);
        GW_LAUNCH_CHECK();
        tc_dimmax_kernel<<<kSmCount, dim3(128, 2), 0, st>>>(T.B, T.m, T.K, mxd + 128);
        GW_LAUNCH_CHECK();
        tc_layout_kernel<<<1, 128, 0, st>>>(mxd, mxd + 128, T.K, split_threshold(prec),
                                            shp_a.Ks, lay);
        GW_LAUNCH_CHECK();
      }
      const float alpha = 16.0f * kLog2e * inv_eps;
      const float beta = 4.0f * kLog2e * inv_eps;
      const int64_t mrows = m_pad > m_pad_a ? m_pad : m_pad_a;
      if (shp.k8 > 0) {
        // FP8: one power-of-two scale per 128-row group of A and of B
        const int64_t ga = n_pad / kFp8Group, gb = m_pad / kFp8Group;
        fp8_scale_kernel<<<ceil_div(ga * 32, 256), 256, 0, st>>>(T.A, T.n, T.K, ga, fsA);
        GW_LAUNCH_CHECK();
        fp8_scale_kernel<<<ceil_div(gb * 32, 256), 256, 0, st>>>(T.B, T.m, T.K, gb, fsB);
        GW_LAUNCH_CHECK();
      }
      dim3 blk(64, 4);
      if (bf16) {
        tc_prep_kernel<__nv_bfloat16><<<ceil_div(n_pad, 4), blk, 0, st>>>(
            T.A, T.sA, nullptr, nullptr, use_est ? T.est : nullptr, T.n, n_pad, shp, 0, alpha,
            beta, inv_eps, mx, reinterpret_cast<__nv_bfloat16*>(opA), kShiftBias, lay, shp_a,
            n_pad, fsA);
        GW_LAUNCH_CHECK();
        tc_prep_kernel<__nv_bfloat16><<<ceil_div(mrows, 4), blk, 0, st>>>(
            T.B, T.sB, T.h, T.logw, nullptr, T.m, m_pad, shp, 1, alpha, beta, inv_eps, mx,
            reinterpret_cast<__nv_bfloat16*>(opB), kShiftBias, lay, shp_a, m_pad_a, fsB);
        GW_LAUNCH_CHECK();
      } else {
        tc_prep_kernel<__half><<<ceil_div(n_pad, 4), blk, 0, st>>>(
            T.A, T.sA, nullptr, nullptr, use_est ? T.est : nullptr, T.n, n_pad, shp, 0, alpha,
            beta, inv_eps, mx, reinterpret_cast<__half*>(opA), kShiftBias, lay, shp_a, n_pad);
        GW_LAUNCH_CHECK();
        tc_prep_kernel<__half><<<ceil_div(mrows, 4), blk, 0, st>>>(
            T.B, T.sB, T.h, T.logw, nullptr, T.m, m_pad, shp, 1, alpha, beta, inv_eps, mx,
            reinterpret_cast<__half*>(opB), kShiftBias, lay, shp_a, m_pad_a);
        GW_LAUNCH_CHECK();
      }
    }
    GW_TRY(make_map(&maps[2 * q], opA, n_pad, shp.KP, bf16, 128));
    GW_TRY(make_map(&maps[2 * q + 1], opB, m_pad, shp.KP, bf16, bn_f));
    TcTask& K = tt[q];
    K.n = T.n;
    K.m = T.m;
    K.ksteps = (shp.used + 15) / 16;
    K.est = use_est ? T.est : nullptr;
    K.flags = flags;
    K.row_tiles = row_tiles[q];
    K.col_tiles = col_tiles[q];
    K.splits = s;
    K.tiles_per_split = tps;
    K.blocks = row_tiles[q] * s;
    K.eps = T.eps;
    K.avg_with = T.avg_with;
    K.out = T.out;
    K.pm = T.pm;
    K.ps = T.ps;
    K.wc = wait_ctl();
    K.gate = nullptr;
    K.gate_on = 0;
    K.K = T.K;
    K.k8 = shp.k8;
    K.fsA = fsA;
    K.fsB = fsB;
    K.alpha8 = 16.0f * kLog2e * inv_eps;
    if (narrow) {
      // the split layout over the same buffers (its rows are kp_a wide)
      GW_TRY(make_map(&maps_a[2 * q], opA, n_pad, kp_a, bf16, 128));
      GW_TRY(make_map(&maps_a[2 * q + 1], opB, m_pad_a, kp_a, bf16, bn_a));
      TcTask& A = ta[q];
      A = K;
      A.ksteps = (shp_a.used + 15) / 16;
      A.col_tiles = col_tiles_a;
      A.tiles_per_split = tps_a;
      A.gate = lay;
      A.gate_on = 1;
      K.gate = lay;
      K.gate_on = 0;
    }
  }
  if (tasks[0].reuse_ops) {
    float* part = ws.take<float>(static_cast<size_t>(2 * 2 * kSmCount));
    GW_REQUIRE(!ws.overflow, GW_ENOMEM, "workspace too small for the tensor-core softmin");
    tc_refresh_max_kernel<<<kSmCount, 256, 0, st>>>(refresh[0], refresh[1], ntasks, part);
    GW_LAUNCH_CHECK();
    int64_t rows = 0;
    for (int q = 0; q < ntasks; ++q) rows += refresh[q].n + refresh[q].m;
    if (bf16) {
      tc_refresh_multi_kernel<__nv_bfloat16><<<ceil_div(rows, 256), 256, 0, st>>>(
          refresh[0], refresh[1], ntasks, shp, part, kSmCount, lay, shp_a);
    } else {
      tc_refresh_multi_kernel<__half><<<ceil_div(rows, 256), 256, 0, st>>>(
          refresh[0], refresh[1], ntasks, shp, part, kSmCount, lay, shp_a);
    }
    GW_LAUNCH_CHECK();
  }
  if (ntasks == 1) {
    maps[2] = maps[0];
    maps[3] = maps[1];
    tt[1] = tt[0];
    tt[1].blocks = 0;
    maps_a[2] = maps_a[0];
    maps_a[3] = maps_a[1];
    ta[1] = ta[0];
    ta[1].blocks = 0;
  }
  // one pass in the layout the device chose (the other launch returns at once)
  auto pass = [&](bool fast) -> int {
    if (narrow) GW_TRY(run_tc(bf16, fast, kp_a, maps_a, ta[0], ta[1], st));
    if (narrow && !two_launches) return GW_OK;
    return run_tc(bf16, fast, shp.KP, maps, tt[0], tt[1], st);
  };
  if (!all_est) {
    // no usable estimate: one safe pass over every CTA
    tt[0].flags = tt[1].flags = nullptr;
    ta[0].flags = ta[1].flags = nullptr;
    GW_TRY(pass(false));
    return run_combine(tt[0], tt[1], 0, st);
  }
  GW_TRY(pass(true));
  GW_TRY(run_combine(tt[0], tt[1], 1, st));
  GW_TRY(pass(false));
  return run_combine(tt[0], tt[1], 2, st);
}

}  // namespace gw
