// Block product of the Kernel PCA subspace iteration on the tensor cores
// (Section 5 "CNT Embeddings"; Appendix B.2):
//   Z_i = sum_k C(x_i, x_k) P_k,   C(x, x') = c(||x - x'||^2) the CNT cost,
// with C never stored.  Each CTA owns 256 rows i (two M = 128 halves) and one
// split of the 64-point source tiles k:
//   1. the epilogue warps generate C'_ik = s_C c(x_i, x_k) from the point
//      coordinates (translated by x_0 and pre-scaled by a power of two, so
//      that max C' <= 2^14) and split it into f16 hi (C' with its mantissa cut
//      to f16 width, exact) + lo (the remainder, rounded once), written to
//      shared memory in the 128-byte swizzled K-major layout of an MMA A
//      operand; two such tiles alternate, so the CUDA cores fill one while
//      the tensor cores read the other;
//   2. P (each column scaled by a power of two, f16 hi + lo, stored
//      feature-major so that a tile of 64 sources is a K-major B operand,
//      loaded by TMA) enters one MMA of N = 2 RP against [P_hi; P_lo], which
//      leaves C_hi P_hi and C_hi P_lo side by side in TMEM, and one of N = RP
//      that adds C_lo P_hi to the first block;
//   3. after its last tile the CTA adds the two blocks, undoes the scales and
//      writes its split partial in FP32; the partials are summed in a fixed
//      order afterwards (deterministic).
// A wait that gives up makes the CTA write NaN rows, which the
// orthonormalisation that follows reports as an error.
#include <algorithm>

#include "gw_tc_ops.cuh"

namespace gw {

namespace {

constexpr int kLtBM = 256;                   // rows per CTA
constexpr int kLtBN = 64;                    // sources per tile
constexpr int kLtEpiWarps = 16;
constexpr int kLtThreads = 64 + 32 * kLtEpiWarps;
constexpr int kLtMaxStages = 4;
constexpr int kLtCHalf = 128 * 128;          // 128 rows x 64 sources of f16 (hi or lo)
constexpr int kLtCBuf = 4 * kLtCHalf;        // [half][hi, lo]
constexpr int kLtXBytes = 4 * kLtBN * 4;     // source coordinates of a tile, [4][64] FP32
constexpr int kLtSmemMax = 232448;           // opt-in shared memory per block
constexpr float kLtCMax = 16384.0f;          // 2^14
constexpr int kLtMaxSplits = 4;

enum LtCost { kLtSqrt = 0, kLtGauss = 1, kLtGeneric = 2 };

struct LtLayout {
  int64_t rows_pad, cols_pad;
  int row_tiles, col_tiles, splits, tiles_per_split;
  int stage_bytes, stages, smem_bytes;
  uint32_t tmem_cols;
};

struct LtTask {
  tc::WaitCtl wc;
  int64_t n;
  int64_t rows_pad;     // row stride of the coordinate table
  int RP;
  int col_tiles, splits, tiles_per_split, stages, stage_bytes;
  uint32_t tmem_cols;
  float gk;             // Gauss: log2(e) / (2 sigma^2); power p: p / 2
  const float* xt;      // [4][rows_pad] translated, scaled coordinates
  const float* uinv;    // [RP] per-column unscale
  float* Zp;            // [splits][n][RP]
};

LtLayout lt_layout(int64_t n, int RP) {
  LtLayout L;
  L.row_tiles = static_cast<int>(ceil_div(n, kLtBM));
  L.col_tiles = static_cast<int>(ceil_div(n, kLtBN));
  L.rows_pad = static_cast<int64_t>(L.row_tiles) * kLtBM;
  L.cols_pad = static_cast<int64_t>(L.col_tiles) * kLtBN;
  // the split count (at most 4, at least 8 tiles per CTA) that fills whole
  // waves of 152 CTAs best
  int smax = L.col_tiles / 8;
  if (smax > kLtMaxSplits) smax = kLtMaxSplits;
  if (smax < 1) smax = 1;
  int s = 1;
  double best = 0.0;
  for (int c = 1; c <= smax; ++c) {
    const double waves = static_cast<double>(L.row_tiles) * c / kSmCount;
    const double eff = waves / ceil(waves);
    if (eff > best + 1e-3) {
      best = eff;
      s = c;
    }
    if (eff > 0.97) break;
  }
  L.tiles_per_split = static_cast<int>(ceil_div(L.col_tiles, s));
  L.splits = static_cast<int>(ceil_div(L.col_tiles, L.tiles_per_split));
  L.stage_bytes = 2 * RP * 128 + kLtXBytes;
  L.stages = (kLtSmemMax - 2 * kLtCBuf - 2048) / L.stage_bytes;
  if (L.stages > kLtMaxStages) L.stages = kLtMaxStages;
  L.smem_bytes = 2 * kLtCBuf + L.stages * L.stage_bytes + 256 + 1024;
  uint32_t tc = 32;
  while (tc < static_cast<uint32_t>(4 * RP)) tc *= 2;
  L.tmem_cols = tc;
  return L;
}

__device__ __forceinline__ float lt_rsqrt(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float lt_lg2(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// C' from the scaled squared distance (the scale is in the coordinates for
// the power costs and in the 2^14 factor for the Gaussian one); the power
// p = 1 is taken in the kernel as d2 rsqrt(d2), two entries at a time
template <int KIND>
__device__ __forceinline__ float lt_cost(float d2, float gk) {
  if (KIND == kLtGauss) return fmaf(-kLtCMax, ex2(-d2 * gk), kLtCMax);
  if (gk == 1.0f) return d2;
  return d2 > 0.0f ? ex2(gk * lt_lg2(d2)) : 0.0f;
}

// Position of point i in the coordinate table: within each block of 64,
// point 8 c + 4 h + e (c < 8, h < 2, e < 4) sits at 32 h + 4 c + e, so the
// eight lanes of a quarter warp that need points 8 c .. 8 c + 3 (then
// 8 c + 4 .. 8 c + 7) read 128 contiguous bytes.
__host__ __device__ __forceinline__ int64_t lt_pos(int64_t i) {
  const int b = static_cast<int>(i & 63);
  return (i - b) + 32 * ((b >> 2) & 1) + 4 * (b >> 3) + (b & 3);
}

// 8 consecutive 32-bit TMEM columns of this thread's lane
__device__ __forceinline__ void lt_tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                 "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}
__device__ __forceinline__ void lt_tmem_wait(uint32_t (&a)[8], uint32_t (&b)[8]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3]), "+r"(a[4]), "+r"(a[5]),
                 "+r"(a[6]), "+r"(a[7]), "+r"(b[0]), "+r"(b[1]), "+r"(b[2]), "+r"(b[3]),
                 "+r"(b[4]), "+r"(b[5]), "+r"(b[6]), "+r"(b[7])
               :
               : "memory");
}

template <int DIM, int KIND>
__global__ void __launch_bounds__(kLtThreads, 1)
    lift_tc_kernel(const __grid_constant__ CUtensorMap mX, const __grid_constant__ CUtensorMap mQh,
                   const __grid_constant__ CUtensorMap mQl, LtTask T) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* Cs = smem;                    // 2 C tiles
  unsigned char* Ss = smem + 2 * kLtCBuf;      // stages: [P_hi; P_lo] tile, then coordinates
  uint64_t* bars = reinterpret_cast<uint64_t*>(Ss + T.stages * T.stage_bytes);
  uint64_t* full = bars;                       // [stages]
  uint64_t* empty = bars + kLtMaxStages;       // [stages]
  uint64_t* cfull = bars + 2 * kLtMaxStages;   // [2] C tile written (one arrival per warp)
  uint64_t* cempty = cfull + 2;                // [2] C tile read by the MMAs
  uint64_t* wdone = cfull + 4;
  uint64_t* drain = cfull + 5;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  __shared__ int consumed;

  const int RP = T.RP;
  const int S = T.stages;
  const int qbytes = RP * 128;                 // one feature-major tile (hi or lo)
  const int rt = blockIdx.x / T.splits;
  const int sp = blockIdx.x % T.splits;
  const int64_t row0 = static_cast<int64_t>(rt) * kLtBM;
  const int tile0 = sp * T.tiles_per_split;
  const int ntiles = min(T.tiles_per_split, T.col_tiles - tile0);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    abort_flag = 0;
    consumed = 0;
    for (int s = 0; s < S; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&cfull[b], kLtEpiWarps);
      tc::mbar_init(&cempty[b], 1);
    }
    tc::mbar_init(wdone, 1);
    tc::mbar_init(drain, 1);
    tc::fence_mbar_init();
  }
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base, T.tmem_cols);
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
      tc::prefetch_tmap(&mX);
      tc::prefetch_tmap(&mQh);
      tc::prefetch_tmap(&mQl);
      int issued = 0;
      for (int t = 0; t < ntiles; ++t) {
        const int s = t % S;
        if (!tc::mbar_wait(&empty[s], ((t / S) & 1) ^ 1, ab, lim)) break;
        tc::mbar_arrive_expect_tx(&full[s], T.stage_bytes);
        unsigned char* st = Ss + s * T.stage_bytes;
        const int k0 = (tile0 + t) * kLtBN;
        tc::tma_load_2d(st, &mQh, k0, 0, &full[s]);
        tc::tma_load_2d(st + qbytes, &mQl, k0, 0, &full[s]);
        tc::tma_load_2d(st + 2 * qbytes, &mX, k0, 0, &full[s]);
        issued = t + 1;
      }
      if (*ab) {
        // wind down: wait for the copies still in flight before leaving
        const int done = *reinterpret_cast<volatile int*>(&consumed);
        for (int t = done; t < issued; ++t) mbar_drain(&full[t % S], (t / S) & 1);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ------------------------------------------------------- MMA issuer
      const uint32_t id2 = tc::f16_idesc(128, 2 * RP, false);
      const uint32_t id1 = tc::f16_idesc(128, RP, false);
      for (int t = 0; t < ntiles; ++t) {
        const int s = t % S, b = t & 1;
        if (!tc::mbar_wait(&cfull[b], (t >> 1) & 1, ab, lim)) break;
        if (!tc::mbar_wait(&full[s], (t / S) & 1, ab, lim)) break;
        *reinterpret_cast<volatile int*>(&consumed) = t + 1;   // this stage's copies landed
        tc::tc_fence_after();
        const unsigned char* Cb = Cs + b * kLtCBuf;
        const uint32_t qaddr = tc::smem_u32(Ss + s * T.stage_bytes);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const uint32_t acc = tbase + static_cast<uint32_t>(h * 2 * RP);
          const uint32_t ahi = tc::smem_u32(Cb + (2 * h) * kLtCHalf);
          const uint32_t alo = tc::smem_u32(Cb + (2 * h + 1) * kLtCHalf);
#pragma unroll
          for (int ks = 0; ks < kLtBN / 16; ++ks) {
            tc::mma_f16(acc, tc::sw128_desc(ahi + ks * 32), tc::sw128_desc(qaddr + ks * 32), id2,
                        (t > 0 || ks > 0) ? 1u : 0u);
            tc::mma_f16(acc, tc::sw128_desc(alo + ks * 32), tc::sw128_desc(qaddr + ks * 32), id1,
                        1u);
          }
        }
        tc::mma_commit(&cempty[b]);
        tc::mma_commit(&empty[s]);
      }
      tc::mma_commit(wdone);
      // every MMA issued above has finished before TMEM is freed
      tc::mma_commit(drain);
      mbar_drain(drain, 0);
    }
  } else {
    // ------------------------------------------------------------ epilogue
    // C tile: warp e covers rows 16 e .. 16 e + 15 of the 256; lane = (row
    // group rg of 4 rows, source chunk cc of 8), so a quarter warp stores the
    // 8 chunks of one row (distinct banks under the swizzle)
    const int e = warp - 2;
    const int cc = lane & 7, rg = lane >> 3;
    const int h = e >> 3;
    const int rbase = (e & 7) * 16 + rg * 4;
    uint64_t nxi[4][DIM];   // (-x_i, -x_i) per row and coordinate
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t i = row0 + h * 128 + rbase + j;
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        const float v = -T.xt[c * T.rows_pad + lt_pos(i)];
        nxi[j][c] = tc::pack2(v, v);
      }
    }
    const uint64_t zero2 = tc::pack2(0.0f, 0.0f);
    const uint64_t tiny2 = tc::pack2(7.888609052210118e-31f, 7.888609052210118e-31f);   // 2^-100
    bool ok = true;
    for (int t = 0; t < ntiles; ++t) {
      const int s = t % S, b = t & 1;
      bool got = tc::mbar_wait(&full[s], (t / S) & 1, ab, lim);
      if (got && t >= 2) got = tc::mbar_wait(&cempty[b], ((t >> 1) & 1) ^ 1, ab, lim);
      if (!__all_sync(0xffffffffu, got)) {
        ok = false;
        break;
      }
      const float* xs = reinterpret_cast<const float*>(Ss + s * T.stage_bytes + 2 * qbytes);
      float xk[DIM][8];
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        const float4 a = *reinterpret_cast<const float4*>(xs + c * kLtBN + cc * 4);
        const float4 a2 = *reinterpret_cast<const float4*>(xs + c * kLtBN + 32 + cc * 4);
        xk[c][0] = a.x; xk[c][1] = a.y; xk[c][2] = a.z; xk[c][3] = a.w;
        xk[c][4] = a2.x; xk[c][5] = a2.y; xk[c][6] = a2.z; xk[c][7] = a2.w;
      }
      unsigned char* Ch = Cs + b * kLtCBuf + (2 * h) * kLtCHalf;
      unsigned char* Cl = Ch + kLtCHalf;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        uint32_t hv[4], lv[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          uint64_t acc = KIND == kLtSqrt ? tiny2 : zero2;
#pragma unroll
          for (int c = 0; c < DIM; ++c) {
            const uint64_t dx = tc::add2(tc::pack2(xk[c][2 * p], xk[c][2 * p + 1]), nxi[j][c]);
            acc = tc::fma2(dx, dx, acc);
          }
          float c0, c1;
          if (KIND == kLtSqrt) {
            // sqrt(d2) = d2 rsqrt(d2), with d2 >= 2^-100 (the accumulator's
            // start) so that the diagonal stays finite (2^-50 instead of 0)
            float d0, d1;
            tc::unpack2(acc, d0, d1);
            tc::unpack2(tc::fma2(acc, tc::pack2(lt_rsqrt(d0), lt_rsqrt(d1)), zero2), c0, c1);
          } else {
            float d0, d1;
            tc::unpack2(acc, d0, d1);
            c0 = lt_cost<KIND>(d0, T.gk);
            c1 = lt_cost<KIND>(d1, T.gk);
          }
          const float h0 = __uint_as_float(__float_as_uint(c0) & 0xFFFFE000u);
          const float h1 = __uint_as_float(__float_as_uint(c1) & 0xFFFFE000u);
          const __half2 hh = __floats2half2_rn(h0, h1);
          const __half2 ll = __floats2half2_rn(c0 - h0, c1 - h1);
          hv[p] = *reinterpret_cast<const uint32_t*>(&hh);
          lv[p] = *reinterpret_cast<const uint32_t*>(&ll);
        }
        const uint32_t r = static_cast<uint32_t>(rbase + j);
        const uint32_t off = (r >> 3) * 1024 + (r & 7) * 128 + ((cc ^ (r & 7)) << 4);
        asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(tc::smem_u32(Ch + off)),
                     "r"(hv[0]), "r"(hv[1]), "r"(hv[2]), "r"(hv[3])
                     : "memory");
        asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(tc::smem_u32(Cl + off)),
                     "r"(lv[0]), "r"(lv[1]), "r"(lv[2]), "r"(lv[3])
                     : "memory");
      }
      // generic-proxy writes become visible to the tensor core's async proxy
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&cfull[b]);
    }
    // partial rows: warp -> (TMEM lane quarter q = warp % 4, half hh, column
    // half ch); thread -> one row
    int fin = (ok && ntiles > 0) ? 1 : 0;
    if (fin && lane == 0) fin = tc::mbar_wait(wdone, 0, ab, lim) ? 1 : 0;
    fin = __shfl_sync(0xffffffffu, fin, 0);
    const bool good = __all_sync(0xffffffffu, fin != 0 && *ab == 0);
    const int q = warp & 3, g = e >> 2, hh = g & 1, ch = g >> 1;
    const int64_t i = row0 + hh * 128 + q * 32 + lane;
    const int half = RP / 2;
    float* out = T.Zp + (static_cast<int64_t>(sp) * T.n + i) * RP;
    tc::tc_fence_after();
    for (int c0 = ch * half; c0 < (ch + 1) * half; c0 += 8) {
      uint32_t a[8] = {0, 0, 0, 0, 0, 0, 0, 0}, b2[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      if (good) {
        const uint32_t ta = tbase + (static_cast<uint32_t>(q * 32) << 16) +
                            static_cast<uint32_t>(hh * 2 * RP + c0);
        lt_tmem_ld8(ta, a);
        lt_tmem_ld8(ta + static_cast<uint32_t>(RP), b2);
        lt_tmem_wait(a, b2);
      }
      if (i < T.n) {
        float v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k)
          v[k] = good ? (__uint_as_float(a[k]) + __uint_as_float(b2[k])) * T.uinv[c0 + k]
                      : __int_as_float(0x7fc00000);
        float4* o4 = reinterpret_cast<float4*>(out + c0);
        o4[0] = make_float4(v[0], v[1], v[2], v[3]);
        o4[1] = make_float4(v[4], v[5], v[6], v[7]);
      }
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0) tc::note_gave_up(T.wc, ab);
  if (warp == 0) {
    __syncwarp();
    tc::tc_fence_after();
    tc::tmem_dealloc(tbase, T.tmem_cols);
  }
}

// r2 = max_i ||x_i - x_0||^2 (non-negative floats order like their bits)
__global__ void lt_radius_kernel(const float* x, int64_t n, int d, unsigned* r2) {
  float v = 0.0f;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    float s = 0.0f;
    for (int c = 0; c < d; ++c) {
      const float df = x[i * d + c] - x[c];
      s = fmaf(df, df, s);
    }
    v = fmaxf(v, s);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) atomicMax(r2, __float_as_uint(v));
}

// scal[0] = s_x (coordinate scale), scal[1] = 1 / s_C (cost unscale).
// Power p: s_x = 2^e with (s_x^2 d2max)^(p/2) <= 2^14 for d2max = 4 r2 (a
// bound on every squared distance), and s_x^2 d2max far from FP32 overflow;
// s_C = s_x^p.  Gauss: s_x = 1, s_C = 2^13 (the cost is at most 2).
__global__ void lt_scale_kernel(const unsigned* r2, int gauss, double p, float* scal) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (gauss) {
    scal[0] = 1.0f;
    scal[1] = 1.0f / 8192.0f;
    return;
  }
  const double d2max = 4.0 * static_cast<double>(__uint_as_float(*r2));
  int e = 0;
  if (d2max > 0.0 && isfinite(d2max)) {
    const double l = log2(d2max);
    double ed = floor(14.0 / p - 0.5 * l);
    const double ecap = floor(0.5 * (120.0 - l));
    if (ed > ecap) ed = ecap;
    if (ed > 100.0) ed = 100.0;
    if (ed < -100.0) ed = -100.0;
    e = static_cast<int>(ed);
  }
  scal[0] = static_cast<float>(ldexp(1.0, e));
  scal[1] = static_cast<float>(exp2(-p * e));
}

// xt[c][lt_pos(i)] = (x_ic - x_0c) s_x for c < d and i < n; 0 elsewhere
__global__ void lt_table_kernel(const float* x, int64_t n, int d, int64_t rows_pad,
                                const float* scal, float* xt) {
  const int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= 4 * rows_pad) return;
  const int c = static_cast<int>(q / rows_pad);
  const int64_t i = q % rows_pad;
  xt[c * rows_pad + lt_pos(i)] = (i < n && c < d) ? (x[i * d + c] - x[c]) * scal[0] : 0.0f;
}

// qmax[r] = max_k |P_kr|  (blockDim.x == RP)
__global__ void lt_qmax_kernel(const float* P, int64_t n, int RP, unsigned* qmax) {
  const int r = threadIdx.x;
  float v = 0.0f;
  for (int64_t k = blockIdx.x; k < n; k += gridDim.x) v = fmaxf(v, fabsf(P[k * RP + r]));
  atomicMax(&qmax[r], __float_as_uint(v));
}

// 2^(14 - e) for max = m 2^e (m in [0.5, 1)): max times it lies in [2^13, 2^14)
__device__ __forceinline__ float lt_qscale(unsigned bits) {
  const float mx = __uint_as_float(bits);
  if (!(mx > 0.0f) || !isfinite(mx)) return 1.0f;
  int e;
  frexpf(mx, &e);
  return ldexpf(1.0f, 14 - e);
}

// Ph / Pl [RP][cols_pad] = P^T scaled per column, f16 hi + lo (64 sources
// per block, transposed through shared memory); uinv[r] = 1 / (scale_r s_C)
__global__ void lt_prep_kernel(const float* P, int64_t n, int RP, int64_t cols_pad,
                               const unsigned* qmax, const float* scal, __half* Ph, __half* Pl,
                               float* uinv) {
  __shared__ float tile[kLtBN][129];
  const int64_t k0 = static_cast<int64_t>(blockIdx.x) * kLtBN;
  for (int idx = threadIdx.x; idx < kLtBN * RP; idx += blockDim.x) {
    const int kk = idx / RP, r = idx % RP;
    tile[kk][r] = k0 + kk < n ? P[(k0 + kk) * RP + r] : 0.0f;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < kLtBN * RP; idx += blockDim.x) {
    const int r = idx / kLtBN, kk = idx % kLtBN;
    const float u = tile[kk][r] * lt_qscale(qmax[r]);
    const __half hi = __float2half_rn(u);
    Ph[r * cols_pad + k0 + kk] = hi;
    Pl[r * cols_pad + k0 + kk] = __float2half_rn(u - __half2float(hi));
  }
  if (blockIdx.x == 0)
    for (int r = threadIdx.x; r < RP; r += blockDim.x) uinv[r] = scal[1] / lt_qscale(qmax[r]);
}

int lt_encode(CUtensorMap* map, CUtensorMapDataType type, void* ptr, int64_t inner, int rows,
              int elem, int box_rows, CUtensorMapSwizzle swz) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  GW_REQUIRE(enc != nullptr, GW_ECUDA, "cuTensorMapEncodeTiled is not available");
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(inner), static_cast<cuuint64_t>(rows)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(inner) * elem};
  cuuint32_t box[2] = {static_cast<cuuint32_t>(kLtBN), static_cast<cuuint32_t>(box_rows)};
  cuuint32_t es[2] = {1, 1};
  CUresult r = enc(map, type, 2, ptr, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  GW_REQUIRE(r == CUDA_SUCCESS, GW_ECUDA, "cuTensorMapEncodeTiled failed (%d)", static_cast<int>(r));
  return GW_OK;
}

template <int DIM, int KIND>
int launch_lt(const CUtensorMap* maps, const LtTask& T, const LtLayout& L, cudaStream_t st) {
  auto kern = lift_tc_kernel<DIM, KIND>;
  // set once, at the largest size any RP needs: launches for different RP
  // may run concurrently on several host threads, and a per-launch setting
  // would let one thread lower the limit under another's launch
  static std::once_flag once;
  static cudaError_t attr_rc = cudaSuccess;
  std::call_once(once, [&] {
    int mx = 0;
    for (int rp : {16, 32, 48, 64, 80, 96, 128}) mx = std::max(mx, lt_layout(kLtBN, rp).smem_bytes);
    attr_rc = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  });
  GW_CUDA_TRY(attr_rc);
  kern<<<L.row_tiles * L.splits, kLtThreads, L.smem_bytes, st>>>(maps[0], maps[1], maps[2], T);
  GW_LAUNCH_CHECK();
  return GW_OK;
}

}  // namespace

LiftTcBufs carve_lift_tc(Carver& c, int64_t n, int RP) {
  const LtLayout L = lt_layout(n, RP);
  LiftTcBufs B;
  B.splits = L.splits;
  B.xt = c.take<float>(static_cast<size_t>(4) * L.rows_pad);
  B.Ph = c.take<uint16_t>(static_cast<size_t>(RP) * L.cols_pad);
  B.Pl = c.take<uint16_t>(static_cast<size_t>(RP) * L.cols_pad);
  B.qmax = c.take<unsigned>(128);
  B.uinv = c.take<float>(128);
  B.scal = c.take<float>(4);
  B.r2 = c.take<unsigned>(4);
  return B;
}

int lift_tc_prepare(const float* x, int64_t n, int d, int kind, float param, int RP,
                    LiftTcBufs& B, cudaStream_t st) {
  const LtLayout L = lt_layout(n, RP);
  GW_CUDA_TRY(cudaMemsetAsync(B.r2, 0, sizeof(unsigned), st));
  lt_radius_kernel<<<kSmCount, 256, 0, st>>>(x, n, d, B.r2);
  GW_LAUNCH_CHECK();
  const double p = kind == GW_PEN_POWER ? static_cast<double>(param) : 2.0;
  lt_scale_kernel<<<1, 32, 0, st>>>(B.r2, kind == GW_PEN_GAUSS ? 1 : 0, p, B.scal);
  GW_LAUNCH_CHECK();
  lt_table_kernel<<<ceil_div(4 * L.rows_pad, 256), 256, 0, st>>>(x, n, d, L.rows_pad, B.scal, B.xt);
  GW_LAUNCH_CHECK();
  return GW_OK;
}

int lift_tc_matvec(const float* P, int64_t n, int d, int kind, float param, int RP,
                   LiftTcBufs& B, float* Zp, cudaStream_t st) {
  const LtLayout L = lt_layout(n, RP);
  GW_CUDA_TRY(cudaMemsetAsync(B.qmax, 0, sizeof(unsigned) * RP, st));
  lt_qmax_kernel<<<2 * kSmCount, RP, 0, st>>>(P, n, RP, B.qmax);
  GW_LAUNCH_CHECK();
  lt_prep_kernel<<<L.col_tiles, 256, 0, st>>>(P, n, RP, L.cols_pad, B.qmax, B.scal,
                                              reinterpret_cast<__half*>(B.Ph),
                                              reinterpret_cast<__half*>(B.Pl), B.uinv);
  GW_LAUNCH_CHECK();
  CUtensorMap maps[3];
  GW_TRY(lt_encode(&maps[0], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, B.xt, L.rows_pad, 4, 4, 4,
                   CU_TENSOR_MAP_SWIZZLE_NONE));
  GW_TRY(lt_encode(&maps[1], CU_TENSOR_MAP_DATA_TYPE_FLOAT16, B.Ph, L.cols_pad, RP, 2, RP,
                   CU_TENSOR_MAP_SWIZZLE_128B));
  GW_TRY(lt_encode(&maps[2], CU_TENSOR_MAP_DATA_TYPE_FLOAT16, B.Pl, L.cols_pad, RP, 2, RP,
                   CU_TENSOR_MAP_SWIZZLE_128B));
  LtTask T;
  T.n = n;
  T.rows_pad = L.rows_pad;
  T.RP = RP;
  T.col_tiles = L.col_tiles;
  T.splits = L.splits;
  T.tiles_per_split = L.tiles_per_split;
  T.stages = L.stages;
  T.stage_bytes = L.stage_bytes;
  T.tmem_cols = L.tmem_cols;
  T.gk = kind == GW_PEN_GAUSS ? kLog2e / (2.0f * param * param)
                              : 0.5f * (kind == GW_PEN_POWER ? param : 2.0f);
  T.xt = B.xt;
  T.uinv = B.uinv;
  T.Zp = Zp;
  T.wc = wait_ctl();
  const int cost = kind == GW_PEN_GAUSS ? kLtGauss
                   : (kind == GW_PEN_POWER && param == 1.0f) ? kLtSqrt
                                                             : kLtGeneric;
  if (d == 4) {
    switch (cost) {
      case kLtSqrt: return launch_lt<4, kLtSqrt>(maps, T, L, st);
      case kLtGauss: return launch_lt<4, kLtGauss>(maps, T, L, st);
      default: return launch_lt<4, kLtGeneric>(maps, T, L, st);
    }
  }
  switch (cost) {
    case kLtSqrt: return launch_lt<3, kLtSqrt>(maps, T, L, st);
    case kLtGauss: return launch_lt<3, kLtGauss>(maps, T, L, st);
    default: return launch_lt<3, kLtGeneric>(maps, T, L, st);
  }
}

}  // namespace gw
