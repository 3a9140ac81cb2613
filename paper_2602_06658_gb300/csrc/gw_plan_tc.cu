// Plan-weighted column reduction on the tensor cores:
//   W_j = sum_i pi_ij [X_i, s_i, 1],   pi_ij = a_i b_j exp((f_i + g_j - c_ij) / eps),
// the cross-covariance step of Algorithm 1 (Xtilde, Gamma_{t+1} = sum_j W_j Y_j^T)
// with both contractions as tcgen05 MMAs, like an attention forward pass:
//   1. exponent: the column-softmin operands (targets j as rows, sources i as
//      columns, shift estimate g, shift bias 12) give, per 128 x 64 tile,
//      out_ji = log2(pi_ij / b_j) + 12 in TMEM (the same 16-bit split product
//      as the softmin);
//   2. the epilogue warps form q = exp2(out) = 2^12 pi_ij / b_j and split it
//      into f16 hi (q with its mantissa cut to f16 width, exact) + lo (the
//      exact remainder, rounded), written to shared memory in the 128-byte
//      swizzled K-major layout of an MMA A operand;
//   3. W accumulates in TMEM as q_hi U_hi + q_hi U_lo + q_lo U_hi, with
//      U = [X, s, 1] (per feature scaled by a power of two, f16 hi + lo,
//      stored feature-major so its tiles are K-major B operands).
// Each CTA owns 256 targets (two M = 128 halves) and one split of the source
// tiles; the split partials go to Wp[split][j][D + 2] in FP32 and are reduced
// in a fixed order (deterministic).  For the energy's KL term the same pass
// also gives, per split and target, A_j = sum_i pi_ij log2(pi_ij / b_j) (the
// epilogue accumulates q (out - 12) beside the exponentials) and
// B_j = sum_i pi_ij log a_i (a fourth U column, log a): KL = sum_j ln2 A_j - B_j,
// a sum of plan entries times their own small log-ratios, with no large
// potentials cancelling.  A q that does not fit f16 (an estimate
// far from the potential) or a wait that gives up sets *flag, and the FP32
// kernel then recomputes every partial (the launch that follows reads it).
#include "gw_tc_ops.cuh"

namespace gw {

namespace {

constexpr int kPlanBM = 256;
constexpr int kPlanBN = 64;
constexpr int kPlanEpiWarps = 16;
constexpr int kPlanThreads = 64 + 32 * kPlanEpiWarps;
constexpr float kPlanShiftBias = 12.0f;    // out = log2(2^12 pi / b)
constexpr float kPlanQScale = 4096.0f;     // 2^12
constexpr uint32_t kHalfMaxBits = 0x477FE000u;   // 65504.0f: larger q (or inf / NaN) do not fit
constexpr uint32_t kPlanWCol = 256;        // W accumulators after 2 buffers x 2 halves x 64

template <int KP, int S, int NW>
struct PlanSmem {
  static constexpr int KB = KP / 64;
  static constexpr int kABytes = 2 * KB * 16384;      // 256 target rows
  static constexpr int kBBlock = kPlanBN * 128;       // 64 source rows x one 64-wide K block
  static constexpr int kBBytes = KB * kBBlock;
  static constexpr int kUBytes = NW * 128;            // NW feature rows x 64 sources (hi or lo)
  static constexpr int kStageBytes = kBBytes + 2 * kUBytes;
  static constexpr int kPBytes = 128 * 128;           // 128 rows x 64 f16 (one half, hi or lo)
  static constexpr int kPOff = kABytes + S * kStageBytes;
  static constexpr int kBarOff = kPOff + 4 * kPBytes;
  static constexpr int kXeOff = kBarOff + 256;        // [256] floats: column-half merge
  static constexpr int kBytes = kXeOff + 1024 + 1024; // + alignment slack of the base
};

struct PlanTask {
  tc::WaitCtl wc;
  int64_t rows;      // targets j
  int ksteps;
  int col_tiles;     // source tiles of 64
  int splits;
  int tiles_per_split;
  int D;
  const float* b;    // target weights
  const float* uinv; // per W column: c_d / 2^12
  float* Wp;         // [splits][rows][D + 2]
  float* Ep;         // [splits][rows][2]: A_j, B_j of the KL term (or null)
  int* flag;
  int k8;            // FP8: leading K-steps of E4M3 features
  const float* fsA;  // FP8: power-of-two scale per 128 targets
  const float* fsB;  // FP8: the same per 128 sources (two source tiles)
  float alpha8;      // FP8: 16 log2(e) / eps, applied in the epilogue
};

template <int KP, int S, int NW, bool BF16, bool F8>
__global__ void __launch_bounds__(kPlanThreads, 1)
    plan_tc_kernel(const __grid_constant__ CUtensorMap mA, const __grid_constant__ CUtensorMap mB,
                   const __grid_constant__ CUtensorMap mUh, const __grid_constant__ CUtensorMap mUl,
                   PlanTask T) {
  using L = PlanSmem<KP, S, NW>;
  constexpr int KB = L::KB;
  constexpr uint32_t kTmemCols = 512;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* As = smem;
  unsigned char* Bs = smem + L::kABytes;
  unsigned char* Ps = smem + L::kPOff;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::kBarOff);
  uint64_t* full = bars;                // [S]
  uint64_t* empty = bars + S;           // [S]
  uint64_t* tfull = bars + 2 * S;       // [2]
  uint64_t* tempty = bars + 2 * S + 2;  // [2]
  uint64_t* pfull = bars + 2 * S + 4;
  uint64_t* pempty = bars + 2 * S + 5;
  uint64_t* afull = bars + 2 * S + 6;
  uint64_t* wdone = bars + 2 * S + 7;
  uint64_t* drain = bars + 2 * S + 8;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  __shared__ int consumed;

  const int rt = blockIdx.x / T.splits;
  const int sp = blockIdx.x % T.splits;
  const int row0 = rt * kPlanBM;
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
      tc::mbar_init(&tfull[b], 1);
      tc::mbar_init(&tempty[b], kPlanEpiWarps);
    }
    tc::mbar_init(pfull, kPlanEpiWarps);
    tc::mbar_init(pempty, 1);
    tc::mbar_init(afull, 1);
    tc::mbar_init(wdone, 1);
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
      tc::prefetch_tmap(&mA);
      tc::prefetch_tmap(&mB);
      tc::prefetch_tmap(&mUh);
      tc::prefetch_tmap(&mUl);
      tc::mbar_arrive_expect_tx(afull, L::kABytes);
      for (int h = 0; h < 2; ++h)
        for (int kb = 0; kb < KB; ++kb)
          tc::tma_load_2d(As + (h * KB + kb) * 16384, &mA, kb * 64, row0 + h * 128, afull);
      int issued = 0;
      for (int t = 0; t < ntiles; ++t) {
        const int s = t % S;
        if (!tc::mbar_wait(&empty[s], ((t / S) & 1) ^ 1, ab, lim)) break;
        tc::mbar_arrive_expect_tx(&full[s], L::kStageBytes);
        unsigned char* st = Bs + s * L::kStageBytes;
        const int c0 = (tile0 + t) * kPlanBN;
        for (int kb = 0; kb < KB; ++kb) tc::tma_load_2d(st + kb * L::kBBlock, &mB, kb * 64, c0, &full[s]);
        tc::tma_load_2d(st + L::kBBytes, &mUh, c0, 0, &full[s]);
        tc::tma_load_2d(st + L::kBBytes + L::kUBytes, &mUl, c0, 0, &full[s]);
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
      const uint32_t idesc = tc::f16_idesc(128, kPlanBN, BF16);
      const uint32_t idesc2 = tc::f16_idesc(128, NW, false);
      constexpr uint32_t idesc8 = tc::f16_idesc(128, kPlanBN, false);   // E4M3 x E4M3
      const int k8 = F8 ? T.k8 : 0;
      const int nks = T.ksteps;
      bool ok = tc::mbar_wait(afull, 0, ab, lim);
      // exponent tile t into TMEM buffer t & 1
      auto issue_e = [&](int t) -> bool {
        const int s = t % S, b = t & 1;
        if (!tc::mbar_wait(&tempty[b], ((t >> 1) & 1) ^ 1, ab, lim)) return false;
        if (!tc::mbar_wait(&full[s], (t / S) & 1, ab, lim)) return false;
        *reinterpret_cast<volatile int*>(&consumed) = t + 1;   // this stage's copies landed
        tc::tc_fence_after();
        const unsigned char* Bst = Bs + s * L::kStageBytes;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
#pragma unroll
          for (int ks = 0; ks < KP / 16; ++ks) {
            if (ks >= nks) break;   // the rest of the operand row is zero padding
            const uint32_t aaddr = tc::smem_u32(As + (h * KB + ks / 4) * 16384 + (ks % 4) * 32);
            const uint32_t baddr = tc::smem_u32(Bst + (ks / 4) * L::kBBlock + (ks % 4) * 32);
            if (F8 && ks < k8)
              tc::mma_f8(tbase + (b * 2 + h) * kPlanBN, tc::sw128_desc(aaddr),
                         tc::sw128_desc(baddr), idesc8, ks > 0 ? 1u : 0u);
            else
              tc::mma_f16(tbase + (b * 2 + h) * kPlanBN, tc::sw128_desc(aaddr),
                          tc::sw128_desc(baddr), idesc, ks > 0 ? 1u : 0u);
          }
        }
        tc::mma_commit(&tfull[b]);
        return true;
      };
      // W += q_hi U_hi + q_hi U_lo + q_lo U_hi for tile t (P written by the epilogue)
      auto issue_w = [&](int t) -> bool {
        const int s = t % S;
        if (!tc::mbar_wait(pfull, t & 1, ab, lim)) return false;
        tc::tc_fence_after();
        const unsigned char* Ust = Bs + s * L::kStageBytes + L::kBBytes;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
#pragma unroll
          for (int prod = 0; prod < 3; ++prod) {
            const unsigned char* Pa = Ps + (h * 2 + (prod == 2 ? 1 : 0)) * L::kPBytes;
            const unsigned char* Ub = Ust + (prod == 1 ? 1 : 0) * L::kUBytes;
#pragma unroll
            for (int ks = 0; ks < kPlanBN / 16; ++ks) {
              tc::mma_f16(tbase + kPlanWCol + h * NW, tc::sw128_desc(tc::smem_u32(Pa + ks * 32)),
                          tc::sw128_desc(tc::smem_u32(Ub + ks * 32)), idesc2,
                          (t > 0 || prod > 0 || ks > 0) ? 1u : 0u);
            }
          }
        }
        tc::mma_commit(pempty);
        tc::mma_commit(&empty[s]);
        return true;
      };
      for (int t = 0; ok && t < ntiles; ++t) {
        ok = issue_e(t);
        if (ok && t > 0) ok = issue_w(t - 1);
      }
      if (ok && ntiles > 0) ok = issue_w(ntiles - 1);
      tc::mma_commit(wdone);
      // every MMA issued above has finished before TMEM is freed
      tc::mma_commit(drain);
      mbar_drain(drain, 0);
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int e = warp - 2;
    const int g = e >> 2;
    const int h = g & 1;    // row half
    const int ch = g >> 1;  // column half of the 64-column tile
    const int q = warp & 3; // TMEM lane quarter
    const int rloc = q * 32 + lane;
    bool ok = true;
    uint32_t qbits = 0;
    float ent = 0.0f;   // sum over this warp's sources of q (out - 12)
    unsigned char* Ph = Ps + (h * 2 + 0) * L::kPBytes;
    unsigned char* Pl = Ps + (h * 2 + 1) * L::kPBytes;
    const uint32_t prow = static_cast<uint32_t>((rloc >> 3) * 1024 + (rloc & 7) * 128);
    // FP8: alpha / the scale of this half's 128 targets (n_pad covered)
    const float a_over = F8 ? T.alpha8 / T.fsA[(row0 >> 7) + h] : 1.0f;
    for (int t = 0; t < ntiles; ++t) {
      const int b = t & 1;
      int got = 0;
      if (lane == 0) got = tc::mbar_wait(&tfull[b], (t >> 1) & 1, ab, lim) ? 1 : 0;
      got = __shfl_sync(0xffffffffu, got, 0);
      if (!got) {
        ok = false;
        break;
      }
      tc::tc_fence_after();
      uint32_t r[32];
      tc::tmem_ld32_issue(tbase + (static_cast<uint32_t>(q * 32) << 16) + (b * 2 + h) * kPlanBN +
                              ch * 32,
                          r);
      tc::tmem_ld_wait(r);
      tc::tc_fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&tempty[b]);
      if constexpr (F8) unscale(r, a_over / T.fsB[(tile0 + t) >> 1]);
      // q = 2^12 pi_ij / b_j as f16 hi + lo, packed in pairs along the sources:
      // hi keeps the top 11 significant bits (exact in f16 for q >= 2^-14),
      // lo = q - hi is exact in FP32 and rounded once
      uint32_t hp[16], lp[16];
#pragma unroll
      for (int k = 0; k < 32; k += 2) {
        const float q0 = ex2(__uint_as_float(r[k]));
        const float q1 = ex2(__uint_as_float(r[k + 1]));
        ent = fmaf(q0, __uint_as_float(r[k]) - kPlanShiftBias, ent);
        ent = fmaf(q1, __uint_as_float(r[k + 1]) - kPlanShiftBias, ent);
        const uint32_t b0 = __float_as_uint(q0), b1 = __float_as_uint(q1);
        qbits = max(qbits, max(b0, b1));   // q > 0: bit order = value order (inf, NaN above)
        const float h0 = __uint_as_float(b0 & 0xFFFFE000u);
        const float h1 = __uint_as_float(b1 & 0xFFFFE000u);
        const __half2 hh = __floats2half2_rn(h0, h1);
        const __half2 ll = __floats2half2_rn(q0 - h0, q1 - h1);
        hp[k / 2] = *reinterpret_cast<const uint32_t*>(&hh);
        lp[k / 2] = *reinterpret_cast<const uint32_t*>(&ll);
      }
      // the P tile is free once the W MMAs of the previous tile are done
      if (t > 0) {
        if (lane == 0) got = tc::mbar_wait(pempty, (t - 1) & 1, ab, lim) ? 1 : 0;
        got = __shfl_sync(0xffffffffu, got, 0);
        if (!got) {
          ok = false;
          break;
        }
      }
#pragma unroll
      for (int c4 = 0; c4 < 4; ++c4) {
        const uint32_t c = static_cast<uint32_t>(ch * 4 + c4);
        const uint32_t off = prow + ((c ^ static_cast<uint32_t>(rloc & 7)) << 4);
        asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(tc::smem_u32(Ph + off)),
                     "r"(hp[4 * c4]), "r"(hp[4 * c4 + 1]), "r"(hp[4 * c4 + 2]), "r"(hp[4 * c4 + 3])
                     : "memory");
        asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(tc::smem_u32(Pl + off)),
                     "r"(lp[4 * c4]), "r"(lp[4 * c4 + 1]), "r"(lp[4 * c4 + 2]), "r"(lp[4 * c4 + 3])
                     : "memory");
      }
      // generic-proxy writes become visible to the tensor core's async proxy
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(pfull);
    }
    // the two column halves of a target row merge their q (out - 12) sums
    // (named barrier of the epilogue warps only; every one of them gets here)
    {
      float* xe = reinterpret_cast<float*>(smem + L::kXeOff);
      const int slot = h * 128 + rloc;
      if (ch == 1) xe[slot] = ent;
      asm volatile("bar.sync 1, %0;" ::"r"(32 * kPlanEpiWarps) : "memory");
      if (ch == 0) ent += xe[slot];
    }
    // final W rows: one warp per (half, lane quarter) reads its 32 rows
    int got = 1;
    if (ok) {
      if (lane == 0) got = tc::mbar_wait(wdone, 0, ab, lim) ? 1 : 0;
      got = __shfl_sync(0xffffffffu, got, 0);
      ok = got != 0;
    }
    int go = (ok && ntiles > 0 && !*ab) ? 1 : 0;
    go = __shfl_sync(0xffffffffu, go, 0);   // tcgen05.ld needs the whole warp
    if (go) {
      tc::tc_fence_after();
      if (ch == 0) {
        // the W row in chunks of 32 columns (the last chunk may run past NW
        // into columns this row does not use; TMEM holds 512)
        const uint32_t wa = tbase + (static_cast<uint32_t>(q * 32) << 16) + kPlanWCol + h * NW;
        const int64_t j = static_cast<int64_t>(row0) + h * 128 + rloc;
        const bool in = j < T.rows;
        const float bj = in ? T.b[j] : 0.0f;
        float* out = T.Wp + (static_cast<int64_t>(sp) * T.rows + (in ? j : 0)) * (T.D + 2);
        float* e2 = T.Ep ? T.Ep + (static_cast<int64_t>(sp) * T.rows + (in ? j : 0)) * 2 : nullptr;
#pragma unroll 1
        for (int c0 = 0; c0 < NW; c0 += 32) {
          uint32_t w[32];
          tc::tmem_ld32_issue(wa + c0, w);
          tc::tmem_ld_wait(w);
          if (!in) continue;
#pragma unroll
          for (int k = 0; k < 32; ++k) {
            const int d = c0 + k;
            const float v = __uint_as_float(w[k]);
            if (d < T.D + 2) {
              out[d] = v * bj * T.uinv[d];
            } else if (d == T.D + 2 && T.Ep != nullptr) {   // the log a column, and the KL sum
              e2[0] = ent * bj * (1.0f / kPlanQScale);
              e2[1] = v * bj * T.uinv[d];
            }
          }
        }
      }
    }
    const bool bad = qbits >= kHalfMaxBits;
    const bool fail = __any_sync(0xffffffffu, bad || !ok || go == 0) != 0;
    if (fail && lane == 0) atomicExch(T.flag, 1);
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

// per W column d (X_d, then s, then 1, then log a): max |U_id| -> umax[d]
// (the constant column D + 1 needs none)
__global__ void u_absmax_kernel(const float* X, const float* s, const float* loga, int64_t n, int D,
                                unsigned* umax) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int d = 0; d < D + 3; ++d) {
    if (d == D + 1) continue;
    float v = 0.f;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride)
      v = fmaxf(v, fabsf(d < D ? X[i * D + d] : (d == D ? s[i] : (isfinite(loga[i]) ? loga[i] : 0.0f))));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) atomicMax(&umax[d], __float_as_uint(v));
  }
}

// Uh / Ul [NW][n_pad]: U_id / c_d split into f16 hi + lo; uinv[d] = c_d / 2^12;
// U = [X, s, 1, log a]
__global__ void u_prep_kernel(const float* X, const float* s, const float* loga, int64_t n,
                              int64_t n_pad, int D, int NW, const unsigned* umax, __half* Uh,
                              __half* Ul, float* uinv) {
  const int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= static_cast<int64_t>(NW) * n_pad) return;
  const int d = static_cast<int>(q / n_pad);
  const int64_t i = q % n_pad;
  float c = 1.0f;
  if (d <= D || d == D + 2) c = pow2_scale(__uint_as_float(umax[d]));
  float u = 0.0f;
  if (i < n && d < D + 3)
    u = (d < D ? X[i * D + d]
               : (d == D ? s[i] : (d == D + 1 ? 1.0f : (isfinite(loga[i]) ? loga[i] : 0.0f)))) / c;
  const __half hi = __float2half_rn(u);
  Uh[q] = hi;
  Ul[q] = __float2half_rn(u - __half2float(hi));
  if (i == 0) uinv[d] = c / kPlanQScale;
}

int make_u_map(CUtensorMap* map, void* ptr, int64_t n_pad, int NW) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  GW_REQUIRE(enc != nullptr, GW_ECUDA, "cuTensorMapEncodeTiled is not available");
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(n_pad), static_cast<cuuint64_t>(NW)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(n_pad) * 2};
  cuuint32_t box[2] = {64, static_cast<cuuint32_t>(NW)};
  cuuint32_t es[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, ptr, dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  GW_REQUIRE(r == CUDA_SUCCESS, GW_ECUDA, "cuTensorMapEncodeTiled failed (%d)", static_cast<int>(r));
  return GW_OK;
}

int plan_nw(int D) {
  return D + 3 <= 16 ? 16 : D + 3 <= 32 ? 32 : D + 3 <= 48 ? 48 : D + 3 <= 64 ? 64 : 80;
}

template <int KP, int S, int NW, bool BF16, bool F8>
int launch_plan(const CUtensorMap* maps, const PlanTask& T, int blocks, cudaStream_t st) {
  using L = PlanSmem<KP, S, NW>;
  auto kern = plan_tc_kernel<KP, S, NW, BF16, F8>;
  static std::once_flag once;
  static cudaError_t attr_rc = cudaSuccess;
  std::call_once(once, [&] {
    attr_rc = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L::kBytes);
  });
  GW_CUDA_TRY(attr_rc);
  kern<<<blocks, kPlanThreads, L::kBytes, st>>>(maps[0], maps[1], maps[2], maps[3], T);
  GW_LAUNCH_CHECK();
  return GW_OK;
}

template <int KP, int S, bool BF16, bool F8 = false>
int launch_plan_nw(int NW, const CUtensorMap* maps, const PlanTask& T, int blocks, cudaStream_t st) {
  switch (NW) {
    case 16: return launch_plan<KP, S, 16, BF16, F8>(maps, T, blocks, st);
    case 32: return launch_plan<KP, S, 32, BF16, F8>(maps, T, blocks, st);
    case 48: return launch_plan<KP, S, 48, BF16, F8>(maps, T, blocks, st);
    case 64: return launch_plan<KP, S, 64, BF16, F8>(maps, T, blocks, st);
    default: break;
  }
  // NW = 80 (D + 3 <= 80): the U tiles take more shared memory, so 128-column
  // operands keep 2 stages
  if constexpr (KP == 64) return launch_plan<64, S, 80, BF16, F8>(maps, T, blocks, st);
  else return launch_plan<KP, 2, 80, BF16, F8>(maps, T, blocks, st);
}

struct PlanLayout {
  int64_t rows_pad, cols_pad;
  int row_tiles, col_tiles, splits, tiles_per_split;
};

PlanLayout plan_layout(int64_t m, int64_t n) {
  PlanLayout Lt;
  Lt.row_tiles = static_cast<int>(ceil_div(m, kPlanBM));
  Lt.col_tiles = static_cast<int>(ceil_div(n, kPlanBN));
  Lt.rows_pad = static_cast<int64_t>(Lt.row_tiles) * kPlanBM;
  Lt.cols_pad = static_cast<int64_t>(Lt.col_tiles) * kPlanBN;
  // At most 128 source tiles (8192 sources) per split: each split's W sums
  // in one FP32 TMEM accumulator, whose rounding over a long chain of MMAs
  // dominates the error of these sums.  Among the counts above that floor
  // (and with at least 8 tiles per CTA to amortise its set-up), the one that
  // fills whole waves of 152 CTAs best.
  const int smax = Lt.col_tiles / 8 > 1 ? Lt.col_tiles / 8 : 1;
  int smin = static_cast<int>(ceil_div(Lt.col_tiles, 128));
  if (smin > smax) smin = smax;
  int s = smin;
  double best = 0.0;
  for (int c = smin; c <= smax && c <= smin + 64; ++c) {
    const double ctas = static_cast<double>(Lt.row_tiles) * c;
    const double waves = ctas / kSmCount;
    const double eff = waves / ceil(waves);
    if (eff > best + 1e-3) {
      best = eff;
      s = c;
    }
    if (eff > 0.97) break;
  }
  Lt.tiles_per_split = static_cast<int>(ceil_div(Lt.col_tiles, s));
  Lt.splits = static_cast<int>(ceil_div(Lt.col_tiles, Lt.tiles_per_split));
  return Lt;
}

struct PlanBufs {
  uint16_t *opA, *opB;
  unsigned *mx, *umax;
  float *loga, *uinv;
  __half *Uh, *Ul;
  int* flag;
  float* Wp;
  float* Ep;
  float *fsA, *fsB;   // FP8 group scales (targets, sources)
};

PlanBufs carve_plan(Carver& c, int64_t n, int64_t m, int D, int prec) {
  const TcOperandShape shp = tc_shape(D, prec);
  const PlanLayout Lt = plan_layout(m, n);
  const int NW = plan_nw(D);
  PlanBufs B;
  B.opA = c.take<uint16_t>(static_cast<size_t>(Lt.rows_pad) * shp.KP);
  B.opB = c.take<uint16_t>(static_cast<size_t>(Lt.cols_pad) * shp.KP);
  B.mx = c.take<unsigned>(8);
  B.umax = c.take<unsigned>(128);
  B.loga = c.take<float>(static_cast<size_t>(n));
  B.uinv = c.take<float>(128);
  B.Uh = c.take<__half>(static_cast<size_t>(NW) * Lt.cols_pad);
  B.Ul = c.take<__half>(static_cast<size_t>(NW) * Lt.cols_pad);
  B.flag = c.take<int>(4);
  B.Wp = c.take<float>(static_cast<size_t>(Lt.splits) * m * (D + 2));
  B.Ep = c.take<float>(static_cast<size_t>(Lt.splits) * m * 2);
  B.fsA = B.fsB = nullptr;
  if (shp.k8 > 0) {
    B.fsA = c.take<float>(static_cast<size_t>(Lt.rows_pad / kFp8Group));
    B.fsB = c.take<float>(static_cast<size_t>(ceil_div(Lt.cols_pad, kFp8Group)));
  }
  return B;
}

}  // namespace

bool plan_tc_supported(int D, int prec) {
  if (prec != GW_PREC_BF16 && prec != GW_PREC_BF16X3 && prec != GW_PREC_F16X3 &&
      prec != GW_PREC_FP8)
    return false;
  return D + 3 <= 80 && tc_shape(D, prec).KP <= 128;
}

size_t plan_tc_ws_bytes(int64_t n, int64_t m, int D, int prec) {
  Carver c(nullptr, ~size_t(0));
  carve_plan(c, n, m, D, prec);
  return c.used();
}

int run_plan_tc(const PlanArgs& p, int prec, const float* V, float** Wp_out, float** Ep_out,
                int* splits_out, int* rows_per_split_out, int** flag_out, Carver& ws,
                cudaStream_t st) {
  GW_REQUIRE(plan_tc_supported(p.D, prec), GW_EUNSUPPORTED, "tensor-core plan sums: D=%d prec=%d",
             p.D, prec);
  const TcOperandShape shp = tc_shape(p.D, prec);
  const PlanLayout Lt = plan_layout(p.m, p.n);
  const int NW = plan_nw(p.D);
  const bool bf16 = tc_is_bf16(prec);
  PlanBufs B = carve_plan(ws, p.n, p.m, p.D, prec);
  GW_REQUIRE(!ws.overflow, GW_ENOMEM, "workspace too small for the tensor-core plan sums");
  GW_CUDA_TRY(cudaMemsetAsync(B.flag, 0, sizeof(int) * 4, st));
  GW_TRY(launch_log(p.a, p.n, B.loga, st));
  // exponent operands: the column softmin's (targets V as rows with the shift
  // estimate g; sources X as columns with the bias f / eps + log a)
  const float inv_eps = 1.0f / p.eps;
  GW_CUDA_TRY(cudaMemsetAsync(B.mx, 0, 8 * sizeof(unsigned), st));
  tc_absmax_kernel<<<2 * kSmCount, 256, 0, st>>>(V, p.m * p.D, p.X, p.n * p.D, p.t, p.m, p.s, p.n,
                                                 p.f, B.loga, p.g, inv_eps, B.mx, kPlanShiftBias);
  GW_LAUNCH_CHECK();
  const float alpha = 16.0f * kLog2e * inv_eps;
  const float beta = 4.0f * kLog2e * inv_eps;
  if (shp.k8 > 0) {
    // FP8: the same 128-row group scales the softmin gives V and X
    const int64_t ga = Lt.rows_pad / kFp8Group, gb = ceil_div(Lt.cols_pad, kFp8Group);
    fp8_scale_kernel<<<ceil_div(ga * 32, 256), 256, 0, st>>>(V, p.m, p.D, ga, B.fsA);
    GW_LAUNCH_CHECK();
    fp8_scale_kernel<<<ceil_div(gb * 32, 256), 256, 0, st>>>(p.X, p.n, p.D, gb, B.fsB);
    GW_LAUNCH_CHECK();
  }
  dim3 blk(64, 4);
  if (bf16) {
    tc_prep_kernel<__nv_bfloat16><<<ceil_div(Lt.rows_pad, 4), blk, 0, st>>>(
        V, p.t, nullptr, nullptr, p.g, p.m, Lt.rows_pad, shp, 0, alpha, beta, inv_eps, B.mx,
        reinterpret_cast<__nv_bfloat16*>(B.opA), kPlanShiftBias, nullptr, TcOperandShape{}, 0,
        B.fsA);
    GW_LAUNCH_CHECK();
    tc_prep_kernel<__nv_bfloat16><<<ceil_div(Lt.cols_pad, 4), blk, 0, st>>>(
        p.X, p.s, p.f, B.loga, nullptr, p.n, Lt.cols_pad, shp, 1, alpha, beta, inv_eps, B.mx,
        reinterpret_cast<__nv_bfloat16*>(B.opB), kShiftBias, nullptr, TcOperandShape{}, 0, B.fsB);
    GW_LAUNCH_CHECK();
  } else {
    tc_prep_kernel<__half><<<ceil_div(Lt.rows_pad, 4), blk, 0, st>>>(
        V, p.t, nullptr, nullptr, p.g, p.m, Lt.rows_pad, shp, 0, alpha, beta, inv_eps, B.mx,
        reinterpret_cast<__half*>(B.opA), kPlanShiftBias);
    GW_LAUNCH_CHECK();
    tc_prep_kernel<__half><<<ceil_div(Lt.cols_pad, 4), blk, 0, st>>>(
        p.X, p.s, p.f, B.loga, nullptr, p.n, Lt.cols_pad, shp, 1, alpha, beta, inv_eps, B.mx,
        reinterpret_cast<__half*>(B.opB));
    GW_LAUNCH_CHECK();
  }
  // U = [X, s, 1, log a], feature-major, per-column power-of-two scales
  GW_CUDA_TRY(cudaMemsetAsync(B.umax, 0, 128 * sizeof(unsigned), st));
  u_absmax_kernel<<<kSmCount, 256, 0, st>>>(p.X, p.s, B.loga, p.n, p.D, B.umax);
  GW_LAUNCH_CHECK();
  u_prep_kernel<<<ceil_div(static_cast<int64_t>(NW) * Lt.cols_pad, 256), 256, 0, st>>>(
      p.X, p.s, B.loga, p.n, Lt.cols_pad, p.D, NW, B.umax, B.Uh, B.Ul, B.uinv);
  GW_LAUNCH_CHECK();
  CUtensorMap maps[4];
  GW_TRY(make_map(&maps[0], B.opA, Lt.rows_pad, shp.KP, bf16, 128));
  GW_TRY(make_map(&maps[1], B.opB, Lt.cols_pad, shp.KP, bf16, kPlanBN));
  GW_TRY(make_u_map(&maps[2], B.Uh, Lt.cols_pad, NW));
  GW_TRY(make_u_map(&maps[3], B.Ul, Lt.cols_pad, NW));
  PlanTask T;
  T.rows = p.m;
  T.ksteps = (shp.used + 15) / 16;
  T.col_tiles = Lt.col_tiles;
  T.splits = Lt.splits;
  T.tiles_per_split = Lt.tiles_per_split;
  T.D = p.D;
  T.b = p.b;
  T.uinv = B.uinv;
  T.Wp = B.Wp;
  T.Ep = Ep_out ? B.Ep : nullptr;
  T.flag = B.flag;
  T.wc = wait_ctl();
  T.k8 = shp.k8;
  T.fsA = B.fsA;
  T.fsB = B.fsB;
  T.alpha8 = alpha;
  const int blocks = Lt.row_tiles * Lt.splits;
  int rc;
  if (shp.k8 > 0) {
    rc = shp.KP == 64 ? launch_plan_nw<64, 4, true, true>(NW, maps, T, blocks, st)
                      : launch_plan_nw<128, 3, true, true>(NW, maps, T, blocks, st);
  } else if (shp.KP == 64) {
    rc = bf16 ? launch_plan_nw<64, 4, true>(NW, maps, T, blocks, st)
              : launch_plan_nw<64, 4, false>(NW, maps, T, blocks, st);
  } else {
    rc = bf16 ? launch_plan_nw<128, 3, true>(NW, maps, T, blocks, st)
              : launch_plan_nw<128, 3, false>(NW, maps, T, blocks, st);
  }
  GW_TRY(rc);
  *Wp_out = B.Wp;
  if (Ep_out) *Ep_out = B.Ep;
  *splits_out = Lt.splits;
  *rows_per_split_out = Lt.tiles_per_split * kPlanBN;
  *flag_out = B.flag;
  return GW_OK;
}

}  // namespace gw
