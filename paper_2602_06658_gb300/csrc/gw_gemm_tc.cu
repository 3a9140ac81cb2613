// Dense FP32-accuracy matrix product on the 5th-generation tensor cores, for
// the exact Kernel-GW mode (Algorithm 5, Appendix B.3), whose cost needs
// K^X pi K^Y every outer step.
//
//   out[r][s] = scale * sum_k A[s][k] Bt[r][k] + coef * u[r] v[s]
//
// Each FP32 operand row is scaled by a power of two (its largest magnitude
// to 2^14) and split into f16 hi + lo; the operands are laid out K-major as
// A3 = [hi | hi | lo] and B3 = [hi | lo | hi], so one K' = 3 K_pad contraction
// gives hi*hi + hi*lo + lo*hi (about 2^-21 relative per product, FP32
// accumulation in TMEM).  The MMA's M side (TMEM lanes, one per epilogue
// thread) is the output's column index s, so the epilogue's stores of one
// output row are contiguous across a warp.
//
// CTA: one 128 x BN output tile (BN = 128), K' streamed by TMA in blocks of
// 64 through an S-stage ring (A and B blocks side by side, 128-byte swizzle),
// warp 0 TMA, warp 1 MMA (one thread), warps 2..5 the epilogue (one TMEM lane
// quarter each).  Every wait is bounded (the launch's WaitCtl).
#include <mutex>

#include "gw_tc_ops.cuh"

namespace gw {

namespace {

constexpr int kGBM = 128;     // output columns s per CTA (MMA M)
constexpr int kGBN = 128;     // output rows r per CTA (MMA N)
constexpr int kGS = 6;        // ring stages
constexpr int kGThreads = 64 + 128;
constexpr int kGABlock = kGBM * 128;   // one 64-wide K block of A: 16 KB
constexpr int kGBBlock = kGBN * 128;   // one 64-wide K block of B: 16 KB
constexpr int kGStage = kGABlock + kGBBlock;
constexpr int kGBarOff = kGS * kGStage;
constexpr int kGBytes = kGBarOff + 256 + 1024;

struct GemmTask {
  tc::WaitCtl wc;
  int kblocks;           // K' / 64
  int tiles_s;           // S_pad / 128
  int64_t R, S;          // output rows / columns
  float scale, coef;
  const float* u;        // R or null
  const float* v;        // S or null
  const float* cA;       // per-row scale of A (S_pad)
  const float* cB;       // per-row scale of B (R_pad)
  float* out;            // R x S row-major
};

__global__ void __launch_bounds__(kGThreads, 1)
    gemm_tc_kernel(const __grid_constant__ CUtensorMap mA, const __grid_constant__ CUtensorMap mB,
                   GemmTask T) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kGBarOff);
  uint64_t* full = bars;             // [S]
  uint64_t* empty = bars + kGS;      // [S]
  uint64_t* done = bars + 2 * kGS;
  uint64_t* drain = bars + 2 * kGS + 1;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  __shared__ int consumed;

  const int ts = blockIdx.x % T.tiles_s;
  const int tr = blockIdx.x / T.tiles_s;
  const int s0 = ts * kGBM, r0 = tr * kGBN;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nkb = T.kblocks;

  if (threadIdx.x == 0) {
    abort_flag = 0;
    consumed = 0;
    for (int s = 0; s < kGS; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    tc::mbar_init(done, 1);
    tc::mbar_init(drain, 1);
    tc::fence_mbar_init();
  }
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base, kGBN);
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
      int issued = 0;
      for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % kGS;
        if (!tc::mbar_wait(&empty[s], ((kb / kGS) & 1) ^ 1, ab, lim)) break;
        tc::mbar_arrive_expect_tx(&full[s], kGStage);
        unsigned char* st = smem + s * kGStage;
        tc::tma_load_2d(st, &mA, kb * 64, s0, &full[s]);
        tc::tma_load_2d(st + kGABlock, &mB, kb * 64, r0, &full[s]);
        issued = kb + 1;
      }
      if (*ab) {
        // wind down: wait for the copies still in flight before leaving
        const int first = *reinterpret_cast<volatile int*>(&consumed);
        for (int kb = first; kb < issued; ++kb) mbar_drain(&full[kb % kGS], (kb / kGS) & 1);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ------------------------------------------------------- MMA issuer
      const uint32_t idesc = tc::f16_idesc(kGBM, kGBN, false);
      for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % kGS;
        if (!tc::mbar_wait(&full[s], (kb / kGS) & 1, ab, lim)) break;
        *reinterpret_cast<volatile int*>(&consumed) = kb + 1;
        tc::tc_fence_after();
        const uint32_t aaddr = tc::smem_u32(smem + s * kGStage);
        const uint32_t baddr = tc::smem_u32(smem + s * kGStage + kGABlock);
#pragma unroll
        for (int ks = 0; ks < 4; ++ks)
          tc::mma_f16(tbase, tc::sw128_desc(aaddr + ks * 32), tc::sw128_desc(baddr + ks * 32), idesc,
                      (kb > 0 || ks > 0) ? 1u : 0u);
        tc::mma_commit(&empty[s]);
      }
      tc::mma_commit(done);
      // every MMA issued above has finished before TMEM is freed
      tc::mma_commit(drain);
      mbar_drain(drain, 0);
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int q = warp & 3;                        // TMEM lane quarter
    const int64_t s = static_cast<int64_t>(s0) + q * 32 + lane;
    int got = 0;
    if (lane == 0) got = tc::mbar_wait(done, 0, ab, lim) ? 1 : 0;
    got = __shfl_sync(0xffffffffu, got, 0);
    got = __shfl_sync(0xffffffffu, (got && !*ab) ? 1 : 0, 0);
    const bool in_s = s < T.S;
    const float csa = in_s ? T.cA[s] : 0.0f;
    const float vs = (in_s && T.v != nullptr) ? T.v[s] : 0.0f;
    tc::tc_fence_after();
    for (int c0 = 0; c0 < kGBN; c0 += 32) {
      uint32_t rr[32];
      if (got) {
        tc::tmem_ld32_issue(tbase + (static_cast<uint32_t>(q * 32) << 16) + c0, rr);
        tc::tmem_ld_wait(rr);
      }
#pragma unroll 4
      for (int k = 0; k < 32; ++k) {
        const int64_t r = static_cast<int64_t>(r0) + c0 + k;
        if (r < T.R && in_s) {
          float val = __int_as_float(0x7fc00000);   // a wait gave up
          if (got) {
            val = T.scale * (__uint_as_float(rr[k]) * (csa * T.cB[r]));
            if (T.u != nullptr) val = fmaf(T.coef * T.u[r], vs, val);
          }
          T.out[r * T.S + s] = val;
        }
      }
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0) tc::note_gave_up(T.wc, ab);
  if (warp == 0) {
    __syncwarp();
    tc::tc_fence_after();
    tc::tmem_dealloc(tbase, kGBN);
  }
}

// Largest |x| of every logical row of a rows x K operand stored row-major
// (trans = 0: src[s][k]) or transposed (trans = 1: src[k][s]) -> mx bits.
__global__ void gemm_rowmax_kernel(const float* src, int trans, int64_t rows, int64_t K,
                                   unsigned* mx) {
  const int64_t total = rows * K;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += stride) {
    const int64_t s = trans ? e % rows : e / K;
    const float v = fabsf(src[e]);
    if (v > 0.0f) atomicMax(&mx[s], __float_as_uint(v));
  }
}

// Power-of-two scale c_s with max |row| / c_s in (2^13, 2^14] (1 for a zero
// or non-finite row).
__device__ __forceinline__ float row_pow2(unsigned bits) {
  const float m = __uint_as_float(bits);
  if (!(m > 0.0f) || !isfinite(m)) return 1.0f;
  int e;
  frexpf(m, &e);          // m = f 2^e, f in [0.5, 1)
  return ldexpf(1.0f, e - 14);
}

// Split layout of one operand, 32 x 32 tiles through shared memory (coalesced
// reads in the source's storage order and writes along K):
// out3[s][k] = hi, out3[s][K_pad + k] = hi (A) / lo (B),
// out3[s][2 K_pad + k] = lo (A) / hi (B), of x = src(s, k) / c_s;
// padding rows and columns are zero.  cs[s] = c_s.
__global__ void gemm_split_kernel(const float* src, int trans, int64_t rows, int64_t K,
                                  int64_t K_pad, int role, const unsigned* mx, __half* out3,
                                  float* cs) {
  __shared__ float tile[32][33];
  const int64_t s0 = static_cast<int64_t>(blockIdx.y) * 32, k0 = static_cast<int64_t>(blockIdx.x) * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
  for (int j = 0; j < 32; j += 8) {
    float v = 0.0f;
    if (trans) {
      const int64_t k = k0 + ty + j, s = s0 + tx;
      if (k < K && s < rows) v = src[k * rows + s];
      tile[tx][ty + j] = v;
    } else {
      const int64_t s = s0 + ty + j, k = k0 + tx;
      if (k < K && s < rows) v = src[s * K + k];
      tile[ty + j][tx] = v;
    }
  }
  __syncthreads();
  const int64_t KP3 = 3 * K_pad;
  for (int j = 0; j < 32; j += 8) {
    const int64_t s = s0 + ty + j, k = k0 + tx;
    const float c = s < rows ? row_pow2(mx[s]) : 1.0f;
    const float x = tile[ty + j][tx] / c;
    const __half hi = __float2half_rn(x);
    const __half lo = __float2half_rn(x - __half2float(hi));
    __half* row = out3 + s * KP3;
    row[k] = hi;
    row[K_pad + k] = role == 0 ? hi : lo;
    row[2 * K_pad + k] = role == 0 ? lo : hi;
    if (k0 == 0 && tx == 0) cs[s] = c;
  }
}

int64_t pad_to(int64_t v, int64_t q) { return (v + q - 1) / q * q; }

struct GemmBufs {
  __half *A3, *B3;
  unsigned *mxA, *mxB;
  float *cA, *cB;
};

GemmBufs carve_gemm(Carver& c, int64_t S, int64_t R, int64_t K) {
  const int64_t Sp = pad_to(S, kGBM), Rp = pad_to(R, kGBN), Kp = pad_to(K, 64);
  GemmBufs B;
  B.A3 = c.take<__half>(static_cast<size_t>(Sp) * 3 * Kp);
  B.B3 = c.take<__half>(static_cast<size_t>(Rp) * 3 * Kp);
  B.mxA = c.take<unsigned>(static_cast<size_t>(Sp));
  B.mxB = c.take<unsigned>(static_cast<size_t>(Rp));
  B.cA = c.take<float>(static_cast<size_t>(Sp));
  B.cB = c.take<float>(static_cast<size_t>(Rp));
  return B;
}

}  // namespace

size_t gemm_tc_ws_bytes(int64_t S, int64_t R, int64_t K) {
  Carver c(nullptr, ~size_t(0));
  carve_gemm(c, S, R, K);
  return c.used();
}

int gemm_tc_f16x3(const float* A, bool a_trans, const float* Bt, bool b_trans, int64_t S,
                  int64_t R, int64_t K, float scale, const float* u, const float* v, float coef,
                  float* out, Carver& ws, cudaStream_t st) {
  GW_REQUIRE(S >= 1 && R >= 1 && K >= 1, GW_EINVAL, "gemm: empty operand");
  const int64_t Sp = pad_to(S, kGBM), Rp = pad_to(R, kGBN), Kp = pad_to(K, 64);
  GW_REQUIRE(3 * Kp <= (int64_t(1) << 31) && Sp <= (int64_t(1) << 31) && Rp <= (int64_t(1) << 31),
             GW_EUNSUPPORTED, "gemm: operands too large");
  GemmBufs B = carve_gemm(ws, S, R, K);
  GW_REQUIRE(!ws.overflow, GW_ENOMEM, "workspace too small for the tensor-core product");
  GW_CUDA_TRY(cudaMemsetAsync(B.mxA, 0, sizeof(unsigned) * Sp, st));
  GW_CUDA_TRY(cudaMemsetAsync(B.mxB, 0, sizeof(unsigned) * Rp, st));
  gemm_rowmax_kernel<<<4 * kSmCount, 256, 0, st>>>(A, a_trans ? 1 : 0, S, K, B.mxA);
  GW_LAUNCH_CHECK();
  gemm_rowmax_kernel<<<4 * kSmCount, 256, 0, st>>>(Bt, b_trans ? 1 : 0, R, K, B.mxB);
  GW_LAUNCH_CHECK();
  gemm_split_kernel<<<dim3(static_cast<unsigned>(Kp / 32), static_cast<unsigned>(Sp / 32)),
                      dim3(32, 8), 0, st>>>(A, a_trans ? 1 : 0, S, K, Kp, 0, B.mxA, B.A3, B.cA);
  GW_LAUNCH_CHECK();
  gemm_split_kernel<<<dim3(static_cast<unsigned>(Kp / 32), static_cast<unsigned>(Rp / 32)),
                      dim3(32, 8), 0, st>>>(Bt, b_trans ? 1 : 0, R, K, Kp, 1, B.mxB, B.B3, B.cB);
  GW_LAUNCH_CHECK();
  CUtensorMap maps[2];
  GW_TRY(make_map(&maps[0], B.A3, Sp, static_cast<int>(3 * Kp), false, kGBM));
  GW_TRY(make_map(&maps[1], B.B3, Rp, static_cast<int>(3 * Kp), false, kGBN));
  GemmTask T;
  T.wc = wait_ctl();
  T.kblocks = static_cast<int>(3 * Kp / 64);
  T.tiles_s = static_cast<int>(Sp / kGBM);
  T.R = R;
  T.S = S;
  T.scale = scale;
  T.coef = coef;
  T.u = u;
  T.v = v;
  T.cA = B.cA;
  T.cB = B.cB;
  T.out = out;
  static std::once_flag once;
  static cudaError_t attr_rc = cudaSuccess;
  std::call_once(once, [] {
    attr_rc = cudaFuncSetAttribute(gemm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   kGBytes);
  });
  GW_CUDA_TRY(attr_rc);
  const int64_t blocks = (Sp / kGBM) * (Rp / kGBN);
  GW_REQUIRE(blocks <= 2147483647, GW_EUNSUPPORTED, "gemm: too many tiles");
  gemm_tc_kernel<<<static_cast<unsigned>(blocks), kGThreads, kGBytes, st>>>(maps[0], maps[1], T);
  GW_LAUNCH_CHECK();
  return GW_OK;
}

}  // namespace gw
