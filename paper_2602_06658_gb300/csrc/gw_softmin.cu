// Softmin on the bilinear cost (discrete Sinkhorn operator, Eq.
// sinkhorn_operators; loop bodies of Algorithms 2 and 3), FP32 CUDA-core form.
//
//   out_i = -eps * LSE_j [ logw_j + (h_j + 16 <A_i, B_j> + 4 sA_i sB_j) / eps ]
//
// Work is tiled flash-style: every CTA keeps 128*R rows of A in registers,
// streams B through shared memory in tiles of kBN columns and keeps a running
// (max, sum) per row in base 2; the N x M cost matrix never exists.  Columns
// can be split across CTAs; the per-split (max, sum) pairs are merged by a
// second small kernel.  Two tasks (the row and the column half-steps of one
// symmetric Sinkhorn iteration) can share one launch.
#include <math.h>
#include <stdio.h>

#include "gw_internal.cuh"

namespace gw {

namespace {

constexpr int kThreads = 128;
constexpr int kBN = 32;      // columns per shared-memory tile
constexpr int kChunk = 8;    // columns per online-max update

template <int KP>
struct RowsPerThread {
  static constexpr int value = KP <= 32 ? 2 : 1;
};

template <int KP, int R>
__global__ void __launch_bounds__(kThreads)
    softmin_fp32_kernel(SoftminTask t0, SoftminTask t1, int blocks0) {
  const bool second = static_cast<int>(blockIdx.x) >= blocks0;
  const SoftminTask T = second ? t1 : t0;
  const int bid = second ? blockIdx.x - blocks0 : blockIdx.x;
  const int rblk = bid / T.splits;
  const int split = bid % T.splits;
  const int tid = threadIdx.x;

  __shared__ __align__(16) float Bs[kBN][KP];
  __shared__ float cw[kBN];
  __shared__ float ct[kBN];

  const float inv_eps = 1.0f / T.eps;
  const float alpha = 16.0f * kLog2e * inv_eps;   // scale of <A_i, B_j>
  const float beta = 4.0f * kLog2e * inv_eps;     // scale of sA_i sB_j
  const float hs = kLog2e * inv_eps;              // scale of h_j

  float a[R][KP];
  float u[R];
  float mrun[R], srun[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int64_t i = static_cast<int64_t>(rblk) * kThreads * R + r * kThreads + tid;
    const bool ok = i < T.n;
#pragma unroll
    for (int k = 0; k < KP; ++k) a[r][k] = (ok && k < T.K) ? T.A[i * T.K + k] * alpha : 0.0f;
    u[r] = ok ? T.sA[i] * beta : 0.0f;
    mrun[r] = kNegBig;
    srun[r] = 0.0f;
  }

  const int64_t c_begin = static_cast<int64_t>(split) * T.cols_per_split;
  const int64_t c_end = c_begin + T.cols_per_split < T.m ? c_begin + T.cols_per_split : T.m;

  for (int64_t c0 = c_begin; c0 < c_end; c0 += kBN) {
    __syncthreads();
    for (int idx = tid; idx < kBN * KP; idx += kThreads) {
      const int jj = idx / KP, k = idx % KP;
      const int64_t j = c0 + jj;
      Bs[jj][k] = (j < c_end && k < T.K) ? T.B[j * T.K + k] : 0.0f;
    }
    if (tid < kBN) {
      const int64_t j = c0 + tid;
      if (j < c_end) {
        cw[tid] = T.h[j] * hs + T.logw[j] * kLog2e;
        ct[tid] = T.sB[j];
      } else {
        cw[tid] = kNegBig;
        ct[tid] = 0.0f;
      }
    }
    __syncthreads();

#pragma unroll 1
    for (int jc = 0; jc < kBN; jc += kChunk) {
      float z[R][kChunk];
#pragma unroll
      for (int c = 0; c < kChunk; ++c) {
        const float4* brow = reinterpret_cast<const float4*>(&Bs[jc + c][0]);
        float acc[R];
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = fmaf(u[r], ct[jc + c], cw[jc + c]);
#pragma unroll
        for (int k4 = 0; k4 < KP / 4; ++k4) {
          const float4 bv = brow[k4];
#pragma unroll
          for (int r = 0; r < R; ++r) {
            acc[r] = fmaf(a[r][4 * k4 + 0], bv.x, acc[r]);
            acc[r] = fmaf(a[r][4 * k4 + 1], bv.y, acc[r]);
            acc[r] = fmaf(a[r][4 * k4 + 2], bv.z, acc[r]);
            acc[r] = fmaf(a[r][4 * k4 + 3], bv.w, acc[r]);
          }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) z[r][c] = acc[r];
      }
#pragma unroll
      for (int r = 0; r < R; ++r) {
        float cm = z[r][0];
#pragma unroll
        for (int c = 1; c < kChunk; ++c) cm = fmaxf(cm, z[r][c]);
        if (cm > mrun[r]) {
          srun[r] *= ex2(mrun[r] - cm);
          mrun[r] = cm;
        }
        float sum = 0.0f;
#pragma unroll
        for (int c = 0; c < kChunk; ++c) sum += ex2(z[r][c] - mrun[r]);
        srun[r] += sum;
      }
    }
  }

#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int64_t i = static_cast<int64_t>(rblk) * kThreads * R + r * kThreads + tid;
    if (i >= T.n) continue;
    if (T.splits == 1) {
      const float lse2 = mrun[r] + log2f(srun[r]);
      float v = -T.eps * kLn2 * lse2;
      if (T.avg_with) v = 0.5f * (T.avg_with[i] + v);
      T.out[i] = v;
    } else {
      T.pm[static_cast<int64_t>(split) * T.n + i] = mrun[r];
      T.ps[static_cast<int64_t>(split) * T.n + i] = srun[r];
    }
  }
}

// Merge the per-split (max, sum) pairs of up to two tasks.
__global__ void softmin_combine_kernel(SoftminTask t0, SoftminTask t1, int64_t n0) {
  const int64_t gi = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const bool second = gi >= n0;
  const SoftminTask T = second ? t1 : t0;
  const int64_t i = second ? gi - n0 : gi;
  if (i >= T.n || T.splits == 1) return;
  float M = kNegBig;
  for (int s = 0; s < T.splits; ++s) M = fmaxf(M, T.pm[static_cast<int64_t>(s) * T.n + i]);
  float S = 0.0f;
  for (int s = 0; s < T.splits; ++s) {
    const int64_t o = static_cast<int64_t>(s) * T.n + i;
    S += T.ps[o] * ex2(T.pm[o] - M);
  }
  float v = -T.eps * kLn2 * (M + log2f(S));
  if (T.avg_with) v = 0.5f * (T.avg_with[i] + v);
  T.out[i] = v;
}

int kpad(int K) {
  if (K <= 4) return 4;
  if (K <= 8) return 8;
  if (K <= 16) return 16;
  if (K <= 32) return 32;
  if (K <= 64) return 64;
  return 128;
}

int rows_per_thread(int KP) { return KP <= 32 ? 2 : 1; }

template <int KP>
void launch_fp32(const SoftminTask& t0, const SoftminTask& t1, int blocks0, int blocks,
                 cudaStream_t st) {
  constexpr int R = RowsPerThread<KP>::value;
  softmin_fp32_kernel<KP, R><<<blocks, kThreads, 0, st>>>(t0, t1, blocks0);
}

}  // namespace

SoftminShape softmin_shape(int64_t n, int64_t m, int K, int prec) {
  (void)prec;
  SoftminShape sh;
  const int KP = kpad(K);
  sh.rows_per_block = kThreads * rows_per_thread(KP);
  sh.row_blocks = n > 0 ? ceil_div(n, sh.rows_per_block) : 0;
  // Aim for ~4 resident CTAs per SM; never split below 128 columns.
  const int target = 4 * kSmCount;
  int splits = sh.row_blocks > 0 ? ceil_div(target, sh.row_blocks) : 1;
  const int max_splits = ceil_div(m, 128);
  if (splits > max_splits) splits = max_splits;
  if (splits < 1) splits = 1;
  int cps = ceil_div(m, splits);
  cps = ((cps + kBN - 1) / kBN) * kBN;
  sh.cols_per_split = cps;
  sh.splits = ceil_div(m, cps);
  return sh;
}

size_t softmin_ws_bytes(int64_t n, int64_t m, int K, int prec) {
  if (prec != GW_PREC_FP32) return softmin_tc_ws_bytes(n, m, K, prec);
  Carver c(nullptr, ~size_t(0));
  const SoftminShape sh = softmin_shape(n, m, K, prec);
  if (sh.splits > 1) {
    c.take<float>(static_cast<size_t>(sh.splits) * n);
    c.take<float>(static_cast<size_t>(sh.splits) * n);
  }
  return c.used();
}

int launch_softmin(SoftminTask* tasks, int ntasks, int prec, Carver& ws, cudaStream_t st) {
  SoftminTask t[2];
  for (int q = 0; q < ntasks; ++q) t[q] = tasks[q];
  GW_REQUIRE(ntasks == 1 || t[0].K == t[1].K, GW_EINVAL, "fused softmin tasks need the same K");
  if (prec != GW_PREC_FP32) {
    return launch_softmin_tc(t, ntasks, prec, ws, st);   // merges its own split partials
  } else {
    int blocks[2] = {0, 0};
    for (int q = 0; q < ntasks; ++q) {
      const SoftminShape sh = softmin_shape(t[q].n, t[q].m, t[q].K, prec);
      t[q].splits = sh.splits;
      t[q].cols_per_split = sh.cols_per_split;
      t[q].pm = t[q].ps = nullptr;
      if (sh.splits > 1) {
        t[q].pm = ws.take<float>(static_cast<size_t>(sh.splits) * t[q].n);
        t[q].ps = ws.take<float>(static_cast<size_t>(sh.splits) * t[q].n);
      }
      blocks[q] = sh.row_blocks * sh.splits;
    }
    GW_REQUIRE(!ws.overflow, GW_ENOMEM, "workspace too small for softmin partials");
    SoftminTask u1 = t[1];
    if (ntasks == 1) {
      u1 = t[0];
      u1.n = 0;
    }
    const int total = blocks[0] + blocks[1];
    if (total > 0) {
      switch (kpad(t[0].K)) {
        case 4: launch_fp32<4>(t[0], u1, blocks[0], total, st); break;
        case 8: launch_fp32<8>(t[0], u1, blocks[0], total, st); break;
        case 16: launch_fp32<16>(t[0], u1, blocks[0], total, st); break;
        case 32: launch_fp32<32>(t[0], u1, blocks[0], total, st); break;
        case 64: launch_fp32<64>(t[0], u1, blocks[0], total, st); break;
        default: launch_fp32<128>(t[0], u1, blocks[0], total, st); break;
      }
      GW_LAUNCH_CHECK();
    }
  }
  if (ntasks == 1) {
    t[1] = t[0];
    t[1].n = 0;
  }
  const bool need_combine = t[0].splits > 1 || (ntasks == 2 && t[1].splits > 1);
  if (need_combine) {
    const int64_t nn = t[0].n + t[1].n;
    const int thr = 256;
    softmin_combine_kernel<<<ceil_div(nn, thr), thr, 0, st>>>(t[0], t[1], t[0].n);
    GW_LAUNCH_CHECK();
  }
  return GW_OK;
}

}  // namespace gw
