// Multiscale-GW (Algorithms 7 and 8, Appendix B.5): K-Means coarsening of
// both measures, a coarse CNT-GW solve, interpolation of the coarse
// potentials to the fine points by one softmin each (Algorithm 8), and the
// fine CNT-GW solve started from Gamma^c and the interpolated potentials.
//
// K-Means is Lloyd's algorithm started from caller-given indices; ties go to
// the lowest centroid index.  Cluster sums are accumulated in 64-bit fixed
// point with integer atomics (associative, so the result is bitwise
// reproducible whatever the order), then divided in float64.  Empty clusters
// are dropped.
#include <math.h>

#include <vector>

#include "gw_internal.cuh"

namespace gw {

namespace {

constexpr int kKmThreads = 128;
constexpr int kKmTile = 32;

// assign[j] = argmin_c (||C_c||^2 - 2 <X_j, C_c>), first minimum
template <int DP>
__global__ void __launch_bounds__(kKmThreads)
    km_assign_kernel(const float* X, int64_t n, int D, const float* C, const float* cn, int64_t k,
                     int* assign) {
  __shared__ __align__(16) float Cs[kKmTile][DP];
  __shared__ float ns[kKmTile];
  const int64_t j = static_cast<int64_t>(blockIdx.x) * kKmThreads + threadIdx.x;
  const bool ok = j < n;
  float x[DP];
#pragma unroll
  for (int d = 0; d < DP; ++d) x[d] = (ok && d < D) ? X[j * D + d] : 0.f;
  float best = INFINITY;
  int bi = 0;
  for (int64_t c0 = 0; c0 < k; c0 += kKmTile) {
    __syncthreads();
    for (int idx = threadIdx.x; idx < kKmTile * DP; idx += kKmThreads) {
      const int cc = idx / DP, d = idx % DP;
      const int64_t c = c0 + cc;
      Cs[cc][d] = (c < k && d < D) ? C[c * D + d] : 0.f;
    }
    if (threadIdx.x < kKmTile) {
      const int64_t c = c0 + threadIdx.x;
      ns[threadIdx.x] = c < k ? cn[c] : INFINITY;
    }
    __syncthreads();
    const int cnt = static_cast<int>(k - c0 < kKmTile ? k - c0 : kKmTile);
    for (int cc = 0; cc < cnt; ++cc) {
      float dot = 0.f;
#pragma unroll
      for (int d = 0; d < DP; ++d) dot = fmaf(x[d], Cs[cc][d], dot);
      const float v = fmaf(-2.0f, dot, ns[cc]);
      if (v < best) {
        best = v;
        bi = static_cast<int>(c0 + cc);
      }
    }
  }
  if (ok) assign[j] = bi;
}

__global__ void km_norms_kernel(const float* C, int64_t k, int D, float* cn) {
  const int64_t c = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (c >= k) return;
  float s = 0.f;
  for (int d = 0; d < D; ++d) s = fmaf(C[c * D + d], C[c * D + d], s);
  cn[c] = s;
}

// initial centroids X[idx]; an index outside [0, n) sets *bad and reads nothing
__global__ void km_gather_kernel(const float* X, int64_t n, int D, const int64_t* idx, int64_t k,
                                 float* C, int64_t* bad) {
  const int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= k * D) return;
  const int64_t j = idx[q / D];
  if (j < 0 || j >= n) {
    *bad = 1;
    C[q] = 0.f;
    return;
  }
  C[q] = X[j * D + q % D];
}

// mx[0] = max |X|, mx[1] = max a (float bits; non-negative, so the bit
// patterns order like the values)
__global__ void km_absmax_kernel(const float* X, int64_t count, const float* a, int64_t n,
                                 unsigned* mx) {
  float v = 0.f, w = 0.f;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < count;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    v = fmaxf(v, fabsf(X[i]));
  if (a) {
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
      w = fmaxf(w, fabsf(a[i]));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    w = fmaxf(w, __shfl_xor_sync(0xffffffffu, w, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(mx, __float_as_uint(v));
    atomicMax(mx + 1, __float_as_uint(w));
  }
}

// Fixed-point scale 2^s: every cluster sum is bounded by max|X| * sum_j a_j
// <= max|X| * n * max a, kept below 2^60 (3 bits of headroom under 2^63).
__device__ __forceinline__ int fixed_shift(const unsigned* mx, int64_t n, bool has_w) {
  const double xm = fmax(static_cast<double>(__uint_as_float(mx[0])), 1.0);
  const double wt = has_w ? fmax(static_cast<double>(__uint_as_float(mx[1])) * n, 1.0) : 1.0;
  int e;
  frexp(xm * wt, &e);   // bound < 2^e
  const int s = 60 - e;
  return s > 56 ? 56 : s;
}

// acc[c][d] += a_j X_jd, acc[c][D] += a_j  (64-bit fixed point, integer atomics)
__global__ void km_accumulate_kernel(const float* X, const float* a, float wu, int64_t n, int D,
                                     const int* assign, const unsigned* mx,
                                     unsigned long long* acc) {
  const int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int s = fixed_shift(mx, n, a != nullptr);
  const double scale = ldexp(1.0, s);
  const double aj = a ? static_cast<double>(a[j]) : static_cast<double>(wu);
  unsigned long long* row = acc + static_cast<int64_t>(assign[j]) * (D + 1);
  for (int d = 0; d < D; ++d) {
    const long long v = llrint(aj * static_cast<double>(X[j * D + d]) * scale);
    atomicAdd(row + d, static_cast<unsigned long long>(v));
  }
  atomicAdd(row + D, static_cast<unsigned long long>(llrint(aj * scale)));
}

// C_c = sum / weight for non-empty clusters (empty ones keep their centroid)
__global__ void km_update_kernel(const unsigned long long* acc, int64_t k, int D,
                                 const unsigned* mx, int64_t n, bool has_w, float* C, float* cn,
                                 double* w) {
  const int64_t c = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (c >= k) return;
  const double inv_scale = ldexp(1.0, -fixed_shift(mx, n, has_w));
  const unsigned long long* row = acc + c * (D + 1);
  const double wc = static_cast<double>(static_cast<long long>(row[D])) * inv_scale;
  w[c] = wc;
  if (wc > 0.0) {
    float s = 0.f;
    for (int d = 0; d < D; ++d) {
      const float v = static_cast<float>(static_cast<double>(static_cast<long long>(row[d])) *
                                         inv_scale / wc);
      C[c * D + d] = v;
      s = fmaf(v, v, s);
    }
    cn[c] = s;
  }
}

// keep the non-empty clusters in order (one block): out rows, weights, norms,
// old -> new cluster index (-1 for dropped ones), count
__global__ void km_compact_kernel(const float* C, const double* w, int64_t k, int D, float* Cout,
                                  float* wout, float* nout, int* remap, int64_t* kout) {
  __shared__ int64_t base;
  __shared__ int64_t cnt[1024];
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  for (int64_t c0 = 0; c0 < k; c0 += blockDim.x) {
    const int64_t c = c0 + threadIdx.x;
    const int keep = (c < k && w[c] > 0.0) ? 1 : 0;
    cnt[threadIdx.x] = keep;
    __syncthreads();
    // inclusive scan (Hillis-Steele) over the block
    for (int o = 1; o < static_cast<int>(blockDim.x); o <<= 1) {
      const int64_t v = threadIdx.x >= static_cast<unsigned>(o) ? cnt[threadIdx.x - o] : 0;
      __syncthreads();
      cnt[threadIdx.x] += v;
      __syncthreads();
    }
    if (c < k) remap[c] = keep ? static_cast<int>(base + cnt[threadIdx.x] - 1) : -1;
    if (keep) {
      const int64_t pos = base + cnt[threadIdx.x] - 1;
      float s = 0.f;
      for (int d = 0; d < D; ++d) {
        const float v = C[c * D + d];
        Cout[pos * D + d] = v;
        s = fmaf(v, v, s);
      }
      wout[pos] = static_cast<float>(w[c]);
      nout[pos] = s;
    }
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) base += cnt[threadIdx.x];
    __syncthreads();
  }
  if (threadIdx.x == 0) *kout = base;
}

__global__ void km_relabel_kernel(const int* assign, const int* remap, int64_t n, int* out) {
  const int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j < n) out[j] = remap[assign[j]];
}

// U_i[e] = sum_d X_i[d] Gamma[d][e]  (n x E), Gamma D x E float64
__global__ void xg_kernel(const float* X, const double* Gamma, int64_t n, int D, int E, float* U) {
  const int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= n * E) return;
  const int64_t i = q / E;
  const int e = static_cast<int>(q % E);
  double acc = 0.0;
  for (int d = 0; d < D; ++d) acc = fma(static_cast<double>(X[i * D + d]), Gamma[d * E + e], acc);
  U[q] = static_cast<float>(acc);
}

struct KmBufs {
  float *C, *cn;
  double* w;
  unsigned long long* acc;
  int* assign;
  int* remap;
  unsigned* mx;
  int64_t* kdev;
};

KmBufs carve_km(Carver& c, int64_t n, int64_t k, int D) {
  KmBufs B;
  B.C = c.take<float>(static_cast<size_t>(k) * D);
  B.cn = c.take<float>(static_cast<size_t>(k));
  B.w = c.take<double>(static_cast<size_t>(k));
  B.acc = c.take<unsigned long long>(static_cast<size_t>(k) * (D + 1));
  B.assign = c.take<int>(static_cast<size_t>(n));
  B.remap = c.take<int>(static_cast<size_t>(k));
  B.mx = c.take<unsigned>(4);
  B.kdev = c.take<int64_t>(2);
  return B;
}

template <int DP>
void launch_assign(const float* X, int64_t n, int D, const KmBufs& B, int64_t k, cudaStream_t st) {
  km_assign_kernel<DP><<<ceil_div(n, kKmThreads), kKmThreads, 0, st>>>(X, n, D, B.C, B.cn, k,
                                                                       B.assign);
}

}  // namespace

size_t coarsen_ws_bytes(int64_t n, int64_t k, int D) {
  Carver c(nullptr, ~size_t(0));
  carve_km(c, n, k, D);
  return c.used();
}

// Lloyd's iterations on the device; returns the number of non-empty clusters.
int run_coarsen(const float* X, const float* a, int64_t n, int D, const int64_t* init_idx,
                int64_t k, int n_iter, float* Xc, float* ac, float* sc, int* assign_out,
                int64_t* k_out, Carver& ws, cudaStream_t st) {
  KmBufs B = carve_km(ws, n, k, D);
  GW_REQUIRE(!ws.overflow, GW_ENOMEM, "workspace too small for K-Means");
  GW_CUDA_TRY(cudaMemsetAsync(B.kdev, 0, sizeof(int64_t) * 2, st));
  km_gather_kernel<<<ceil_div(k * D, 256), 256, 0, st>>>(X, n, D, init_idx, k, B.C, B.kdev + 1);
  GW_LAUNCH_CHECK();
  km_norms_kernel<<<ceil_div(k, 256), 256, 0, st>>>(B.C, k, D, B.cn);
  GW_LAUNCH_CHECK();
  GW_CUDA_TRY(cudaMemsetAsync(B.mx, 0, sizeof(unsigned) * 4, st));
  km_absmax_kernel<<<kSmCount, 256, 0, st>>>(X, n * D, a, n, B.mx);
  GW_LAUNCH_CHECK();
  const float wu = 1.0f / static_cast<float>(n);
  for (int it = 0; it <= n_iter; ++it) {
    const int DP = D <= 4 ? 4 : (D <= 8 ? 8 : (D <= 16 ? 16 : (D <= 32 ? 32 : (D <= 64 ? 64 : 128))));
    switch (DP) {
      case 4: launch_assign<4>(X, n, D, B, k, st); break;
      case 8: launch_assign<8>(X, n, D, B, k, st); break;
      case 16: launch_assign<16>(X, n, D, B, k, st); break;
      case 32: launch_assign<32>(X, n, D, B, k, st); break;
      case 64: launch_assign<64>(X, n, D, B, k, st); break;
      default: launch_assign<128>(X, n, D, B, k, st); break;
    }
    GW_LAUNCH_CHECK();
    GW_CUDA_TRY(cudaMemsetAsync(B.acc, 0, sizeof(unsigned long long) * k * (D + 1), st));
    km_accumulate_kernel<<<ceil_div(n, 256), 256, 0, st>>>(X, a, wu, n, D, B.assign, B.mx, B.acc);
    GW_LAUNCH_CHECK();
    km_update_kernel<<<ceil_div(k, 256), 256, 0, st>>>(B.acc, k, D, B.mx, n, a != nullptr, B.C,
                                                       B.cn, B.w);
    GW_LAUNCH_CHECK();
  }
  km_compact_kernel<<<1, 1024, 0, st>>>(B.C, B.w, k, D, Xc, ac, sc, B.remap, B.kdev);
  GW_LAUNCH_CHECK();
  if (assign_out) {
    km_relabel_kernel<<<ceil_div(n, 256), 256, 0, st>>>(B.assign, B.remap, n, assign_out);
    GW_LAUNCH_CHECK();
  }
  int64_t h[2] = {0, 0};
  GW_CUDA_TRY(cudaMemcpyAsync(h, B.kdev, sizeof(h), cudaMemcpyDeviceToHost, st));
  GW_CUDA_TRY(cudaStreamSynchronize(st));
  GW_REQUIRE(h[1] == 0, GW_EINVAL, "an initial index lies outside [0, n)");
  *k_out = h[0];
  return GW_OK;
}

namespace {

// device buffers of Multiscale-GW that outlive the steps (carved first)
struct MsBufs {
  float *Xc, *Yc, *ac, *sc, *lac, *bc, *tcn, *lbc, *fc, *gc, *f0, *g0, *Vc, *Uc;
  double *Gc, *Gcp, *enc;
};

MsBufs carve_ms(Carver& c, int64_t n, int64_t m, int D, int E, int64_t kx, int64_t ky) {
  MsBufs B;
  B.Xc = c.take<float>(static_cast<size_t>(kx) * D);
  B.Yc = c.take<float>(static_cast<size_t>(ky) * E);
  B.ac = c.take<float>(static_cast<size_t>(kx));
  B.sc = c.take<float>(static_cast<size_t>(kx));
  B.lac = c.take<float>(static_cast<size_t>(kx));
  B.bc = c.take<float>(static_cast<size_t>(ky));
  B.tcn = c.take<float>(static_cast<size_t>(ky));
  B.lbc = c.take<float>(static_cast<size_t>(ky));
  B.fc = c.take<float>(static_cast<size_t>(kx));
  B.gc = c.take<float>(static_cast<size_t>(ky));
  B.f0 = c.take<float>(static_cast<size_t>(n));
  B.g0 = c.take<float>(static_cast<size_t>(m));
  B.Gc = c.take<double>(static_cast<size_t>(D) * E);
  B.Gcp = c.take<double>(static_cast<size_t>(D) * E);
  B.enc = c.take<double>(GW_EN_LEN);
  B.Vc = c.take<float>(static_cast<size_t>(ky) * D);   // Gamma^c Y^c
  B.Uc = c.take<float>(static_cast<size_t>(kx) * E);   // X^c Gamma^c
  return B;
}

}  // namespace

size_t multiscale_ws_bytes(int64_t n, int64_t m, int D, int E, int64_t kx, int64_t ky, int prec) {
  Carver c(nullptr, ~size_t(0));
  carve_ms(c, n, m, D, E, kx, ky);
  const size_t fixed = c.used();
  size_t scratch = coarsen_ws_bytes(n, kx, D);
  const size_t cy = coarsen_ws_bytes(m, ky, E);
  const size_t coarse = gw_workspace_size(GW_OP_SOLVE, kx, ky, D, E, prec);
  const size_t fine = gw_workspace_size(GW_OP_SOLVE, n, m, D, E, prec);
  const size_t interp = softmin_ws_bytes(n, ky, D, prec) + softmin_ws_bytes(m, kx, E, prec) + 512;
  for (size_t v : {cy, coarse, fine, interp})
    if (v > scratch) scratch = v;
  return fixed + scratch;
}

int run_multiscale(const gw_problem& p, const gw_options& oc, const gw_options& of,
                   const int64_t* init_x, int64_t kx, const int64_t* init_y, int64_t ky,
                   int km_iter, gw_result& r, double* coarse_energy, void* ws, size_t ws_bytes,
                   cudaStream_t st) {
  Carver c(ws, ws_bytes);
  const MsBufs M = carve_ms(c, p.n, p.m, p.D, p.E, kx, ky);
  float *Xc = M.Xc, *Yc = M.Yc, *ac = M.ac, *sc = M.sc, *lac = M.lac, *bc = M.bc, *tcn = M.tcn,
        *lbc = M.lbc, *fc = M.fc, *gc = M.gc, *f0 = M.f0, *g0 = M.g0, *Vc = M.Vc, *Uc = M.Uc;
  double *Gc = M.Gc, *Gcp = M.Gcp, *enc = M.enc;
  GW_TRY(check_ws(c, ws));
  const size_t mark = c.used();
  char* base = static_cast<char*>(ws);
  // Coarsen (K-Means) both measures
  int64_t kx2 = 0, ky2 = 0;
  {
    Carver sub(base + mark, ws_bytes - mark);
    GW_TRY(run_coarsen(p.X, p.a, p.n, p.D, init_x, kx, km_iter, Xc, ac, sc, nullptr, &kx2, sub, st));
  }
  {
    Carver sub(base + mark, ws_bytes - mark);
    GW_TRY(run_coarsen(p.Y, p.b, p.m, p.E, init_y, ky, km_iter, Yc, bc, tcn, nullptr, &ky2, sub, st));
  }
  GW_REQUIRE(kx2 >= 1 && ky2 >= 1, GW_ENONFINITE, "K-Means left no non-empty cluster");
  // coarse CNT-GW
  gw_problem Pc{Xc, Yc, sc, tcn, ac, bc, kx2, ky2, p.D, p.E};
  gw_result Rc{Gc, Gcp, fc, gc, enc, nullptr};
  gw_options occ = oc;
  occ.record = 0;
  GW_TRY(gw_solve(&Pc, &occ, &Rc, base + mark, ws_bytes - mark, reinterpret_cast<gw_stream_t>(st)));
  if (coarse_energy) {
    GW_CUDA_TRY(cudaMemcpyAsync(coarse_energy, enc, sizeof(double) * GW_EN_LEN,
                                cudaMemcpyDeviceToDevice, st));
  }
  // Interpolate (Algorithm 8): f from g^c over Y^c, g from f^c over X^c
  GW_TRY(launch_gamma_y(Gc, Yc, ky2, p.D, p.E, Vc, st));
  xg_kernel<<<ceil_div(kx2 * p.E, 256), 256, 0, st>>>(Xc, Gc, kx2, p.D, p.E, Uc);
  GW_LAUNCH_CHECK();
  GW_TRY(launch_log(bc, ky2, lbc, st));
  GW_TRY(launch_log(ac, kx2, lac, st));
  {
    Carver sub(base + mark, ws_bytes - mark);
    SoftminTask T{};
    T.A = p.X;
    T.B = Vc;
    T.sA = p.s;
    T.sB = tcn;
    T.h = gc;
    T.logw = lbc;
    T.out = f0;
    T.n = p.n;
    T.m = ky2;
    T.K = p.D;
    T.eps = of.eps;
    GW_TRY(launch_softmin(&T, 1, of.prec, sub, st));
  }
  {
    Carver sub(base + mark, ws_bytes - mark);
    SoftminTask T{};
    T.A = p.Y;
    T.B = Uc;
    T.sA = p.t;
    T.sB = sc;
    T.h = fc;
    T.logw = lac;
    T.out = g0;
    T.n = p.m;
    T.m = kx2;
    T.K = p.E;
    T.eps = of.eps;
    GW_TRY(launch_softmin(&T, 1, of.prec, sub, st));
  }
  // fine CNT-GW from Gamma^c and the interpolated potentials
  gw_options off = of;
  off.Gamma0 = Gc;
  off.f0 = f0;
  off.g0 = g0;
  return gw_solve(&p, &off, &r, base + mark, ws_bytes - mark, reinterpret_cast<gw_stream_t>(st));
}

}  // namespace gw
