/*
 * gw.h -- C ABI of libgw, the GB300 (sm_103a) hot path of the CNT-GW
 * entropic Gromov-Wasserstein solver of "Gromov-Wasserstein at Scale,
 * Beyond Squared Norms" (arXiv 2602.06658).
 *
 * Notation (the paper's, Section 5 "Notations" and Algorithm 1):
 *   a (N), b (M)         probability weights of the source / target measures
 *   X (N x D), Y (M x E) centered embeddings: sum_i a_i X_i = 0,
 *                        c_X(x_i, x_k) = ||X_i - X_k||^2 (Eqs. embedding_X/Y)
 *   s_i = ||X_i||^2, t_j = ||Y_j||^2
 *   Gamma (D x E)        the linear map of Theorems 3.2-3.4
 *   f (N), g (M)         dual potentials; the plan is never stored:
 *                        pi_ij = a_i b_j exp((f_i + g_j - C_ij)/eps)
 *                        (Eq. sinkhorn_pi)
 *   C_ij = c_Gamma(i,j) = -16 X_i^T Gamma Y_j - 4 s_i t_j
 *                        (Remark after Theorem 3.2, Eq. egw_otherform)
 *
 * Conventions for every entry point:
 *   - Pointers are DEVICE pointers unless the argument name starts with h_.
 *   - Matrices are dense row-major; features and potentials are float32,
 *     Gamma and energy terms float64.
 *   - The caller owns and allocates every input, output and workspace
 *     buffer.  The library allocates no device memory.  Scratch comes from
 *     the caller's workspace `ws` of `ws_bytes` bytes, sized by
 *     gw_workspace_size(); a smaller workspace returns GW_ENOMEM.
 *     Workspace pointers must be 256-byte aligned.
 *   - All device work is enqueued on `stream` (a cudaStream_t; NULL is the
 *     legacy default stream) and is asynchronous unless stated.  Calls on
 *     different streams with disjoint workspaces may run concurrently.
 *   - Every function returns an int status (GW_OK = 0).  Arguments are
 *     validated on the host before anything is enqueued; on error nothing is
 *     enqueued and gw_last_error() describes the problem (per host thread).
 *     No C++ exception or abort crosses this interface.
 */
#ifndef GW_H_
#define GW_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* gw_stream_t;

/* status codes */
#define GW_OK 0
#define GW_EINVAL 1        /* bad shape, null pointer, eps <= 0, bad option */
#define GW_ENOMEM 2        /* workspace too small or misaligned */
#define GW_ECUDA 3         /* a CUDA launch or API call failed */
#define GW_ENONFINITE 4    /* NaN/Inf met in potentials or energy */
#define GW_ETIMEOUT 5      /* a bounded device wait expired */
#define GW_EUNSUPPORTED 6  /* feature dimension or precision not supported */
#define GW_ECANCELED 7     /* a server request was cancelled (gw_server_cancel) */

/* cost-tile precision of the softmin / plan kernels.  The log-sum-exp, the
 * potentials and all accumulations stay float32 (Gamma and energies float64)
 * in every mode. */
#define GW_PREC_FP32 0     /* FP32 dot products on the CUDA cores */
#define GW_PREC_BF16 1     /* BF16 operands on tcgen05, FP32 accumulate (a speed reference:
                            * its exponent error grows as 1 / eps; with D + 3 > 80 its plan
                            * sums run in FP32 on the exact features) */
#define GW_PREC_BF16X3 2   /* split BF16 (hi*hi + hi*lo + lo*hi) on tcgen05 */
#define GW_PREC_F16X3 3    /* split FP16 with scaling (hi*hi + hi*lo + lo*hi) on tcgen05 */
#define GW_PREC_FP8 4      /* E4M3 features on tcgen05 (kind::f8f6f4): each feature matrix
                            * rounded under one power-of-two scale per 128-row group (the
                            * same rounding in the row and column softmins and the plan
                            * sums), the rank-one, bias and shift columns as split BF16 in
                            * the same FP32 accumulator, 16 log2(e) / eps applied in the
                            * epilogue.  The softmin takes K <= 128; the plan sums, the
                            * solve and the energy take D <= 77 (GW_EUNSUPPORTED beyond,
                            * where no plan kernel rounds the same features).
                            * A measured mode: e4m3's 3 mantissa bits move the
                            * exponent by whole log2 units already at eps = 0.1 on
                            * unit-scale features (the error is stated per eps beside the
                            * other modes); not an accuracy-preserving form. */

/* CNT penalties accepted by gw_lift (Section 2, "Embeddable costs") */
#define GW_PEN_SQEUCLID 0  /* ||x - x'||^2: the lift is a centering */
#define GW_PEN_POWER 1     /* ||x - x'||^p, 0 < p <= 2, p = param */
#define GW_PEN_GAUSS 2     /* 2 (1 - exp(-||x - x'||^2 / (2 param^2))) */

/* workspace queries (gw_workspace_size's `op`) */
#define GW_OP_SOFTMIN 0
#define GW_OP_CROSS_COV 1
#define GW_OP_ENERGY 2
#define GW_OP_SOLVE 3
#define GW_OP_LIFT 4
#define GW_OP_GRAD 5
#define GW_OP_COARSEN 6  /* gw_workspace_size(GW_OP_COARSEN, n points, k clusters, D, 1, 0) */
#define GW_OP_ITERATION 7 /* gw_sinkhorn_iteration(n, m, K): both half-steps */

#define GW_MAX_FEATURES 128 /* largest D, E (and K) the kernels accept */

/* Layout of the float64 energy record written by gw_energy and gw_solve. */
#define GW_EN_E 0          /* L + eps KL  (objective of Eq. entropic_gromov_wasserstein) */
#define GW_EN_L 1          /* C - 8 ||Gamma_{t+1}||^2 - 4 T  (Lemma, Appendix C.1) */
#define GW_EN_KL 2         /* KL(pi | a x b) */
#define GW_EN_C 3          /* C(alpha, beta) of the Lemma */
#define GW_EN_GAMMA2 4     /* ||Gamma_{t+1}||_F^2 */
#define GW_EN_T 5          /* T = sum_ij pi_ij s_i t_j */
#define GW_EN_ROW_L1 6     /* ||pi 1 - a||_1 */
#define GW_EN_COL_L1 7     /* ||pi^T 1 - b||_1 */
#define GW_EN_ROW_RELMAX 8 /* max_i |(pi 1)_i - a_i| / a_i */
#define GW_EN_COL_RELMAX 9 /* max_j |(pi^T 1)_j - b_j| / b_j */
#define GW_EN_MASS 10      /* sum_ij pi_ij */
#define GW_EN_DGAMMA 11    /* ||Gamma_{t+1} - Gamma_t||_F */
#define GW_EN_EPS 12       /* eps used */
#define GW_EN_STATUS 13    /* 0, GW_ENONFINITE when a term is not finite, or
                              (gw_solve) GW_ETIMEOUT when a bounded wait gave up */
#define GW_EN_NINNER 14    /* gw_solve: Sinkhorn iterations run in this outer step */
#define GW_EN_STOPERR 15   /* gw_solve: Err of the stop rule's last check, -1 if none */
#define GW_EN_LEN 16

/*
 * gw_sinkhorn_softmin -- one Sinkhorn half-step on the bilinear cost
 * (discrete Sinkhorn operator, Eq. sinkhorn_operators; the loop bodies of
 * Algorithms 2 and 3):
 *
 *   out_i = -eps * log sum_j exp( logw_j + (h_j + 16 <A_i, B_j> + 4 sA_i sB_j) / eps )
 *
 * and, when avg_with != NULL, the Jacobi average of Algorithm 3,
 *   out_i = (avg_with_i + out_i) / 2.
 * Row update (f): A = X, B = V = Gamma Y (rows V_j = Gamma Y_j), sA = s,
 *   sB = t, h = g, logw = log b.  Column update (g): A = V, B = X, sA = t,
 *   sB = s, h = f, logw = log a.
 *   A: n x K, B: m x K (row-major float32), sA, out, avg_with: n; sB, h, logw: m.
 *   avg_with may alias out.  logw_j = -inf (zero weight) is allowed.
 *   1 <= K <= GW_MAX_FEATURES, m >= 1, n >= 0 (n == 0 is a no-op), eps > 0.
 *   prec: GW_PREC_*.  Tensor-core modes need 6 + K (BF16) or 6 + 3K (BF16X3,
 *   F16X3) <= 192 and |exponent| < 1e9 (base 2) for real cells.
 * Errors: GW_EINVAL, GW_ENOMEM, GW_EUNSUPPORTED, GW_ECUDA.
 */
int gw_sinkhorn_softmin(const float* A, const float* B, const float* sA, const float* sB,
                        const float* h, const float* logw, float eps, int64_t n, int64_t m,
                        int K, int prec, const float* avg_with, float* out, void* ws,
                        size_t ws_bytes, gw_stream_t stream);

/*
 * gw_sinkhorn_softmin_noalloc -- gw_sinkhorn_softmin for callers that cannot
 * allocate device memory.  The paper has no counterpart; this is a service
 * of the library.
 *
 * Some callers can't call cudaMalloc or pass a workspace: runtimes that
 * reserve all device memory up front and forbid allocation afterwards, host
 * code that runs where an allocation's implicit device synchronisation is
 * not allowed, and plug-in hosts that give their plug-ins no allocator.  This
 * entry point takes the same arguments as gw_sinkhorn_softmin minus the
 * workspace and computes the same result with the same kernels; its scratch
 * (the per-split partial maxima and sums) lives in a 2 MiB static device
 * array inside the library, which every GPU that loads the library holds
 * until the process exits.  It calls no allocating function.
 *   - Sizes whose scratch exceeds 2 MiB (gw_workspace_size(GW_OP_SOFTMIN,
 *     ...) > 2 MiB, e.g. n above ~131k when the columns are split) return
 *     GW_ENOMEM with the sizes in gw_last_error().
 *   - The first call on a device looks up the array's device address with
 *     that device current; make that first call before any stream capture.
 *     The current device must be the device of `stream`.  The address is
 *     kept for the life of the process and is not looked up again after a
 *     cudaDeviceReset: do not call this entry point after resetting a device.
 *   - All calls on a device share the one array: calls that overlap on the
 *     GPU (different streams, or host threads) race and give wrong results.
 *     Serialise them, e.g. on one stream.
 *   - The array keeps the last call's contents; nothing in it needs to start
 *     at zero.
 *   Only GW_PREC_FP32.  Errors: GW_EINVAL, GW_ENOMEM, GW_EUNSUPPORTED, GW_ECUDA.
 */
int gw_sinkhorn_softmin_noalloc(const float* A, const float* B, const float* sA,
                                const float* sB, const float* h, const float* logw, float eps,
                                int64_t n, int64_t m, int K, int prec, const float* avg_with,
                                float* out, gw_stream_t stream);

/*
 * gw_cross_cov -- the plan-weighted reduction of Algorithm 1 (its Xtilde and
 * Gamma_{t+1} lines; Theorem 3.3): with pi built from (f, g) on c_{Gamma_t}
 * at temperature eps,
 *   W_j         = sum_i pi_ij [X_i, s_i, 1]               (float32 -> float64)
 *   Gamma_out   = sum_j W_j[0:D] Y_j^T = sum_ij pi_ij X_i Y_j^T   (D x E float64)
 *   stats[0]    = T = sum_ij pi_ij s_i t_j
 *   stats[1]    = sum_j g_j (pi^T 1)_j
 *   stats[2]    = sum_ij pi_ij
 *   stats[3]    = ||pi^T 1 - b||_1
 *   stats[4]    = max_j |(pi^T 1)_j - b_j| / b_j
 *   (stats: device, 8 float64).  W_opt (m x (D+2) float64, or NULL) receives
 *   W.  X: n x D, Y: m x E, s, a, f: n; t, b, g: m; Gamma_t: D x E float64.
 *   a, b must be > 0 (their logs enter the exponent).
 * Errors: GW_EINVAL, GW_ENOMEM, GW_EUNSUPPORTED, GW_ECUDA.
 */
int gw_cross_cov(const float* X, const float* Y, const float* s, const float* t,
                 const float* a, const float* b, const float* f, const float* g,
                 const double* Gamma_t, float eps, int64_t n, int64_t m, int D, int E,
                 int prec, double* Gamma_out, double* stats, double* W_opt, void* ws,
                 size_t ws_bytes, gw_stream_t stream);

/*
 * gw_energy -- energy terms of the plan encoded by (f, g) on c_{Gamma_t}
 * (Lemma in Appendix C.1; Eq. entropic_gromov_wasserstein):
 *   C(alpha,beta) from the centered moments of X and Y,
 *   L = C - 8 ||Gamma_{t+1}||^2 - 4 T,
 *   eps KL = sum_i f_i (pi 1)_i + sum_j g_j (pi^T 1)_j + 16 <Gamma_t, Gamma_{t+1}> + 4 T,
 *   E = L + eps KL,
 * with (pi 1)_i = a_i exp((f_i - S_b(g)_i)/eps) from one extra row softmin.
 * Writes GW_EN_LEN float64 values (layout GW_EN_*) to `energy` (device) and
 * Gamma_{t+1} to Gamma_out (device, D x E float64, may be NULL).
 * X, Y must be centered (sum a X = 0, sum b Y = 0).
 * Errors: GW_EINVAL, GW_ENOMEM, GW_EUNSUPPORTED, GW_ECUDA.
 */
int gw_energy(const float* X, const float* Y, const float* s, const float* t, const float* a,
              const float* b, const float* f, const float* g, const double* Gamma_t, float eps,
              int64_t n, int64_t m, int D, int E, int prec, double* energy, double* Gamma_out,
              void* ws, size_t ws_bytes, gw_stream_t stream);

/* Problem and options of gw_solve (Algorithm 1 with Algorithm 3). */
typedef struct gw_problem {
  const float* X;  /* n x D centered features */
  const float* Y;  /* m x E centered features */
  const float* s;  /* n squared norms ||X_i||^2 */
  const float* t;  /* m squared norms ||Y_j||^2 */
  const float* a;  /* n weights (> 0, sum 1) */
  const float* b;  /* m weights (> 0, sum 1) */
  int64_t n, m;
  int D, E;
} gw_problem;

typedef struct gw_options {
  float eps;          /* temperature of the first outer step (> 0) */
  float eps_final;    /* <= 0: constant eps; else geometric eps_t from eps to eps_final */
  int n_outer;        /* outer (Gamma) steps, >= 1 */
  int n_inner;        /* Sinkhorn iterations per outer step, >= 1 */
  int symmetric;      /* 1: Algorithm 3 (Jacobi averaging); 0: Algorithm 2 */
  int prec;           /* GW_PREC_* for the cost tiles */
  int record;         /* 1: energy record after every outer step into history */
  int use_graph;      /* 1: capture the whole solve as one CUDA graph; 2: per outer step,
                       * run the first Sinkhorn iteration directly and replay the others
                       * from a graph of up to 10 iterations captured for that step (the
                       * host enqueues O(n_outer) work instead of O(n_outer n_inner));
                       * 0: direct launches.  All three enqueue the same kernels with the
                       * same arguments: results are bitwise equal.  Graphs need a
                       * non-null stream (else direct launches). */
  const double* Gamma0; /* D x E initial map, NULL = 0 (the start of Algorithm 1) */
  const float* f0;    /* initial potentials (warm start), NULL = 0 */
  const float* g0;
  /* Algorithm 6 (Appendix B.4) applied to CNT-GW: 1 = n_inner is the initial
     count, doubled (up to n_inner_max) after every outer step whose energy E
     exceeds the previous step's by more than adapt_rtol * |E_prev|
     (adapt_rtol = 0 is the paper's strict test). */
  int adaptive;
  int n_inner_max;    /* cap of the adaptive count (<= 0: n_inner) */
  float adapt_rtol;   /* >= 0 */
  /* Hybrid stop (Appendix D.1): > 0 = after every stop_every-th iteration,
     end the outer step's Sinkhorn loop once Err (Appendix A) of the plan that
     iteration measured is below stop_tol: (f^n, g^n) for Algorithm 3,
     (f^{n+1}, g^n) for Algorithm 2.  n_inner stays the maximum. */
  float stop_tol;
  int stop_every;
  /* Checkpoint / resume (the warm start of Appendix B.1 across calls): the
     call runs outer steps outer_offset .. outer_offset + n_outer - 1 of an
     eps schedule of outer_total steps (outer_total <= 0: n_outer, offset 0).
     A solve split into consecutive calls, each started from the previous
     call's Gamma, f and g (Gamma0, f0, g0 = its result), runs the same
     kernels on the same values as one call over all steps: its final
     record is bitwise the same.  (Algorithm 6's doubled count is not
     carried across calls.) */
  int outer_offset;
  int outer_total;
} gw_options;

typedef struct gw_result {
  double* Gamma;      /* out: D x E, the last Gamma_{t+1} */
  double* Gamma_plan; /* out or NULL: D x E, the Gamma_t whose cost c_{Gamma_t} encodes the
                         final plan together with (f, g) */
  float* f;           /* out: n potentials */
  float* g;           /* out: m potentials */
  double* energy;     /* out: GW_EN_LEN energy record of the last plan */
  double* history;    /* out or NULL: n_outer x GW_EN_LEN records (needs record = 1) */
} gw_result;

/*
 * gw_solve -- CNT-GW (Algorithm 1) on device: for t = 0..n_outer-1,
 *   V = Gamma_t Y; n_inner symmetrized (or standard) Sinkhorn iterations on
 *   c_{Gamma_t} at eps_t, warm-started from the previous potentials;
 *   Gamma_{t+1} = sum_ij pi_ij X_i Y_j^T; energy record of pi_{t+1}.
 * All outputs are device buffers owned by the caller; nothing is read back
 * to the host.  Asynchronous on `stream`, except with adaptive = 1 or
 * stop_tol > 0: those decisions are taken on the host, which waits for each
 * outer step's energy (adaptive) or each stop check (and no CUDA graph is
 * used).  Records carry the iterations run (GW_EN_NINNER) and the last
 * checked Err (GW_EN_STOPERR).
 * Errors: GW_EINVAL, GW_ENOMEM, GW_EUNSUPPORTED, GW_ECUDA.
 */
int gw_solve(const gw_problem* p, const gw_options* o, gw_result* r, void* ws, size_t ws_bytes,
             gw_stream_t stream);

/*
 * gw_lift -- embeddings feeding Algorithm 1 (Section 5, "CNT Embeddings";
 * Appendix B.2).
 *   GW_PEN_SQEUCLID: X = x - sum_i w_i x_i (D must equal d; Section 3 example).
 *   GW_PEN_POWER / GW_PEN_GAUSS: Kernel PCA of the kernel of Prop. 2.3,
 *     centered as in Algorithm 4, computed matrix-free by block subspace
 *     iteration (n_iter iterations, 0 = default) with Rayleigh-Ritz:
 *     X = V sqrt(Lambda) for the D largest eigenpairs.  Each eigenvector's
 *     entry of largest magnitude is made positive.
 *   x: n x d raw points (float32); w: n weights or NULL (uniform).
 *   Outputs: X (n x D), sqn (n) = ||X_i||^2, basis_opt (n x D, V) and
 *   eigvals_opt (D, Lambda) may be NULL.  `seed` seeds the start block.
 *   Asynchronous on `stream` like the other calls: every step, the small
 *   r x r Cholesky, triangular inverse and Rayleigh-Ritz eigen-solve
 *   included, runs on the device, and nothing is read back (a first call
 *   outside any stream capture sets the kernels' shared-memory limits; later
 *   calls may be captured).  A degenerate block (the Gram matrix of a
 *   subspace iterate not positive definite, e.g. from NaN points) leaves X,
 *   sqn (and basis_opt) as NaN, which a solve on them reports as
 *   GW_ENONFINITE.
 * Errors: GW_EINVAL, GW_ENOMEM, GW_EUNSUPPORTED, GW_ECUDA.
 */
int gw_lift(const float* x, int64_t n, int d, const float* w, int kind, float param, int D,
            int n_iter, uint64_t seed, float* X, float* sqn, float* basis_opt,
            float* eigvals_opt, void* ws, size_t ws_bytes, gw_stream_t stream);

/*
 * gw_grad_x -- gradient of the EGW energy with respect to the source points
 * through the converged plan (envelope theorem, Appendix B.6):
 *   dX_i = 8 a_i [(s_i + m2_X) X_i + 2 Sigma_X X_i - mu3_X] - 8 a_i m2_Y X_i
 *          - 16 Gamma_pi w_i - 8 q_i X_i,
 *   w_i = sum_j pi_ij Y_j, q_i = sum_j pi_ij t_j (pi from f, g on c_{Gamma_t}),
 *   then the adjoint of the centering, dX_i <- dX_i - a_i sum_k dX_k.
 *   If x != NULL (lifted features, Algorithm 12), additionally
 *   dx_i = sum_d dX_id grad_x Pi_d(x_i) with Kernel-Proj (Algorithm 13)
 *   frozen at the training points x (n x dx_dim), basis V (n x D) and
 *   eigvals Lambda (D), for the penalty (kind, param).
 *   For squared features (x == NULL) dx may equal NULL and dX is the answer.
 * Errors: GW_EINVAL, GW_ENOMEM, GW_EUNSUPPORTED, GW_ECUDA.
 */
int gw_grad_x(const gw_problem* p, const float* f, const float* g, const double* Gamma_t,
              const double* Gamma_pi, float eps, int prec, const float* x, int dx_dim, int kind,
              float param, const float* basis, const float* eigvals, float* dX, float* dx,
              void* ws, size_t ws_bytes, gw_stream_t stream);

/*
 * gw_sinkhorn_iteration -- one Sinkhorn iteration on c_Gamma, both halves in
 * one launch, as gw_solve runs it (Algorithm 3: f' = (f + S_b(g))/2,
 * g' = (g + S_a(f))/2; Algorithm 2 with symmetric = 0: f' = S_b(g),
 * g' = S_a(f')).  Cost c_ij = -16 <X_i, V_j> - 4 s_i t_j with V = Gamma Y
 * (m x K); loga = log a (n), logb = log b (m); f, g in, f_out, g_out out (all
 * device; f_out / g_out must not alias f / g).  f and g double as the shift
 * estimates of the tensor-core forms.  reuse = 1: X, V, s, t, eps and prec
 * are those of the previous call on the same workspace, which the caller has
 * left untouched, so the tensor-core forms keep their 16-bit operands and
 * refresh only the potential columns (how gw_solve runs the iterations of an
 * outer step).  Enqueued on `stream`.  Workspace: GW_OP_ITERATION.
 */
int gw_sinkhorn_iteration(const float* X, const float* V, const float* s, const float* t,
                          const float* loga, const float* logb, const float* f, const float* g,
                          float* f_out, float* g_out, float eps, int64_t n, int64_t m, int K,
                          int prec, int symmetric, int reuse, void* ws, size_t ws_bytes,
                          gw_stream_t stream);

/*
 * gw_coarsen -- Coarsen of Multiscale-GW (Appendix B.5): K-Means of the
 * features X (n x D, weights a; NULL = uniform) by Lloyd's iterations from
 * the k caller-given point indices init_idx (device, int64), ties to the
 * lowest centroid index, n_iter update rounds followed by a last assignment
 * and update.  Writes the non-empty clusters in order: centroids Xc (k x D),
 * aggregated weights ac (k), squared norms sc (k), their count to *h_k_out
 * (host), and, when assign (device, n) is not NULL, each point's cluster in
 * that order (from the last assignment).  Weights must be non-negative.  An
 * index of init_idx outside [0, n) returns GW_EINVAL (checked on the device,
 * nothing is read out of bounds).  Workspace: GW_OP_COARSEN.  Synchronous.  Cluster sums use 64-bit fixed point with
 * integer atomics, so the result is bitwise reproducible.
 * Errors: GW_EINVAL, GW_ENOMEM, GW_ECUDA.
 */
int gw_coarsen(const float* X, const float* a, int64_t n, int D, const int64_t* init_idx,
               int64_t k, int n_iter, float* Xc, float* ac, float* sc, int* assign,
               int64_t* h_k_out, void* ws, size_t ws_bytes, gw_stream_t stream);

/*
 * gw_multiscale -- Multiscale-GW (Algorithm 7): coarsen both measures
 * (gw_coarsen with init_x (kx indices) / init_y (ky indices) and km_iter
 * rounds), CNT-GW on the coarse measures with options `coarse` (Gamma0 /
 * f0 / g0 honoured, record ignored), Interpolate (Algorithm 8: one softmin per
 * side at the fine solve's first eps, with the coarse Gamma), then CNT-GW on
 * the fine measures with options `fine`, started from Gamma^c and the
 * interpolated potentials (its Gamma0 / f0 / g0 are replaced).  Results as
 * gw_solve; coarse_energy (device, GW_EN_LEN, may be NULL) receives the
 * coarse solve's final record.  Synchronous up to the fine solve, which is
 * enqueued on `stream`.  Workspace: gw_multiscale_workspace_size().
 */
int gw_multiscale(const gw_problem* p, const gw_options* coarse, const gw_options* fine,
                  const int64_t* init_x, int64_t kx, const int64_t* init_y, int64_t ky,
                  int km_iter, gw_result* r, double* coarse_energy, void* ws, size_t ws_bytes,
                  gw_stream_t stream);
size_t gw_multiscale_workspace_size(int64_t n, int64_t m, int D, int E, int64_t kx, int64_t ky,
                                    int prec);

/*
 * gw_transfer -- color / UV transfer (Appendix E): the barycentric projection
 *   out_j = sum_i pi_ij U_i / b_j  of source attributes U (n x k, device,
 *   1 <= k <= 16) through the plan pi_ij = a_i b_j exp((f_i + g_j - c_ij)/eps)
 *   on c_{Gamma_t} (the state gw_solve returns: f, g, Gamma_plan).  out (m x k,
 *   device); mass (m, device, may be NULL) receives the column sums of pi.
 *   Enqueued on `stream`; deterministic.
 * Workspace: gw_transfer_workspace_size(n, m, D, k).
 * Errors: GW_EINVAL, GW_ENOMEM, GW_EUNSUPPORTED, GW_ECUDA.
 */
int gw_transfer(const gw_problem* p, const float* f, const float* g, const double* Gamma_t,
                float eps, const float* U, int k, float* out, float* mass, void* ws,
                size_t ws_bytes, gw_stream_t stream);
size_t gw_transfer_workspace_size(int64_t n, int64_t m, int D, int k);

/*
 * gw_kernel_gw -- Kernel-GW (Algorithm 5, Appendix B.3): the exact
 * kernelised EGW scheme for small N with dense matrices.  CX (n x n) and
 * CY (m x m): CNT cost matrices (device, FP32, row-major); a, b: weights.
 * K^X, K^Y = Algorithm 4 (base index 0, weighted double centering); pi^0 =
 * a b^T; each outer step: C = -4 K^X_ii K^Y_jj - 16 K^X pi K^Y, n_inner
 * Sinkhorn iterations on C (Algorithm 3, or 2 with symmetric = 0), warm
 * started, then pi = a b^T exp((f + g - C)/eps).  Options used: eps,
 * eps_final, n_outer, n_inner, symmetric, record, f0, g0 (prec, Gamma0 and
 * the adaptive / stop fields are ignored).  The two dense products per step
 * run on the tensor cores at FP32 accuracy (split f16 operands, three
 * products per term, FP32 accumulation), in this library's own kernel.
 * Outputs (device): pi
 * (n x m), f, g, energy (GW_EN_LEN record of the final plan, Lemma in kernel
 * form), history (n_outer x GW_EN_LEN when record = 1).  Enqueued on
 * `stream`.  Memory: O(n m + n^2 + m^2), n m <= 2^31.
 * Workspace: gw_kernel_gw_workspace_size(n, m).
 */
int gw_kernel_gw(const float* CX, const float* CY, const float* a, const float* b, int64_t n,
                 int64_t m, const gw_options* o, float* pi, float* f, float* g, double* energy,
                 double* history, void* ws, size_t ws_bytes, gw_stream_t stream);
size_t gw_kernel_gw_workspace_size(int64_t n, int64_t m);

/*
 * gw_sgw -- Sinkhorn GW divergence (Section 4.1):
 *   SGW_eps(alpha, beta) = GW_eps(alpha, beta) - (GW_eps(alpha, alpha) + GW_eps(beta, beta)) / 2,
 * each GW_eps the final energy E (GW_EN_E) of a gw_solve with options `o`
 * (record ignored; Gamma0 / f0 / g0 apply to the alpha-beta solve only, the
 * two self solves start from zero).  Writes sgw (device, 4 doubles): SGW,
 * GW(alpha,beta), GW(alpha,alpha), GW(beta,beta); records (device,
 * 3 x GW_EN_LEN, may be NULL): the three final energy records.
 * Gradient (dX not NULL): d SGW / d X (n x D, device) with every plan held at
 * its optimum (envelope theorem, Appendix B.6) at the schedule's last eps;
 * the self term is differentiated through both of its sides.  With x (raw
 * points, n x dx_dim) and the lift's basis/eigvals also d SGW / d x into dx,
 * as gw_grad_x.  Enqueued on `stream` (the three solves in sequence).
 * Workspace: gw_sgw_workspace_size(n, m, D, E, prec, want_grad, dx_dim).
 * Errors: as gw_solve and gw_grad_x.
 */
int gw_sgw(const gw_problem* p, const gw_options* o, double* sgw, double* records, float* dX,
           const float* x, int dx_dim, int kind, float param, const float* basis,
           const float* eigvals, float* dx, void* ws, size_t ws_bytes, gw_stream_t stream);
size_t gw_sgw_workspace_size(int64_t n, int64_t m, int D, int E, int prec, int want_grad,
                             int dx_dim);

/*
 * gw_solve_batch -- many small CNT-GW problems in one persistent launch
 * (Algorithm 1 with the symmetric Sinkhorn loop of Algorithm 3, or
 * Algorithm 2 when symmetric == 0; FP32 softmins on the CUDA cores, FP64
 * cross-covariance and energy, the math of gw_solve's GW_PREC_FP32 path).
 *   Problem q owns sources [xo[q], xo[q+1]) and targets [yo[q], yo[q+1]) of
 *   packed arrays: X ((sum n) x D), s, a, f per source; Y ((sum m) x E),
 *   t, b, g per target.  xo, yo: nprob + 1 non-decreasing int64 offsets
 *   (device).  eps0[q] > 0 (device); eps1 NULL (constant eps) or eps1[q] > 0,
 *   the geometric schedule of gw_solve's eps_final.  Every problem starts
 *   from f = g = 0, Gamma = 0 and runs n_outer x n_inner iterations.
 *   Outputs (device): f, g (packed like s, t), Gamma and Gamma_plan
 *   (nprob x D x E float64: the last update and the Gamma of the last plan,
 *   as gw_result), energy (nprob x GW_EN_LEN: the record of the last plan),
 *   history (NULL, or nprob x n_outer x GW_EN_LEN: every outer step).
 *   A device work queue hands problems to CTAs; each problem is solved by one
 *   CTA entirely in shared memory, so results do not depend on the batch
 *   (bitwise).  Sizes: 1 <= D, E <= 4; n_max, m_max (host) bound every
 *   problem's n and m and size the shared memory, which must hold
 *   (n_max + m_max) (D + 7) floats plus padding (about 7000 points in all at
 *   D = 2); a problem outside the bounds (or with n or m = 0, or an eps0 /
 *   eps1 that is not finite and > 0) gets a record of NaN terms with
 *   GW_EINVAL in GW_EN_STATUS, and its other outputs are left untouched.
 * Workspace: gw_solve_batch_workspace_size() bytes (the queue counter),
 *   256-byte aligned.
 * Errors: GW_EINVAL (nprob < 1, n_outer / n_inner < 1, a null pointer),
 *   GW_EUNSUPPORTED (D or E outside 1..4, sizes that do not fit), GW_ENOMEM,
 *   GW_ECUDA.
 */
int gw_solve_batch(int nprob, const int64_t* xo, const int64_t* yo, int64_t n_max, int64_t m_max,
                   int D, int E, const float* X, const float* Y, const float* s, const float* t,
                   const float* a, const float* b, const float* eps0, const float* eps1,
                   int n_outer, int n_inner, int symmetric, float* f, float* g, double* Gamma,
                   double* Gamma_plan, double* energy, double* history, void* ws,
                   size_t ws_bytes, gw_stream_t stream);
size_t gw_solve_batch_workspace_size(void);

/*
 * Request server (continuous batching; no counterpart in the paper, which
 * solves one problem at a time).  Requests are admitted in arrival order as
 * soon as a worker slot is free and their device memory fits in the pool the
 * caller gives at creation (the server allocates no device memory).  Each
 * admitted request runs on its own stream: copy in, gw_lift, gw_solve as one
 * CUDA graph, energy record out; admitted requests overlap on the device.
 * Results are deterministic: the same request gives the same record alone
 * or among others.  Weights are uniform.  Host arrays are copied at submit.
 */
typedef struct gw_server gw_server;

typedef struct gw_request {
  uint64_t id;          /* caller's tag, also seeds the Kernel PCA start block */
  int64_t n, m;         /* source / target points */
  int d;                /* point dimension (1..4) */
  int kind;             /* GW_PEN_* */
  float param;          /* penalty parameter */
  int D;                /* feature dimension for lifted penalties */
  float eps, eps_final; /* temperature schedule (eps_final <= 0: constant) */
  int n_outer, n_inner;
  int prec;             /* GW_PREC_*; requests with n * m < 8e6 run the FP32 kernels (faster
                           there, and at least as accurate) */
} gw_request;

typedef struct gw_response {
  uint64_t id;
  int status;                 /* GW_OK or an error code */
  double energy[GW_EN_LEN];   /* energy record of the final plan */
  double t_submit, t_admit, t_done;   /* seconds on a monotonic host clock (t_admit: the
                                         first admission) */
  int preempted;              /* times the request was checkpointed and re-queued */
} gw_response;

/* pool: 256-byte aligned device buffer owned by the caller; max_active:
 * worker slots (1..256); device: CUDA ordinal the workers use.  NULL on error. */
gw_server* gw_server_create(void* pool, size_t pool_bytes, int max_active, int device);
/* Queue a request (h_x: n x d, h_y: m x d, host float32, copied).  GW_ENOMEM
 * if the request can never fit in the pool. */
int gw_server_submit(gw_server* s, const gw_request* r, const float* h_x, const float* h_y);
/* Time slicing with checkpoint / resume: an admitted request runs at most
 * outer_steps outer steps at a time (0, the default: all of them).  When a
 * slice ends while other requests wait for admission, the request is
 * checkpointed — its lifted features and solver state (Gamma_t, f, g) are
 * copied to host memory and its device memory and slot released — and
 * queued again behind them; readmitted, it resumes from that state through
 * gw_solve's outer_offset, with the same result as an uninterrupted run.
 * Applies to requests admitted after the call. */
int gw_server_set_slice(gw_server* s, int outer_steps);
/* Batch lane (on by default): small squared-penalty requests (d <= 4,
 * n m <= 1.5e6, both clouds in one CTA's shared memory) skip the worker
 * slots; those waiting when the lane is free (the same d, n_outer, n_inner)
 * are solved together in one gw_solve_batch launch, one CTA each, on the
 * lane's own thread and stream, after a per-problem centering on the device.
 * Results: gw_solve_batch's (FP32 arithmetic), independent of the batch.
 * on = 0 sends every request through the slots (gw_solve). */
int gw_server_set_batching(gw_server* s, int on);
/* Cancel request `id`: a pending request is answered at once, a running one
 * at its next slice boundary (with time slicing; without it, when its solve
 * ends), in both cases with status GW_ECANCELED.  GW_EINVAL if no request
 * with that id is in flight. */
int gw_server_cancel(gw_server* s, uint64_t id);
/* Host watchdog: a request not finished `seconds` after its submission
 * (<= 0: no limit, the default) is stopped at its next slice boundary, or
 * instead of being admitted, and answered with GW_ETIMEOUT.  With time
 * slicing every slice ends with a stream synchronisation, so the check
 * follows the request's progress on the device (its heartbeat). */
int gw_server_set_deadline(gw_server* s, double seconds);
/* Move up to max_out finished responses to out.  wait_ms: 0 = do not wait,
 * < 0 = wait until one is ready or nothing is in flight, > 0 = bounded wait.
 * Returns the number written. */
int gw_server_poll(gw_server* s, gw_response* out, int max_out, int wait_ms);
/* Device bytes the server reserves in its pool for this request. */
size_t gw_server_request_bytes(const gw_request* r);
/* Requests waiting for admission and requests running. */
int gw_server_stats(gw_server* s, int* pending, int* active);
/* Finish the running requests, drop the pending ones, free the server. */
void gw_server_destroy(gw_server* s);

/* Bytes of workspace `op` needs for these sizes (0 on invalid arguments). */
size_t gw_workspace_size(int op, int64_t n, int64_t m, int D, int E, int prec);

/* Description of the last error on this host thread ("" if none). */
const char* gw_last_error(void);

/* Library version, major * 10000 + minor * 100 + patch. */
int gw_version(void);

/* Number of kernels this library has enqueued in the process (kernels
 * captured into a CUDA graph count once, at capture).  reset != 0 returns the
 * count and sets it to zero.  Diagnostic only. */
unsigned long long gw_kernel_launches(int reset);

/*
 * Bounded device waits (failure detection).  The tensor-core kernels run a
 * pipeline of copy, MMA and epilogue roles inside each CTA that wait on one
 * another through shared-memory barriers.  No wait is unbounded: a wait that
 * has not been satisfied after the limit below (nanoseconds of the GPU's
 * global timer; default 2 s) gives up, the CTA waits (at most 2 s more) for
 * its own copies and MMAs already in flight, frees its tensor memory, writes
 * NaN for its rows and adds 1 to a per-device counter.  The context stays
 * usable.  Because the potentials then hold NaN, a solve's energy record
 * reports it: gw_solve sets GW_EN_STATUS to GW_ETIMEOUT when the counter
 * moved during the call (a give-up in a call that ran at the same time on
 * another stream of the device is attributed to both).  The tensor-core
 * plan sums recompute their partials on the CUDA cores instead.
 *
 * gw_set_wait_limit_ns: limit for kernels enqueued after the call (process-
 *   wide; kernels already captured in a CUDA graph keep theirs).  1 ns ..
 *   600 s, else GW_EINVAL.  A limit far below a kernel's run time makes its
 *   waits give up: that is how the failure path is exercised.
 * gw_wait_limit_ns: the current limit.
 * gw_wait_status: synchronizes the current device, then returns GW_ETIMEOUT
 *   if its counter is non-zero (else GW_OK); reset != 0 sets it to zero.
 *   The counter's address is looked up once per device and kept for the
 *   life of the process (not again after a cudaDeviceReset).
 */
int gw_set_wait_limit_ns(unsigned long long ns);
unsigned long long gw_wait_limit_ns(void);
int gw_wait_status(int reset);

/*
 * gw_probe_ex2 -- measurement aid, not part of the method: enqueues one
 * kernel of `blocks` x 512 threads in which every thread evaluates 8
 * independent register chains x <- 2^-x with ex2.approx (the instruction
 * the softmin epilogue spends one of per cell), `iters` x 4 steps each.
 * *h_ops receives the number of exponentials the launch evaluates; timing
 * the launch (CUDA events on `stream`) gives the measured exponential
 * throughput that bounds the softmin.  out: blocks x 512 floats (device).
 * Errors: GW_EINVAL, GW_ECUDA.
 */
int gw_probe_ex2(int blocks, int iters, float* out, unsigned long long* h_ops, gw_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* GW_H_ */
