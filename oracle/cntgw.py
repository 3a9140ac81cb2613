"""FP64 CPU oracle of CNT-GW (arXiv 2602.06658), written from the paper.

TEST INFRASTRUCTURE ONLY: imported by tests, smoke() and bench.py's cpu
baseline leg; never by the product path.

Conventions (the paper's notation):
  * alpha = sum_i a_i delta_{x_i}, beta = sum_j b_j delta_{y_j}  (Section 5,
    "Notations"); X (N x D) and Y (M x E) are centered embeddings,
    sum_i a_i X_i = 0, c_X(x_i, x_k) = ||X_i - X_k||^2 (Eqs. embedding_X/Y).
  * s_i = ||X_i||^2, t_j = ||Y_j||^2.
  * The linear map Gamma is D x E.  The entropic OT problem solved at every
    outer step uses the bilinear cost of the Remark after Theorem 3.2
    (Eq. egw_otherform):  c_Gamma(i, j) = -16 X_i^T Gamma Y_j - 4 s_i t_j,
    at temperature eps.  Algorithm 1 states the same problem as Sinkhorn at
    eps/8 on ||Xbar_i - Zbar_j||^2; the two differ by a factor 8 and
    separable terms, which leave the plan unchanged.
  * Potentials f (N), g (M) encode the plan,
    pi_ij = a_i b_j exp((f_i + g_j - C_ij) / eps)   (Eq. sinkhorn_pi).
"""

from __future__ import annotations

import itertools
import math

import numpy as np

__all__ = [
    "pairwise_sqdist", "cnt_cost", "cnt_cost_grad1", "center", "sqnorms",
    "kernel_from_cost", "kernel_pca", "lift", "kernel_proj", "kernel_proj_vjp",
    "cost_gamma", "softmin", "softmin_bilinear_one", "sinkhorn", "plan",
    "marginal_error", "row_marginal_from_potentials",
    "gw_loss_bruteforce", "gw_constant_pairwise", "gw_constant_moments",
    "gw_loss_lemma", "kl_divergence", "egw_energy", "energy_from_potentials",
    "cross_covariance", "cnt_gw", "eps_schedule", "dual_function",
    "entropic_gw_step", "kernel_gw",
    "grad_features", "center_vjp", "grad_x_squared", "grad_x_lifted",
    "grad_x_bruteforce", "permutation_ot",
    "kmeans_coarsen", "kmeans_objective", "interpolate", "multiscale_gw", "sinkhorn_stop",
    "final_plan", "sgw", "sgw_grad_features", "barycentric_transfer",
]

F64 = np.float64


# --------------------------------------------------------------------------
# Costs and embeddings (Section 2 "Embeddable costs", Section 3 example,
# Appendix B.2 "Kernel matrices computations")
# --------------------------------------------------------------------------

def pairwise_sqdist(x, y):
    """||x_i - y_j||^2 for all pairs, by its definition."""
    x = np.asarray(x, F64)
    y = np.asarray(y, F64)
    diff = x[:, None, :] - y[None, :, :]
    return np.einsum("ijd,ijd->ij", diff, diff)


def cnt_cost(x, y, kind="sqeuclid", param=2.0):
    """Pairwise CNT cost matrix c(x_i, y_j) (Section 2, "Embeddable costs").

    kind = "sqeuclid": ||x - y||^2.
    kind = "power":    ||x - y||^p with p = param in (0, 2]; p = 1 is the
                       Euclidean cost of the paper's benchmarks (Section 6).
    kind = "gauss":    2 (1 - exp(-||x - y||^2 / (2 sigma^2))), sigma = param;
                       a squared RKHS distance, hence CNT (Theorem 2.2 (ii)).
    """
    d2 = pairwise_sqdist(x, y)
    if kind == "sqeuclid":
        return d2
    if kind == "power":
        return np.power(d2, param / 2.0)
    if kind == "gauss":
        return 2.0 * (1.0 - np.exp(-d2 / (2.0 * param * param)))
    raise ValueError(kind)


def cnt_cost_grad1(x, y, kind="sqeuclid", param=2.0):
    """Gradient of c(x, y_k) with respect to its first argument x (one point x
    of shape (d,), all y_k): returns (K, d).  Used by the gradient pins."""
    x = np.asarray(x, F64)
    y = np.asarray(y, F64)
    diff = x[None, :] - y
    d2 = np.einsum("kd,kd->k", diff, diff)
    if kind == "sqeuclid":
        return 2.0 * diff
    if kind == "power":
        p = param
        with np.errstate(divide="ignore", invalid="ignore"):
            coef = np.where(d2 > 0, p * np.power(d2, p / 2.0 - 1.0), 0.0)
        return coef[:, None] * diff
    if kind == "gauss":
        s2 = param * param
        return (2.0 / s2) * np.exp(-d2 / (2.0 * s2))[:, None] * diff
    raise ValueError(kind)


def center(x, a):
    """x - x_alpha with x_alpha = sum_i a_i x_i (Section 3, "Example")."""
    x = np.asarray(x, F64)
    a = np.asarray(a, F64)
    return x - a @ x


def sqnorms(X):
    X = np.asarray(X, F64)
    return np.einsum("nd,nd->n", X, X)


def kernel_from_cost(C, a):
    """Algorithm 4 (Kernel): K_ij = (C_i1 + C_1j - C_ij)/2 with base index 1
    (Prop. 2.3), then the weighted double centering that Algorithm 4 applies."""
    C = np.asarray(C, F64)
    a = np.asarray(a, F64)
    K = (C[:, :1] + C[:1, :] - C) / 2.0
    col = a @ K                 # sum_i a_i K_ij
    row = K @ a                 # sum_j a_j K_ij
    tot = a @ K @ a
    return K - col[None, :] - row[:, None] + tot


def kernel_pca(K, D):
    """Kernel PCA (Appendix B.2): the D largest eigenpairs (Lambda, V) of the
    centered kernel matrix and X_i = V_{i,1:D} sqrt(Lambda_{1:D}).

    Sign reading (the paper is silent): each eigenvector is flipped so that
    its entry of largest magnitude is positive.  Returns (X, V, lam)."""
    K = np.asarray(K, F64)
    lam, V = np.linalg.eigh(0.5 * (K + K.T))
    order = np.argsort(lam)[::-1][:D]
    lam = lam[order]
    V = V[:, order]
    for d in range(V.shape[1]):
        k = np.argmax(np.abs(V[:, d]))
        if V[k, d] < 0:
            V[:, d] = -V[:, d]
    lam_pos = np.clip(lam, 0.0, None)
    X = V * np.sqrt(lam_pos)[None, :]
    return X, V, lam


def lift(x, a, kind="sqeuclid", param=2.0, D=None):
    """The embedding step feeding Algorithm 1.

    Squared-Euclidean cost: X = x - x_alpha (Section 3, "Example").
    Other CNT costs: Kernel PCA of the kernel of Prop. 2.3 centered by
    Algorithm 4 (Section 5, "CNT Embeddings"; Appendix B.2).
    Returns dict(X, s, V, lam) (V, lam are None in the squared case)."""
    x = np.asarray(x, F64)
    a = np.asarray(a, F64)
    if kind == "sqeuclid" and D is None:
        X = center(x, a)
        return {"X": X, "s": sqnorms(X), "V": None, "lam": None}
    C = cnt_cost(x, x, kind, param)
    K = kernel_from_cost(C, a)
    X, V, lam = kernel_pca(K, D)
    return {"X": X, "s": sqnorms(X), "V": V, "lam": lam}


def _centered_kernel_row(xq, x, a, kind, param):
    """k~(xq, x_i) for all i: the kernel of Prop. 2.3 (base point x_1),
    centered against the training measure the way Algorithm 4 centers it.
    The terms that do not depend on xq are evaluated once from the training
    cost matrix."""
    x = np.asarray(x, F64)
    a = np.asarray(a, F64)
    xq = np.atleast_2d(np.asarray(xq, F64))
    C_qx = cnt_cost(xq, x, kind, param)            # (Q, N)
    C_q0 = C_qx[:, :1]                              # c(xq, x_1)
    C_xx = cnt_cost(x, x, kind, param)
    C_0x = C_xx[:1, :]                              # c(x_1, x_i)
    k_qx = (C_q0 + C_0x - C_qx) / 2.0               # k(xq, x_i)
    K = (C_xx[:, :1] + C_xx[:1, :] - C_xx) / 2.0    # k(x_l, x_i)
    col = a @ K                                     # sum_l a_l k(x_l, x_i)
    tot = a @ K @ a
    row_q = k_qx @ a                                # sum_l a_l k(xq, x_l)
    return k_qx - col[None, :] - row_q[:, None] + tot


def kernel_proj(xq, x, a, V, lam, kind="power", param=1.0):
    """Algorithm 13 (Kernel-Proj): Pi_X(xq)_d = Lambda_d^{-1/2}
    sum_i k(xq, x_i) V_{id}, with k the centered kernel (the centering of a
    moving point is our reading: the paper is silent)."""
    k = _centered_kernel_row(xq, x, a, kind, param)
    return (k @ V) / np.sqrt(lam)[None, :]


def kernel_proj_vjp(G, xq, x, a, V, lam, kind="power", param=1.0):
    """Vector-Jacobian product of Kernel-Proj at points xq (Appendix B.6,
    "Approximation with Kernel PCA"): returns sum_d G_{qd} grad_x Pi_d(xq).

    grad_x k~(x, x_i) = (-grad_1 c(x, x_i) + sum_l a_l grad_1 c(x, x_l)) / 2,
    since the base-point terms cancel against the centering."""
    xq = np.atleast_2d(np.asarray(xq, F64))
    a = np.asarray(a, F64)
    W = (np.asarray(G, F64) / np.sqrt(lam)[None, :]) @ np.asarray(V, F64).T  # (Q, N)
    out = np.zeros_like(xq)
    for q in range(xq.shape[0]):
        dc = cnt_cost_grad1(xq[q], x, kind, param)          # (N, d)
        mean_dc = a @ dc
        dk = 0.5 * (-dc + mean_dc[None, :])                 # grad_x k~(xq, x_i)
        out[q] = W[q] @ dk
    return out


# --------------------------------------------------------------------------
# Entropic OT (Appendix A "Sinkhorn"; Appendix B.1, Algorithms 2 and 3)
# --------------------------------------------------------------------------

def cost_gamma(X, Y, Gamma, s=None, t=None):
    """Bilinear cost of the Remark after Theorem 3.2 (Eq. egw_otherform):
    C_ij = -16 X_i^T Gamma Y_j - 4 ||X_i||^2 ||Y_j||^2."""
    X = np.asarray(X, F64)
    Y = np.asarray(Y, F64)
    s = sqnorms(X) if s is None else np.asarray(s, F64)
    t = sqnorms(Y) if t is None else np.asarray(t, F64)
    return -16.0 * (X @ np.asarray(Gamma, F64) @ Y.T) - 4.0 * np.outer(s, t)


def softmin(eps, logw, h, C):
    """Discrete Sinkhorn operator (Eq. sinkhorn_operators; first line of the
    loop of Algorithm 2):
        out_i = -eps log sum_j exp(logw_j + (h_j - C_ij) / eps),
    each log-sum-exp taken with an exact max shift."""
    Z = np.asarray(logw, F64)[None, :] + (np.asarray(h, F64)[None, :] - np.asarray(C, F64)) / eps
    m = Z.max(axis=1)
    return -eps * (m + np.log(np.exp(Z - m[:, None]).sum(axis=1)))


def softmin_bilinear_one(i, A, B, sA, sB, h, logw, eps):
    """One output of the softmin on the bilinear cost, computed alone:
        out_i = -eps LSE_j [logw_j + (h_j + 16 <A_i, B_j> + 4 sA_i sB_j) / eps].
    With A = X, B = Gamma Y (rows), sA = s, sB = t, h = g, logw = log b this is
    the row update of Algorithm 3 on c_Gamma; with the roles swapped it is the
    column update.  Used for sampled checks at sizes where no dense matrix
    fits."""
    A = np.asarray(A, F64)
    B = np.asarray(B, F64)
    c = -16.0 * (B @ A[i]) - 4.0 * float(sA[i]) * np.asarray(sB, F64)
    z = np.asarray(logw, F64) + (np.asarray(h, F64) - c) / eps
    m = z.max()
    return -eps * (m + math.log(np.exp(z - m).sum()))


def sinkhorn(a, b, C, eps, n_inner, f0=None, g0=None, symmetric=True):
    """Algorithm 3 (Sinkhorn-symm) when symmetric, else Algorithm 2.

    Symmetric: both halves read iterate n (Jacobi averaging):
        f^{n+1} = (f^n + S_b(g^n)) / 2,   g^{n+1} = (g^n + S_a(f^n)) / 2.
    Standard: f^{n+1} = S_b(g^n), g^{n+1} = S_a(f^{n+1}).
    Initial potentials default to zero (the paper leaves them open)."""
    a = np.asarray(a, F64)
    b = np.asarray(b, F64)
    C = np.asarray(C, F64)
    f = np.zeros(C.shape[0]) if f0 is None else np.array(f0, F64)
    g = np.zeros(C.shape[1]) if g0 is None else np.array(g0, F64)
    la, lb = np.log(a), np.log(b)
    for _ in range(n_inner):
        if symmetric:
            f_new = 0.5 * (f + softmin(eps, lb, g, C))
            g_new = 0.5 * (g + softmin(eps, la, f, C.T))
            f, g = f_new, g_new
        else:
            f = softmin(eps, lb, g, C)
            g = softmin(eps, la, f, C.T)
    return f, g


def plan(a, b, f, g, C, eps):
    """pi_ij = a_i b_j exp((f_i + g_j - C_ij) / eps)  (Eq. sinkhorn_pi)."""
    a = np.asarray(a, F64)
    b = np.asarray(b, F64)
    return np.outer(a, b) * np.exp((np.asarray(f, F64)[:, None] + np.asarray(g, F64)[None, :]
                                    - np.asarray(C, F64)) / eps)


def marginal_error(pi, a, b):
    """Err(pi) = ||pi 1 - a||_1 + ||pi^T 1 - b||_1 (Appendix A)."""
    return float(np.abs(pi.sum(1) - a).sum() + np.abs(pi.sum(0) - b).sum())


def row_marginal_from_potentials(a, b, f, g, C, eps):
    """r_i = sum_j pi_ij, written through one extra softmin:
    r_i = a_i exp((f_i - S_b(g)_i) / eps)."""
    return np.asarray(a, F64) * np.exp((np.asarray(f, F64) - softmin(eps, np.log(b), g, C)) / eps)


# --------------------------------------------------------------------------
# GW loss and energy (Eq. GW_loss; Eq. entropic_gromov_wasserstein; Lemma in
# Appendix C.1; Theorem 3.3)
# --------------------------------------------------------------------------

def gw_loss_bruteforce(pi, CX, CY):
    """L(pi) = sum_{ijkl} (CX_ik - CY_jl)^2 pi_ij pi_kl  (Eq. GW_loss), summed
    term by term over (i, j) with a vectorised inner sum over (k, l)."""
    pi = np.asarray(pi, F64)
    CX = np.asarray(CX, F64)
    CY = np.asarray(CY, F64)
    N, M = pi.shape
    total = 0.0
    for i in range(N):
        for j in range(M):
            if pi[i, j] == 0.0:
                continue
            D = CX[i][:, None] - CY[j][None, :]          # (k, l)
            total += pi[i, j] * float(np.sum(D * D * pi))
    return total


def gw_constant_pairwise(X, Y, a, b):
    """C(alpha, beta) of the Lemma, by its definition:
    sum_ik a_i a_k ||X_i - X_k||^4 + sum_jl b_j b_l ||Y_j - Y_l||^4
    - 4 (sum_i a_i ||X_i||^2)(sum_j b_j ||Y_j||^2)."""
    DX = pairwise_sqdist(X, X)
    DY = pairwise_sqdist(Y, Y)
    a = np.asarray(a, F64)
    b = np.asarray(b, F64)
    return float(a @ (DX * DX) @ a + b @ (DY * DY) @ b
                 - 4.0 * (a @ sqnorms(X)) * (b @ sqnorms(Y)))


def gw_constant_moments(X, Y, a, b):
    """C(alpha, beta) expanded with the centering of X and Y:
    [2 m4_X + 2 m2_X^2 + 4 ||Sigma_X||^2] + [same for Y] - 4 m2_X m2_Y,
    m2 = sum a ||X||^2, m4 = sum a ||X||^4, Sigma_X = sum a X X^T.
    (For alpha = beta it reduces to 8 ||Sigma||^2 + 4 m4, the direct
    computation in the proof of Prop. 4.3.)"""
    a = np.asarray(a, F64)
    b = np.asarray(b, F64)
    X = np.asarray(X, F64)
    Y = np.asarray(Y, F64)
    s, t = sqnorms(X), sqnorms(Y)
    m2x, m4x = a @ s, a @ (s * s)
    m2y, m4y = b @ t, b @ (t * t)
    Sx = (X * a[:, None]).T @ X
    Sy = (Y * b[:, None]).T @ Y
    cx = 2 * m4x + 2 * m2x ** 2 + 4 * np.sum(Sx * Sx)
    cy = 2 * m4y + 2 * m2y ** 2 + 4 * np.sum(Sy * Sy)
    return float(cx + cy - 4 * m2x * m2y)


def cross_covariance(pi, X, Y):
    """Gamma*(pi) = sum_ij pi_ij X_i Y_j^T (Theorem 3.3)."""
    return np.asarray(X, F64).T @ np.asarray(pi, F64) @ np.asarray(Y, F64)


def gw_loss_lemma(pi, X, Y, a, b):
    """L(pi) = C(alpha, beta) - 8 ||Gamma_pi||^2 - 4 sum_ij pi_ij ||X_i||^2 ||Y_j||^2
    (Lemma in Appendix C.1; valid for pi in Pi(a, b) and centered X, Y)."""
    G = cross_covariance(pi, X, Y)
    T = float(sqnorms(X) @ np.asarray(pi, F64) @ sqnorms(Y))
    return gw_constant_pairwise(X, Y, a, b) - 8.0 * float(np.sum(G * G)) - 4.0 * T


def kl_divergence(pi, a, b):
    """KL(pi | a x b) = sum_ij pi_ij log(pi_ij / (a_i b_j)), with 0 log 0 = 0."""
    pi = np.asarray(pi, F64)
    ab = np.outer(a, b)
    mask = pi > 0
    return float(np.sum(pi[mask] * np.log(pi[mask] / ab[mask])))


def egw_energy(pi, X, Y, a, b, eps):
    """Objective of Eq. entropic_gromov_wasserstein at pi: L(pi) + eps KL.
    Returns dict(E, L, KL, C)."""
    L = gw_loss_lemma(pi, X, Y, a, b)
    KL = kl_divergence(pi, a, b)
    return {"E": L + eps * KL, "L": L, "KL": KL, "C": gw_constant_pairwise(X, Y, a, b)}


def energy_from_potentials(a, b, f, g, Gamma_t, X, Y, eps):
    """Energy terms of the plan encoded by (f, g) on c_{Gamma_t}, with every
    sum taken over the dense plan.  Returns dict(E, L, KL, C, Gamma, T,
    row, col) where Gamma = Gamma_{t+1}."""
    C = cost_gamma(X, Y, Gamma_t)
    pi = plan(a, b, f, g, C, eps)
    out = egw_energy(pi, X, Y, a, b, eps)
    out["Gamma"] = cross_covariance(pi, X, Y)
    out["T"] = float(sqnorms(X) @ pi @ sqnorms(Y))
    out["row"] = pi.sum(1)
    out["col"] = pi.sum(0)
    return out


# --------------------------------------------------------------------------
# CNT-GW (Algorithm 1) and its dual function (Prop. 4.5)
# --------------------------------------------------------------------------

def eps_schedule(eps0, eps_final, n_outer):
    """Temperature per outer step.  Constant when eps_final is None or equal
    to eps0; otherwise geometric, eps_t = eps0 (eps_final/eps0)^(t/(T-1)).
    (Our reading of an annealed run from 1e-1 to 1e-3: the paper's per-
    iteration eps0/sqrt(n) schedule of Appendix B.1 cannot span two decades
    within one Sinkhorn call.)"""
    if eps_final is None or eps_final == eps0 or n_outer == 1:
        return [float(eps0)] * n_outer
    return [float(eps0 * (eps_final / eps0) ** (t / (n_outer - 1))) for t in range(n_outer)]


def sinkhorn_stop(a, b, C, eps, n_max, f0=None, g0=None, symmetric=True, tol=0.0, every=1,
                  trace=None):
    """Sinkhorn with the hybrid stop of Appendix D.1 (a fixed maximum of
    iterations and early stopping on the marginal error): after every
    `every`-th iteration the error Err (Appendix A) of the last plan whose
    marginals that iteration measured is compared with tol, and the loop ends
    once it is below.  The measured plan is (f^n, g^n) for Algorithm 3 (its
    row and column softmins were just evaluated) and (f^{n+1}, g^n) for
    Algorithm 2 (exact rows; columns from S_a(f^{n+1})).  The paper prints a
    weighted form of the error next to the plain one of Appendix A; this uses
    the plain one.  Every check appends (iteration, Err) to `trace` when it is
    a list.  Returns (f, g, iterations run, last measured Err or None)."""
    a = np.asarray(a, F64)
    b = np.asarray(b, F64)
    C = np.asarray(C, F64)
    f = np.zeros(C.shape[0]) if f0 is None else np.array(f0, F64)
    g = np.zeros(C.shape[1]) if g0 is None else np.array(g0, F64)
    err = None
    for it in range(n_max):
        f_new, g_new = sinkhorn(a, b, C, eps, 1, f, g, symmetric)
        if (it + 1) % every == 0:
            measured = (f, g) if symmetric else (f_new, g)
            err = marginal_error(plan(a, b, measured[0], measured[1], C, eps), a, b)
            if trace is not None:
                trace.append((it + 1, err))
        f, g = f_new, g_new
        if err is not None and (it + 1) % every == 0 and err < tol:
            return f, g, it + 1, err
    return f, g, n_max, err


def cnt_gw(a, b, X, Y, eps, n_outer, n_inner, Gamma0=None, f0=None, g0=None,
           symmetric=True, eps_final=None, record=True, adaptive=False, n_inner_max=None,
           stop_tol=None, stop_every=1, adapt_rtol=0.0):
    """Algorithm 1 (CNT-GW) with Algorithm 3 as SinkhornOT, on c_Gamma.

    For t = 0 .. n_outer-1:
      1. C = c_{Gamma_t}  (Zbar_j = [Gamma_t Y_j, ||Y_j||^2 / 2] in Alg. 1);
      2. (f, g) <- n_inner Sinkhorn iterations at eps_t, warm-started (App. B.1);
      3. Xtilde_j = sum_i a_i X_i exp((f_i + g_j - C_ij) / eps_t);
      4. Gamma_{t+1} = sum_j b_j Xtilde_j Y_j^T.
    Gamma_0 = 0 unless given.  Each step records the energy of pi_{t+1}
    (E = L + eps_t KL), its marginal error and ||Gamma_{t+1} - Gamma_t||_F.

    adaptive: Algorithm 6 applied to CNT-GW (Appendix B.4): n_inner is the
    initial count; when the energy of pi_{t+1} exceeds that of pi_t the next
    steps run twice as many iterations (capped at n_inner_max).  The loss
    compared is E = L + eps_t KL on the lifted features; "exceeds" means
    E(pi_{t+1}) > E(pi_t) + adapt_rtol |E(pi_t)| (0: the paper's strict test,
    which near convergence also fires on rounding noise).
    stop_tol: the hybrid stop of sinkhorn_stop inside every outer step, with
    n_inner (or the adaptive count) as the maximum.
    Returns dict(Gamma, f, g, history, eps)."""
    a = np.asarray(a, F64)
    b = np.asarray(b, F64)
    X = np.asarray(X, F64)
    Y = np.asarray(Y, F64)
    D, E = X.shape[1], Y.shape[1]
    Gamma = np.zeros((D, E)) if Gamma0 is None else np.array(Gamma0, F64)
    f = np.zeros(X.shape[0]) if f0 is None else np.array(f0, F64)
    g = np.zeros(Y.shape[0]) if g0 is None else np.array(g0, F64)
    sched = eps_schedule(eps, eps_final, n_outer)
    cap = n_inner_max if n_inner_max is not None else n_inner
    n_cur = n_inner
    E_prev = None
    hist = []
    for t in range(n_outer):
        e = sched[t]
        C = cost_gamma(X, Y, Gamma)
        trace = []
        if stop_tol is not None and stop_tol > 0:
            f, g, n_run, serr = sinkhorn_stop(a, b, C, e, n_cur, f, g, symmetric, stop_tol,
                                              stop_every, trace)
        else:
            f, g = sinkhorn(a, b, C, e, n_cur, f, g, symmetric)
            n_run, serr = n_cur, None
        K = np.exp((f[:, None] + g[None, :] - C) / e)
        Xtilde = K.T @ (a[:, None] * X)                  # (M, D): Xtilde_j
        Gamma_next = (Xtilde * b[:, None]).T @ Y         # sum_j b_j Xtilde_j Y_j^T
        if record or adaptive:
            pi = plan(a, b, f, g, C, e)
            en = egw_energy(pi, X, Y, a, b, e)
        if record:
            hist.append({
                "eps": e, "E": en["E"], "L": en["L"], "KL": en["KL"], "C": en["C"],
                "err": marginal_error(pi, a, b),
                "row": pi.sum(1), "col": pi.sum(0),
                "dGamma": float(np.linalg.norm(Gamma_next - Gamma)),
                "Gamma": Gamma_next.copy(),
                "n_inner": n_run, "stop_err": serr, "stop_trace": trace,
            })
        if adaptive:
            if E_prev is not None and en["E"] > E_prev + adapt_rtol * abs(E_prev):
                n_cur = min(2 * n_cur, cap)
            E_prev = en["E"]
        Gamma = Gamma_next
    return {"Gamma": Gamma, "f": f, "g": g, "history": hist, "eps": sched}


def dual_function(Gamma, a, b, X, Y, eps, n_inner=2000):
    """D_eps(Gamma) = ||Gamma||^2 + OT_eps^{c_Gamma} / 8 (proof of Prop. 4.5),
    with OT_eps evaluated by its dual value <a, f> + <b, g> at Sinkhorn
    convergence (Appendix A).  Returns (value, f, g)."""
    C = cost_gamma(X, Y, Gamma)
    f, g = sinkhorn(a, b, C, eps, n_inner, symmetric=False)
    ot = float(np.asarray(a) @ f + np.asarray(b) @ g)
    return float(np.sum(np.asarray(Gamma) ** 2)) + ot / 8.0, f, g


# --------------------------------------------------------------------------
# Comparison solvers used only as cross-checks
# --------------------------------------------------------------------------

def entropic_gw_step(pi_t, CX, CY, a, b, eps, n_inner):
    """One update of Eq. entropic_cgd_sequence: entropic OT for the cost
    grad_{pi_t} L = 2 sum_kl (CX_ik - CY_jl)^2 pi_t[k, l] (proof of
    Prop. 4.4).  Cubic; tiny N only.  Returns the new plan."""
    CX = np.asarray(CX, F64)
    CY = np.asarray(CY, F64)
    pi_t = np.asarray(pi_t, F64)
    # sum_kl (CX_ik - CY_jl)^2 p_kl = sum_k CX_ik^2 p_k. + sum_l CY_jl^2 p_.l - 2 (CX p CY^T)_ij
    G = 2.0 * ((CX ** 2) @ pi_t.sum(1)[:, None] + ((CY ** 2) @ pi_t.sum(0))[None, :]
               - 2.0 * CX @ pi_t @ CY.T)
    f, g = sinkhorn(a, b, G, eps, n_inner, symmetric=False)
    return plan(a, b, f, g, G, eps)


def kernel_gw(a, b, CX, CY, eps, n_outer, n_inner, pi0=None, symmetric=True):
    """Algorithm 5 (Kernel-GW): the exact kernelised scheme with a dense
    N x M cost  C = -4 K^X_ii K^Y_jj - 16 K^X pi K^Y.  Tiny N only.
    Returns (pi, f, g)."""
    a = np.asarray(a, F64)
    b = np.asarray(b, F64)
    KX = kernel_from_cost(CX, a)
    KY = kernel_from_cost(CY, b)
    pi = np.outer(a, b) if pi0 is None else np.array(pi0, F64)
    f = np.zeros(len(a))
    g = np.zeros(len(b))
    for _ in range(n_outer):
        C = -4.0 * np.outer(np.diag(KX), np.diag(KY)) - 16.0 * KX @ pi @ KY
        f, g = sinkhorn(a, b, C, eps, n_inner, f, g, symmetric)
        pi = plan(a, b, f, g, C, eps)
    return pi, f, g


def permutation_ot(C):
    """Brute-force optimal assignment by enumeration (N <= 8)."""
    C = np.asarray(C, F64)
    n = C.shape[0]
    best, best_p = None, None
    for p in itertools.permutations(range(n)):
        v = sum(C[i, p[i]] for i in range(n))
        if best is None or v < best:
            best, best_p = v, p
    return best, best_p


# --------------------------------------------------------------------------
# Gradients (Appendix B.6, envelope theorem)
# --------------------------------------------------------------------------

def grad_features(pi, Gamma, X, Y, a, b):
    """Gradient of E = L(pi) + eps KL with pi held at the converged plan
    (envelope theorem, Appendix B.6), with respect to the centered features
    X_i, from the Lemma:
      dC/dX_i     = 8 a_i [(s_i + m2_X) X_i + 2 Sigma_X X_i - mu3_X] - 8 a_i m2_Y X_i
      d(-8||G||^2) = -16 Gamma w_i,   w_i = sum_j pi_ij Y_j
      d(-4 T)      = -8 q_i X_i,      q_i = sum_j pi_ij t_j
    with mu3_X = sum_k a_k s_k X_k and Gamma = Gamma_pi."""
    X = np.asarray(X, F64)
    Y = np.asarray(Y, F64)
    a = np.asarray(a, F64)
    b = np.asarray(b, F64)
    pi = np.asarray(pi, F64)
    s, t = sqnorms(X), sqnorms(Y)
    m2x = a @ s
    m2y = b @ t
    Sx = (X * a[:, None]).T @ X
    mu3 = (a * s) @ X
    dC = 8.0 * a[:, None] * ((s + m2x)[:, None] * X + 2.0 * X @ Sx - mu3[None, :]) \
        - 8.0 * (a * m2y)[:, None] * X
    w = pi @ Y
    q = pi @ t
    return dC - 16.0 * w @ np.asarray(Gamma, F64).T - 8.0 * q[:, None] * X


def center_vjp(G, a):
    """Adjoint of X = x - sum_k a_k x_k:  grad_x_i = G_i - a_i sum_k G_k."""
    G = np.asarray(G, F64)
    return G - np.asarray(a, F64)[:, None] * G.sum(0)[None, :]


def grad_x_squared(pi, Gamma, X, Y, a, b):
    """Gradient of the EGW energy w.r.t. source points for the squared cost
    (features = centered points): center_vjp(grad_features)."""
    return center_vjp(grad_features(pi, Gamma, X, Y, a, b), a)


def grad_x_lifted(pi, Gamma, X, Y, a, b, x, V, lam, kind, param):
    """Algorithm 12 (EGW-Grad with Kernel PCA): features X = center(Pi_X(x))
    with Kernel-Proj frozen at the training points, so
    grad_x = Pi_X'^T center^T grad_features.  X must be the re-centered
    Kernel-Proj features of x (equal to the Kernel PCA features at the
    training points)."""
    G = center_vjp(grad_features(pi, Gamma, X, Y, a, b), a)
    return kernel_proj_vjp(G, x, x, a, V, lam, kind, param)


def grad_x_bruteforce(pi, x, y, a, b, kind="sqeuclid", param=2.0):
    """grad_{x_i} L(pi) with pi fixed, from Eq. GW_loss term by term:
    4 sum_{j,k,l} (c_X(x_i, x_k) - c_Y(y_j, y_l)) pi_ij pi_kl grad_1 c_X(x_i, x_k)."""
    x = np.asarray(x, F64)
    pi = np.asarray(pi, F64)
    CX = cnt_cost(x, x, kind, param)
    CY = cnt_cost(y, y, kind, param)
    N, M = pi.shape
    out = np.zeros_like(x)
    for i in range(N):
        dc = cnt_cost_grad1(x[i], x, kind, param)      # (k, d)
        coef = np.zeros(N)
        for j in range(M):
            if pi[i, j] == 0.0:
                continue
            Dkl = CX[i][:, None] - CY[j][None, :]       # (k, l)
            coef += pi[i, j] * (Dkl * pi).sum(1)
        out[i] = 4.0 * coef @ dc
    return out


# --------------------------------------------------------------------------
# Color / UV transfer (Appendix E, "Transport plan visualizations")
# --------------------------------------------------------------------------

def barycentric_transfer(pi, U, b):
    """C_Y(y_j) = sum_i C_X(x_i) pi_ij / (a_i b_j) a_i = (pi^T U)_j / b_j for
    source attributes U (colors, UV coordinates; N x k)."""
    return (np.asarray(pi, F64).T @ np.asarray(U, F64)) / np.asarray(b, F64)[:, None]


# --------------------------------------------------------------------------
# Sinkhorn GW divergence (Section 4.1, "Entropic Bias and Symmetric Debiasing")
# --------------------------------------------------------------------------

def final_plan(res, a, b, X, Y, Gamma0=None):
    """The plan a cnt_gw result (record=True) ends on: its potentials on the
    cost of the Gamma that preceded the last update."""
    hist = res["history"]
    if len(hist) >= 2:
        Gt = hist[-2]["Gamma"]
    else:
        Gt = np.zeros((X.shape[1], Y.shape[1])) if Gamma0 is None else np.asarray(Gamma0, F64)
    return plan(a, b, res["f"], res["g"], cost_gamma(X, Y, Gt), res["eps"][-1])


def sgw(a, b, X, Y, eps, n_outer, n_inner, **kw):
    """SGW_eps(alpha, beta) = GW_eps(alpha, beta) - (GW_eps(alpha, alpha)
    + GW_eps(beta, beta)) / 2, each GW_eps the final energy E = L + eps KL of a
    CNT-GW solve with the same options.  Returns dict(SGW, ab, aa, bb)."""
    ab = cnt_gw(a, b, X, Y, eps, n_outer, n_inner, **kw)
    aa = cnt_gw(a, a, X, X, eps, n_outer, n_inner, **kw)
    bb = cnt_gw(b, b, Y, Y, eps, n_outer, n_inner, **kw)
    E = lambda r: r["history"][-1]["E"]
    return {"SGW": E(ab) - 0.5 * (E(aa) + E(bb)), "ab": ab, "aa": aa, "bb": bb}


def sgw_grad_features(pi_ab, pi_aa, X, Y, a, b):
    """Gradient of SGW with respect to the source features X with every plan
    held at its optimum (envelope theorem, Appendix B.6).  GW_eps(alpha,
    alpha) depends on X through both of its sides: the target side is the
    source side of the transposed problem (plan pi^T)."""
    g_ab = grad_features(pi_ab, cross_covariance(pi_ab, X, Y), X, Y, a, b)
    g_src = grad_features(pi_aa, cross_covariance(pi_aa, X, X), X, X, a, a)
    pt = np.asarray(pi_aa, F64).T
    g_tgt = grad_features(pt, cross_covariance(pt, X, X), X, X, a, a)
    return g_ab - 0.5 * (g_src + g_tgt)


# --------------------------------------------------------------------------
# Multiscale-GW (Algorithms 7 and 8, Appendix B.5)
# --------------------------------------------------------------------------

def kmeans_coarsen(X, a, init_idx, n_iter):
    """Coarsen (Appendix B.5): K-Means centroids of the features with the
    aggregated weights a^c_i = sum_{j in C_i} a_j.  Lloyd's iterations (the
    paper does not say which K-Means): assign every point to its nearest
    centroid (ties to the lowest index), then move each centroid to the
    a-weighted mean of its points; the centroids start at X[init_idx] (the
    caller draws the indices).  A last assignment follows the last update, and
    the final centroids are the weighted means of that assignment.  Empty
    clusters are dropped.  Returns (Xc, ac, assign) with assign indexing Xc."""
    X = np.asarray(X, F64)
    a = np.asarray(a, F64)
    C = X[np.asarray(init_idx)].copy()
    for _ in range(n_iter + 1):
        d2 = pairwise_sqdist(X, C)
        assign = np.argmin(d2, axis=1)          # first minimum
        k = C.shape[0]
        wsum = np.bincount(assign, weights=a, minlength=k)
        for d in range(X.shape[1]):
            num = np.bincount(assign, weights=a * X[:, d], minlength=k)
            C[:, d] = np.where(wsum > 0, num / np.where(wsum > 0, wsum, 1.0), C[:, d])
    keep = np.flatnonzero(wsum > 0)
    remap = -np.ones(C.shape[0], dtype=np.int64)
    remap[keep] = np.arange(len(keep))
    return C[keep], wsum[keep], remap[assign]


def kmeans_objective(X, a, C, assign):
    """sum_j a_j ||X_j - C_{assign(j)}||^2"""
    X = np.asarray(X, F64)
    return float(np.asarray(a, F64) @ np.sum((X - np.asarray(C, F64)[assign]) ** 2, axis=1))


def interpolate(g_c, X, Yc, b_c, Gamma, eps):
    """Algorithm 8 (Interpolate): f_i = -eps log sum_j exp(log b^c_j +
    (g^c_j - C_ij)/eps) with C_ij = -4 ||X_i||^2 ||Y^c_j||^2 - 16 X_i^T Gamma Y^c_j
    (Gamma the coarse linear map: our reading of the free Gamma of the listing)."""
    C = cost_gamma(X, Yc, Gamma)
    return softmin(eps, np.log(np.asarray(b_c, F64)), g_c, C)


def multiscale_gw(a, b, X, Y, eps, init_x, init_y, km_iter, coarse_outer, coarse_inner,
                  fine_outer, fine_inner, eps_final=None, symmetric=True, Gamma0=None):
    """Algorithm 7 (Multiscale-GW): coarsen both measures by K-Means, solve
    CNT-GW on the coarse measures, interpolate the coarse potentials to the
    fine points (Algorithm 8), then run CNT-GW on the fine measures from
    Gamma^c and the interpolated potentials.  The coarse solve runs at the
    fine solve's first temperature.  Returns the fine result plus the coarse
    one under "coarse"."""
    Xc, ac, _ = kmeans_coarsen(X, a, init_x, km_iter)
    Yc, bc, _ = kmeans_coarsen(Y, b, init_y, km_iter)
    coarse = cnt_gw(ac, bc, Xc, Yc, eps, coarse_outer, coarse_inner, Gamma0=Gamma0,
                    symmetric=symmetric)
    Gc = coarse["Gamma"]
    f0 = interpolate(coarse["g"], X, Yc, bc, Gc, eps)
    g0 = interpolate(coarse["f"], Y, Xc, ac, np.asarray(Gc).T, eps)
    fine = cnt_gw(a, b, X, Y, eps, fine_outer, fine_inner, Gamma0=Gc, f0=f0, g0=g0,
                  symmetric=symmetric, eps_final=eps_final)
    fine["coarse"] = coarse
    fine["Xc"], fine["ac"], fine["Yc"], fine["bc"] = Xc, ac, Yc, bc
    return fine
