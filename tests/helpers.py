"""Shared test helpers: numpy <-> device tensors and derived tolerances."""

import math

import numpy as np


def dev(x, dtype=None):
    import torch
    t = torch.as_tensor(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def f32(x):
    import torch
    return dev(np.asarray(x, np.float32), torch.float32)


def f64(x):
    import torch
    return dev(np.asarray(x, np.float64), torch.float64)


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def softmin_tolerance(A, B, sA, sB, h, logw, eps):
    """Per-output bound on |GPU FP32 - FP64| for the softmin, derived from the
    arithmetic of the FP32 kernel:
      * every exponent z_ij is a sum of K+2 FP32 products/terms, so its
        rounding error is at most (K+2) 2^-24 sum|terms|; out_i moves by at
        most eps*ln2 times the largest exponent error (the LSE is 1-Lipschitz
        in the max norm), i.e. (K+2) 2^-24 S_i with
        S_i = max_j (16 sum_k |A_ik B_jk| + 4 |sA_i sB_j| + |h_j| + eps |logw_j|);
      * ex2.approx has relative error below 2^-22 and the running FP32 sum of
        m terms adds a relative error of about sqrt(m) 2^-24 (rounding
        errors of a long sum behave like a random walk): eps (2^-21 + sqrt(m) 2^-22).
    A factor 2 covers the conversion of the scaled terms to base 2."""
    A = np.asarray(A, np.float64)
    B = np.asarray(B, np.float64)
    K = A.shape[1]
    m = B.shape[0]
    lw = np.where(np.isfinite(logw), np.abs(logw), 0.0)
    S = (16.0 * np.abs(A) @ np.abs(B).T + 4.0 * np.abs(np.outer(sA, sB))
         + np.abs(h)[None, :] + eps * lw[None, :]).max(axis=1)
    return 2.0 * ((K + 2) * 2.0 ** -24 * S + eps * (2.0 ** -21 + math.sqrt(m) * 2.0 ** -22))


# Relative error of one product term of the exponent in each cost-tile mode:
# F16X3 keeps hi*hi + hi*lo + lo*hi of 11-bit halves (dropped lo*lo and the
# rounding of lo: ~3 * 2^-22); BF16X3 the same with 8-bit halves (~3 * 2^-17);
# BF16 a single 8-bit product (2^-8 with the operand roundings).
TERM_REL = {0: 2.0 ** -23, 1: 2.0 ** -7, 2: 2.0 ** -15, 3: 2.0 ** -20}


# Relative error of a single 16-bit product (both operands rounded once).
SINGLE_REL = {2: 2.0 ** -7, 3: 2.0 ** -10}


def narrow_layout_bound(A, B, prec):
    """Per-row bound (output units) of the dims the split precisions may run
    as one product when their full operand layout is wider than 128 columns
    (K >= 40): those with P_k = max|A_k| max|B_k| at most
    TERM_REL[prec] / SINGLE_REL[prec] times the largest P.  Each of their
    terms carries SINGLE_REL[prec] relative error; in the output
    (eps ln2 times the base-2 exponent, whose product scale is
    16 log2(e) / eps) that is 16 SINGLE_REL sum_k |A_ik B_jk|."""
    A = np.asarray(A, np.float64)
    B = np.asarray(B, np.float64)
    K = A.shape[1]
    if prec not in (2, 3) or 3 * K + 10 <= 128:
        return np.zeros(A.shape[0])
    P = np.abs(A).max(axis=0) * np.abs(B).max(axis=0)
    small = P <= TERM_REL[prec] / SINGLE_REL[prec] * P.max() * (1.0 + 1e-6)
    if not small.any():
        return np.zeros(A.shape[0])
    return 16.0 * SINGLE_REL[prec] * (np.abs(A[:, small]) @ np.abs(B[:, small]).T).max(axis=1)


def softmin_tolerance_prec(A, B, sA, sB, h, logw, eps, prec):
    """softmin_tolerance for the tensor-core modes: the exponent terms carry
    TERM_REL[prec] relative error each (summed over K + 2 terms) and the
    bias columns an absolute error below 2^-8 (base 2) from the 16-bit
    splitting times the 2^15 constant."""
    if prec == 0:
        return softmin_tolerance(A, B, sA, sB, h, logw, eps)
    A = np.asarray(A, np.float64)
    B = np.asarray(B, np.float64)
    K = A.shape[1]
    m = B.shape[0]
    lw = np.where(np.isfinite(logw), np.abs(logw), 0.0)
    S = (16.0 * np.abs(A) @ np.abs(B).T + 4.0 * np.abs(np.outer(sA, sB))
         + np.abs(h)[None, :] + eps * lw[None, :]).max(axis=1)
    return 2.0 * ((K + 2) * TERM_REL[prec] * S + narrow_layout_bound(A, B, prec)
                  + eps * (2.0 ** -8 + 2.0 ** -21 + math.sqrt(m) * 2.0 ** -22))


def noisy_cnt_gw(a, b, X, Y, eps0, n_outer, n_inner, prec, seed, eps_final=None,
                 Gamma0=None, f0=None, g0=None, states=None):
    """The FP64 oracle's Algorithm 1 with Algorithm 3 (oracle.cnt_gw), except
    that every softmin's exponent carries fresh uniform noise of the per-cell
    error bound the GPU arithmetic of precision `prec` has (the bound behind
    softmin_tolerance_prec): the exponent (h_j - C_ij) / eps of cell (i, j)
    moves by up to (K + 2) TERM_REL[prec] S_ij / eps, with
    S_ij = |h_j| + 16 sum_k |X_ik V_jk| + 4 |s_i t_j| + eps |log w_j|, in
    both half-steps of every iteration.  The spread of its energies against
    the noiseless oracle is the error that arithmetic alone implies for the
    annealed solve.  Returns the per-step energy records (E, L, KL) of the
    plans pi_{t+1}, as cnt_gw's history, and (when `states` is a list) the
    state (Gamma_t, f, g) each outer step started from."""
    import oracle as O
    rng = np.random.default_rng(seed)
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    X = np.asarray(X, np.float64)
    Y = np.asarray(Y, np.float64)
    n, m, K = X.shape[0], Y.shape[0], X.shape[1]
    la, lb = np.log(a), np.log(b)
    s, t = (X * X).sum(1), (Y * Y).sum(1)
    Gamma = np.zeros((K, Y.shape[1])) if Gamma0 is None else np.array(Gamma0, np.float64)
    f = np.zeros(n) if f0 is None else np.array(f0, np.float64)
    g = np.zeros(m) if g0 is None else np.array(g0, np.float64)
    rel = (K + 2) * TERM_REL[prec]
    hist = []
    for e in O.eps_schedule(eps0, eps_final, n_outer):
        if states is not None:
            states.append((Gamma.copy(), f.copy(), g.copy()))
        C = O.cost_gamma(X, Y, Gamma, s, t)
        V = Y @ Gamma.T
        Sdot = 16.0 * np.abs(X) @ np.abs(V).T + 4.0 * np.outer(s, t)
        for _ in range(n_inner):
            Sr = Sdot + np.abs(g)[None, :] + e * np.abs(lb)[None, :]
            Sc = Sdot + np.abs(f)[:, None] + e * np.abs(la)[:, None]
            fh = O.softmin(e, lb, g, C + rel * Sr * rng.uniform(-1.0, 1.0, Sr.shape))
            gh = O.softmin(e, la, f, (C + rel * Sc * rng.uniform(-1.0, 1.0, Sc.shape)).T)
            f, g = 0.5 * (f + fh), 0.5 * (g + gh)
        pi = O.plan(a, b, f, g, C, e)
        en = O.egw_energy(pi, X, Y, a, b, e)
        hist.append({"eps": e, "E": en["E"], "L": en["L"], "KL": en["KL"]})
        Gamma = O.cross_covariance(pi, X, Y)
    return hist


def grad_tolerance(pi, X, Y, a, eps):
    """Relative bound (times the largest term) of the FP32 adjoint's feature
    gradient: each plan entry carries ~(D+4) 2^-24 |C| / eps of relative error
    from its exponent, each sum over N or M terms ~sqrt(N) 2^-24; a factor 8
    for the closed form's combination of terms."""
    X = np.asarray(X, np.float64)
    Y = np.asarray(Y, np.float64)
    scale = 16 * np.abs(X).max() * np.abs(Y).max() + 8 * (X * X).sum(1).max() * (Y * Y).sum(1).max()
    rel = (X.shape[1] + 4) * 2.0 ** -24 * scale / eps + np.sqrt(max(X.shape[0], Y.shape[0])) * 2.0 ** -22
    return 8.0 * rel
