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


# --------------------------------------------------------------- FP8 mode
E4M3_MAX = 448.0
LOG2E_F32 = np.float32(1.4426950408889634)


def round_e4m3(x):
    """Round to the nearest e4m3 value (bias 7: normals down to 2^-6 with 3
    mantissa bits, subnormals in steps of 2^-9, largest finite 448); ties to
    even.  |x| <= 448 is assumed (the scales guarantee it)."""
    x = np.asarray(x, np.float64)
    ax = np.abs(x)
    e = np.maximum(np.floor(np.log2(np.maximum(ax, 2.0 ** -9))), -6.0)
    step = 2.0 ** (e - 3.0)
    return np.sign(x) * np.minimum(np.round(ax / step) * step, E4M3_MAX)


def e4m3_group_scale(m):
    """The power of two 2^e, e in [-40, 40], largest with m 2^e <= 448 (the
    scale GW_PREC_FP8 gives a group of operand values of largest magnitude
    m); 1 for m = 0 or a non-finite m."""
    m = float(m)
    if not (m > 0.0) or not math.isfinite(m):
        return 1.0
    fr, E = math.frexp(m)                       # m = fr 2^E, fr in [0.5, 1)
    e = (9 if fr <= 0.875 else 8) - E           # fr 2^9 <= 448 iff fr <= 0.875
    return 2.0 ** min(max(e, -40), 40)


def fp8_operands(A, B, eps=None, group=128, scales=False):
    """The feature operands GW_PREC_FP8 multiplies, from the mode's
    definition (gw.h): each matrix (as FP32) gets one power-of-two scale per
    group of `group` rows (e4m3_group_scale of the group's largest |value|)
    and is rounded to e4m3; the same rounding whichever side of the product
    the matrix takes.  Returns (Ahat, Bhat), the rounded values in the units
    of A and B: the mode's exponent is 16 <Ahat_i, Bhat_j> / eps (up to FP32
    rounding of the coefficient).  scales=True also returns the per-row
    factors that take Ahat and Bhat to the e4m3 values.  (eps is accepted for
    symmetry with the callers; the rounding does not depend on it.)"""
    out, facs = [], []
    for M in (A, B):
        M32 = np.asarray(M, np.float32)
        grp = np.arange(len(M32)) // group
        fg = np.array([e4m3_group_scale(np.abs(M32[grp == q]).max()) for q in range(grp.max() + 1)])
        fr = fg[grp]
        out.append(round_e4m3(M32.astype(np.float64) * fr[:, None]) / fr[:, None])
        facs.append(fr)
    if scales:
        return out[0], out[1], facs[0], facs[1]
    return out[0], out[1]


def softmin_tolerance_fp8_emulated(Ahat, Bhat, sA, sB, h, logw, eps):
    """Bound for GW_PREC_FP8 against the oracle on the rounded operands
    (fp8_operands): the e4m3 products are exact, what remains is the FP32
    accumulation, the split-BF16 bias and rank-one columns (relative 2^-15
    per term, as the split BF16 mode's), the FP32 coefficient alpha and its
    quotient by the scales (a few 2^-24 of each term)."""
    Ahat = np.asarray(Ahat, np.float64)
    Bhat = np.asarray(Bhat, np.float64)
    K = Ahat.shape[1]
    m = Bhat.shape[0]
    lw = np.where(np.isfinite(logw), np.abs(logw), 0.0)
    S = (16.0 * np.abs(Ahat) @ np.abs(Bhat).T + 4.0 * np.abs(np.outer(sA, sB))
         + np.abs(h)[None, :] + eps * lw[None, :]).max(axis=1)
    return 2.0 * ((K + 2) * 2.0 ** -15 * S
                  + eps * (2.0 ** -8 + 2.0 ** -21 + math.sqrt(m) * 2.0 ** -22))
