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
    return 2.0 * ((K + 2) * TERM_REL[prec] * S
                  + eps * (2.0 ** -8 + 2.0 ** -21 + math.sqrt(m) * 2.0 ** -22))
