"""Parity at the bench's sizes: the tensor-core kernels in the launch
configuration the benchmark times (N = M = 100k, D = 32: one fused Sinkhorn
iteration of Algorithm 3 with every column split and both the fast and the
safe pass; the plan-weighted sums of Algorithm 1 with many source splits),
checked element by element on sampled outputs that the FP64 oracle computes
one by one over all 100k points of the other side.

Inputs are seeded, with the shapes of the lifted workload: centered features
with a decaying spectrum (as Kernel PCA features have), Gamma_t near a
rotation times the feature covariance, an annealed eps = 5e-3.  The shift
estimates the kernels take (the potential of the output side) are made on the
CPU from the exact maximum exponent of every row, so the log-sum-exp lies in
[max, max + log M] of them: the fast pass runs, and rows whose estimate is
moved by 300 eps (2^+-430) go through the safe pass."""

import math

import numpy as np
import pytest

import oracle as O
import workloads as W
from helpers import SINGLE_REL, TERM_REL, f32, f64, host

pytestmark = pytest.mark.gpu

N = 100_000
D = 32
EPS = 5e-3
r32 = lambda x: np.asarray(x, np.float32).astype(np.float64)


def lifted_shape_features(n, seed):
    g = W.rng(seed)
    sig = (1.0 + np.arange(D)) ** -0.8
    sig *= math.sqrt(0.3 / float((sig ** 2).sum()))      # E ||X||^2 = 0.3 (radius-1 clouds)
    X = g.standard_normal((n, D)) * sig
    return X - X.mean(0), sig


def max_exponent(A, B, sA, sB, h, logw, eps, chunk=512):
    """max_j z_ij with z_ij = logw_j + (h_j + 16 <A_i, B_j> + 4 sA_i sB_j) / eps
    (natural log), one FP32 product of augmented rows per chunk of rows."""
    Ap = np.concatenate([16.0 / eps * A, (4.0 / eps * sA)[:, None], np.ones((len(A), 1))],
                        axis=1).astype(np.float32)
    Bp = np.concatenate([B, sB[:, None], (logw + h / eps)[:, None]], axis=1).astype(np.float32)
    out = np.empty(len(A))
    for i0 in range(0, len(A), chunk):
        out[i0:i0 + chunk] = (Ap[i0:i0 + chunk] @ Bp.T).max(axis=1)
    return out


@pytest.fixture(scope="module")
def big():
    X, sig = lifted_shape_features(N, 101)
    Y, _ = lifted_shape_features(N, 102)
    g = W.rng(103)
    Q, _ = np.linalg.qr(g.standard_normal((D, D)))
    Gamma = (sig ** 2)[:, None] * Q                     # near an isometry's cross-covariance
    X, Y = r32(X), r32(Y)
    V = r32(Y @ Gamma.T)                                # V_j = Gamma Y_j
    s, t = r32((X * X).sum(1)), r32((Y * Y).sum(1))
    a = r32(W.random_weights(N, 104, 0.3))
    b = r32(W.random_weights(N, 105, 0.3))
    la, lb = r32(np.log(a)), r32(np.log(b))
    h = r32(0.1 * g.standard_normal(N))                 # target potential g
    zmax = max_exponent(X, V, s, t, h, lb, EPS)
    f = -EPS * (zmax + 0.5 * math.log(N))               # row estimate: S_b(g) within eps log(N) / 2
    far = g.random(N) < 0.02
    f = r32(np.where(far, f + 300.0 * EPS * np.sign(g.standard_normal(N)), f))
    # a column potential for the plan sums with pi_ij / b_j <= 1 (its
    # exponent's maximum over the sources is 0), as the plan kernel's f16
    # range needs: g_plan_j = -eps max_i [log a_i + (f_i - c_ij) / eps]
    zc = max_exponent(V, X, t, s, f, la, EPS)
    g_plan = r32(-EPS * zc)
    return dict(X=X, Y=Y, V=V, s=s, t=t, a=a, b=b, la=la, lb=lb, h=h, f=f, far=far,
                Gamma=Gamma, g_plan=g_plan)


def sampled(n, k, seed, must=()):
    g = W.rng(seed)
    idx = set(int(i) for i in g.choice(n, k, replace=False))
    idx.update(int(i) for i in must)
    idx.update((0, 255, 256, n - 161, n - 1))           # first tile, tile edge, ragged last tile
    return np.array(sorted(idx))


def tol_rows(A, B, sA, sB, h, logw, eps, prec, rows):
    """helpers.softmin_tolerance_prec for the sampled rows only (the same
    derivation: TERM_REL[prec] per exponent term, the dims the split
    precisions may run as one product, bias columns, ex2, sum)."""
    Ar = np.abs(A[rows])
    lw = np.where(np.isfinite(logw), np.abs(logw), 0.0)
    S = (16.0 * Ar @ np.abs(B).T + 4.0 * np.abs(np.outer(sA[rows], sB))
         + np.abs(h)[None, :] + eps * lw[None, :]).max(axis=1)
    single = np.zeros(len(rows))
    if prec in (2, 3) and 3 * A.shape[1] + 10 > 128:
        P = np.abs(A).max(axis=0) * np.abs(B).max(axis=0)
        small = P <= TERM_REL[prec] / SINGLE_REL[prec] * P.max() * (1.0 + 1e-6)
        if small.any():
            single = 16.0 * SINGLE_REL[prec] * (Ar[:, small] @ np.abs(B[:, small]).T).max(axis=1)
    m = len(B)
    return 2.0 * ((A.shape[1] + 2) * TERM_REL[prec] * S + single
                  + eps * (2.0 ** -8 + 2.0 ** -21 + math.sqrt(m) * 2.0 ** -22))


@pytest.mark.parametrize("prec", [3, 2, 1])
def test_fused_iteration_at_bench_size(gw, big, prec):
    P = big
    fo, go = gw.gw_sinkhorn_iteration(f32(P["X"]), f32(P["V"]), f32(P["s"]), f32(P["t"]),
                                      f32(P["la"]), f32(P["lb"]), f32(P["f"]), f32(P["h"]), EPS,
                                      prec=prec, symmetric=True)
    fo, go = host(fo), host(go)
    far_rows = np.flatnonzero(P["far"])[:40]
    I = sampled(N, 200, 7, must=far_rows)
    want_f = np.array([0.5 * (P["f"][i] + O.softmin_bilinear_one(i, P["X"], P["V"], P["s"], P["t"],
                                                                  P["h"], P["lb"], EPS)) for i in I])
    tf = 0.5 * tol_rows(P["X"], P["V"], P["s"], P["t"], P["h"], P["lb"], EPS, prec, I) \
        + 1e-7 * np.abs(want_f)
    ef = np.abs(fo[I] - want_f)
    assert np.all(ef <= tf), (prec, ef.max(), I[np.argmax(ef - tf)])
    J = sampled(N, 200, 8)
    want_g = np.array([0.5 * (P["h"][j] + O.softmin_bilinear_one(j, P["V"], P["X"], P["t"], P["s"],
                                                                  P["f"], P["la"], EPS)) for j in J])
    tg = 0.5 * tol_rows(P["V"], P["X"], P["t"], P["s"], P["f"], P["la"], EPS, prec, J) \
        + 1e-7 * np.abs(want_g)
    eg = np.abs(go[J] - want_g)
    assert np.all(eg <= tg), (prec, eg.max(), J[np.argmax(eg - tg)])
    assert np.isfinite(fo).all() and np.isfinite(go).all()


@pytest.mark.parametrize("prec", [3, 2])
def test_plan_sums_at_bench_size(gw, big, prec):
    """W_j = sum_i pi_ij [X_i, s_i, 1] with 100k sources (13 source splits of
    at most 128 tiles) for sampled targets j, against the oracle's plan
    column over all sources; bound as in test_gpu_plan's tensor-core test,
    with S the largest sum of absolute exponent terms of the sampled columns."""
    P = big
    G, stats, Wd = gw.gw_cross_cov(f32(P["X"]), f32(P["Y"]), f32(P["s"]), f32(P["t"]), f32(P["a"]),
                                   f32(P["b"]), f32(P["f"]), f32(P["g_plan"]), f64(P["Gamma"]), EPS,
                                   prec=prec, want_W=True)
    Wd = host(Wd)
    J = sampled(N, 128, 9)
    U = np.concatenate([P["X"], P["s"][:, None], np.ones((N, 1))], axis=1)
    C = O.cost_gamma(P["X"], P["Y"][J], P["Gamma"], P["s"], P["t"][J])
    pi = O.plan(P["a"], P["b"][J], P["f"], P["g_plan"][J], C, EPS)     # N x |J|
    W_ref = pi.T @ U
    S = (16.0 * np.abs(P["X"]) @ np.abs(P["V"][J]).T + 4.0 * np.outer(P["s"], P["t"][J])
         + np.abs(P["f"])[:, None] + np.abs(P["g_plan"][J])[None, :]
         + EPS * (np.abs(P["la"])[:, None] + np.abs(P["lb"][J])[None, :])).max()
    rel = 2.0 * ((D + 4) * TERM_REL[prec] * S / EPS + math.sqrt(N) * 2.0 ** -23 + 2.0 ** -20)
    Wb = rel * (pi.T @ np.abs(U))
    err = np.abs(Wd[J] - W_ref)
    assert np.all(err <= Wb + 1e-15), (prec, np.max(err / (Wb + 1e-15)))
    assert np.isfinite(host(G)).all()


def test_fp8_fused_iteration_at_bench_size(gw, big):
    """The FP8 mode's fused iteration at N = M = 100k, D = 32 on sampled rows
    (fast pass and the far rows' safe pass) against the oracle over all 100k
    points of the other side on the features helpers.fp8_operands rounds
    (one power-of-two scale per 128 rows of X and of V, e4m3), within the
    FP32-accumulation and split-BF16 bound; beside it, the rounding's own
    effect against the exact features is at most eps times the largest
    exponent change it makes in the row."""
    from helpers import fp8_operands, softmin_tolerance_fp8_emulated
    P = big
    Xh, Vh = fp8_operands(P["X"], P["V"])
    fo, go = gw.gw_sinkhorn_iteration(f32(P["X"]), f32(P["V"]), f32(P["s"]), f32(P["t"]),
                                      f32(P["la"]), f32(P["lb"]), f32(P["f"]), f32(P["h"]), EPS,
                                      prec=4, symmetric=True)
    fo, go = host(fo), host(go)
    far_rows = np.flatnonzero(P["far"])[:40]
    I = sampled(N, 160, 17, must=far_rows)
    want_f = np.array([0.5 * (P["f"][i] + O.softmin_bilinear_one(i, Xh, Vh, P["s"], P["t"],
                                                                  P["h"], P["lb"], EPS)) for i in I])
    tf = np.array([0.5 * softmin_tolerance_fp8_emulated(Xh[i:i + 1], Vh, P["s"][i:i + 1], P["t"],
                                                        P["h"], P["lb"], EPS)[0] for i in I]) \
        + 1e-7 * np.abs(want_f)
    ef = np.abs(fo[I] - want_f)
    assert np.all(ef <= tf), (ef.max(), I[np.argmax(ef - tf)])
    J = sampled(N, 160, 18)
    want_g = np.array([0.5 * (P["h"][j] + O.softmin_bilinear_one(j, Vh, Xh, P["t"], P["s"],
                                                                  P["f"], P["la"], EPS)) for j in J])
    tg = np.array([0.5 * softmin_tolerance_fp8_emulated(Vh[j:j + 1], Xh, P["t"][j:j + 1], P["s"],
                                                        P["f"], P["la"], EPS)[0] for j in J]) \
        + 1e-7 * np.abs(want_g)
    eg = np.abs(go[J] - want_g)
    assert np.all(eg <= tg), (eg.max(), J[np.argmax(eg - tg)])
    # the rounding's own error on the row half against the exact features
    exact = np.array([0.5 * (P["f"][i] + O.softmin_bilinear_one(i, P["X"], P["V"], P["s"], P["t"],
                                                                 P["h"], P["lb"], EPS)) for i in I[:40]])
    dz = np.array([16.0 * np.abs(Xh[i] @ Vh.T - P["X"][i] @ P["V"].T).max() for i in I[:40]])
    assert np.all(np.abs(fo[I[:40]] - exact) <= 0.5 * dz + tf[:40])


def test_fp8_plan_sums_at_bench_size(gw, big):
    """The FP8 plan sums with 100k sources (many source splits) for sampled
    targets, against the oracle's plan columns over all sources on the
    e4m3-rounded features (helpers.fp8_operands); Gamma_t = I / 4 so that
    V = Gamma_t Y is exact in FP32 and both sides round the same V.  The
    column potential makes pi_ij / b_j <= 1 on the rounded cost, as in the
    16-bit test."""
    from helpers import fp8_operands
    P = big
    Gt = 0.25 * np.eye(D)
    V4 = 0.25 * P["Y"]
    Xh, Vh = fp8_operands(P["X"], V4)
    zc = max_exponent(Vh, Xh, P["t"], P["s"], P["f"], P["la"], EPS)
    g_plan = r32(-EPS * zc)
    G, stats, Wd = gw.gw_cross_cov(f32(P["X"]), f32(P["Y"]), f32(P["s"]), f32(P["t"]), f32(P["a"]),
                                   f32(P["b"]), f32(P["f"]), f32(g_plan), f64(Gt), EPS, prec=4,
                                   want_W=True)
    Wd = host(Wd)
    J = sampled(N, 96, 19)
    U = np.concatenate([P["X"], P["s"][:, None], np.ones((N, 1))], axis=1)
    C = -16.0 * Xh @ Vh[J].T - 4.0 * np.outer(P["s"], P["t"][J])
    pi = O.plan(P["a"], P["b"][J], P["f"], g_plan[J], C, EPS)
    W_ref = pi.T @ U
    S = (16.0 * np.abs(Xh) @ np.abs(Vh[J]).T + 4.0 * np.outer(P["s"], P["t"][J])
         + np.abs(P["f"])[:, None] + np.abs(g_plan[J])[None, :]
         + EPS * (np.abs(P["la"])[:, None] + np.abs(P["lb"][J])[None, :])).max()
    rel = 2.0 * ((D + 4) * 2.0 ** -15 * S / EPS + math.sqrt(N) * 2.0 ** -23 + 2.0 ** -20)
    Wb = rel * (pi.T @ np.abs(U))
    err = np.abs(Wd[J] - W_ref)
    assert np.all(err <= Wb + 1e-15), np.max(err / (Wb + 1e-15))
    assert np.isfinite(host(G)).all()
