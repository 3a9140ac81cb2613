"""GW_PREC_FP8 (E4M3 features with one power-of-two scale per 128-row group
on tcgen05 kind::f8f6f4, split-BF16 bias columns, the coefficient 16 log2(e) /
eps in the epilogue) against the FP64 oracle.  Parity: the mode computes the
softmin of the Sinkhorn operator on c_Gamma (Eq. sinkhorn_operators with the
bilinear cost) and the plan-weighted sums of Algorithm 1 on the features
helpers.fp8_operands rounds from the mode's definition, so the oracle on those
features must agree within the FP32 accumulation and split-BF16 bound.  The
error of the rounding itself (against the oracle on the exact features) is
measured beside it and checked against its analytic size."""

import numpy as np
import pytest

import oracle as O
import workloads as W
from helpers import f32, fp8_operands, host, softmin_tolerance_fp8_emulated

pytestmark = pytest.mark.gpu

PREC_FP8 = 4


def make_inputs(n, m, K, seed, scale=0.5, zero_cols=0):
    g = W.rng(seed)
    A = scale * g.standard_normal((n, K))
    B = scale * g.standard_normal((m, K))
    sA, sB = (A * A).sum(1), (B * B).sum(1)
    h = 0.3 * g.standard_normal(m)
    logw = np.log(W.random_weights(m, seed + 1))
    if zero_cols:
        logw[g.choice(m, zero_cols, replace=False)] = -np.inf
    r = lambda x: np.asarray(x, np.float32).astype(np.float64)
    return r(A), r(B), r(sA), r(sB), r(h), r(logw)


def oracle_softmin(A, B, sA, sB, h, logw, eps):
    C = -16.0 * A @ B.T - 4.0 * np.outer(sA, sB)
    return O.softmin(eps, logw, h, C)


@pytest.mark.parametrize("n,m,K", [(3000, 2500, 32), (1100, 700, 64), (513, 2049, 20),
                                   (300, 517, 3), (257, 300, 128), (200, 333, 100),
                                   (1, 1, 1)])
@pytest.mark.parametrize("eps", [0.05, 0.01])
def test_fp8_softmin_matches_oracle_on_rounded_operands(gw, n, m, K, eps):
    A, B, sA, sB, h, logw = make_inputs(n, m, K, seed=n + 3 * m + K, zero_cols=min(5, m - 1))
    out = host(gw.gw_sinkhorn_softmin(f32(A), f32(B), f32(sA), f32(sB), f32(h), f32(logw), eps,
                                      prec=PREC_FP8))
    Ah, Bh = fp8_operands(A, B, eps)
    want = oracle_softmin(Ah, Bh, sA, sB, h, logw, eps)
    tol = softmin_tolerance_fp8_emulated(Ah, Bh, sA, sB, h, logw, eps)
    err = np.abs(out - want)
    assert np.all(err <= tol), (err.max(), tol[np.argmax(err - tol)], np.argmax(err - tol))
    # the rounding's own error against the exact operands: at most eps times
    # the largest exponent change it makes in the row (softmin is 1-Lipschitz
    # in the max norm), and here well above the split-f16 bar
    exact = oracle_softmin(A, B, sA, sB, h, logw, eps)
    dz = 16.0 * np.abs(Ah @ Bh.T - A @ B.T).max(axis=1)
    assert np.all(np.abs(out - exact) <= dz + tol)


@pytest.mark.parametrize("quality", ["good", "far", "mixed"])
def test_fp8_shift_estimate_paths(gw, quality):
    """The fast pass (estimate folded into the MMA, scaled with the row) and
    the safe pass for rows whose estimate is off by 2^+-430."""
    n, m, K, eps = 3000, 2000, 32, 0.05
    A, B, sA, sB, h, logw = make_inputs(n, m, K, seed=31)
    Ah, Bh = fp8_operands(A, B, eps)
    ref = oracle_softmin(Ah, Bh, sA, sB, h, logw, eps)
    g = W.rng(77)
    if quality == "good":
        prev = ref + 1e-3 * eps * g.standard_normal(n)
    elif quality == "far":
        prev = ref + 300.0 * eps * np.sign(g.standard_normal(n))
    else:
        prev = ref + np.where(g.random(n) < 0.02, 300.0 * eps, 0.01 * eps)
    prev = np.asarray(prev, np.float32).astype(np.float64)
    out = gw.gw_sinkhorn_softmin(f32(A), f32(B), f32(sA), f32(sB), f32(h), f32(logw), eps,
                                 prec=PREC_FP8, avg_with=f32(prev))
    want = 0.5 * (prev + ref)
    tol = 0.5 * softmin_tolerance_fp8_emulated(Ah, Bh, sA, sB, h, logw, eps) + 1e-7 * np.abs(want)
    err = np.abs(host(out) - want)
    assert np.all(err <= tol), (quality, err.max())


def test_fp8_iteration_and_reuse(gw):
    """gw_sinkhorn_iteration in FP8 (both halves in one launch) against the
    oracle on the rounded operands; with reuse = 1 after a call on other
    potentials (the bias and shift columns refreshed under the kept scales)
    the result equals a fresh preparation bitwise."""
    n, m, K, eps = 1500, 1300, 32, 0.05
    A, B, sA, sB, _, _ = make_inputs(n, m, K, seed=5)
    g0 = W.rng(6)
    la = np.log(np.asarray(W.random_weights(n, 7), np.float32)).astype(np.float64)
    lb = np.log(np.asarray(W.random_weights(m, 8), np.float32)).astype(np.float64)
    f = np.asarray(0.2 * g0.standard_normal(n), np.float32).astype(np.float64)
    g = np.asarray(0.2 * g0.standard_normal(m), np.float32).astype(np.float64)
    fo, go = gw.gw_sinkhorn_iteration(f32(A), f32(B), f32(sA), f32(sB), f32(la), f32(lb), f32(f),
                                      f32(g), eps, prec=PREC_FP8, symmetric=True)
    Ah, Bh = fp8_operands(A, B, eps)
    Bh2, Ah2 = fp8_operands(B, A, eps)          # the column half: B as the row side
    C = -16.0 * Ah @ Bh.T - 4.0 * np.outer(sA, sB)
    C2 = -16.0 * Bh2 @ Ah2.T - 4.0 * np.outer(sB, sA)
    want_f = 0.5 * (f + O.softmin(eps, lb, g, C))
    want_g = 0.5 * (g + O.softmin(eps, la, f, C2))
    tol_f = 0.5 * softmin_tolerance_fp8_emulated(Ah, Bh, sA, sB, g, lb, eps)
    tol_g = 0.5 * softmin_tolerance_fp8_emulated(Bh2, Ah2, sB, sA, f, la, eps)
    assert np.all(np.abs(host(fo) - want_f) <= tol_f)
    assert np.all(np.abs(host(go) - want_g) <= tol_g)
    ws = gw.workspace(gw.gw_workspace_size(gw.OP_ITERATION, n, m, K, 1, PREC_FP8), "cuda")
    gw.gw_sinkhorn_iteration(f32(A), f32(B), f32(sA), f32(sB), f32(la), f32(lb), f32(0.5 * f),
                             f32(-g), eps, prec=PREC_FP8, symmetric=True, ws=ws)
    fr, gr = gw.gw_sinkhorn_iteration(f32(A), f32(B), f32(sA), f32(sB), f32(la), f32(lb), f32(f),
                                      f32(g), eps, prec=PREC_FP8, symmetric=True, reuse=True,
                                      ws=ws)
    assert bool((fr == fo).all()) and bool((gr == go).all())


@pytest.mark.parametrize("D", [16, 64])
def test_cross_cov_fp8_matches_oracle_on_rounded_operands(gw, D):
    """The plan-weighted sums with the exponent on E4M3 features: W_j =
    sum_i pi_ij [X_i, s_i, 1] and Gamma_{t+1} against the dense FP64 plan of
    the cost on the rounded features (Gamma_t = I / 4 so that V = Gamma_t Y is
    exact in FP32 and both sides round the same V), potentials from oracle
    Sinkhorn iterations on that cost.  D = 64 takes the plan kernel's widest
    W accumulator (D + 3 columns in 80)."""
    from helpers import f64
    n, m, eps = 1500, 1300, 0.05
    g = W.rng(9)
    a, b = W.random_weights(n, 10, 0.3), W.random_weights(m, 11, 0.3)
    r32 = lambda x: np.asarray(x, np.float32).astype(np.float64)
    X = g.standard_normal((n, D)) / np.sqrt(D)
    Y = g.standard_normal((m, D)) / np.sqrt(D)
    X, Y, a, b = r32(X - a @ X), r32(Y - b @ Y), r32(a), r32(b)
    s, t = r32((X * X).sum(1)), r32((Y * Y).sum(1))
    Gt = 0.25 * np.eye(D)
    Xh, Vh = fp8_operands(X, 0.25 * Y)
    C = -16.0 * Xh @ Vh.T - 4.0 * np.outer(s, t)
    f, gg = O.sinkhorn(a, b, C, eps, 30)
    f, gg = r32(f), r32(gg)
    G, stats, Wd = gw.gw_cross_cov(f32(X), f32(Y), f32(s), f32(t), f32(a), f32(b), f32(f),
                                   f32(gg), f64(Gt), eps, prec=PREC_FP8, want_W=True)
    pi = O.plan(a, b, f, gg, C, eps)
    S = (16 * np.abs(Xh) @ np.abs(Vh).T + 4 * np.outer(s, t) + np.abs(f)[:, None]
         + np.abs(gg)[None, :] + eps * (np.abs(np.log(a))[:, None] + np.abs(np.log(b))[None, :])).max()
    rel = 2.0 * ((D + 4) * 2.0 ** -15 * S / eps + np.sqrt(n) * 2.0 ** -23 + 2.0 ** -20)
    W_ref = np.concatenate([pi.T @ X, (pi.T @ s)[:, None], pi.sum(0)[:, None]], axis=1)
    Wb = rel * np.concatenate([pi.T @ np.abs(X), (pi.T @ s)[:, None], pi.sum(0)[:, None]], axis=1)
    err = np.abs(host(Wd) - W_ref)
    assert np.all(err <= Wb + 1e-15), np.max(err / (Wb + 1e-15))
    bound = rel * (np.abs(X).T @ pi @ np.abs(Y)) + 1e-12
    assert np.all(np.abs(host(G) - X.T @ pi @ Y) <= bound)


def test_fp8_solve_runs_and_states_its_error(gw):
    """A lifted solve in FP8 (softmin and plan sums on E4M3 features, the same
    rounding in every kernel): finite, status clean, and an energy error
    against the FP64 oracle far above the split-f16 form's on the same
    problem (the statement the mode's docs make)."""
    import torch
    w = W.gmm_rigid(1000, seed=8, m=900)
    a = np.full(1000, 1 / 1000)
    b = np.full(900, 1 / 900)
    X = O.lift(w["x"], a, "power", 1.0, D=16)["X"]
    Y = O.lift(w["y"], b, "power", 1.0, D=16)["X"]
    r32 = lambda v: np.asarray(v, np.float32).astype(np.float64)
    X, Y = r32(X), r32(Y)
    s, t = (X * X).sum(1), (Y * Y).sum(1)
    ref = O.cnt_gw(a, b, X, Y, 0.1, 6, 40, eps_final=0.02, symmetric=True, record=True)
    e_ref = ref["history"][-1]["E"]
    dev = lambda v: torch.tensor(np.ascontiguousarray(v, np.float32), device="cuda")
    errs = {}
    for prec in (3, PREC_FP8):
        res = gw.gw_solve(dev(X), dev(Y), dev(s), dev(t), dev(a), dev(b), 0.1, 6, 40,
                          eps_final=0.02, prec=prec, record=False)
        en = res["energy"].cpu().numpy()
        assert np.isfinite(en[gw.EN["E"]]) and en[gw.EN["status"]] == 0.0
        errs[prec] = abs(en[gw.EN["E"]] - e_ref) / abs(e_ref)
    print("relative energy error: F16X3 %.3g, FP8 %.3g" % (errs[3], errs[PREC_FP8]))
    assert errs[3] < 1e-3
    assert errs[PREC_FP8] > 10.0 * errs[3]


def test_fp8_solve_at_d64_runs(gw):
    """An FP8 solve with D = 64 (the large-scale configuration's width): the
    plan sums run on tcgen05 with the same rounded features, so the annealed
    solve stays finite with a clean status down to eps = 5e-3."""
    import torch
    g = W.rng(12)
    n, D = 3000, 64
    sig = (1.0 + np.arange(D)) ** -1.0
    X = g.standard_normal((n, D)) * sig
    Y = g.standard_normal((n, D)) * sig
    X, Y = X - X.mean(0), Y - Y.mean(0)
    dev = lambda v: torch.tensor(np.ascontiguousarray(v, np.float32), device="cuda")
    X, Y = dev(X), dev(Y)
    s, t = (X * X).sum(1).contiguous(), (Y * Y).sum(1).contiguous()
    a = torch.full((n,), 1.0 / n, device="cuda")
    res = gw.gw_solve(X, Y, s, t, a, a.clone(), 0.1, 8, 40, eps_final=0.005, prec=PREC_FP8,
                      record=True)
    h = res["history"].cpu().numpy()
    assert np.isfinite(h[:, gw.EN["E"]]).all() and (h[:, gw.EN["status"]] == 0).all()
