"""GPU softmin (gw_sinkhorn_softmin through the C-ABI) against the FP64 oracle."""

import math

import numpy as np
import pytest

import oracle as O
import workloads as W
from helpers import f32, host, softmin_tolerance

pytestmark = pytest.mark.gpu


def make_inputs(n, m, K, seed, scale=0.5, zero_cols=0):
    g = W.rng(seed)
    A = scale * g.standard_normal((n, K))
    B = scale * g.standard_normal((m, K))
    sA = (A * A).sum(1)
    sB = (B * B).sum(1)
    h = 0.3 * g.standard_normal(m)
    w = W.random_weights(m, seed + 1)
    logw = np.log(w)
    if zero_cols:
        logw[g.choice(m, zero_cols, replace=False)] = -np.inf
    # round to the FP32 values the GPU sees, so both sides take the same inputs
    r = lambda x: np.asarray(x, np.float32).astype(np.float64)
    return r(A), r(B), r(sA), r(sB), r(h), r(logw)


def oracle_softmin(A, B, sA, sB, h, logw, eps):
    C = -16.0 * A @ B.T - 4.0 * np.outer(sA, sB)
    return O.softmin(eps, logw, h, C)


SHAPES = [(1, 1, 1), (7, 5, 2), (300, 517, 3), (1000, 1000, 2), (513, 2049, 16),
          (1200, 700, 32), (257, 300, 64), (100, 90, 128), (4099, 33, 5), (31, 5000, 8)]


@pytest.mark.parametrize("n,m,K", SHAPES)
@pytest.mark.parametrize("eps", [1.0, 0.05])
def test_softmin_matches_oracle(gw, n, m, K, eps):
    A, B, sA, sB, h, logw = make_inputs(n, m, K, seed=n + 7 * m + K)
    out = gw.gw_sinkhorn_softmin(f32(A), f32(B), f32(sA), f32(sB), f32(h), f32(logw), eps)
    ref = oracle_softmin(A, B, sA, sB, h, logw, eps)
    tol = softmin_tolerance(A, B, sA, sB, h, logw, eps)
    err = np.abs(host(out) - ref)
    assert np.all(err <= tol), (err.max(), tol[np.argmax(err - tol)])


def test_softmin_average_and_alias(gw):
    A, B, sA, sB, h, logw = make_inputs(640, 900, 4, seed=3)
    eps = 0.1
    prev = W.rng(9).standard_normal(640).astype(np.float32)
    out = f32(prev)
    gw.gw_sinkhorn_softmin(f32(A), f32(B), f32(sA), f32(sB), f32(h), f32(logw), eps,
                           avg_with=out, out=out)
    ref = 0.5 * (prev.astype(np.float64) + oracle_softmin(A, B, sA, sB, h, logw, eps))
    tol = 0.5 * softmin_tolerance(A, B, sA, sB, h, logw, eps) + 1e-7 * np.abs(ref)
    assert np.all(np.abs(host(out) - ref) <= tol)


def test_softmin_zero_weight_columns(gw):
    A, B, sA, sB, h, logw = make_inputs(300, 400, 3, seed=5, zero_cols=150)
    eps = 0.2
    out = gw.gw_sinkhorn_softmin(f32(A), f32(B), f32(sA), f32(sB), f32(h), f32(logw), eps)
    ref = oracle_softmin(A, B, sA, sB, h, logw, eps)
    assert np.all(np.abs(host(out) - ref) <= softmin_tolerance(A, B, sA, sB, h, logw, eps))


def test_softmin_small_eps_large_cost(gw):
    """eps = 1e-3 with radius-1 features (the paper's setting): exponents in
    the tens of thousands, still within the derived FP32 bound."""
    A, B, sA, sB, h, logw = make_inputs(777, 1500, 32, seed=11, scale=1.0 / math.sqrt(32))
    eps = 1e-3
    out = gw.gw_sinkhorn_softmin(f32(A), f32(B), f32(sA), f32(sB), f32(h), f32(logw), eps)
    ref = oracle_softmin(A, B, sA, sB, h, logw, eps)
    assert np.all(np.abs(host(out) - ref) <= softmin_tolerance(A, B, sA, sB, h, logw, eps))


def test_softmin_empty_rows_and_validation(gw):
    import torch
    z = torch.zeros(0, 3, device="cuda")
    B = torch.randn(5, 3, device="cuda")
    out = gw.gw_sinkhorn_softmin(z, B, torch.zeros(0, device="cuda"), torch.ones(5, device="cuda"),
                                 torch.zeros(5, device="cuda"), torch.zeros(5, device="cuda"), 0.1)
    assert out.numel() == 0
    with pytest.raises(gw.GWError) as e:
        gw.gw_sinkhorn_softmin(B, B, torch.ones(5, device="cuda"), torch.ones(5, device="cuda"),
                               torch.zeros(5, device="cuda"), torch.zeros(5, device="cuda"), 0.0)
    assert e.value.code == 1
    with pytest.raises(gw.GWError) as e:
        ws = torch.empty(256, dtype=torch.uint8, device="cuda")
        A = torch.randn(5000, 3, device="cuda")
        gw.gw_sinkhorn_softmin(A, torch.randn(5000, 3, device="cuda"), torch.ones(5000, device="cuda"),
                               torch.ones(5000, device="cuda"), torch.zeros(5000, device="cuda"),
                               torch.zeros(5000, device="cuda"), 0.1, ws=ws)
    assert e.value.code == 2


def test_softmin_is_deterministic(gw):
    A, B, sA, sB, h, logw = make_inputs(3000, 2500, 16, seed=21)
    args = [f32(v) for v in (A, B, sA, sB, h, logw)]
    o1 = gw.gw_sinkhorn_softmin(*args, 0.07)
    o2 = gw.gw_sinkhorn_softmin(*args, 0.07)
    assert bool((o1 == o2).all())


TC_SHAPES = [(1, 1, 1), (7, 5, 2), (300, 517, 3), (513, 2049, 16), (1200, 700, 32),
             (257, 300, 60), (4099, 33, 5), (31, 5000, 8), (2000, 2000, 32), (300, 400, 64),
             (700, 1500, 64)]


@pytest.mark.parametrize("prec", [1, 2, 3])
@pytest.mark.parametrize("n,m,K", TC_SHAPES)
@pytest.mark.parametrize("eps", [1.0, 0.05])
def test_tensor_core_softmin_matches_oracle(gw, prec, n, m, K, eps):
    from helpers import softmin_tolerance_prec
    if prec in (2, 3) and 3 * K + 10 > 256:
        pytest.skip("split modes take K <= 82")
    A, B, sA, sB, h, logw = make_inputs(n, m, K, seed=n + 7 * m + K)
    out = gw.gw_sinkhorn_softmin(f32(A), f32(B), f32(sA), f32(sB), f32(h), f32(logw), eps, prec=prec)
    ref = oracle_softmin(A, B, sA, sB, h, logw, eps)
    tol = softmin_tolerance_prec(A, B, sA, sB, h, logw, eps, prec)
    err = np.abs(host(out) - ref)
    assert np.all(err <= tol), (prec, err.max(), tol[np.argmax(err - tol)], np.argmax(err - tol))


@pytest.mark.parametrize("prec", [2, 3])
def test_tensor_core_small_eps_and_zero_weights(gw, prec):
    from helpers import softmin_tolerance_prec
    A, B, sA, sB, h, logw = make_inputs(777, 1500, 32, seed=11, scale=1.0 / math.sqrt(32),
                                        zero_cols=100)
    eps = 1e-3
    out = gw.gw_sinkhorn_softmin(f32(A), f32(B), f32(sA), f32(sB), f32(h), f32(logw), eps, prec=prec)
    ref = oracle_softmin(A, B, sA, sB, h, logw, eps)
    assert np.all(np.abs(host(out) - ref) <= softmin_tolerance_prec(A, B, sA, sB, h, logw, eps, prec))


def test_tensor_core_average_alias_and_determinism(gw):
    A, B, sA, sB, h, logw = make_inputs(3000, 2500, 16, seed=21)
    args = [f32(v) for v in (A, B, sA, sB, h, logw)]
    o1 = gw.gw_sinkhorn_softmin(*args, 0.07, prec=3)
    o2 = gw.gw_sinkhorn_softmin(*args, 0.07, prec=3)
    assert bool((o1 == o2).all())
    prev = o1.clone()
    gw.gw_sinkhorn_softmin(*args, 0.07, prec=3, avg_with=prev, out=prev)
    assert bool((prev == o1).all())   # (x + x) / 2 == x exactly


@pytest.mark.parametrize("prec", [1, 3])
@pytest.mark.parametrize("quality", ["good", "far", "mixed"])
def test_tensor_core_shift_estimate_paths(gw, prec, quality):
    """avg_with (not aliased to out) doubles as the per-row shift estimate of
    the fast pass.  Good estimates take the fast path; estimates off by more
    than the safe range (some or all rows) send their CTAs through the safe
    pass.  Every case must match the oracle."""
    from helpers import softmin_tolerance_prec
    n, m, K, eps = 3000, 2000, 16, 0.05
    A, B, sA, sB, h, logw = make_inputs(n, m, K, seed=31)
    ref = oracle_softmin(A, B, sA, sB, h, logw, eps)
    g = W.rng(77)
    if quality == "good":
        prev = ref + 1e-3 * eps * g.standard_normal(n)
    elif quality == "far":
        prev = ref + 300.0 * eps * np.sign(g.standard_normal(n))   # 2^+-430: out of range
    else:
        prev = ref + np.where(g.random(n) < 0.02, 300.0 * eps, 0.01 * eps)
    prev = np.asarray(prev, np.float32).astype(np.float64)
    out = gw.gw_sinkhorn_softmin(f32(A), f32(B), f32(sA), f32(sB), f32(h), f32(logw), eps,
                                 prec=prec, avg_with=f32(prev))
    want = 0.5 * (prev + ref)
    tol = 0.5 * softmin_tolerance_prec(A, B, sA, sB, h, logw, eps, prec) + 1e-7 * np.abs(want)
    err = np.abs(host(out) - want)
    assert np.all(err <= tol), (quality, err.max())


@pytest.mark.parametrize("prec", [0, 3])
@pytest.mark.parametrize("symmetric", [True, False])
def test_sinkhorn_iteration_matches_oracle_and_reuse(gw, prec, symmetric):
    """gw_sinkhorn_iteration: one iteration of Algorithm 3 (or 2) against the
    oracle's, each half within its softmin tolerance (for Algorithm 2 the
    column half reads the device's own f'); with reuse = 1 after a call on
    other potentials, the result equals a fresh preparation."""
    from helpers import softmin_tolerance_prec
    n, m, K = 1500, 1300, 16
    A, B, sA, sB, _, _ = make_inputs(n, m, K, seed=5)
    g0 = W.rng(6)
    la = np.log(np.asarray(W.random_weights(n, 7), np.float32)).astype(np.float64)
    lb = np.log(np.asarray(W.random_weights(m, 8), np.float32)).astype(np.float64)
    f = np.asarray(0.2 * g0.standard_normal(n), np.float32).astype(np.float64)
    g = np.asarray(0.2 * g0.standard_normal(m), np.float32).astype(np.float64)
    eps = 0.05
    fo, go = gw.gw_sinkhorn_iteration(f32(A), f32(B), f32(sA), f32(sB), f32(la), f32(lb), f32(f),
                                      f32(g), eps, prec=prec, symmetric=symmetric)
    C = -16.0 * A @ B.T - 4.0 * np.outer(sA, sB)
    Sf = O.softmin(eps, lb, g, C)
    tol_f = softmin_tolerance_prec(A, B, sA, sB, g, lb, eps, prec)
    if symmetric:
        Sg = O.softmin(eps, la, f, C.T)
        want_f, want_g = 0.5 * (f + Sf), 0.5 * (g + Sg)
        tol_f = 0.5 * tol_f
        tol_g = 0.5 * softmin_tolerance_prec(B, A, sB, sA, f, la, eps, prec)
    else:
        fd = host(fo)
        want_f, want_g = Sf, O.softmin(eps, la, fd, C.T)
        tol_g = softmin_tolerance_prec(B, A, sB, sA, fd, la, eps, prec)
    assert np.all(np.abs(host(fo) - want_f) <= tol_f)
    assert np.all(np.abs(host(go) - want_g) <= tol_g)
    # reuse: prepare on other potentials, then iterate on (f, g) with reuse = 1
    ws = gw.workspace(gw.gw_workspace_size(gw.OP_ITERATION, n, m, K, 1, prec), "cuda")
    gw.gw_sinkhorn_iteration(f32(A), f32(B), f32(sA), f32(sB), f32(la), f32(lb), f32(0.5 * f),
                             f32(-g), eps, prec=prec, symmetric=symmetric, ws=ws)
    fr, gr = gw.gw_sinkhorn_iteration(f32(A), f32(B), f32(sA), f32(sB), f32(la), f32(lb), f32(f),
                                      f32(g), eps, prec=prec, symmetric=symmetric, reuse=True,
                                      ws=ws)
    assert bool((fr == fo).all()) and bool((gr == go).all())


def decaying_inputs(n, m, K, seed, eps):
    """Features with a decaying spectrum, as Kernel PCA features and
    V = Gamma Y have: A_k ~ (k + 1)^-1.5, B_k ~ (k + 1)^-3."""
    g = W.rng(seed)
    k = np.arange(K) + 1.0
    A = 0.6 * g.standard_normal((n, K)) * k ** -1.5
    B = 0.3 * g.standard_normal((m, K)) * k ** -3.0
    sA, sB = (A * A).sum(1), (B * B).sum(1)
    h = 0.05 * g.standard_normal(m)
    logw = np.log(W.random_weights(m, seed + 1))
    r = lambda x: np.asarray(x, np.float32).astype(np.float64)
    return r(A), r(B), r(sA), r(sB), r(h), r(logw)


@pytest.mark.parametrize("prec", [2, 3])
@pytest.mark.parametrize("K", [48, 64])
@pytest.mark.parametrize("eps", [0.5, 0.02])
def test_tensor_core_narrow_layout_matches_oracle(gw, prec, K, eps):
    """K >= 40 in the split precisions: with a decaying spectrum only the few
    dims of largest product bound need three products, so the 128-column
    layout runs (the rest as one product each).  Ragged sizes, a far-off
    estimate on some rows (safe pass) and the bound of helpers
    (softmin_tolerance_prec, which adds the one-product dims' error)."""
    from helpers import softmin_tolerance_prec
    n, m = 2051, 1537
    A, B, sA, sB, h, logw = decaying_inputs(n, m, K, seed=K + 3, eps=eps)
    ref = oracle_softmin(A, B, sA, sB, h, logw, eps)
    g = W.rng(5)
    prev = ref + np.where(g.random(n) < 0.03, 300.0 * eps, 0.01 * eps)
    prev = np.asarray(prev, np.float32).astype(np.float64)
    out = gw.gw_sinkhorn_softmin(f32(A), f32(B), f32(sA), f32(sB), f32(h), f32(logw), eps,
                                 prec=prec, avg_with=f32(prev))
    want = 0.5 * (prev + ref)
    tol = 0.5 * softmin_tolerance_prec(A, B, sA, sB, h, logw, eps, prec) + 1e-7 * np.abs(want)
    err = np.abs(host(out) - want)
    assert np.all(err <= tol), (prec, K, err.max(), np.argmax(err - tol))


@pytest.mark.parametrize("prec", [2, 3])
def test_narrow_layout_iteration_and_reuse(gw, prec):
    """The fused iteration (both half-steps, both tasks in one launch) at
    K = 64 with decaying spectra, and the per-iteration refresh of the bias
    and shift columns in the narrow layout (reuse = 1 equals a fresh
    preparation bitwise)."""
    from helpers import softmin_tolerance_prec
    n, m, K, eps = 1500, 1300, 64, 0.05
    A, B, sA, sB, _, _ = decaying_inputs(n, m, K, seed=11, eps=eps)
    g0 = W.rng(6)
    la = np.log(np.asarray(W.random_weights(n, 7), np.float32)).astype(np.float64)
    lb = np.log(np.asarray(W.random_weights(m, 8), np.float32)).astype(np.float64)
    f = np.asarray(0.05 * g0.standard_normal(n), np.float32).astype(np.float64)
    g = np.asarray(0.05 * g0.standard_normal(m), np.float32).astype(np.float64)
    fo, go = gw.gw_sinkhorn_iteration(f32(A), f32(B), f32(sA), f32(sB), f32(la), f32(lb), f32(f),
                                      f32(g), eps, prec=prec)
    C = -16.0 * A @ B.T - 4.0 * np.outer(sA, sB)
    want_f = 0.5 * (f + O.softmin(eps, lb, g, C))
    want_g = 0.5 * (g + O.softmin(eps, la, f, C.T))
    tol_f = 0.5 * softmin_tolerance_prec(A, B, sA, sB, g, lb, eps, prec) + 1e-7 * np.abs(want_f)
    tol_g = 0.5 * softmin_tolerance_prec(B, A, sB, sA, f, la, eps, prec) + 1e-7 * np.abs(want_g)
    assert np.all(np.abs(host(fo) - want_f) <= tol_f)
    assert np.all(np.abs(host(go) - want_g) <= tol_g)
    ws = gw.workspace(gw.gw_workspace_size(gw.OP_ITERATION, n, m, K, 1, prec), "cuda")
    gw.gw_sinkhorn_iteration(f32(A), f32(B), f32(sA), f32(sB), f32(la), f32(lb), f32(0.5 * f),
                             f32(-g), eps, prec=prec, ws=ws)
    fr, gr = gw.gw_sinkhorn_iteration(f32(A), f32(B), f32(sA), f32(sB), f32(la), f32(lb), f32(f),
                                      f32(g), eps, prec=prec, reuse=True, ws=ws)
    assert bool((fr == fo).all()) and bool((gr == go).all())
