"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a brute-force
sum, a closed form, an enumeration, an invariant or an independent solver.
"""

import itertools
import math

import numpy as np
import pytest

import oracle as O
import workloads as W


def nw_coupling(a, b, perm_a=None, perm_b=None):
    """Exact coupling in Pi(a, b) by the north-west corner rule on permuted
    index orders (test helper)."""
    N, M = len(a), len(b)
    pa = np.arange(N) if perm_a is None else perm_a
    pb = np.arange(M) if perm_b is None else perm_b
    ra, rb = a[pa].astype(float).copy(), b[pb].astype(float).copy()
    pi = np.zeros((N, M))
    i = j = 0
    while i < N and j < M:
        m = min(ra[i], rb[j])
        pi[pa[i], pb[j]] += m
        ra[i] -= m
        rb[j] -= m
        if ra[i] <= rb[j]:
            i += 1
        else:
            j += 1
    return pi


def centered(n, d, seed, w):
    x = W.random_features(n, d, seed)
    return x - w @ x


def small_problem(N=7, M=6, D=3, E=2, seed=0):
    a = W.random_weights(N, seed + 1)
    b = W.random_weights(M, seed + 2)
    X = centered(N, D, seed + 3, a)
    Y = centered(M, E, seed + 4, b)
    return a, b, X, Y


# ---------------------------------------------------------------- the Lemma

@pytest.mark.parametrize("seed", [0, 1, 2])
def test_lemma_matches_bruteforce_quartic(seed):
    a, b, X, Y = small_problem(seed=seed)
    g = W.rng(seed + 10)
    pi = 0.3 * np.outer(a, b) + 0.7 * nw_coupling(a, b, g.permutation(len(a)), g.permutation(len(b)))
    CX = O.pairwise_sqdist(X, X)
    CY = O.pairwise_sqdist(Y, Y)
    brute = O.gw_loss_bruteforce(pi, CX, CY)
    lemma = O.gw_loss_lemma(pi, X, Y, a, b)
    assert brute > 0
    assert abs(brute - lemma) <= 1e-12 * abs(brute)


def test_constant_moments_match_pairwise_definition():
    for seed in range(3):
        a, b, X, Y = small_problem(N=9, M=11, D=4, E=3, seed=seed)
        c1 = O.gw_constant_pairwise(X, Y, a, b)
        c2 = O.gw_constant_moments(X, Y, a, b)
        assert abs(c1 - c2) <= 1e-12 * abs(c1)


def test_constant_self_is_eight_sigma_plus_four_m4():
    """C(alpha, alpha) = 8 ||Sigma_alpha||_F^2 + 4 int ||x||^4 (proof of Prop. 4.3)."""
    a = W.random_weights(10, 5)
    X = centered(10, 3, 6, a)
    Sig = (X * a[:, None]).T @ X
    m4 = a @ (np.sum(X * X, 1) ** 2)
    direct = 8 * np.sum(Sig * Sig) + 4 * m4
    assert abs(O.gw_constant_pairwise(X, X, a, a) - direct) <= 1e-12 * direct


def test_zero_distortion_identity_coupling():
    """Prop. 2.1: alpha matched to itself by the identity coupling has L = 0."""
    a = W.random_weights(8, 3)
    X = centered(8, 3, 4, a)
    pi = np.diag(a)
    CX = O.pairwise_sqdist(X, X)
    assert O.gw_loss_bruteforce(pi, CX, CX) == 0.0
    assert abs(O.gw_loss_lemma(pi, X, X, a, a)) <= 1e-12 * O.gw_constant_pairwise(X, X, a, a)


# ------------------------------------------------------------ Sinkhorn pins

def test_softmin_limits():
    g = W.rng(0)
    N, M = 5, 7
    C = g.standard_normal((N, M))
    h = g.standard_normal(M)
    b = W.random_weights(M, 1)
    # eps -> infinity: -eps log sum b exp((h - C)/eps) -> sum_j b_j (C_ij - h_j)
    big = O.softmin(1e7, np.log(b), h, C)
    assert np.allclose(big, (C - h[None, :]) @ b, atol=1e-5)
    # eps -> 0: -> min_j (C_ij - h_j), at rate eps log(1/b)
    small = O.softmin(1e-4, np.log(b), h, C)
    assert np.allclose(small, (C - h[None, :]).min(1), atol=1e-4 * (np.abs(np.log(b)).max() + 1))
    # one column: exact
    one = O.softmin(0.3, np.log(b[:1] / b[:1].sum()), h[:1], C[:, :1])
    assert np.allclose(one, C[:, 0] - h[0], atol=1e-14)


def test_standard_sinkhorn_row_update_gives_exact_row_marginal():
    """After the f-update of Algorithm 2 the plan's rows sum to a exactly."""
    g = W.rng(1)
    a, b = W.random_weights(6, 2), W.random_weights(9, 3)
    C = g.standard_normal((6, 9))
    f = O.softmin(0.2, np.log(b), np.zeros(9), C)
    pi = O.plan(a, b, f, np.zeros(9), C, 0.2)
    assert np.allclose(pi.sum(1), a, rtol=1e-13, atol=0)


@pytest.mark.parametrize("symmetric", [False, True])
def test_sinkhorn_converges_to_marginals(symmetric):
    g = W.rng(2)
    a, b = W.random_weights(12, 4), W.random_weights(10, 5)
    C = g.standard_normal((12, 10))
    f, gg = O.sinkhorn(a, b, C, 0.5, 400, symmetric=symmetric)
    pi = O.plan(a, b, f, gg, C, 0.5)
    assert O.marginal_error(pi, a, b) < 1e-12


def test_row_marginal_from_potentials():
    g = W.rng(3)
    a, b = W.random_weights(8, 6), W.random_weights(5, 7)
    C = g.standard_normal((8, 5))
    f, gg = g.standard_normal(8), g.standard_normal(5)
    r = O.row_marginal_from_potentials(a, b, f, gg, C, 0.7)
    assert np.allclose(r, O.plan(a, b, f, gg, C, 0.7).sum(1), rtol=1e-13)


def test_small_eps_plan_is_optimal_permutation():
    """eps -> 0 with uniform weights: the entropic plan concentrates on the
    optimal assignment (found by enumeration)."""
    n = 6
    g = W.rng(4)
    C = g.random((n, n))
    a = b = W.uniform_weights(n)
    _, perm = O.permutation_ot(C)
    f, gg = O.sinkhorn(a, b, C, 2e-3, 3000, symmetric=False)
    pi = O.plan(a, b, f, gg, C, 2e-3)
    P = np.zeros((n, n))
    P[np.arange(n), perm] = 1.0 / n
    assert np.abs(pi - P).sum() < 1e-3


def test_large_eps_plan_is_product_and_gamma_vanishes():
    """eps -> infinity: pi -> a x b (proof of Theorem 4.1) and then
    Gamma_1 = (sum a X)(sum b Y)^T = 0 by centering."""
    a, b, X, Y = small_problem(N=9, M=8, D=3, E=3, seed=7)
    res = O.cnt_gw(a, b, X, Y, eps=1e8, n_outer=1, n_inner=5, Gamma0=W.rng(0).standard_normal((3, 3)))
    f, g = res["f"], res["g"]
    C = O.cost_gamma(X, Y, W.rng(0).standard_normal((3, 3)))
    pi = O.plan(a, b, f, g, C, 1e8)
    assert np.abs(pi - np.outer(a, b)).max() < 1e-6
    assert np.abs(res["Gamma"]).max() < 1e-6


# --------------------------------------------------- the solver's structure

def converged_cntgw(a, b, X, Y, eps, n_outer, Gamma0, n_inner=600):
    return O.cnt_gw(a, b, X, Y, eps, n_outer, n_inner, Gamma0=Gamma0, symmetric=False)


def test_cntgw_step_equals_entropic_gw_step():
    """Prop. 4.4: for CNT costs the coupling produced by one alternate step from
    Gamma_t = Gamma(pi_t) equals Entropic-GW's update from pi_t."""
    a, b, X, Y = small_problem(N=7, M=8, D=3, E=2, seed=11)
    g = W.rng(12)
    pi_t = 0.5 * np.outer(a, b) + 0.5 * nw_coupling(a, b, g.permutation(7), g.permutation(8))
    Gamma_t = O.cross_covariance(pi_t, X, Y)
    eps = 0.05
    C = O.cost_gamma(X, Y, Gamma_t)
    f, gg = O.sinkhorn(a, b, C, eps, 3000, symmetric=False)
    pi_cnt = O.plan(a, b, f, gg, C, eps)
    pi_egw = O.entropic_gw_step(pi_t, O.pairwise_sqdist(X, X), O.pairwise_sqdist(Y, Y), a, b, eps, 3000)
    assert np.abs(pi_cnt - pi_egw).max() < 1e-10


def test_kernel_gw_matches_cntgw_with_full_rank_kernel_pca():
    """Algorithm 5 (Kernel-GW) and Algorithm 1 on exact (full-rank) Kernel PCA
    features of the Euclidean cost ||x - x'|| produce the same potentials and
    plans from the same starting plan."""
    N, M = 9, 8
    g = W.rng(13)
    x, y = g.standard_normal((N, 3)), g.standard_normal((M, 3))
    a, b = W.uniform_weights(N), W.uniform_weights(M)
    CX, CY = O.cnt_cost(x, x, "power", 1.0), O.cnt_cost(y, y, "power", 1.0)
    LX = O.lift(x, a, "power", 1.0, D=N - 1)
    LY = O.lift(y, b, "power", 1.0, D=M - 1)
    eps = 0.3
    pi0 = 0.5 * np.outer(a, b) + 0.5 * nw_coupling(a, b, g.permutation(N), g.permutation(M))
    Gamma0 = O.cross_covariance(pi0, LX["X"], LY["X"])
    pi_k, f_k, g_k = O.kernel_gw(a, b, CX, CY, eps, 3, 800, pi0=pi0, symmetric=False)
    res = O.cnt_gw(a, b, LX["X"], LY["X"], eps, 3, 800, Gamma0=Gamma0, symmetric=False)
    assert np.abs(res["f"] - f_k).max() < 1e-9
    assert np.abs(res["g"] - g_k).max() < 1e-9
    assert np.abs(res["history"][-1]["row"] - pi_k.sum(1)).max() < 1e-9
    assert np.abs(res["Gamma"] - O.cross_covariance(pi_k, LX["X"], LY["X"])).max() < 1e-9


def test_dual_gradient_step():
    """Prop. 4.5: grad D_eps(Gamma_t) = 2 Gamma_t - 2 Gamma_{t+1}, checked with
    central finite differences of D_eps."""
    a, b, X, Y = small_problem(N=8, M=7, D=2, E=2, seed=21)
    eps = 0.2
    Gt = W.rng(22).standard_normal((2, 2)) * 0.1
    res = O.cnt_gw(a, b, X, Y, eps, 1, 3000, Gamma0=Gt, symmetric=False, record=False)
    analytic = 2 * Gt - 2 * res["Gamma"]
    h = 1e-5
    fd = np.zeros_like(Gt)
    for p in range(2):
        for q in range(2):
            Gp, Gm = Gt.copy(), Gt.copy()
            Gp[p, q] += h
            Gm[p, q] -= h
            fd[p, q] = (O.dual_function(Gp, a, b, X, Y, eps, 3000)[0]
                        - O.dual_function(Gm, a, b, X, Y, eps, 3000)[0]) / (2 * h)
    assert np.abs(fd - analytic).max() < 1e-7 * max(1.0, np.abs(analytic).max())


def test_step_norm_bound_and_monotone_energy():
    """Theorem 4.6: sum_k ||Gamma_k - Gamma_{k+1}||^2 <= D(Gamma_0) - D(Gamma_t);
    Prop. 4.4: the EGW energy decreases at every step (converged inner loops)."""
    a, b, X, Y = small_problem(N=10, M=9, D=3, E=3, seed=31)
    X, Y = 0.3 * X, 0.3 * Y
    eps = 0.05
    G0 = W.rng(32).standard_normal((3, 3)) * 0.05
    res = O.cnt_gw(a, b, X, Y, eps, 6, 3000, Gamma0=G0, symmetric=False)
    assert max(h["err"] for h in res["history"]) < 1e-10
    gammas = [G0] + [h["Gamma"] for h in res["history"]]
    steps = sum(np.sum((gammas[k] - gammas[k + 1]) ** 2) for k in range(6))
    D0 = O.dual_function(gammas[0], a, b, X, Y, eps, 3000)[0]
    Dt = O.dual_function(gammas[6], a, b, X, Y, eps, 3000)[0]
    assert steps > 0
    assert steps <= D0 - Dt + 1e-12
    E = [h["E"] for h in res["history"]]
    assert all(E[k + 1] <= E[k] + 1e-12 for k in range(len(E) - 1))


def test_dual_identity_at_fixed_point():
    """Remark (Eq. egw_otherform): at a fixed point, GW_eps = C + 8||Gamma||^2
    + <a, f> + <b, g>, while the primal value is L + eps KL of the plan."""
    a, b, X, Y = small_problem(N=8, M=8, D=2, E=2, seed=41)
    eps = 0.1
    G0 = W.rng(42).standard_normal((2, 2)) * 0.1
    res = O.cnt_gw(a, b, X, Y, eps, 80, 400, Gamma0=G0, symmetric=False, record=False)
    G = res["Gamma"]
    C = O.cost_gamma(X, Y, G)
    f, g = O.sinkhorn(a, b, C, eps, 4000, res["f"], res["g"], symmetric=False)
    pi = O.plan(a, b, f, g, C, eps)
    assert np.linalg.norm(O.cross_covariance(pi, X, Y) - G) < 1e-10
    primal = O.egw_energy(pi, X, Y, a, b, eps)["E"]
    dual = O.gw_constant_pairwise(X, Y, a, b) + 8 * np.sum(G * G) + a @ f + b @ g
    assert abs(primal - dual) < 1e-10 * abs(primal)


def test_two_point_closed_form():
    """alpha = beta = uniform on {0, 1} (squared cost).  Couplings are
    [[p, 1/2 - p], [1/2 - p, p]]; by Eq. GW_loss L(p) = 8 p (1/2 - p) and the
    EGW objective is E(p) = 8p(1/2-p) + eps [2p log 4p + (1-2p) log(2-4p)].
    Its minimiser on (1/4, 1/2) solves 4 - 16 p + 2 eps log(4p/(2-4p)) = 0,
    found here by bisection; CNT-GW from a positive Gamma_0 must reach it."""
    eps = 0.1
    lo, hi = 0.25 + 1e-12, 0.5 - 1e-15

    def dE(p):
        return 4 - 16 * p + 2 * eps * math.log(4 * p / (2 - 4 * p))
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if dE(mid) < 0:
            lo = mid
        else:
            hi = mid
    p = 0.5 * (lo + hi)
    E_star = 8 * p * (0.5 - p) + eps * (2 * p * math.log(4 * p) + (1 - 2 * p) * math.log(2 - 4 * p))
    x = np.array([[0.0], [1.0]])
    a = b = np.array([0.5, 0.5])
    X = O.center(x, a)
    res = O.cnt_gw(a, b, X, X, eps, 60, 500, Gamma0=np.array([[0.01]]), symmetric=False)
    last = res["history"][-1]
    assert abs(last["E"] - E_star) < 1e-10
    # also the unstable critical point: Gamma_0 = 0 keeps pi = a x b, E = 1/2
    res0 = O.cnt_gw(a, b, X, X, eps, 3, 200, symmetric=False)
    assert abs(res0["history"][-1]["E"] - 0.5) < 1e-12


def test_energy_invariant_under_isometries():
    """The costs depend only on pairwise distances, so E(Qx + c, y) = E(x, y)
    and the solve is equivariant: Gamma -> Q Gamma (rotation/reflection)."""
    g = W.rng(51)
    N, M = 12, 10
    x, y = g.standard_normal((N, 2)), g.standard_normal((M, 2))
    a, b = W.uniform_weights(N), W.uniform_weights(M)
    Q = W.random_orthogonal(2, g)
    X, Y = O.center(x, a), O.center(y, b)
    X2 = O.center(x @ Q.T + np.array([3.0, -1.0]), a)
    G0 = g.standard_normal((2, 2)) * 0.05
    r1 = O.cnt_gw(a, b, X, Y, 0.05, 5, 300, Gamma0=G0)
    r2 = O.cnt_gw(a, b, X2, Y, 0.05, 5, 300, Gamma0=Q @ G0)
    assert abs(r1["history"][-1]["E"] - r2["history"][-1]["E"]) < 1e-10 * abs(r1["history"][-1]["E"])
    assert np.allclose(Q @ r1["Gamma"], r2["Gamma"], atol=1e-10)


# ---------------------------------------------------------------- the lift

def test_squared_lift_is_centering_and_kernel_pca_agrees():
    g = W.rng(61)
    x = g.standard_normal((15, 3))
    a = W.random_weights(15, 62)
    L = O.lift(x, a)
    assert np.allclose(a @ L["X"], 0, atol=1e-14)
    Lk = O.lift(x, a, "sqeuclid", 2.0, D=3)
    # same Gram matrix, i.e. the same features up to an orthogonal map
    assert np.allclose(L["X"] @ L["X"].T, Lk["X"] @ Lk["X"].T, atol=1e-10)


def test_kernel_pca_full_rank_reproduces_cost():
    """At D = rank the Kernel PCA features satisfy ||X_i - X_k||^2 = c(x_i, x_k)
    exactly (Theorem 2.2 with Eqs. embedding_X)."""
    g = W.rng(71)
    x = g.standard_normal((20, 3))
    a = W.uniform_weights(20)
    for kind, param in [("power", 1.0), ("power", 0.5), ("gauss", 0.7)]:
        L = O.lift(x, a, kind, param, D=19)
        C = O.cnt_cost(x, x, kind, param)
        assert np.allclose(O.pairwise_sqdist(L["X"], L["X"]), C, atol=1e-9), kind
        assert np.allclose(a @ L["X"], 0, atol=1e-12)


def test_kernel_pca_is_rotation_invariant_up_to_sign():
    g = W.rng(72)
    x = g.standard_normal((30, 3))
    a = W.uniform_weights(30)
    Q = W.random_orthogonal(3, g)
    L1 = O.lift(x, a, "power", 1.0, D=5)
    L2 = O.lift(x @ Q.T + 2.0, a, "power", 1.0, D=5)
    assert np.allclose(L1["lam"], L2["lam"], rtol=1e-10)
    assert np.allclose(np.abs(L1["X"]), np.abs(L2["X"]), atol=1e-8)


def test_kernel_proj_reproduces_training_features():
    g = W.rng(73)
    x = g.standard_normal((25, 3))
    a = W.uniform_weights(25)
    L = O.lift(x, a, "power", 1.0, D=6)
    P = O.kernel_proj(x, x, a, L["V"], L["lam"], "power", 1.0)
    assert np.allclose(P, L["X"], atol=1e-10)


def test_kernel_proj_vjp_matches_finite_differences():
    g = W.rng(74)
    x = g.standard_normal((18, 3))
    a = W.uniform_weights(18)
    L = O.lift(x, a, "power", 1.0, D=4)
    xq = g.standard_normal((3, 3))
    G = g.standard_normal((3, 4))
    vjp = O.kernel_proj_vjp(G, xq, x, a, L["V"], L["lam"], "power", 1.0)
    h = 1e-6
    fd = np.zeros_like(xq)
    for q in range(3):
        for d in range(3):
            xp, xm = xq.copy(), xq.copy()
            xp[q, d] += h
            xm[q, d] -= h
            Pp = O.kernel_proj(xp, x, a, L["V"], L["lam"], "power", 1.0)
            Pm = O.kernel_proj(xm, x, a, L["V"], L["lam"], "power", 1.0)
            fd[q, d] = np.sum(G * (Pp - Pm)) / (2 * h)
    assert np.allclose(vjp, fd, atol=1e-7)


def test_kernel_proj_vjp_matches_finite_differences_gaussian_cost():
    """The same finite-difference pin for the Gaussian CNT cost
    2 (1 - exp(-||x - x'||^2 / (2 sigma^2))), whose cost gradient (the
    chain rule through the exponential) the power cost does not exercise."""
    g = W.rng(75)
    x = g.standard_normal((20, 3)) * 0.7
    a = W.uniform_weights(20)
    L = O.lift(x, a, "gauss", 0.8, D=5)
    xq = g.standard_normal((4, 3)) * 0.7
    G = g.standard_normal((4, 5))
    vjp = O.kernel_proj_vjp(G, xq, x, a, L["V"], L["lam"], "gauss", 0.8)
    h = 1e-6
    fd = np.zeros_like(xq)
    for q in range(4):
        for d in range(3):
            xp, xm = xq.copy(), xq.copy()
            xp[q, d] += h
            xm[q, d] -= h
            Pp = O.kernel_proj(xp, x, a, L["V"], L["lam"], "gauss", 0.8)
            Pm = O.kernel_proj(xm, x, a, L["V"], L["lam"], "gauss", 0.8)
            fd[q, d] = np.sum(G * (Pp - Pm)) / (2 * h)
    assert np.abs(vjp).max() > 1e-3          # the check is not vacuous
    assert np.allclose(vjp, fd, atol=1e-7)


def test_gaussian_cost_gradient_matches_finite_differences():
    """cnt_cost_grad1 of the Gaussian cost against central differences of
    cnt_cost (the derivative both the adjoint and the VJP take)."""
    g = W.rng(76)
    x = g.standard_normal((5, 3))
    y = g.standard_normal((6, 3))
    h = 1e-6
    for i in range(5):
        Gd = O.cnt_cost_grad1(x[i], y, "gauss", 0.9)    # (6, 3): d c(x_i, y_k) / d x_i
        assert np.abs(Gd).max() > 1e-3
        for d in range(3):
            xp, xm = x[i:i + 1].copy(), x[i:i + 1].copy()
            xp[0, d] += h
            xm[0, d] -= h
            fd = (O.cnt_cost(xp, y, "gauss", 0.9) - O.cnt_cost(xm, y, "gauss", 0.9))[0] / (2 * h)
            assert np.allclose(Gd[:, d], fd, atol=1e-8)


# ------------------------------------------------------------- gradients

def _converged_state(x, y, a, b, eps, G0, kind="sqeuclid", n_outer=60):
    X, Y = O.center(x, a), O.center(y, b)
    res = O.cnt_gw(a, b, X, Y, eps, n_outer, 400, Gamma0=G0, symmetric=False, record=False)
    C = O.cost_gamma(X, Y, res["Gamma"])
    f, g = O.sinkhorn(a, b, C, eps, 3000, res["f"], res["g"], symmetric=False)
    pi = O.plan(a, b, f, g, C, eps)
    return X, Y, res, pi


def test_gradient_closed_form_matches_bruteforce_quartic():
    g = W.rng(81)
    N, M = 9, 8
    x, y = g.standard_normal((N, 2)), g.standard_normal((M, 2))
    a, b = W.random_weights(N, 82), W.random_weights(M, 83)
    X, Y, res, pi = _converged_state(x, y, a, b, 0.1, g.standard_normal((2, 2)) * 0.1)
    G = O.cross_covariance(pi, X, Y)
    closed = O.grad_x_squared(pi, G, X, Y, a, b)
    brute = O.grad_x_bruteforce(pi, x, y, a, b)
    assert np.abs(closed - brute).max() < 1e-10 * np.abs(brute).max()
    assert np.abs(closed.sum(0)).max() < 1e-12 * np.abs(closed).max()   # translation invariance


def _energy_of_points(x, y, a, b, eps, G0, f0, g0, n_outer=80):
    X, Y = O.center(x, a), O.center(y, b)
    res = O.cnt_gw(a, b, X, Y, eps, n_outer, 300, Gamma0=G0, f0=f0, g0=g0, symmetric=False)
    return res["history"][-1]["E"]


def test_gradient_matches_finite_differences_of_resolved_energy():
    """Envelope theorem (Appendix B.6): the closed-form gradient equals the
    derivative of the re-solved EGW value."""
    g = W.rng(91)
    N, M = 7, 6
    x, y = g.standard_normal((N, 2)), g.standard_normal((M, 2))
    a, b = W.uniform_weights(N), W.uniform_weights(M)
    eps = 0.2
    X, Y, res, pi = _converged_state(x, y, a, b, eps, g.standard_normal((2, 2)) * 0.1)
    G = O.cross_covariance(pi, X, Y)
    closed = O.grad_x_squared(pi, G, X, Y, a, b)
    h = 1e-5
    for (i, d) in [(0, 0), (3, 1), (6, 0)]:
        xp, xm = x.copy(), x.copy()
        xp[i, d] += h
        xm[i, d] -= h
        Ep = _energy_of_points(xp, y, a, b, eps, res["Gamma"], res["f"], res["g"])
        Em = _energy_of_points(xm, y, a, b, eps, res["Gamma"], res["f"], res["g"])
        fd = (Ep - Em) / (2 * h)
        assert abs(fd - closed[i, d]) < 1e-6 * max(1.0, np.abs(closed).max()), (i, d, fd, closed[i, d])


def test_lifted_gradient_matches_finite_differences():
    """Algorithm 12: with Kernel-Proj frozen at the training points, the
    chained gradient equals the finite-difference derivative of
    x -> E(center(Pi(x)), Y)."""
    g = W.rng(95)
    N, M = 10, 9
    x, y = g.standard_normal((N, 3)), g.standard_normal((M, 3))
    a, b = W.uniform_weights(N), W.uniform_weights(M)
    eps = 0.2
    LX = O.lift(x, a, "power", 1.0, D=4)
    LY = O.lift(y, b, "power", 1.0, D=4)
    Y = LY["X"]

    def feats(xx):
        return O.center(O.kernel_proj(xx, x, a, LX["V"], LX["lam"], "power", 1.0), a)

    X = feats(x)
    assert np.allclose(X, LX["X"], atol=1e-10)
    res = O.cnt_gw(a, b, X, Y, eps, 60, 400, Gamma0=g.standard_normal((4, 4)) * 0.1, symmetric=False,
                   record=False)
    C = O.cost_gamma(X, Y, res["Gamma"])
    f, gg = O.sinkhorn(a, b, C, eps, 3000, res["f"], res["g"], symmetric=False)
    pi = O.plan(a, b, f, gg, C, eps)
    grad = O.grad_x_lifted(pi, O.cross_covariance(pi, X, Y), X, Y, a, b, x, LX["V"], LX["lam"], "power", 1.0)
    h = 1e-5
    for (i, d) in [(0, 0), (4, 2), (9, 1)]:
        xp, xm = x.copy(), x.copy()
        xp[i, d] += h
        xm[i, d] -= h
        Ep = O.cnt_gw(a, b, feats(xp), Y, eps, 60, 300, Gamma0=res["Gamma"], f0=f, g0=gg,
                      symmetric=False)["history"][-1]["E"]
        Em = O.cnt_gw(a, b, feats(xm), Y, eps, 60, 300, Gamma0=res["Gamma"], f0=f, g0=gg,
                      symmetric=False)["history"][-1]["E"]
        fd = (Ep - Em) / (2 * h)
        assert abs(fd - grad[i, d]) < 1e-6 * max(1.0, np.abs(grad).max()), (i, d, fd, grad[i, d])


def test_softmin_bilinear_one_matches_dense_definition():
    """The one-output form agrees with the dense operator on c_Gamma."""
    g = W.rng(99)
    X, V = g.standard_normal((6, 4)), g.standard_normal((9, 4))
    s, t = (X * X).sum(1), g.random(9)
    h, lw = g.standard_normal(9), np.log(W.random_weights(9, 5))
    C = -16 * X @ V.T - 4 * np.outer(s, t)
    dense = O.softmin(0.3, lw, h, C)
    one = [O.softmin_bilinear_one(i, X, V, s, t, h, lw, 0.3) for i in range(6)]
    assert np.allclose(dense, one, rtol=1e-13, atol=1e-13)


def test_eps_schedule():
    s = O.eps_schedule(1e-1, 1e-3, 20)
    assert len(s) == 20 and abs(s[0] - 1e-1) < 1e-15 and abs(s[-1] - 1e-3) < 1e-15
    r = [s[k + 1] / s[k] for k in range(19)]
    assert max(r) - min(r) < 1e-12
    assert O.eps_schedule(0.02, None, 3) == [0.02] * 3


def test_symmetric_sinkhorn_is_exchange_symmetric():
    """Algorithm 3: exchanging the roles of alpha and beta exchanges the
    returned pair at every iteration count (Appendix B.1); the Gauss-Seidel
    order of Algorithm 2 does not have this property."""
    g = W.rng(101)
    a, b = W.random_weights(7, 102), W.random_weights(5, 103)
    C = g.standard_normal((7, 5))
    for n in (1, 2, 7):
        f, gg = O.sinkhorn(a, b, C, 0.3, n, symmetric=True)
        g2, f2 = O.sinkhorn(b, a, C.T, 0.3, n, symmetric=True)
        assert np.allclose(f, f2, rtol=0, atol=1e-14) and np.allclose(gg, g2, rtol=0, atol=1e-14)
    f, gg = O.sinkhorn(a, b, C, 0.3, 2, symmetric=False)
    g2, f2 = O.sinkhorn(b, a, C.T, 0.3, 2, symmetric=False)
    assert not np.allclose(f, f2, atol=1e-6)


# ----------------------------------------------------------- Multiscale-GW

def test_kmeans_recovers_separated_blob_means():
    """Well-separated blobs, one initial centroid in each: Lloyd's iterations
    stop at the blobs' weighted means, and the weights aggregate exactly."""
    g = W.rng(201)
    centers = np.array([[0.0, 0.0], [10.0, 0.0], [0.0, 10.0], [10.0, 10.0]])
    lab = np.repeat(np.arange(4), 30)
    X = centers[lab] + 0.3 * g.standard_normal((120, 2))
    a = W.random_weights(120, 202)
    init = [0, 30, 60, 90]
    C, ac, assign = O.kmeans_coarsen(X, a, init, 5)
    assert np.array_equal(assign, lab)
    for c in range(4):
        m = lab == c
        assert np.allclose(C[c], (a[m] @ X[m]) / a[m].sum(), atol=1e-13)
        assert abs(ac[c] - a[m].sum()) < 1e-15
    assert abs(ac.sum() - 1.0) < 1e-14


def test_kmeans_objective_decreases_and_centering_is_kept():
    g = W.rng(203)
    X = g.standard_normal((400, 3))
    a = W.random_weights(400, 204)
    X = X - a @ X
    init = g.choice(400, 25, replace=False)
    objs = []
    for it in range(0, 8):
        C, ac, assign = O.kmeans_coarsen(X, a, init, it)
        objs.append(O.kmeans_objective(X, a, C, assign))
        # centroids are weighted means, so the coarse measure stays centered
        assert np.abs(ac @ C).max() < 1e-13
        # every centroid is the weighted mean of the points assigned to it
        for c in range(len(ac)):
            m = assign == c
            assert np.allclose(C[c], (a[m] @ X[m]) / a[m].sum(), atol=1e-13)
    assert all(objs[k + 1] <= objs[k] + 1e-15 for k in range(len(objs) - 1))


def test_interpolate_with_identical_coarse_measure_is_the_softmin():
    """Coarse = fine (every point its own cluster): Interpolate is the row
    update S_b(g) of Algorithm 2 on c_Gamma."""
    a, b, X, Y = small_problem(N=9, M=8, D=3, E=2, seed=205)
    G = W.rng(206).standard_normal((3, 2)) * 0.1
    g = W.rng(207).standard_normal(8)
    f = O.interpolate(g, X, Y, b, G, 0.3)
    assert np.allclose(f, O.softmin(0.3, np.log(b), g, O.cost_gamma(X, Y, G)), atol=1e-14)


def test_multiscale_reaches_the_direct_solution():
    """A multiscale solve (rho = 0.1) lands on the energy of the direct fine
    solve when both converge to the same critical point."""
    w = W.square_rotated(300, seed=4)
    a, b = w["a"], w["b"]
    X, Y = O.center(w["x"], a), O.center(w["y"], b)
    eps = w["eps"]
    g = W.rng(208)
    ix, iy = g.choice(300, 30, replace=False), g.choice(300, 30, replace=False)
    ms = O.multiscale_gw(a, b, X, Y, eps, ix, iy, 10, 20, 50, 20, 50)
    direct = O.cnt_gw(a, b, X, Y, eps, 40, 50)
    assert abs(ms["history"][-1]["E"] - direct["history"][-1]["E"]) < 1e-4 * abs(direct["history"][-1]["E"])
    assert ms["coarse"]["history"][-1]["E"] > 0
    assert len(ms["ac"]) <= 30 and abs(ms["ac"].sum() - 1) < 1e-12


# ---------------------------------------------------------------- Algorithm 6 and the hybrid stop

def small_uniform_problem(seed=3, n=40, m=35):
    g = W.rng(seed)
    x = g.uniform(0, 1, (n, 2)) * [1.0, 0.6]
    y = g.uniform(0, 1, (m, 2)) * [0.9, 0.7]
    a, b = np.full(n, 1 / n), np.full(m, 1 / m)
    return a, b, O.center(x, a), O.center(y, b)


def test_adaptive_never_doubles_on_converged_sinkhorn_and_reaches_the_converged_energy():
    """Algorithm 6 (Appendix B.4): with Sinkhorn converged at every step the
    energy cannot increase (Prop. 4.4), so the count never doubles; from
    n_inner^0 = 1 the schedule grows (doubling only after an increase) and
    reaches the energy of the converged solver (the paper's convergence
    guarantee; this problem has one minimum reachable from Gamma_0 = 0)."""
    a, b, X, Y = small_uniform_problem()
    eps = 0.05
    ref = O.cnt_gw(a, b, X, Y, eps, 60, 500)
    same = O.cnt_gw(a, b, X, Y, eps, 60, 500, adaptive=True, n_inner_max=4096, adapt_rtol=1e-12)
    assert all(h["n_inner"] == 500 for h in same["history"])
    ad = O.cnt_gw(a, b, X, Y, eps, 60, 1, adaptive=True, n_inner_max=4096)
    n_seq = [h["n_inner"] for h in ad["history"]]
    E_seq = [h["E"] for h in ad["history"]]
    assert n_seq[0] == 1 and n_seq[-1] > 64
    for t in range(1, len(n_seq)):
        assert n_seq[t] in (n_seq[t - 1], min(2 * n_seq[t - 1], 4096))
        if t >= 2 and n_seq[t] > n_seq[t - 1]:
            assert E_seq[t - 1] > E_seq[t - 2]        # a doubling follows an increase
    assert abs(ad["history"][-1]["E"] - ref["history"][-1]["E"]) <= 1e-10 * ref["history"][-1]["E"]


@pytest.mark.parametrize("symmetric", [True, False])
def test_hybrid_stop_rule(symmetric):
    """Appendix D.1 hybrid stop: below tol at the stop and not at the check
    before; tol = 0 runs the maximum and equals plain Sinkhorn.  The measured
    plan is the one whose marginals the last iteration evaluated: for
    Algorithm 3 the row sums of (f^n, g^n) are a exp(2 (f^n - f^{n+1}) / eps)
    (f^{n+1} averages f^n with S_b(g^n)); for Algorithm 2 the rows of
    (f^{n+1}, g^n) are exact."""
    a, b, X, Y = small_uniform_problem()
    eps = 0.05
    C = O.cost_gamma(X, Y, O.cnt_gw(a, b, X, Y, eps, 10, 300)["Gamma"])
    f0, g0 = np.zeros(len(a)), np.zeros(len(b))
    f, g, n_run, err = O.sinkhorn_stop(a, b, C, eps, 3000, f0, g0, symmetric, 1e-8, 7)
    assert n_run % 7 == 0 and n_run < 3000 and err < 1e-8
    _, _, n_prev, err_prev = O.sinkhorn_stop(a, b, C, eps, n_run - 7, f0, g0, symmetric, 0.0, 7)
    assert n_prev == n_run - 7 and err_prev >= 1e-8
    fz, gz, nz, _ = O.sinkhorn_stop(a, b, C, eps, 50, f0, g0, symmetric, 0.0, 5)
    fs, gs = O.sinkhorn(a, b, C, eps, 50, f0, g0, symmetric)
    assert nz == 50 and np.array_equal(fz, fs) and np.array_equal(gz, gs)
    fn, gn = O.sinkhorn(a, b, C, eps, 12, f0, g0, symmetric)
    f1, g1 = O.sinkhorn(a, b, C, eps, 1, fn, gn, symmetric)
    if symmetric:
        rows = O.plan(a, b, fn, gn, C, eps).sum(1)
        np.testing.assert_allclose(rows, a * np.exp(2 * (fn - f1) / eps), rtol=1e-12)
    else:
        np.testing.assert_allclose(O.plan(a, b, f1, gn, C, eps).sum(1), a, rtol=1e-12)
        cols = O.plan(a, b, f1, gn, C, eps).sum(0)
        np.testing.assert_allclose(cols, b * np.exp((gn - g1) / eps), rtol=1e-12)


# ---------------------------------------------------------------- SGW divergence (Section 4.1)

def _sgw_converged(a, b, X, Y, eps, n_outer=80):
    return O.sgw(a, b, X, Y, eps, n_outer, 300, symmetric=False)


def test_sgw_is_nonnegative_and_vanishes_for_isometric_measures():
    """Section 4.1 theorem on SGW: for CNT costs SGW_eps >= 0, and = 0 when
    alpha and beta are isometric (here a rotated, reflected, translated and
    reordered copy with the same weights)."""
    for seed in range(4):
        g = W.rng(200 + seed)
        n, m = 12, 10
        x = g.standard_normal((n, 2)) * [0.4, 0.2]       # scaled so the plans converge
        y = g.standard_normal((m, 2)) * [0.28, 0.24]
        a, b = W.random_weights(n, 300 + seed, 0.3), W.random_weights(m, 400 + seed, 0.3)
        res = _sgw_converged(a, b, O.center(x, a), O.center(y, b), 0.1)
        assert res["SGW"] >= -1e-9, (seed, res["SGW"])
        assert res["SGW"] > 1e-4                      # these clouds are not isometric
    g = W.rng(9)
    n = 11
    x = g.standard_normal((n, 3)) * [0.4, 0.24, 0.12]
    a = W.random_weights(n, 10, 0.3)
    Q = W.random_orthogonal(3, W.rng(11))
    perm = g.permutation(n)
    y = (x @ Q.T + [0.3, -1.0, 2.0])[perm]
    res = _sgw_converged(a, a[perm], O.center(x, a), O.center(y, a[perm]), 0.1)
    assert abs(res["SGW"]) < 1e-9


def test_sgw_gradient_matches_finite_differences():
    """Envelope theorem for the three solves: the closed-form SGW gradient
    (the self term differentiated through both of its sides) equals central
    differences of the re-solved divergence."""
    g = W.rng(93)
    N, M = 7, 6
    x, y = g.standard_normal((N, 2)) * 0.4, g.standard_normal((M, 2)) * 0.32
    a, b = W.uniform_weights(N), W.uniform_weights(M)
    eps = 0.2

    def solve(xx, warm=None):
        X, Y = O.center(xx, a), O.center(y, b)
        kw = dict(symmetric=False)
        if warm is None:
            return O.sgw(a, b, X, Y, eps, 80, 300, **kw), X, Y
        ab = O.cnt_gw(a, b, X, Y, eps, 60, 300, Gamma0=warm["ab"]["Gamma"], f0=warm["ab"]["f"],
                      g0=warm["ab"]["g"], **kw)
        aa = O.cnt_gw(a, a, X, X, eps, 60, 300, Gamma0=warm["aa"]["Gamma"], f0=warm["aa"]["f"],
                      g0=warm["aa"]["g"], **kw)
        return ab["history"][-1]["E"] - 0.5 * (aa["history"][-1]["E"] + warm["bb"]["history"][-1]["E"])

    res, X, Y = solve(x)
    # converge the final plans tightly, then differentiate
    Cab = O.cost_gamma(X, Y, res["ab"]["Gamma"])
    f, gg = O.sinkhorn(a, b, Cab, eps, 3000, res["ab"]["f"], res["ab"]["g"], symmetric=False)
    pi_ab = O.plan(a, b, f, gg, Cab, eps)
    Caa = O.cost_gamma(X, X, res["aa"]["Gamma"])
    f, gg = O.sinkhorn(a, a, Caa, eps, 3000, res["aa"]["f"], res["aa"]["g"], symmetric=False)
    pi_aa = O.plan(a, a, f, gg, Caa, eps)
    closed = O.center_vjp(O.sgw_grad_features(pi_ab, pi_aa, X, Y, a, b), a)
    h = 1e-5
    for (i, d) in [(0, 0), (2, 1), (5, 0)]:
        xp, xm = x.copy(), x.copy()
        xp[i, d] += h
        xm[i, d] -= h
        fd = (solve(xp, res) - solve(xm, res)) / (2 * h)
        assert abs(fd - closed[i, d]) < 1e-6 * max(1.0, np.abs(closed).max()), (i, d, fd, closed[i, d])


def test_barycentric_transfer_closed_forms():
    """Appendix E transfer: the identity coupling diag(a) (a = b) returns the
    source attributes; the independent coupling a b^T returns their
    a-weighted mean at every target point; a permutation coupling permutes."""
    g = W.rng(61)
    n = 9
    a = W.random_weights(n, 62)
    U = g.standard_normal((n, 3))
    assert np.allclose(O.barycentric_transfer(np.diag(a), U, a), U, atol=1e-14)
    b = W.random_weights(7, 63)
    T = O.barycentric_transfer(np.outer(a, b), U, b)
    assert np.allclose(T, np.tile(a @ U, (7, 1)), atol=1e-14)
    perm = g.permutation(n)
    P = np.zeros((n, n))
    P[np.arange(n), perm] = a
    assert np.allclose(O.barycentric_transfer(P, U, a[np.argsort(perm)]), U[np.argsort(perm)], atol=1e-14)
