"""GPU plan-weighted reduction (gw_cross_cov) and energy (gw_energy) through the
C-ABI, against the FP64 oracle's dense plan."""

import numpy as np
import pytest

import oracle as O
import workloads as W
from helpers import f32, f64, host

pytestmark = pytest.mark.gpu

r32 = lambda x: np.asarray(x, np.float32).astype(np.float64)


def plan_inputs(n, m, D, E, eps, seed, sinkhorn_iters=30):
    """Centered features, weights and potentials from a few oracle Sinkhorn
    iterations on c_{Gamma_t} (so the plan is a sensible near-coupling)."""
    g = W.rng(seed)
    a, b = W.random_weights(n, seed + 1, 0.3), W.random_weights(m, seed + 2, 0.3)
    X = g.standard_normal((n, D)) / np.sqrt(D)
    Y = g.standard_normal((m, E)) / np.sqrt(E)
    X, Y = r32(X - a @ X), r32(Y - b @ Y)
    a, b = r32(a), r32(b)
    s, t = r32((X * X).sum(1)), r32((Y * Y).sum(1))
    Gt = 0.2 * g.standard_normal((D, E)) / np.sqrt(D * E)
    C = O.cost_gamma(X, Y, Gt, s, t)
    f, gg = O.sinkhorn(a, b, C, eps, sinkhorn_iters)
    return dict(X=X, Y=Y, s=s, t=t, a=a, b=b, f=r32(f), g=r32(gg), Gamma_t=Gt, eps=eps)


def dev_args(P):
    return [f32(P[k]) for k in ("X", "Y", "s", "t", "a", "b", "f", "g")] + [f64(P["Gamma_t"]), P["eps"]]


def dense_plan(P):
    C = O.cost_gamma(P["X"], P["Y"], P["Gamma_t"], P["s"], P["t"])
    return O.plan(P["a"], P["b"], P["f"], P["g"], C, P["eps"])


def plan_tolerance(P, pi, D):
    """|GPU - FP64| bound for sums of the plan against weights |w_ij|:
    each exponent carries a rounding error of at most (D+4) 2^-24 S / eps in
    natural-log units (S the largest sum of absolute exponent terms), so each
    plan entry is off by that relative amount; FP32 accumulation over a row
    split adds about sqrt(n) 2^-23 relative.  Returns the relative factor."""
    X, Y, s, t, f, g = (P[k] for k in ("X", "Y", "s", "t", "f", "g"))
    V = Y @ P["Gamma_t"].T
    S = (16 * np.abs(X) @ np.abs(V).T + 4 * np.outer(s, t) + np.abs(f)[:, None] + np.abs(g)[None, :]
         + P["eps"] * (np.abs(np.log(P["a"]))[:, None] + np.abs(np.log(P["b"]))[None, :])).max()
    return 2.0 * ((D + 4) * 2.0 ** -24 * S / P["eps"] + np.sqrt(X.shape[0]) * 2.0 ** -23)


@pytest.mark.parametrize("n,m,D,E,eps", [(300, 257, 2, 2, 0.2), (1000, 1000, 3, 3, 0.05),
                                         (777, 1500, 16, 16, 0.1), (513, 600, 32, 32, 0.05),
                                         (130, 95, 64, 64, 0.3), (2000, 129, 5, 7, 0.1)])
def test_cross_cov_matches_oracle(gw, n, m, D, E, eps):
    P = plan_inputs(n, m, D, E, eps, seed=n + m + D)
    G, stats, Wd = gw.gw_cross_cov(*dev_args(P), want_W=True)
    pi = dense_plan(P)
    rel = plan_tolerance(P, pi, D)
    X, Y = P["X"], P["Y"]
    G_ref = X.T @ pi @ Y
    bound = rel * (np.abs(X).T @ pi @ np.abs(Y)) + 1e-12
    assert np.all(np.abs(host(G) - G_ref) <= bound), np.max(np.abs(host(G) - G_ref) / bound)
    W_ref = np.concatenate([pi.T @ X, (pi.T @ P["s"])[:, None], pi.sum(0)[:, None]], axis=1)
    Wb = rel * np.concatenate([pi.T @ np.abs(X), (pi.T @ P["s"])[:, None], pi.sum(0)[:, None]], axis=1)
    assert np.all(np.abs(host(Wd) - W_ref) <= Wb + 1e-15)
    st = host(stats)
    T_ref = P["s"] @ pi @ P["t"]
    assert abs(st[0] - T_ref) <= rel * T_ref
    col = pi.sum(0)
    assert abs(st[2] - pi.sum()) <= rel * pi.sum()
    assert abs(st[1] - P["g"] @ col) <= rel * (np.abs(P["g"]) @ col)
    assert abs(st[3] - np.abs(col - P["b"]).sum()) <= rel * col.sum() + 1e-12


@pytest.mark.parametrize("n,m,D,E,eps", [(400, 350, 2, 2, 0.1), (900, 1100, 32, 32, 0.05)])
def test_energy_matches_oracle(gw, n, m, D, E, eps):
    P = plan_inputs(n, m, D, E, eps, seed=5 * n + D, sinkhorn_iters=60)
    en, G = gw.gw_energy(*dev_args(P))
    en = host(en)
    pi = dense_plan(P)
    X, Y, a, b = P["X"], P["Y"], P["a"], P["b"]
    ref = O.egw_energy(pi, X, Y, a, b, eps)
    # The GPU's C takes the Lemma's moments, which assume sum a X = 0; the
    # oracle's C is the pairwise definition (translation invariant).  The FP32
    # inputs are centered only up to the FP32 rounding of X (mu ~ 2^-24 |X|),
    # which moves the moment form by about 16 |mu| m3 ~ 1e-7 relative.
    mu = max(np.abs(a @ X).max(), np.abs(b @ Y).max())
    assert abs(en[gw.EN["C"]] - ref["C"]) <= (1e-12 + 64 * mu) * abs(ref["C"])
    rel = plan_tolerance(P, pi, D)
    scale = ref["C"] + 8 * np.sum(O.cross_covariance(pi, X, Y) ** 2) + 4 * (P["s"] @ pi @ P["t"])
    tol_L = 4 * rel * scale
    tol_KL = 4 * rel * (scale / eps + abs(ref["KL"])) + 1e-9
    assert abs(en[gw.EN["L"]] - ref["L"]) <= tol_L
    assert abs(en[gw.EN["KL"]] - ref["KL"]) <= tol_KL
    # E = L + eps KL: the sum of the two bounds (these are arbitrary,
    # unconverged states; the 1e-4 target applies to converged solves)
    assert abs(en[gw.EN["E"]] - ref["E"]) <= tol_L + eps * tol_KL
    row, col = pi.sum(1), pi.sum(0)
    assert abs(en[gw.EN["row_l1"]] - np.abs(row - a).sum()) <= 4 * rel + 1e-9
    assert abs(en[gw.EN["col_l1"]] - np.abs(col - b).sum()) <= 4 * rel + 1e-9
    assert abs(en[gw.EN["mass"]] - pi.sum()) <= rel
    assert en[gw.EN["status"]] == 0.0
    assert np.allclose(host(G), X.T @ pi @ Y, rtol=0, atol=rel * np.abs(X).T @ pi @ np.abs(Y) + 1e-12)


def test_cross_cov_is_deterministic(gw):
    P = plan_inputs(3000, 2000, 16, 16, 0.1, seed=77, sinkhorn_iters=5)
    args = dev_args(P)
    G1, s1, _ = gw.gw_cross_cov(*args)
    G2, s2, _ = gw.gw_cross_cov(*args)
    assert bool((G1 == G2).all()) and bool((s1 == s2).all())


def tc_plan_tolerance(P, pi, D, prec):
    """plan_tolerance for the tensor-core path: every product term of the
    exponent carries TERM_REL[prec] relative error instead of 2^-24, and the
    plan and the features each enter the second product as two f16 parts
    (about 2^-21 relative)."""
    from helpers import TERM_REL
    X, Y, s, t, f, g = (P[k] for k in ("X", "Y", "s", "t", "f", "g"))
    V = Y @ P["Gamma_t"].T
    S = (16 * np.abs(X) @ np.abs(V).T + 4 * np.outer(s, t) + np.abs(f)[:, None] + np.abs(g)[None, :]
         + P["eps"] * (np.abs(np.log(P["a"]))[:, None] + np.abs(np.log(P["b"]))[None, :])).max()
    return 2.0 * ((D + 4) * TERM_REL[prec] * S / P["eps"] + np.sqrt(X.shape[0]) * 2.0 ** -23
                  + 2.0 ** -20)


@pytest.mark.parametrize("prec", [2, 3])
@pytest.mark.parametrize("n,m,D,E,eps", [(300, 257, 2, 2, 0.2), (1000, 1000, 3, 3, 0.05),
                                         (777, 1500, 16, 16, 0.1), (513, 600, 32, 32, 0.05),
                                         (2000, 129, 5, 7, 0.1), (4100, 3000, 32, 32, 0.05)])
def test_cross_cov_tensor_cores_match_oracle(gw, prec, n, m, D, E, eps):
    """The tensor-core plan sums (both contractions on tcgen05) against the
    dense FP64 plan: Gamma_{t+1}, W and the column statistics."""
    P = plan_inputs(n, m, D, E, eps, seed=n + m + D)
    G, stats, Wd = gw.gw_cross_cov(*dev_args(P), prec=prec, want_W=True)
    pi = dense_plan(P)
    rel = tc_plan_tolerance(P, pi, D, prec)
    X, Y = P["X"], P["Y"]
    bound = rel * (np.abs(X).T @ pi @ np.abs(Y)) + 1e-12
    assert np.all(np.abs(host(G) - X.T @ pi @ Y) <= bound), np.max(np.abs(host(G) - X.T @ pi @ Y) / bound)
    W_ref = np.concatenate([pi.T @ X, (pi.T @ P["s"])[:, None], pi.sum(0)[:, None]], axis=1)
    Wb = rel * np.concatenate([pi.T @ np.abs(X), (pi.T @ P["s"])[:, None], pi.sum(0)[:, None]], axis=1)
    err = np.abs(host(Wd) - W_ref)
    assert np.all(err <= Wb + 1e-15), np.max(err / (Wb + 1e-15))
    st = host(stats)
    assert abs(st[0] - P["s"] @ pi @ P["t"]) <= rel * (P["s"] @ pi @ P["t"])
    assert abs(st[2] - pi.sum()) <= rel * pi.sum()


def test_cross_cov_tensor_core_overflow_falls_back_to_fp32(gw):
    """A target potential far above its Sinkhorn value (g + 20 eps) scales
    pi_ij / b_j by e^20, beyond what f16 holds: the tensor-core pass flags it
    and the FP32 kernel recomputes the partials, so the result still meets
    the FP32 bound of the plan the inputs define."""
    P = plan_inputs(600, 500, 8, 8, 0.1, seed=17)
    P["g"] = r32(P["g"] + 20 * P["eps"])
    G, stats, Wd = gw.gw_cross_cov(*dev_args(P), prec=3, want_W=True)
    pi = dense_plan(P)
    rel = plan_tolerance(P, pi, 8)
    W_ref = np.concatenate([pi.T @ P["X"], (pi.T @ P["s"])[:, None], pi.sum(0)[:, None]], axis=1)
    Wb = rel * np.concatenate([pi.T @ np.abs(P["X"]), (pi.T @ P["s"])[:, None], pi.sum(0)[:, None]],
                              axis=1)
    assert np.all(np.abs(host(Wd) - W_ref) <= Wb + 1e-12)
    assert np.isfinite(host(G)).all()
