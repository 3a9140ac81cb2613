"""Color / UV transfer (gw_transfer, Appendix E) against the FP64 oracle, on
the same (f, g, Gamma_t) state.

Bound: every plan entry is exp2 of an FP32 exponent that is a sum of D + 3
terms, so its relative error is at most
delta_j = ln2 (D + 3) 2^-24 max_i S_ij + 2^-22 (S_ij the sum of the terms'
magnitudes, in base 2, plus ex2.approx); the projection of column j then
moves by at most delta_j sum_i pi_ij |U_i| / b_j, plus the FP32 running sum
(sqrt(n) 2^-24 relative).  A factor 4 covers the FP32 inputs' own rounding.
"""

import math

import numpy as np
import pytest

import oracle as O
import workloads as W
from helpers import f32, f64, host

pytestmark = pytest.mark.gpu

r32 = lambda x: np.asarray(x, np.float32).astype(np.float64)


def state(n, m, D, seed, eps):
    g = W.rng(seed)
    X = r32(g.standard_normal((n, D)) * 0.3 * math.sqrt(2.0 / D))   # cost scale independent of D
    Y = r32(g.standard_normal((m, D)) * 0.3 * math.sqrt(2.0 / D))
    a, b = r32(W.random_weights(n, seed + 1, 0.3)), r32(W.random_weights(m, seed + 2, 0.3))
    X, Y = r32(O.center(X, a)), r32(O.center(Y, b))
    res = O.cnt_gw(a, b, X, Y, eps, 4, 40, record=True)
    Gt = res["history"][-2]["Gamma"]
    return X, Y, a, b, r32(res["f"]), r32(res["g"]), Gt


def bound(X, Y, a, b, f, g, Gt, eps, pi, U):
    s, t = (X * X).sum(1), (Y * Y).sum(1)
    V = Y @ np.asarray(Gt).T
    S = (16 * np.abs(X) @ np.abs(V).T + 4 * np.outer(s, t) + np.abs(f)[:, None]
         + np.abs(g)[None, :]) / eps * 1.4426950408889634 \
        + np.abs(np.log2(a))[:, None] + np.abs(np.log2(b))[None, :]
    delta = math.log(2) * (X.shape[1] + 3) * 2.0 ** -24 * S.max(0) + 2.0 ** -22
    mag = (pi.T @ np.abs(U)) / b[:, None]
    return 4 * (delta[:, None] * mag + math.sqrt(X.shape[0]) * 2.0 ** -24 * mag)


@pytest.mark.parametrize("n,m,D,k", [(1000, 777, 2, 3), (700, 900, 33, 2), (513, 300, 8, 16)])
def test_transfer_matches_oracle(gw, n, m, D, k):
    eps = 0.05
    X, Y, a, b, f, g, Gt = state(n, m, D, n + k, eps)
    U = r32(W.rng(k).uniform(0, 1, (n, k)))
    pi = O.plan(a, b, f, g, O.cost_gamma(X, Y, Gt), eps)
    want = O.barycentric_transfer(pi, U, b)
    s, t = r32((X * X).sum(1)), r32((Y * Y).sum(1))
    out, mass = gw.gw_transfer(f32(X), f32(Y), f32(s), f32(t), f32(a), f32(b), f32(f), f32(g),
                               f64(Gt), eps, f32(U))
    got = host(out)
    tol = bound(X, Y, a, b, f, g, Gt, eps, pi, U)
    assert np.all(np.abs(got - want) <= tol), np.abs(got - want).max()
    np.testing.assert_allclose(host(mass), pi.sum(0), rtol=1e-4)


def test_transfer_of_the_independent_plan_is_the_weighted_mean(gw):
    """Gamma_t = 0, f = g = 0: pi = a b^T, so every target gets sum_i a_i U_i."""
    n, m, D = 400, 300, 3
    g0 = W.rng(2)
    X = r32(g0.standard_normal((n, D)))
    Y = r32(g0.standard_normal((m, D)))
    a, b = r32(W.random_weights(n, 3)), r32(W.random_weights(m, 4))
    U = r32(g0.uniform(0, 1, (n, 3)))
    # with s = t = 0 the cost vanishes too
    zn, zm = np.zeros(n), np.zeros(m)
    out, mass = gw.gw_transfer(f32(X), f32(Y), f32(zn), f32(zm), f32(a), f32(b), f32(zn), f32(zm),
                               f64(np.zeros((D, D))), 0.1, f32(U))
    want = a @ U
    assert np.abs(host(out) - want[None, :]).max() <= 1e-5
    np.testing.assert_allclose(host(mass), b, rtol=1e-5)
