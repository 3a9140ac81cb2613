"""Kernel-GW exact mode (gw_kernel_gw, Algorithm 5) against the FP64 oracle.

Tolerances: the final energy within 1e-4 relative and the marginals within
1e-3 (as for gw_solve); plan entries within 1e-3 of the largest entry (an
FP32 Sinkhorn on an FP32 cost whose exponent carries ~n 2^-24 |C| / eps of
rounding).  The reference energy is the Lemma on exact full-rank Kernel PCA
features, which Algorithm 5 reproduces (pinned on the oracle side).
"""

import numpy as np
import pytest

import oracle as O
import workloads as W
from helpers import f32, host

pytestmark = pytest.mark.gpu

r32 = lambda x: np.asarray(x, np.float32).astype(np.float64)


def problem(n, m, seed, scale=0.5):
    g = W.rng(seed)
    x = g.standard_normal((n, 3)) * scale
    y = g.standard_normal((m, 3)) * [0.6 * scale, 0.9 * scale, 0.4 * scale]
    a, b = r32(W.random_weights(n, seed + 1, 0.3)), r32(W.random_weights(m, seed + 2, 0.3))
    CX, CY = r32(O.cnt_cost(x, x, "power", 1.0)), r32(O.cnt_cost(y, y, "power", 1.0))
    return x, y, a, b, CX, CY


@pytest.mark.parametrize("symmetric", [True, False])
def test_kernel_gw_matches_oracle(gw, symmetric):
    n, m = 233, 190                 # ragged against every 32-wide tile
    x, y, a, b, CX, CY = problem(n, m, 3)
    eps = 0.05
    pi, f, g = O.kernel_gw(a, b, CX, CY, eps, 8, 60, symmetric=symmetric)
    LX = O.lift(x, a, "power", 1.0, D=n - 1)
    LY = O.lift(y, b, "power", 1.0, D=m - 1)
    E_ref = O.egw_energy(pi, LX["X"], LY["X"], a, b, eps)["E"]
    out = gw.gw_kernel_gw(f32(CX), f32(CY), f32(a), f32(b), eps, 8, 60, symmetric=symmetric)
    P = host(out["pi"])
    assert np.abs(P - pi).max() <= 1e-3 * pi.max()
    en = host(out["energy"])
    assert en[gw.EN["status"]] == 0
    assert abs(en[gw.EN["E"]] - E_ref) <= 1e-4 * abs(E_ref)
    assert en[gw.EN["row_relmax"]] <= 1e-3 or np.abs(P.sum(1) - pi.sum(1)).max() <= 1e-3 * a.max()
    np.testing.assert_allclose(P.sum(0), pi.sum(0), rtol=0, atol=1e-3 * b.max())
    hist = host(out["history"])
    assert np.all(hist[:, gw.EN["n_inner"]] == 60)
    assert hist[-1, gw.EN["E"]] == en[gw.EN["E"]]


def test_kernel_gw_equals_cnt_gw_for_squared_costs(gw):
    """For the squared Euclidean cost the centered kernel is the Gram matrix
    of the centered points, so Algorithm 5 and Algorithm 1 on D = 2 features
    take the same steps from pi^0 = a b^T (Gamma_0 = 0): same energy history,
    same potentials up to the FP32 arithmetic of two different paths."""
    w = W.square_rotated(300, 7)
    a, b = r32(w["a"]), r32(w["b"])
    X, Y = r32(O.center(w["x"], a)), r32(O.center(w["y"], b))
    CX, CY = r32(O.pairwise_sqdist(X, X)), r32(O.pairwise_sqdist(Y, Y))
    eps = float(np.float32(w["eps"]))
    k = gw.gw_kernel_gw(f32(CX), f32(CY), f32(a), f32(b), eps, 6, 50)
    s, t = r32((X * X).sum(1)), r32((Y * Y).sum(1))
    c = gw.gw_solve(f32(X), f32(Y), f32(s), f32(t), f32(a), f32(b), eps, 6, 50)
    hk, hc = host(k["history"]), host(c["history"])
    E = gw.EN["E"]
    assert np.all(np.abs(hk[:, E] - hc[:, E]) <= 1e-4 * np.abs(hc[:, E]))
    assert np.all(np.abs(hk[:, gw.EN["Gamma2"]] - hc[:, gw.EN["Gamma2"]])
                  <= 1e-4 * np.abs(hc[:, gw.EN["Gamma2"]]).max())
    fk, fc = host(k["f"]), host(c["f"])
    assert np.abs(fk - fc).max() <= 1e-3 * np.abs(fc).max()


def test_kernel_gw_rejects_bad_options(gw):
    _, _, a, b, CX, CY = problem(40, 30, 1)
    with pytest.raises(gw.GWError) as e:
        gw.gw_kernel_gw(f32(CX), f32(CY), f32(a), f32(b), -1.0, 2, 5)
    assert e.value.code == 1


def test_kernel_gw_at_a_thousand_points(gw):
    """n = 1100, m = 900: many 128-wide tiles and 64-wide K blocks of the
    tensor-core products (K' = 3 x 1152 / 3 x 960), ragged in every
    direction; the same bars as the small case."""
    n, m = 1100, 900
    x, y, a, b, CX, CY = problem(n, m, 11)
    eps = 0.05
    pi, f, g = O.kernel_gw(a, b, CX, CY, eps, 4, 40, symmetric=True)
    LX = O.lift(x, a, "power", 1.0, D=n - 1)
    LY = O.lift(y, b, "power", 1.0, D=m - 1)
    E_ref = O.egw_energy(pi, LX["X"], LY["X"], a, b, eps)["E"]
    out = gw.gw_kernel_gw(f32(CX), f32(CY), f32(a), f32(b), eps, 4, 40)
    P = host(out["pi"])
    assert np.abs(P - pi).max() <= 1e-3 * pi.max()
    en = host(out["energy"])
    assert en[gw.EN["status"]] == 0
    assert abs(en[gw.EN["E"]] - E_ref) <= 1e-4 * abs(E_ref)
    np.testing.assert_allclose(P.sum(0), pi.sum(0), rtol=0, atol=1e-3 * b.max())
