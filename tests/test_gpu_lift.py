"""gw_lift (centering / matrix-free Kernel PCA) against the FP64 oracle."""

import numpy as np
import pytest

import oracle as O
import workloads as W
from helpers import f32, host

pytestmark = pytest.mark.gpu

r32 = lambda x: np.asarray(x, np.float32).astype(np.float64)


def test_squared_lift_is_centering(gw):
    w = W.square_rotated(777, 4)
    x = r32(w["x"])
    a = r32(W.random_weights(777, 5))
    out = gw.gw_lift(f32(x), 2, kind=gw.PEN_SQEUCLID, w=f32(a))
    ref = O.lift(x, a)
    assert np.allclose(host(out["X"]), ref["X"], atol=1e-6)
    assert np.allclose(host(out["s"]), ref["s"], rtol=1e-5, atol=1e-7)


@pytest.mark.parametrize("kind,param,n,D", [(1, 1.0, 600, 16), (1, 1.0, 1500, 32), (1, 0.5, 500, 8),
                                            (2, 0.7, 700, 12)])
def test_kernel_pca_matches_dense_eigendecomposition(gw, kind, param, n, D):
    w = W.gmm_rigid(n, seed=n + D)
    x = r32(w["x"])
    a = r32(w["a"])
    kname = {1: "power", 2: "gauss"}[kind]
    out = gw.gw_lift(f32(x), D, kind=kind, param=param, want_basis=True, seed=3)
    ref = O.lift(x, a, kname, param, D=D)
    lam_g, lam_o = host(out["lam"]), ref["lam"]
    assert np.all(np.abs(lam_g - lam_o) <= 2e-5 * lam_o[0]), (lam_g[:5], lam_o[:5])
    # columns with a clear eigen-gap are unique up to sign, fixed by the same
    # convention on both sides (largest-magnitude entry positive)
    lam_all = np.linalg.eigvalsh(O.kernel_from_cost(O.cnt_cost(x, x, kname, param), a))[::-1]
    Xg, Xo = host(out["X"]), ref["X"]
    for d in range(D):
        gap = min(abs(lam_all[d] - lam_all[d + 1]), abs(lam_all[d] - lam_all[d - 1]) if d else np.inf)
        if gap < 1e-2 * lam_all[d]:
            continue
        tol = 1e-3 * np.abs(Xo[:, d]).max() * lam_all[0] / gap
        assert np.abs(Xg[:, d] - Xo[:, d]).max() <= tol, d
    # the features are centered and s = ||X||^2
    assert np.abs(a @ Xg).max() <= 1e-5 * np.abs(Xg).max()
    assert np.allclose(host(out["s"]), (Xg * Xg).sum(1), rtol=1e-5, atol=1e-7)


def test_kernel_pca_reproduces_cost_at_high_rank(gw):
    """With D close to the numerical rank, ||X_i - X_k||^2 approaches c(x_i, x_k)
    (Theorem 2.2 with Eqs. embedding_X); compare with the oracle at the same D."""
    n, D = 300, 64
    x = r32(W.gmm_rigid(n, seed=9)["x"])
    a = r32(W.uniform_weights(n))
    out = gw.gw_lift(f32(x), D, kind=1, param=1.0)
    Xg = host(out["X"])
    ref = O.lift(x, a, "power", 1.0, D=D)
    Dg = O.pairwise_sqdist(Xg, Xg)
    Do = O.pairwise_sqdist(ref["X"], ref["X"])
    assert np.abs(Dg - Do).max() <= 1e-3 * Do.max()


@pytest.mark.parametrize("d,kind,param,n,D", [(2, 1, 1.0, 900, 8), (4, 1, 1.5, 800, 10),
                                              (4, 2, 0.5, 700, 8), (1, 1, 1.0, 400, 4),
                                              (3, 0, 2.0, 1100, 3)])
def test_kernel_pca_point_dims_and_costs(gw, d, kind, param, n, D):
    """Point dimensions 1-4 and every cost form of the block product (sqrt,
    general power, Gaussian, squared distance through Kernel PCA) against the
    oracle's dense eigendecomposition; eigenvalues as in the test above."""
    x = r32(W.normalize_radius(W.random_features(n, d, seed=n + d)))
    a = r32(W.uniform_weights(n))
    kname = {0: "sqeuclid", 1: "power", 2: "gauss"}[kind]
    out = gw.gw_lift(f32(x), D, kind=kind, param=param, want_basis=True, seed=5)
    ref = O.lift(x, a, kname, param, D=D)
    lam_g, lam_o = host(out["lam"]), ref["lam"]
    assert np.all(np.abs(lam_g - lam_o) <= 2e-5 * lam_o[0]), (lam_g[:5], lam_o[:5])
    assert np.abs(a @ host(out["X"])).max() <= 1e-5 * np.abs(host(out["X"])).max()


@pytest.mark.parametrize("kind,param", [(1, 1.0), (2, 0.5)])
def test_full_size_lift_satisfies_the_eigen_equation(gw, kind, param):
    """The lift of the bench's 100k-point 8-blob cloud (D = 32, the launch
    configuration the bench prepares its features with).  K~ v = lam v holds
    row by row, and (K~ v)_i = -1/2 ((C v~)_i - w^T C v~) with v~ = v - w (1^T v),
    so y_i - lam v_i is the same constant for every row (y = -1/2 C v~).
    The oracle evaluates (C v~)_i exactly (FP64) for 256 sampled rows over all
    100k sources; the spread of y_i - lam v_i must be small against lam |v|."""
    n, D = 100_000, 32
    w = W.gmm_rigid(n, seed=0)
    x, a = w["x"], w["a"]
    kname = {1: "power", 2: "gauss"}[kind]
    out = gw.gw_lift(f32(x), D, kind=kind, param=param, w=f32(a), want_basis=True, seed=1)
    V, lam = host(out["V"]), host(out["lam"])
    assert np.all(np.isfinite(V)) and np.all(np.diff(lam) <= 0)
    rows = W.rng(7).choice(n, 256, replace=False)
    xs = r32(x)
    Crow = O.cnt_cost(xs[rows], xs, kname, param)          # (256, n), FP64
    a64 = r32(a)
    for c in range(3):
        v = V[:, c]
        vt = v - a64 * v.sum()
        y = -0.5 * (Crow @ vt)
        r = y - lam[c] * v[rows]
        spread = r.max() - r.min()
        assert spread <= 2e-4 * lam[c] * np.abs(v).max(), (c, spread, lam[c] * np.abs(v).max())
