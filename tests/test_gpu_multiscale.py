"""Multiscale-GW (Algorithms 7 and 8) and its K-Means coarsening on device
against the FP64 oracle.

K-Means assignments are argmins decided in FP32 on the device and in FP64 in
the oracle.  A test that compares them element-wise first shows, from the
oracle's own centroids, that every point's nearest centroid beats the
runner-up by more than twice the FP32 error bound of the device's distance
(below), so the assignment is unique and both sides must agree exactly; the
centroids then agree to FP32 rounding.  Device distance v = ||c||^2 - 2 x.c:
the two FMA chains over D terms and the final FMA round within
(D + 1) u (||c||^2 + 2 ||x|| ||c||), and the device's centroid (its FP32
rounding of the weighted mean) moves v by at most 2 u (||c||^2 + ||x|| ||c||),
u = 2^-24.
"""

import numpy as np
import pytest

import oracle as O
import workloads as W
from helpers import f32, f64, host

pytestmark = pytest.mark.gpu

r32 = lambda x: np.asarray(x, np.float32).astype(np.float64)
U = 2.0 ** -24


def idx(v):
    import torch
    return torch.as_tensor(np.asarray(v, np.int64)).cuda()


def assignment_is_unique(X, a, init, n_iter):
    """True when, in every assignment pass of the oracle's K-Means, each
    point's nearest centroid wins by more than twice the FP32 bound."""
    D = X.shape[1]
    xn = np.sqrt((X * X).sum(1))
    C = X[init]
    for p in range(n_iter + 1):
        if p > 0:
            C, _, _ = O.kmeans_coarsen(X, a, init, p - 1)
            if C.shape[0] != len(init):
                return False
        d2 = O.pairwise_sqdist(X, C)
        srt = np.sort(d2, axis=1)
        cn = np.sqrt((C * C).sum(1))
        bound = ((D + 3) * U * (cn[None, :] ** 2 + 2 * xn[:, None] * cn[None, :])).max(1)
        if np.any(srt[:, 1] - srt[:, 0] <= 2 * bound):
            return False
    return True


def square(n, seed):
    w = W.square_rotated(n, seed)
    a = r32(w["a"])
    return r32(O.center(w["x"], a)), a


@pytest.mark.parametrize("n,k,n_iter,seed", [(1200, 60, 3, 3), (4000, 37, 2, 1)])
def test_coarsen_matches_oracle(gw, n, k, n_iter, seed):
    X, a = square(n, seed)
    init = W.rng(seed + 77).choice(n, k, replace=False)
    assert assignment_is_unique(X, a, init, n_iter)   # precondition of the exact comparison
    Xc, ac, asg = O.kmeans_coarsen(X, a, init, n_iter)
    gXc, gac, gsc, gasg = gw.gw_coarsen(f32(X), idx(init), n_iter, a=f32(a))
    assert gXc.shape[0] == Xc.shape[0]
    np.testing.assert_array_equal(host(gasg).astype(np.int64), asg)
    scale = np.abs(X).max()
    np.testing.assert_allclose(host(gXc), Xc, rtol=0, atol=4 * U * scale)
    np.testing.assert_allclose(host(gac), ac, rtol=4 * U, atol=0)
    np.testing.assert_allclose(host(gsc), (host(gXc) ** 2).sum(1), rtol=4 * U * X.shape[1], atol=0)


def test_coarsen_centroids_are_weighted_means_in_high_dimension(gw):
    """D = 33 features (one past a 32-wide tile), random weights, ragged point
    count: whatever the FP32 argmins decided, every returned centroid is the
    weighted mean of the points the device assigned to it, the weights are
    the cluster masses, and each point's cluster is nearest up to the bound."""
    g = W.rng(9)
    n, D, k = 3001, 33, 70
    X = r32(g.standard_normal((n, D)))
    a = r32(W.random_weights(n, 19))
    init = g.choice(n, k, replace=False)
    gXc, gac, gsc, gasg = gw.gw_coarsen(f32(X), idx(init), 4, a=f32(a))
    C, wc, asg = host(gXc), host(gac), host(gasg).astype(np.int64)
    kk = C.shape[0]
    assert asg.min() >= 0 and asg.max() < kk
    mass = np.bincount(asg, weights=a, minlength=kk)
    assert np.all(mass > 0)
    np.testing.assert_allclose(wc, mass, rtol=1e-6)
    means = np.stack([np.bincount(asg, weights=a * X[:, d], minlength=kk) for d in range(D)], 1)
    means /= mass[:, None]
    np.testing.assert_allclose(C, means, rtol=0, atol=4 * U * np.abs(X).max() * 4)


def test_coarsen_drops_empty_clusters_and_k_equals_n(gw):
    X, a = square(500, 5)
    init = np.arange(40)
    init[7] = init[3]          # a duplicate start: exact ties go to cluster 3, cluster 7 stays empty
    keep = np.delete(np.arange(40), 7)
    assert assignment_is_unique(X, a, init[keep], 0)
    gXc, gac, _, gasg = gw.gw_coarsen(f32(X), idx(init), 0, a=f32(a))
    Xc, ac, asg = O.kmeans_coarsen(X, a, init, 0)
    assert gXc.shape[0] == Xc.shape[0] == 39
    np.testing.assert_array_equal(host(gasg).astype(np.int64), asg)
    np.testing.assert_allclose(host(gXc), Xc, rtol=0, atol=4 * U * np.abs(X).max())
    # k = n: every point is its own cluster
    n = 300
    Xs, as_ = square(n, 6)
    gXc, gac, _, gasg = gw.gw_coarsen(f32(Xs), idx(np.arange(n)), 1, a=f32(as_))
    np.testing.assert_array_equal(host(gasg).astype(np.int64), np.arange(n))
    np.testing.assert_allclose(host(gXc), Xs, rtol=0, atol=2 * U * np.abs(Xs).max())
    np.testing.assert_allclose(host(gac), as_, rtol=2 * U)


def test_coarsen_is_bitwise_reproducible_and_checks_indices(gw):
    g = W.rng(4)
    X = r32(g.standard_normal((20000, 8)))
    init = g.choice(20000, 500, replace=False)
    r1 = gw.gw_coarsen(f32(X), idx(init), 5)
    r2 = gw.gw_coarsen(f32(X), idx(init), 5)
    for u, v in zip(r1, r2):
        assert bool((u == v).all())
    bad = init.copy()
    bad[17] = 20000
    with pytest.raises(gw.GWError) as e:
        gw.gw_coarsen(f32(X), idx(bad), 1)
    assert e.value.code == 1


def test_multiscale_matches_oracle(gw):
    """Config-1 geometry (rotated square), 1500 points coarsened to 80
    clusters; the coarse and the fine energies within 1e-4 relative, the fine
    marginals within 1e-3, like a direct solve."""
    n, k = 1500, 80
    X, a = square(n, 2)
    Y, b = square(n, 12)
    eps = float(np.float32(W.square_rotated(n, 2)["eps"]))
    s, t = r32((X * X).sum(1)), r32((Y * Y).sum(1))
    g = W.rng(31)
    ix, iy = g.choice(n, k, replace=False), g.choice(n, k, replace=False)
    assert assignment_is_unique(X, a, ix, 3) and assignment_is_unique(Y, b, iy, 3)
    ref = O.multiscale_gw(a, b, X, Y, eps, ix, iy, 3, 15, 50, 4, 30)
    out = gw.gw_multiscale(f32(X), f32(Y), f32(s), f32(t), f32(a), f32(b), eps, idx(ix), idx(iy),
                           3, 15, 50, 4, 30)
    ce, en = host(out["coarse_energy"]), host(out["energy"])
    E = gw.EN["E"]
    assert en[gw.EN["status"]] == 0 and ce[gw.EN["status"]] == 0
    ref_c = ref["coarse"]["history"][-1]["E"]
    ref_f = ref["history"][-1]["E"]
    assert abs(ce[E] - ref_c) <= 1e-4 * abs(ref_c)
    assert abs(en[E] - ref_f) <= 1e-4 * abs(ref_f)
    assert en[gw.EN["row_relmax"]] <= 1e-3 and en[gw.EN["col_relmax"]] <= 1e-3
    hist = host(out["history"])
    assert hist.shape == (4, gw.EN_LEN) and np.all(np.isfinite(hist[:, E]))


def test_multiscale_start_beats_a_cold_start(gw):
    """Algorithm 7's purpose: from the interpolated start, a few fine outer
    steps reach (within 1e-3) the energy a cold start needs many more for."""
    n, k = 6000, 200
    w = W.gmm_rigid(n, seed=5)
    wa = np.full(n, 1.0 / n)
    lx = gw.gw_lift(f32(w["x"]), 8, w=f32(wa))
    ly = gw.gw_lift(f32(w["y"]), 8, w=f32(wa))
    g = W.rng(2)
    ix, iy = g.choice(n, k, replace=False), g.choice(n, k, replace=False)
    a = f32(wa)
    eps = 0.02
    cold = gw.gw_solve(lx["X"], ly["X"], lx["s"], ly["s"], a, a, eps, 40, 50, record=False)
    ms = gw.gw_multiscale(lx["X"], ly["X"], lx["s"], ly["s"], a, a, eps, idx(ix), idx(iy), 5, 40,
                          50, 6, 50, record=False)
    Ec, Em = host(cold["energy"])[gw.EN["E"]], host(ms["energy"])[gw.EN["E"]]
    assert Em <= Ec + 1e-3 * abs(Ec)
