"""Sinkhorn GW divergence (gw_sgw, Section 4.1) against the FP64 oracle.

SGW is a difference of three energies, so its tolerance is the energy
tolerance (1e-4 relative) carried through the difference:
|dSGW| <= 1e-4 (|E_ab| + |E_aa| / 2 + |E_bb| / 2).
"""

import numpy as np
import pytest

import oracle as O
import workloads as W
from helpers import grad_tolerance, f32, host

pytestmark = pytest.mark.gpu

r32 = lambda x: np.asarray(x, np.float32).astype(np.float64)


def clouds(n, m, seed, scale=0.4):
    g = W.rng(seed)
    x = r32(g.standard_normal((n, 2)) * [scale, 0.5 * scale])
    y = r32(g.standard_normal((m, 2)) * [0.7 * scale, 0.6 * scale])
    a, b = r32(W.random_weights(n, seed + 1, 0.3)), r32(W.random_weights(m, seed + 2, 0.3))
    return x, y, a, b


def run(gw, X, Y, a, b, eps, n_outer, n_inner, **kw):
    s, t = r32((X * X).sum(1)), r32((Y * Y).sum(1))
    return gw.gw_sgw(f32(X), f32(Y), f32(s), f32(t), f32(a), f32(b), eps, n_outer, n_inner, **kw)


def test_sgw_value_matches_oracle(gw):
    x, y, a, b = clouds(300, 250, 5)
    X, Y = r32(O.center(x, a)), r32(O.center(y, b))
    eps = 0.02
    ref = O.sgw(a, b, X, Y, eps, 20, 100)
    out = run(gw, X, Y, a, b, eps, 20, 100)
    v = host(out["sgw"])
    E = [ref[k]["history"][-1]["E"] for k in ("ab", "aa", "bb")]
    for k in range(3):
        assert abs(v[1 + k] - E[k]) <= 1e-4 * abs(E[k]), k
    bound = 1e-4 * (abs(E[0]) + 0.5 * abs(E[1]) + 0.5 * abs(E[2]))
    assert abs(v[0] - ref["SGW"]) <= bound
    assert v[0] > 0.0
    rec = host(out["records"])
    assert np.all(rec[:, gw.EN["status"]] == 0)
    np.testing.assert_array_equal(rec[:, gw.EN["E"]], v[1:])


def test_sgw_vanishes_for_isometric_clouds(gw):
    """A rotated, reflected, translated and reordered copy with the same
    weights: SGW = 0 within the energy tolerance (Section 4.1 theorem)."""
    x, _, a, _ = clouds(400, 400, 8)
    Q = W.random_orthogonal(2, W.rng(3))
    perm = W.rng(4).permutation(400)
    y = r32((x @ Q.T + [0.5, -0.2])[perm])
    b = a[perm]
    X, Y = r32(O.center(x, a)), r32(O.center(y, b))
    out = run(gw, X, Y, a, b, 0.02, 30, 100, prec=3)
    v = host(out["sgw"])
    assert abs(v[0]) <= 1e-4 * (abs(v[1]) + 0.5 * abs(v[2]) + 0.5 * abs(v[3]))


def test_sgw_gradient_matches_oracle(gw):
    """Converged plans on both sides (Algorithm 2, many iterations); the
    device gradient of SGW with respect to the (centered) features against
    the oracle's closed form followed by the centering adjoint.  SGW's
    gradient is a difference of three adjoint gradients, so the FP32 error
    bound of the adjoint (helpers.grad_tolerance, as for gw_grad_x) applies
    to each term: sum_t rel_t |g_t| with weights 1, 1/2, 1/2."""
    x, y, a, b = clouds(200, 180, 11)
    X, Y = r32(O.center(x, a)), r32(O.center(y, b))
    eps = 0.05
    ref = O.sgw(a, b, X, Y, eps, 40, 300, symmetric=False)

    def tight(res, A, B, wa, wb):
        C = O.cost_gamma(A, B, res["history"][-2]["Gamma"])
        f, g = O.sinkhorn(wa, wb, C, eps, 3000, res["f"], res["g"], symmetric=False)
        return O.plan(wa, wb, f, g, C, eps)

    pi_ab = tight(ref["ab"], X, Y, a, b)
    pi_aa = tight(ref["aa"], X, X, a, a)
    want = O.center_vjp(O.sgw_grad_features(pi_ab, pi_aa, X, Y, a, b), a)
    terms = [O.grad_features(pi_ab, O.cross_covariance(pi_ab, X, Y), X, Y, a, b),
             O.grad_features(pi_aa, O.cross_covariance(pi_aa, X, X), X, X, a, a),
             O.grad_features(pi_aa.T, O.cross_covariance(pi_aa.T, X, X), X, X, a, a)]
    rel_ab = grad_tolerance(pi_ab, X, Y, a, eps)
    rel_aa = grad_tolerance(pi_aa, X, X, a, eps)
    tol = (rel_ab * np.abs(terms[0]).max() + 0.5 * rel_aa * np.abs(terms[1]).max()
           + 0.5 * rel_aa * np.abs(terms[2]).max())
    out = run(gw, X, Y, a, b, eps, 40, 300, symmetric=False, grad=True)
    dX = host(out["dX"])
    assert np.abs(dX - want).max() <= tol
    assert np.abs(dX.sum(0)).max() <= 1e-5 * np.abs(dX).sum(0).max()   # centering adjoint


def test_sgw_lifted_gradient_runs_through_the_lift(gw):
    """Lifted features (Kernel PCA of ||x - x'||): the raw-point gradient is
    the Kernel-Proj VJP (Algorithm 13, training points frozen) of the
    feature gradient, since every term of the combination goes through the
    same linear map."""
    import torch
    w = W.gmm_rigid(1500, seed=2)
    n = 1500
    a = torch.full((n,), 1.0 / n, device="cuda")
    xt = f32(w["x"])
    lx = gw.gw_lift(xt, 8, kind=gw.PEN_POWER, param=1.0, w=a, want_basis=True)
    ly = gw.gw_lift(f32(w["y"]), 8, kind=gw.PEN_POWER, param=1.0, w=a)
    out = gw.gw_sgw(lx["X"], ly["X"], lx["s"], ly["s"], a, a, 0.05, 8, 50, prec=3, grad=True,
                    x=xt, kind=gw.PEN_POWER, param=1.0, basis=lx["V"], eigvals=lx["lam"])
    dx = host(out["dx"])
    assert np.isfinite(dx).all() and np.abs(dx).max() > 0
    xr = r32(w["x"])
    want = O.kernel_proj_vjp(host(out["dX"]), xr, xr, host(a), host(lx["V"]), host(lx["lam"]),
                             "power", 1.0)
    assert np.abs(dx - want).max() <= 2e-3 * np.abs(want).max()


def test_sgw_autograd_flow_step_decreases_the_divergence(gw):
    """SGWDivergence through torch.autograd: a finite gradient, and a small
    step against it on the source points lowers SGW (one step of the gradient
    flows the divergence is meant for)."""
    import torch
    from paper_2602_06658_gb300.autograd import sgw_fn
    x, y, a, b = clouds(300, 260, 21)
    xt = torch.tensor(x, dtype=torch.float32, device="cuda", requires_grad=True)
    yt, at, bt = f32(y), f32(a), f32(b)
    S = sgw_fn(xt, yt, at, bt, 0.05, 20, 100)
    (gx,) = torch.autograd.grad(S, xt)
    assert torch.isfinite(gx).all() and gx.abs().max() > 0
    step = 0.1 * S.item() / (gx * gx).sum().item()
    x2 = (xt.detach() - step * gx).requires_grad_(True)
    S2 = sgw_fn(x2, yt, at, bt, 0.05, 20, 100)
    assert S2.item() < S.item()
