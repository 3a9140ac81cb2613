"""Adaptive Sinkhorn iterations (Algorithm 6 applied to CNT-GW) and the
hybrid marginal-error stop (Appendix D.1) in gw_solve, against the oracle.

Both are discrete decisions taken from floating-point values (an energy
comparison, Err < tol), so each test first shows on the oracle that every
decision has a clear margin: every checked Err is at least 25% away from tol
(the device measures Err from FP32 potentials, a relative error far below
that), and every energy change that decides a doubling exceeds 1e-5
relative (the FP32 solve reproduces energies to ~1e-6).  The iteration
counts must then agree exactly, and the energies within 1e-4.
"""

import numpy as np
import pytest

import oracle as O
import workloads as W
from helpers import f32, host

pytestmark = pytest.mark.gpu

r32 = lambda x: np.asarray(x, np.float32).astype(np.float64)


def config(n=600, seed=4):
    w = W.square_rotated(n, seed)
    a, b = r32(w["a"]), r32(w["b"])
    X, Y = r32(O.center(w["x"], a)), r32(O.center(w["y"], b))
    return dict(X=X, Y=Y, s=r32((X * X).sum(1)), t=r32((Y * Y).sum(1)), a=a, b=b,
                eps=float(np.float32(w["eps"])))


def solve(gw, P, n_outer, n_inner, **kw):
    return gw.gw_solve(f32(P["X"]), f32(P["Y"]), f32(P["s"]), f32(P["t"]), f32(P["a"]),
                       f32(P["b"]), P["eps"], n_outer, n_inner, **kw)


@pytest.mark.parametrize("symmetric", [True, False])
def test_stop_rule_matches_oracle(gw, symmetric):
    P = config()
    tol = 3e-3
    ref = O.cnt_gw(P["a"], P["b"], P["X"], P["Y"], P["eps"], 6, 400, symmetric=symmetric,
                   stop_tol=tol, stop_every=10)
    margins = [abs(np.log(e / tol)) for h in ref["history"] for _, e in h["stop_trace"]]
    assert min(margins) > np.log(1.25)        # precondition: clear decisions
    out = solve(gw, P, 6, 400, symmetric=symmetric, stop_tol=tol, stop_every=10)
    hist = host(out["history"])
    n_gpu = hist[:, gw.EN["n_inner"]].astype(int).tolist()
    assert n_gpu == [h["n_inner"] for h in ref["history"]]
    for t, h in enumerate(ref["history"]):
        assert hist[t, gw.EN["stop_err"]] < tol
        assert abs(hist[t, gw.EN["stop_err"]] - h["stop_err"]) <= 0.02 * h["stop_err"] + 1e-5
        assert abs(hist[t, gw.EN["E"]] - h["E"]) <= 1e-4 * abs(h["E"])


def test_adaptive_matches_oracle(gw):
    P = config()
    ref = O.cnt_gw(P["a"], P["b"], P["X"], P["Y"], P["eps"], 8, 2, adaptive=True,
                   n_inner_max=512)
    E = [h["E"] for h in ref["history"]]
    assert min(abs(E[t] - E[t - 1]) / abs(E[t - 1]) for t in range(1, len(E))) > 1e-5
    n_ref = [h["n_inner"] for h in ref["history"]]
    assert n_ref[-1] > 2                      # the schedule did double
    out = solve(gw, P, 8, 2, adaptive=True, n_inner_max=512)
    hist = host(out["history"])
    assert hist[:, gw.EN["n_inner"]].astype(int).tolist() == n_ref
    assert np.all(hist[:, gw.EN["stop_err"]] == -1.0)
    for t in range(len(E)):
        assert abs(hist[t, gw.EN["E"]] - E[t]) <= 1e-4 * abs(E[t])
    # without a history the decisions are the same (records go to scratch)
    out2 = solve(gw, P, 8, 2, adaptive=True, n_inner_max=512, record=False)
    assert host(out2["energy"])[gw.EN["n_inner"]] == n_ref[-1]
    assert host(out2["energy"])[gw.EN["E"]] == hist[-1, gw.EN["E"]]


def test_fixed_mode_records_the_count_and_adaptive_with_tensor_cores(gw):
    P = config(n=1000, seed=0)
    out = solve(gw, P, 3, 25)                 # graph-captured fixed mode
    hist = host(out["history"])
    assert np.all(hist[:, gw.EN["n_inner"]] == 25) and np.all(hist[:, gw.EN["stop_err"]] == -1.0)
    # adaptive + stop together on the F16X3 tensor-core path: counts are
    # powers-of-two multiples bounded by the cap, and every stop is valid
    out = solve(gw, P, 10, 4, adaptive=True, n_inner_max=64, stop_tol=1e-3, stop_every=2,
                prec=3)
    hist = host(out["history"])
    n = hist[:, gw.EN["n_inner"]]
    assert np.all((n >= 2) & (n <= 64)) and np.all(n % 2 == 0)
    se = hist[:, gw.EN["stop_err"]]
    assert np.all(se >= 0.0)                  # stop_every = 2 <= every count: always checked
    full = se >= 1e-3                         # not stopped: the step ran its whole count
    assert np.all(np.isin(n[full], [4, 8, 16, 32, 64]))
    assert np.all(hist[:, gw.EN["status"]] == 0)


def test_invalid_stop_options_are_rejected(gw):
    P = config(n=200)
    with pytest.raises(gw.GWError) as e:
        solve(gw, P, 2, 10, stop_tol=1e-3, stop_every=0)
    assert e.value.code == 1
    with pytest.raises(gw.GWError) as e:
        solve(gw, P, 2, 10, adaptive=True, adapt_rtol=-1.0)
    assert e.value.code == 1
