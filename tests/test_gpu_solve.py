"""gw_solve (Algorithm 1 with Algorithm 3) on device against the FP64 oracle.

Tolerances (FP32 GPU vs FP64 oracle): max relative error 1e-4 on the energy
and 1e-3 on the marginals, read as max_i |r_i^GPU - r_i^oracle| / a_i (and
likewise for columns).  Several GW minima may exist for symmetric data, so
end-to-end runs compare quantities that are the same in every basin reached
from the same start (energy, marginals, singular values of Gamma); step runs
start both sides from the same (Gamma_t, f, g) and compare everything.
"""

import numpy as np
import pytest

import oracle as O
import workloads as W
from helpers import f32, f64, host

pytestmark = pytest.mark.gpu

r32 = lambda x: np.asarray(x, np.float32).astype(np.float64)


def config1(n=1000, seed=0):
    w = W.square_rotated(n, seed)
    a, b = r32(w["a"]), r32(w["b"])
    X, Y = r32(O.center(w["x"], a)), r32(O.center(w["y"], b))
    return dict(X=X, Y=Y, s=r32((X * X).sum(1)), t=r32((Y * Y).sum(1)), a=a, b=b,
                eps=float(np.float32(w["eps"])))


def gpu_marginals(gw, P, out):
    """Row and column sums of the GPU's final plan, rebuilt from its (f, g,
    Gamma_plan) by the library's own softmin and cross-covariance."""
    import torch
    X, Y = f32(P["X"]), f32(P["Y"])
    Gp = out["Gamma_plan"]
    V = (Gp @ f64(P["Y"]).T).T.float().contiguous()   # host-side check helper, not the product
    fhat = gw.gw_sinkhorn_softmin(X, V, f32(P["s"]), f32(P["t"]), out["g"],
                                  torch.log(f32(P["b"])), P["eps"])
    row = P["a"] * np.exp((host(out["f"]) - host(fhat)) / P["eps"])
    _, _, Wd = gw.gw_cross_cov(X, Y, f32(P["s"]), f32(P["t"]), f32(P["a"]), f32(P["b"]),
                               out["f"], out["g"], Gp, P["eps"], want_W=True)
    return row, host(Wd)[:, -1]


@pytest.fixture(scope="module")
def cfg1_oracle():
    P = config1()
    res = O.cnt_gw(P["a"], P["b"], P["X"], P["Y"], P["eps"], 20, 50, symmetric=True)
    return P, res


@pytest.mark.parametrize("use_graph", [True, False])
def test_config1_end_to_end(gw, cfg1_oracle, use_graph):
    P, res = cfg1_oracle
    out = gw.gw_solve(f32(P["X"]), f32(P["Y"]), f32(P["s"]), f32(P["t"]), f32(P["a"]), f32(P["b"]),
                      P["eps"], 20, 50, use_graph=use_graph)
    en = host(out["energy"])
    last = res["history"][-1]
    assert en[gw.EN["status"]] == 0
    assert abs(en[gw.EN["E"]] - last["E"]) <= 1e-4 * abs(last["E"])
    hist = host(out["history"])
    E_or = np.array([h["E"] for h in res["history"]])
    assert np.all(np.abs(hist[:, gw.EN["E"]] - E_or) <= 1e-4 * np.abs(E_or))
    sv_g = np.linalg.svd(host(out["Gamma"]), compute_uv=False)
    sv_o = np.linalg.svd(res["Gamma"], compute_uv=False)
    assert np.allclose(sv_g, sv_o, rtol=1e-3)
    row, col = gpu_marginals(gw, P, out)
    assert np.max(np.abs(row - last["row"]) / P["a"]) <= 1e-3
    assert np.max(np.abs(col - last["col"]) / P["b"]) <= 1e-3


def test_config1_graph_equals_stream(gw):
    P = config1(400, seed=3)
    args = [f32(P[k]) for k in ("X", "Y", "s", "t", "a", "b")]
    o1 = gw.gw_solve(*args, P["eps"], 4, 20, use_graph=True)
    o2 = gw.gw_solve(*args, P["eps"], 4, 20, use_graph=False)
    for k in ("Gamma", "f", "g", "energy"):
        assert bool((o1[k] == o2[k]).all()), k


@pytest.mark.parametrize("symmetric", [True, False])
def test_one_outer_step_from_shared_state(gw, cfg1_oracle, symmetric):
    """Step parity: from the oracle's (Gamma_t, f, g) after 3 outer steps, one
    GPU outer step matches the oracle's next step."""
    P, _ = cfg1_oracle
    pre = O.cnt_gw(P["a"], P["b"], P["X"], P["Y"], P["eps"], 3, 50, symmetric=symmetric, record=False)
    G0, f0, g0 = pre["Gamma"], r32(pre["f"]), r32(pre["g"])
    nxt = O.cnt_gw(P["a"], P["b"], P["X"], P["Y"], P["eps"], 1, 50, Gamma0=G0, f0=f0, g0=g0,
                   symmetric=symmetric)
    out = gw.gw_solve(*[f32(P[k]) for k in ("X", "Y", "s", "t", "a", "b")], P["eps"], 1, 50,
                      symmetric=symmetric, Gamma0=f64(G0), f0=f32(f0), g0=f32(g0))
    scale_f = np.abs(nxt["f"]).max() + P["eps"]
    assert np.max(np.abs(host(out["f"]) - nxt["f"])) <= 1e-5 * scale_f
    assert np.max(np.abs(host(out["g"]) - nxt["g"])) <= 1e-5 * scale_f
    assert np.allclose(host(out["Gamma"]), nxt["Gamma"], rtol=0, atol=1e-5 * np.abs(nxt["Gamma"]).max())
    assert abs(host(out["energy"])[gw.EN["E"]] - nxt["history"][-1]["E"]) <= 1e-5 * abs(nxt["history"][-1]["E"])


def test_annealed_schedule_and_lifted_dims(gw):
    """Geometric eps schedule and D = E = 16 features (shape of the lifted
    workloads) on a small problem, compared step for step."""
    g = W.rng(123)
    n, m, D = 300, 280, 16
    a, b = r32(W.uniform_weights(n)), r32(W.uniform_weights(m))
    X = g.standard_normal((n, D)) * 0.25
    Y = g.standard_normal((m, D)) * 0.25
    X, Y = r32(X - a @ X), r32(Y - b @ Y)
    s, t = r32((X * X).sum(1)), r32((Y * Y).sum(1))
    G0 = 0.05 * g.standard_normal((D, D))
    res = O.cnt_gw(a, b, X, Y, 0.1, 5, 40, Gamma0=G0, eps_final=0.02, symmetric=True)
    out = gw.gw_solve(f32(X), f32(Y), f32(s), f32(t), f32(a), f32(b), 0.1, 5, 40, eps_final=0.02,
                      Gamma0=f64(G0))
    hist = host(out["history"])
    for k, h in enumerate(res["history"]):
        assert abs(hist[k, gw.EN["eps"]] - h["eps"]) <= 1e-7 * h["eps"]
        assert abs(hist[k, gw.EN["E"]] - h["E"]) <= 1e-4 * abs(h["E"]), k


@pytest.mark.parametrize("prec", [3, 2])
def test_config1_end_to_end_tensor_core(gw, cfg1_oracle, prec):
    """The split tensor-core modes reach the FP32 bar on the 2D workload."""
    P, res = cfg1_oracle
    out = gw.gw_solve(f32(P["X"]), f32(P["Y"]), f32(P["s"]), f32(P["t"]), f32(P["a"]), f32(P["b"]),
                      P["eps"], 20, 50, prec=prec)
    en = host(out["energy"])
    last = res["history"][-1]
    assert en[gw.EN["status"]] == 0
    assert abs(en[gw.EN["E"]] - last["E"]) <= 1e-4 * abs(last["E"])
    row, col = gpu_marginals(gw, P, out)
    assert np.max(np.abs(row - last["row"]) / P["a"]) <= 1e-3
    assert np.max(np.abs(col - last["col"]) / P["b"]) <= 1e-3


@pytest.mark.parametrize("D,prec", [(64, 3), (64, 0), (32, 2)])
def test_solve_wide_features_tensor_core(gw, D, prec):
    """D = 64 (the widest configuration: 64-column tiles, K' = 256 in the
    split modes) and BF16X3 at D = 32, against the oracle step by step."""
    g = W.rng(321 + D)
    n, m = 700, 650
    a, b = r32(W.uniform_weights(n)), r32(W.uniform_weights(m))
    X = g.standard_normal((n, D)) * (0.6 / np.sqrt(D))
    Y = g.standard_normal((m, D)) * (0.6 / np.sqrt(D))
    X, Y = r32(X - a @ X), r32(Y - b @ Y)
    s, t = r32((X * X).sum(1)), r32((Y * Y).sum(1))
    G0 = 0.2 * g.standard_normal((D, D)) / D
    res = O.cnt_gw(a, b, X, Y, 0.05, 4, 40, Gamma0=G0, eps_final=0.01, symmetric=True)
    out = gw.gw_solve(f32(X), f32(Y), f32(s), f32(t), f32(a), f32(b), 0.05, 4, 40, eps_final=0.01,
                      Gamma0=f64(G0), prec=prec)
    hist = host(out["history"])
    for k, h in enumerate(res["history"]):
        assert abs(hist[k, gw.EN["E"]] - h["E"]) <= 1e-4 * abs(h["E"]), (k, hist[k, 0], h["E"])


@pytest.mark.parametrize("prec", [0, 3])
def test_graph_modes_are_bitwise_equal(gw, prec):
    """use_graph 0 (direct launches), 1 (the whole solve as one graph) and 2
    (per outer step: the first iteration direct, the others replayed from a
    captured graph of 10 or 2 iterations, the remainder direct) enqueue the
    same kernels with the same arguments: records, Gamma and potentials are
    bitwise equal, for inner counts that take each branch."""
    import torch
    w = W.gmm_rigid(1200, seed=4, m=1100)
    dev = lambda v: torch.tensor(np.ascontiguousarray(v, np.float32), device="cuda")
    a = torch.full((1200,), 1 / 1200, device="cuda")
    b = torch.full((1100,), 1 / 1100, device="cuda")
    lx = gw.gw_lift(dev(w["x"]), 16, kind=gw.PEN_POWER, param=1.0, w=a)
    ly = gw.gw_lift(dev(w["y"]), 16, kind=gw.PEN_POWER, param=1.0, w=b)
    args = (lx["X"], ly["X"], lx["s"], ly["s"], a, b)
    side = torch.cuda.Stream()
    torch.cuda.synchronize()
    for n_inner in (2, 3, 25):
        outs = []
        for mode in (0, 1, 2):
            with torch.cuda.stream(side):
                o = gw.gw_solve(*args, 0.1, 3, n_inner, eps_final=0.03, prec=prec, record=True,
                                use_graph=mode)
            side.synchronize()
            outs.append(o)
        for o in outs[1:]:
            for k in ("energy", "history", "Gamma", "f", "g"):
                assert bool((o[k] == outs[0][k]).all()), (prec, n_inner, k)
