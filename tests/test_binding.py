"""Host-side marshalling of the Python binding (no GPU needed): the packed
layout gw_solve_batch reads."""

import numpy as np
import torch


def load_binding():
    import importlib.util
    import os
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location(
        "gw_build", os.path.join(root, "paper_2602_06658_gb300", "_build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.build()
    import paper_2602_06658_gb300 as gw
    return gw


def test_pack_problems_offsets_and_order():
    gw = load_binding()
    g = np.random.default_rng(0)
    sizes = [(3, 5), (1, 2), (4, 1)]
    probs = []
    for n, m in sizes:
        probs.append(dict(X=g.standard_normal((n, 2)), Y=g.standard_normal((m, 2)),
                          s=g.random(n), t=g.random(m), a=np.full(n, 1.0 / n),
                          b=torch.full((m,), 1.0 / m, dtype=torch.float64)))
    P = gw.pack_problems(probs, device="cpu")
    assert P["xo"].tolist() == [0, 3, 4, 8] and P["yo"].tolist() == [0, 5, 7, 8]
    assert P["xo"].dtype == torch.int64 and P["yo"].dtype == torch.int64
    assert (P["n_max"], P["m_max"]) == (4, 5)
    assert P["X"].shape == (8, 2) and P["Y"].shape == (8, 2) and P["s"].shape == (8,)
    for k in ("X", "Y", "s", "t", "a", "b"):
        assert P[k].dtype == torch.float32 and P[k].is_contiguous()
    for q, p in enumerate(probs):
        xs, ys = slice(P["xo"][q], P["xo"][q + 1]), slice(P["yo"][q], P["yo"][q + 1])
        assert np.allclose(P["X"][xs].numpy(), np.float32(p["X"]))
        assert np.allclose(P["t"][ys].numpy(), np.float32(p["t"]))
        assert np.allclose(P["b"][ys].numpy(), np.float32(np.asarray(p["b"])))
