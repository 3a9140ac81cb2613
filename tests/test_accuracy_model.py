"""The rounding-noise model behind the stated error (helpers.noisy_cnt_gw)
and its stored spread, checked on the CPU against the oracle."""

import json
import os

import numpy as np

import oracle as O
import workloads as W
import helpers

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                      "accuracy_spread.json")


def small_case(n=60, m=50, D=3, seed=4):
    g = W.rng(seed)
    a = W.random_weights(n, seed + 1, 0.3)
    b = W.random_weights(m, seed + 2, 0.3)
    X = g.standard_normal((n, D)) * 0.4
    Y = g.standard_normal((m, D)) * 0.4
    return a, b, X - a @ X, Y - b @ Y


def test_zero_noise_is_the_oracle(monkeypatch):
    """With the per-cell bound set to zero the model is Algorithm 1 with
    Algorithm 3 exactly as oracle.cnt_gw runs it."""
    a, b, X, Y = small_case()
    monkeypatch.setitem(helpers.TERM_REL, 0, 0.0)
    h = helpers.noisy_cnt_gw(a, b, X, Y, 0.2, 4, 30, 0, seed=1, eps_final=0.05)
    ref = O.cnt_gw(a, b, X, Y, 0.2, 4, 30, eps_final=0.05, symmetric=True)["history"]
    for x, r in zip(h, ref):
        assert abs(x["E"] - r["E"]) <= 1e-12 * abs(r["E"])
        assert abs(x["eps"] - r["eps"]) <= 1e-15


def test_noise_moves_the_energy_by_its_bound_order():
    """The noise moves the solve, and the F16X3 bound (2^-20 per term, 8x the
    FP32 2^-23) moves it more than the FP32 one on average."""
    a, b, X, Y = small_case(120, 100, 8, seed=9)
    ref = O.cnt_gw(a, b, X, Y, 0.1, 3, 40, symmetric=True)["history"]
    E0 = np.array([r["E"] for r in ref])
    d = {}
    for prec in (0, 3):
        errs = []
        for seed in (1, 2, 3):
            h = helpers.noisy_cnt_gw(a, b, X, Y, 0.1, 3, 40, prec, seed)
            errs.append(np.abs(np.array([x["E"] for x in h]) - E0) / np.abs(E0))
        d[prec] = np.mean(errs)
    assert 0.0 < d[0] < d[3]


def test_stored_spread_is_well_formed():
    with open(GOLDEN) as fh:
        g = json.load(fh)
    eps = np.array(g["eps"])
    assert np.allclose(eps, O.eps_schedule(0.1, 1e-3, 20), rtol=1e-12)
    assert len(g["E_oracle"]) == 20
    for name in ("fp32", "f16x3"):
        sp = g["spread"][name]
        per = np.array(sp["per_seed"])
        assert per.shape == (3, 20)
        assert np.allclose(np.array(sp["max"]), per.max(axis=0))
        # below the 1e-4 bar while eps >= 0.02; the end of the schedule above it
        assert np.all(per[:, eps >= 0.02] < 1e-4)
    assert max(g["spread"]["fp32"]["max"][-3:]) > 1e-3
