"""Stated error of the annealed solve against the FP64 oracle, on the shape of
the lifted 3D workload (8-blob mixture vs a rigid copy, ||x - x'|| lifted by
Kernel PCA to D = 32, eps geometric 0.1 -> 1e-3 over 20 outer x 100
symmetric Sinkhorn iterations) at N = M = 1000, where the oracle solves it
in about a minute.  The features come from the oracle's own Kernel PCA.

The energy's relative error per outer step, measured once and asserted here
as the statement: FP32 stays within 1e-4 (the parity bar) while eps >= 2.5e-3
and F16X3 within 2e-4; at the end of the schedule (eps down to 1e-3, where
the O(1) terms of E cancel to ~6e-3 and 100 iterations no longer converge
Sinkhorn) both reach ~2.5e-3, and 5e-3 bounds them.
"""

import numpy as np
import pytest

import oracle as O
import workloads as W
from helpers import f32, host

pytestmark = pytest.mark.gpu

r32 = lambda x: np.asarray(x, np.float32).astype(np.float64)


@pytest.fixture(scope="module")
def annealed_case():
    n, D = 1000, 32
    w = W.gmm_rigid(n, seed=0)
    a = np.full(n, 1.0 / n)
    X = r32(O.lift(w["x"], a, "power", 1.0, D=D)["X"])
    Y = r32(O.lift(w["y"], a, "power", 1.0, D=D)["X"])
    a = r32(a)
    ref = O.cnt_gw(a, a, X, Y, 0.1, 20, 100, eps_final=1e-3, symmetric=True)
    return X, Y, a, ref


@pytest.mark.parametrize("prec,early", [(0, 1e-4), (3, 2e-4)])
def test_annealed_energy_error_statement(gw, annealed_case, prec, early):
    X, Y, a, ref = annealed_case
    s, t = r32((X * X).sum(1)), r32((Y * Y).sum(1))
    out = gw.gw_solve(f32(X), f32(Y), f32(s), f32(t), f32(a), f32(a), 0.1, 20, 100,
                      eps_final=1e-3, prec=prec, record=True)
    h = host(out["history"])
    assert np.all(h[:, gw.EN["status"]] == 0)
    for k, r in enumerate(ref["history"]):
        rel = abs(h[k, gw.EN["E"]] - r["E"]) / abs(r["E"])
        bound = early if r["eps"] >= 2.5e-3 else 5e-3
        assert rel <= bound, (prec, k, r["eps"], rel)
        assert abs(h[k, gw.EN["eps"]] - r["eps"]) <= 1e-6 * r["eps"]
