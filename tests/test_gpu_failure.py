"""Failure detection on the GPU without a GPU fault.

* Bounded waits: with a wait limit far below a kernel's run time the
  tensor-core pipeline waits give up; the solve reports GW_ETIMEOUT in its
  energy record and the device counter says so, and the next call with the
  default limit on the same context returns the undisturbed result.
* Non-finite inputs injected on the host surface as GW_ENONFINITE.
* In the request server a malformed request fails alone: every other
  request of the mix finishes with the result it has alone.
(The paper's own reaction to non-convergence is Algorithm 6's n_inner
doubling, App. B.4; these are the library's bounded-wait and input checks.)
"""

import numpy as np
import pytest

import workloads as W
from helpers import f32

pytestmark = pytest.mark.gpu

ETIMEOUT, ENONFINITE = 5, 4


def features(n, D, seed):
    g = W.rng(seed)
    Z = g.standard_normal((n, D)) * (0.5 / np.sqrt(D))
    Z -= Z.mean(0)
    Z = Z.astype(np.float32)
    return Z, (Z.astype(np.float64) ** 2).sum(1).astype(np.float32)


def problem(n, m, D, seed):
    X, s = features(n, D, seed)
    Y, t = features(m, D, seed + 1)
    a = np.full(n, 1.0 / n, np.float32)
    b = np.full(m, 1.0 / m, np.float32)
    return [f32(v) for v in (X, Y, s, t, a, b)]


@pytest.mark.parametrize("prec", [3, 2])
def test_wait_timeout_is_reported_and_the_context_survives(gw, prec):
    import torch
    X, Y, s, t, a, b = problem(3000, 2600, 16, seed=41)
    kw = dict(prec=prec, record=False, use_graph=False)
    assert gw.gw_wait_status(reset=True) in (0, ETIMEOUT)
    ref = gw.gw_solve(X, Y, s, t, a, b, 0.05, 2, 5, **kw)
    torch.cuda.synchronize()
    e_ref = ref["energy"].cpu().numpy().copy()
    assert e_ref[gw.EN["status"]] == 0 and gw.gw_wait_status() == 0
    prev = gw.gw_set_wait_limit_ns(1)
    try:
        bad = gw.gw_solve(X, Y, s, t, a, b, 0.05, 2, 5, **kw)
        torch.cuda.synchronize()
    finally:
        gw.gw_set_wait_limit_ns(prev)
    assert gw.gw_wait_limit_ns() == prev
    e_bad = bad["energy"].cpu().numpy()
    assert e_bad[gw.EN["status"]] == ETIMEOUT
    assert gw.gw_wait_status(reset=True) == ETIMEOUT
    assert gw.gw_wait_status() == 0
    # the same context, the default limit: the undisturbed result, bitwise
    again = gw.gw_solve(X, Y, s, t, a, b, 0.05, 2, 5, **kw)
    torch.cuda.synchronize()
    e_again = again["energy"].cpu().numpy()
    assert e_again[gw.EN["status"]] == 0
    assert e_again[gw.EN["E"]] == e_ref[gw.EN["E"]]
    assert gw.gw_wait_status() == 0


def test_wait_limit_is_validated(gw):
    with pytest.raises(gw.GWError) as e:
        gw.gw_set_wait_limit_ns(0)
    assert e.value.code == 1
    assert gw.gw_wait_limit_ns() >= 1


@pytest.mark.parametrize("prec", [0, 3])
def test_nonfinite_input_reports_enonfinite(gw, prec):
    import torch
    X, Y, s, t, a, b = problem(2000, 1800, 16, seed=7)
    X[17, 3] = float("nan")
    out = gw.gw_solve(X, Y, s, t, a, b, 0.05, 2, 5, prec=prec, record=False)
    torch.cuda.synchronize()
    en = out["energy"].cpu().numpy()
    assert en[gw.EN["status"]] == ENONFINITE
    # the next problem on the same context is unaffected
    X2, Y2, s2, t2, a2, b2 = problem(2000, 1800, 16, seed=8)
    ok = gw.gw_solve(X2, Y2, s2, t2, a2, b2, 0.05, 2, 5, prec=prec, record=False)
    torch.cuda.synchronize()
    assert ok["energy"].cpu().numpy()[gw.EN["status"]] == 0


def test_malformed_request_fails_alone_in_the_server(gw):
    import time
    g = W.rng(77)
    reqs = []
    for k in range(8):
        n, m = (int(v) for v in np.exp(g.uniform(np.log(800), np.log(3000), 2)))
        w = W.gmm_rigid(n, seed=500 + k, m=m)
        kind = k % 2
        reqs.append(dict(x=w["x"], y=w["y"], id=k, kind=kind, param=1.0 if kind else 2.0,
                         D=16 if kind else 0, eps=0.05, n_outer=4, n_inner=20, prec=3))
    bad = dict(reqs[3])
    bad["id"] = 99
    bad["x"] = np.array(bad["x"], copy=True)
    bad["x"][5, 1] = np.nan

    def run(srv, rs):
        for r in rs:
            srv.submit(**r)
        out = {}
        t_end = time.time() + 300
        while len(out) < len(rs) and time.time() < t_end:
            for res in srv.poll(16, wait_ms=100):
                out[res["id"]] = res
        assert len(out) == len(rs)
        return out

    srv = gw.Server(pool_bytes=2 << 30, max_active=4)
    try:
        alone = run(srv, reqs)
        mixed = run(srv, reqs[:4] + [bad] + reqs[4:])
    finally:
        srv.close()
    assert mixed[99]["status"] != 0
    for k in range(8):
        assert alone[k]["status"] == 0 and mixed[k]["status"] == 0, k
        assert mixed[k]["energy"][0] == alone[k]["energy"][0], k
