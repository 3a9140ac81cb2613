"""gw_sinkhorn_softmin_noalloc: the softmin for callers that cannot allocate
device memory (runtimes that reserve all memory up front, hosts that forbid
an allocation's implicit synchronisation, plug-in hosts without an allocator).

It must return what gw_sinkhorn_softmin returns, within the softmin tests'
derived FP32 tolerance, on two calls in a row (the static scratch array keeps
the previous call's contents).  This file is collected last on purpose, and
passes alone in a fresh process as well as after the other tests.
"""

import numpy as np
import pytest

import workloads as W
from helpers import f32, host, softmin_tolerance

pytestmark = pytest.mark.gpu


def inputs(n, m, K, seed):
    g = W.rng(seed)
    A = 0.5 * g.standard_normal((n, K))
    B = 0.5 * g.standard_normal((m, K))
    r = lambda x: np.asarray(x, np.float32).astype(np.float64)
    return (r(A), r(B), r((A * A).sum(1)), r((B * B).sum(1)), r(0.3 * g.standard_normal(m)),
            r(np.log(W.random_weights(m, seed + 1))))


@pytest.mark.parametrize("n,m,K,eps", [(1000, 1000, 2, 0.05), (5000, 3000, 32, 0.1),
                                       (60_000, 600, 32, 0.01)])
def test_noalloc_matches_workspace_entry_point(gw, n, m, K, eps):
    host_in = inputs(n, m, K, seed=n + m + K)
    A, B, sA, sB, h, logw = (f32(v) for v in host_in)
    ref = host(gw.gw_sinkhorn_softmin(A, B, sA, sB, h, logw, eps))
    tol = softmin_tolerance(*host_in, eps)
    for _ in range(2):
        out = host(gw.gw_sinkhorn_softmin_noalloc(A, B, sA, sB, h, logw, eps))
        assert np.all(np.abs(out - ref) <= tol)
    # a different shape in between must not disturb the next call
    A2, B2, sA2, sB2, h2, lw2 = (f32(v) for v in inputs(700, 333, 3, seed=1))
    gw.gw_sinkhorn_softmin_noalloc(A2, B2, sA2, sB2, h2, lw2, 0.2)
    out = host(gw.gw_sinkhorn_softmin_noalloc(A, B, sA, sB, h, logw, eps))
    assert np.all(np.abs(out - ref) <= tol)


def test_noalloc_rejects_scratch_beyond_the_static_array(gw):
    import torch
    n, m = 140_000, 1000
    assert gw.gw_workspace_size(gw.OP_SOFTMIN, n, m, 2, 1) > 2 << 20
    z = torch.zeros(n, 2, device="cuda")
    w = torch.zeros(m, 2, device="cuda")
    with pytest.raises(gw.GWError) as e:
        gw.gw_sinkhorn_softmin_noalloc(z, w, torch.zeros(n, device="cuda"),
                                       torch.zeros(m, device="cuda"), torch.zeros(m, device="cuda"),
                                       torch.zeros(m, device="cuda"), 0.1)
    assert e.value.code == 2 and "static scratch" in str(e.value)
