"""Plain FP64 CPU oracle for the CNT-GW hot path.

THIS PACKAGE IS TEST INFRASTRUCTURE.  Only the test suite, the smoke check in
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference leg of
``bench.py`` may import it.  The product path (the C-ABI library and its Python
binding) never imports, links or executes anything here, and nothing here
imports the product path.

Everything is written with numpy in float64, step by step in the paper's
order and notation ("Gromov-Wasserstein at Scale, Beyond Squared Norms",
arXiv 2602.06658).  The functions cite the section, equation or algorithm they
follow.  Dense N x M matrices are formed freely: the oracle is meant to be read
against the paper, not to be fast.

Parity status: every function in ``cntgw.py`` is pinned by the not-gpu tests
(closed forms, brute force, invariants, special cases) except where the
function's own docstring says "parity unpinned".
"""

from .cntgw import *  # noqa: F401,F403
