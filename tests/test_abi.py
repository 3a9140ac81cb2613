"""The C-ABI library builds, loads and exports every entry point gw.h declares
(no GPU needed: no compute call is made)."""

import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "gw.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:int|void|size_t|unsigned long long|const char\s*\*|gw_server\s*\*)\s+(gw_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("gw_lift", "gw_sinkhorn_softmin", "gw_cross_cov", "gw_energy", "gw_solve",
                     "gw_grad_x", "gw_workspace_size", "gw_last_error"):
        assert required in names


def builder():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "gw_build", os.path.join(ROOT, "paper_2602_06658_gb300", "_build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_library_exports_every_declared_symbol():
    path = builder().build()
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_host_side_queries_without_gpu():
    lib = ctypes.CDLL(builder().build())
    lib.gw_workspace_size.restype = ctypes.c_size_t
    lib.gw_workspace_size.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                                      ctypes.c_int, ctypes.c_int]
    assert lib.gw_workspace_size(3, 1000, 1000, 2, 2, 0) > 0
    assert lib.gw_workspace_size(3, 1000, 1000, 0, 2, 0) == 0      # invalid D
    assert lib.gw_workspace_size(0, 10, 0, 2, 1, 0) == 0           # empty target
    lib.gw_version.restype = ctypes.c_int
    assert lib.gw_version() >= 100
    # argument validation happens on the host before any launch
    lib.gw_sinkhorn_softmin.restype = ctypes.c_int
    p = ctypes.c_void_p
    lib.gw_sinkhorn_softmin.argtypes = [p, p, p, p, p, p, ctypes.c_float, ctypes.c_int64,
                                        ctypes.c_int64, ctypes.c_int, ctypes.c_int, p, p, p,
                                        ctypes.c_size_t, p]
    rc = lib.gw_sinkhorn_softmin(None, None, None, None, None, None, -1.0, 4, 4, 2, 0, None, None,
                                 None, 0, None)
    assert rc == 1  # GW_EINVAL: eps <= 0
    lib.gw_last_error.restype = ctypes.c_char_p
    assert b"eps" in lib.gw_last_error()
    rc = lib.gw_sinkhorn_softmin(None, None, None, None, None, None, 1.0, 4, 4, 200, 0, None, None,
                                 None, 0, None)
    assert rc == 6  # GW_EUNSUPPORTED: K > 128


def test_batched_solver_validates_on_the_host():
    """gw_solve_batch refuses bad arguments before any CUDA call (dummy
    pointers are never dereferenced)."""
    lib = ctypes.CDLL(builder().build())
    p, i32, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
    lib.gw_solve_batch.restype = i32
    lib.gw_solve_batch.argtypes = [i32, p, p, i64, i64, i32, i32, p, p, p, p, p, p, p, p, i32, i32,
                                   i32, p, p, p, p, p, p, p, ctypes.c_size_t, p]
    lib.gw_solve_batch_workspace_size.restype = ctypes.c_size_t
    lib.gw_last_error.restype = ctypes.c_char_p
    d = p(0x1000)

    def call(nprob=2, n_max=100, m_max=100, D=2, E=2, n_outer=2, n_inner=3, X=d, ws_bytes=4096,
             ws=d):
        return lib.gw_solve_batch(nprob, d, d, n_max, m_max, D, E, X, d, d, d, d, d, d, None,
                                  n_outer, n_inner, 1, d, d, d, d, d, None, ws, ws_bytes, None)

    assert lib.gw_solve_batch_workspace_size() >= 4
    assert call(nprob=0) == 1                      # GW_EINVAL: empty batch
    assert call(X=None) == 1 and b"X" in lib.gw_last_error()
    assert call(n_inner=0) == 1
    assert call(D=5) == 6                          # GW_EUNSUPPORTED: feature width above 4
    assert call(E=0) == 6
    assert call(n_max=40000, m_max=40000) == 6     # shared memory of one problem does not fit
    assert b"shared memory" in lib.gw_last_error()
    assert call(ws_bytes=8) == 2                   # GW_ENOMEM: workspace too small
    assert call(ws=p(0x1010)) == 2                 # GW_ENOMEM: workspace not 256-byte aligned
    assert b"aligned" in lib.gw_last_error()


def test_wait_limit_is_validated_on_the_host():
    """The bounded-wait limit is a host setting: out-of-range values are
    refused, a valid one is kept (no device is touched)."""
    lib = ctypes.CDLL(builder().build())
    lib.gw_set_wait_limit_ns.argtypes = [ctypes.c_ulonglong]
    lib.gw_set_wait_limit_ns.restype = ctypes.c_int
    lib.gw_wait_limit_ns.restype = ctypes.c_ulonglong
    prev = lib.gw_wait_limit_ns()
    assert prev == 2_000_000_000                   # default 2 s
    assert lib.gw_set_wait_limit_ns(0) == 1        # GW_EINVAL
    assert lib.gw_set_wait_limit_ns(601 * 10**9) == 1
    assert lib.gw_wait_limit_ns() == prev
    assert lib.gw_set_wait_limit_ns(5_000_000) == 0
    assert lib.gw_wait_limit_ns() == 5_000_000
    assert lib.gw_set_wait_limit_ns(prev) == 0


def test_solve_schedule_offset_is_validated_on_the_host():
    """gw_solve refuses an outer_offset / outer_total that does not contain
    the call's steps, before any CUDA call (dummy pointers)."""
    lib = ctypes.CDLL(builder().build())
    p, i32, i64, f = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_float

    class Problem(ctypes.Structure):
        _fields_ = [("X", p), ("Y", p), ("s", p), ("t", p), ("a", p), ("b", p),
                    ("n", i64), ("m", i64), ("D", i32), ("E", i32)]

    class Options(ctypes.Structure):
        _fields_ = [("eps", f), ("eps_final", f), ("n_outer", i32), ("n_inner", i32),
                    ("symmetric", i32), ("prec", i32), ("record", i32), ("use_graph", i32),
                    ("Gamma0", p), ("f0", p), ("g0", p), ("adaptive", i32), ("n_inner_max", i32),
                    ("adapt_rtol", f), ("stop_tol", f), ("stop_every", i32),
                    ("outer_offset", i32), ("outer_total", i32)]

    class Result(ctypes.Structure):
        _fields_ = [("Gamma", p), ("Gamma_plan", p), ("f", p), ("g", p), ("energy", p),
                    ("history", p)]

    d = p(0x1000)
    P = Problem(d, d, d, d, d, d, 100, 100, 2, 2)
    R = Result(d, d, d, d, d, None)
    lib.gw_solve.restype = i32
    lib.gw_solve.argtypes = [ctypes.POINTER(Problem), ctypes.POINTER(Options),
                             ctypes.POINTER(Result), p, ctypes.c_size_t, p]
    lib.gw_last_error.restype = ctypes.c_char_p
    bad = Options(0.1, 0.01, 4, 10, 1, 0, 0, 0, None, None, None, 0, 0, 0.0, 0.0, 1, 5, 8)
    assert lib.gw_solve(ctypes.byref(P), ctypes.byref(bad), ctypes.byref(R), d, 1 << 30, None) == 1
    assert b"outer_offset" in lib.gw_last_error()
    neg = Options(0.1, 0.01, 4, 10, 1, 0, 0, 0, None, None, None, 0, 0, 0.0, 0.0, 1, -1, 8)
    assert lib.gw_solve(ctypes.byref(P), ctypes.byref(neg), ctypes.byref(R), d, 1 << 30, None) == 1
    # an FP8 solve needs the tensor-core plan sums (D + 3 <= 80): refused beyond, on the host
    P64 = Problem(d, d, d, d, d, d, 100, 100, 96, 96)
    fp8 = Options(0.1, 0.01, 4, 10, 1, 4, 0, 0, None, None, None, 0, 0, 0.0, 0.0, 1, 0, 0)
    assert lib.gw_solve(ctypes.byref(P64), ctypes.byref(fp8), ctypes.byref(R), d, 1 << 30, None) == 6
    assert b"GW_PREC_FP8" in lib.gw_last_error()


def test_server_controls_refuse_a_null_server():
    """gw_server_cancel / gw_server_set_deadline / gw_server_set_slice check
    their arguments on the host (no server, no device touched)."""
    lib = ctypes.CDLL(builder().build())
    lib.gw_server_cancel.argtypes = [ctypes.c_void_p, ctypes.c_uint64]
    lib.gw_server_set_deadline.argtypes = [ctypes.c_void_p, ctypes.c_double]
    lib.gw_server_set_slice.argtypes = [ctypes.c_void_p, ctypes.c_int]
    assert lib.gw_server_cancel(None, 1) == 1
    assert lib.gw_server_set_deadline(None, 1.0) == 1
    assert lib.gw_server_set_slice(None, 1) == 1
