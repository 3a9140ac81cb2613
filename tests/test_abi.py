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
