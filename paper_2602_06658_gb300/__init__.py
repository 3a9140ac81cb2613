"""Python binding of libgw, the GB300 hot path of CNT-GW (arXiv 2602.06658).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of ``libgw.so`` through its C ABI (``include/gw.h``).  PyTorch is
used for device memory and streams.  There is no CPU fallback: importing this
package fails if the library is missing, and every call raises if the
library reports an error.
"""

from __future__ import annotations

import ctypes
import os

import torch

from ._build import LIB as _LIB_PATH

__all__ = [
    "GW_OK", "PREC_FP32", "PREC_BF16", "PREC_BF16X3", "PREC_F16X3", "PREC_FP8", "PEN_SQEUCLID", "PEN_POWER", "PEN_GAUSS",
    "EN", "GWError", "lib", "gw_sinkhorn_softmin", "gw_cross_cov", "gw_energy", "gw_solve",
    "gw_lift", "gw_grad_x", "gw_workspace_size", "gw_last_error", "gw_version", "workspace",
    "gw_kernel_launches", "gw_sinkhorn_softmin_noalloc", "Server", "gw_coarsen", "gw_multiscale", "gw_sgw", "gw_kernel_gw", "gw_transfer", "gw_sinkhorn_iteration",
    "gw_set_wait_limit_ns", "gw_wait_limit_ns", "gw_wait_status", "gw_probe_ex2",
]

GW_OK = 0
PREC_FP32, PREC_BF16, PREC_BF16X3, PREC_F16X3, PREC_FP8 = 0, 1, 2, 3, 4
PEN_SQEUCLID, PEN_POWER, PEN_GAUSS = 0, 1, 2
OP_SOFTMIN, OP_CROSS_COV, OP_ENERGY, OP_SOLVE, OP_LIFT, OP_GRAD, OP_COARSEN, OP_ITERATION = range(8)
EN_LEN = 16
# index of each term of the float64 energy record
EN = {"E": 0, "L": 1, "KL": 2, "C": 3, "Gamma2": 4, "T": 5, "row_l1": 6, "col_l1": 7,
      "row_relmax": 8, "col_relmax": 9, "mass": 10, "dGamma": 11, "eps": 12, "status": 13,
      "n_inner": 14, "stop_err": 15}
_STATUS = {1: "GW_EINVAL", 2: "GW_ENOMEM", 3: "GW_ECUDA", 4: "GW_ENONFINITE", 5: "GW_ETIMEOUT",
           6: "GW_EUNSUPPORTED", 7: "GW_ECANCELED"}


def _graph_mode(use_graph) -> int:
    """gw_options.use_graph: False / 0 direct launches, True / 1 the whole
    solve as one CUDA graph, 2 per-outer-step replay of captured iterations."""
    if isinstance(use_graph, bool):
        return int(use_graph)
    v = int(use_graph)
    if v not in (0, 1, 2):
        raise ValueError("use_graph must be 0, 1 or 2")
    return v


class GWError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_STATUS.get(code, code)}: {msg}")
        self.code = code


if not os.path.exists(_LIB_PATH):
    raise ImportError(f"{_LIB_PATH} is not built: run `python -c 'import __graft_entry__ as g; g.build()'`")

lib = ctypes.CDLL(_LIB_PATH)

_p = ctypes.c_void_p
_i64 = ctypes.c_int64
_int = ctypes.c_int
_f = ctypes.c_float
_sz = ctypes.c_size_t


class GwProblem(ctypes.Structure):
    _fields_ = [("X", _p), ("Y", _p), ("s", _p), ("t", _p), ("a", _p), ("b", _p),
                ("n", _i64), ("m", _i64), ("D", _int), ("E", _int)]


class GwOptions(ctypes.Structure):
    _fields_ = [("eps", _f), ("eps_final", _f), ("n_outer", _int), ("n_inner", _int),
                ("symmetric", _int), ("prec", _int), ("record", _int), ("use_graph", _int),
                ("Gamma0", _p), ("f0", _p), ("g0", _p), ("adaptive", _int), ("n_inner_max", _int),
                ("adapt_rtol", _f), ("stop_tol", _f), ("stop_every", _int),
                ("outer_offset", _int), ("outer_total", _int)]


class GwResult(ctypes.Structure):
    _fields_ = [("Gamma", _p), ("Gamma_plan", _p), ("f", _p), ("g", _p), ("energy", _p),
                ("history", _p)]


lib.gw_sinkhorn_softmin.argtypes = [_p, _p, _p, _p, _p, _p, _f, _i64, _i64, _int, _int, _p, _p,
                                    _p, _sz, _p]
lib.gw_sinkhorn_softmin_noalloc.argtypes = [_p, _p, _p, _p, _p, _p, _f, _i64, _i64, _int, _int,
                                            _p, _p, _p]
lib.gw_sinkhorn_softmin_noalloc.restype = _int
lib.gw_cross_cov.argtypes = [_p, _p, _p, _p, _p, _p, _p, _p, _p, _f, _i64, _i64, _int, _int, _int,
                             _p, _p, _p, _p, _sz, _p]
lib.gw_energy.argtypes = [_p, _p, _p, _p, _p, _p, _p, _p, _p, _f, _i64, _i64, _int, _int, _int, _p,
                          _p, _p, _sz, _p]
lib.gw_solve.argtypes = [ctypes.POINTER(GwProblem), ctypes.POINTER(GwOptions),
                         ctypes.POINTER(GwResult), _p, _sz, _p]
lib.gw_lift.argtypes = [_p, _i64, _int, _p, _int, _f, _int, _int, ctypes.c_uint64, _p, _p, _p, _p,
                        _p, _sz, _p]
lib.gw_grad_x.argtypes = [ctypes.POINTER(GwProblem), _p, _p, _p, _p, _f, _int, _p, _int, _int, _f,
                          _p, _p, _p, _p, _p, _sz, _p]
lib.gw_coarsen.argtypes = [_p, _p, _i64, _int, _p, _i64, _int, _p, _p, _p, _p,
                           ctypes.POINTER(_i64), _p, _sz, _p]
lib.gw_multiscale.argtypes = [ctypes.POINTER(GwProblem), ctypes.POINTER(GwOptions),
                              ctypes.POINTER(GwOptions), _p, _i64, _p, _i64, _int,
                              ctypes.POINTER(GwResult), _p, _p, _sz, _p]
lib.gw_sinkhorn_iteration.argtypes = [_p, _p, _p, _p, _p, _p, _p, _p, _p, _p, _f, _i64, _i64, _int,
                                      _int, _int, _int, _p, _sz, _p]
lib.gw_transfer.argtypes = [ctypes.POINTER(GwProblem), _p, _p, _p, _f, _p, _int, _p, _p, _p, _sz,
                            _p]
lib.gw_transfer_workspace_size.argtypes = [_i64, _i64, _int, _int]
lib.gw_transfer_workspace_size.restype = _sz
lib.gw_kernel_gw.argtypes = [_p, _p, _p, _p, _i64, _i64, ctypes.POINTER(GwOptions), _p, _p, _p, _p,
                             _p, _p, _sz, _p]
lib.gw_kernel_gw_workspace_size.argtypes = [_i64, _i64]
lib.gw_kernel_gw_workspace_size.restype = _sz
lib.gw_sgw.argtypes = [ctypes.POINTER(GwProblem), ctypes.POINTER(GwOptions), _p, _p, _p, _p, _int,
                       _int, _f, _p, _p, _p, _p, _sz, _p]
lib.gw_sgw_workspace_size.argtypes = [_i64, _i64, _int, _int, _int, _int, _int]
lib.gw_sgw_workspace_size.restype = _sz
lib.gw_multiscale_workspace_size.argtypes = [_i64, _i64, _int, _int, _i64, _i64, _int]
lib.gw_multiscale_workspace_size.restype = _sz
lib.gw_solve_batch.argtypes = [_int, _p, _p, _i64, _i64, _int, _int, _p, _p, _p, _p, _p, _p, _p,
                               _p, _int, _int, _int, _p, _p, _p, _p, _p, _p, _p, _sz, _p]
lib.gw_solve_batch.restype = _int
lib.gw_solve_batch_workspace_size.argtypes = []
lib.gw_solve_batch_workspace_size.restype = _sz
class GwRequest(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("n", _i64), ("m", _i64), ("d", _int), ("kind", _int),
                ("param", _f), ("D", _int), ("eps", _f), ("eps_final", _f), ("n_outer", _int),
                ("n_inner", _int), ("prec", _int)]


class GwResponse(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("status", _int), ("energy", ctypes.c_double * 16),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_done", ctypes.c_double), ("preempted", _int)]


lib.gw_server_create.argtypes = [_p, _sz, _int, _int]
lib.gw_server_create.restype = _p
lib.gw_server_submit.argtypes = [_p, ctypes.POINTER(GwRequest), _p, _p]
lib.gw_server_submit.restype = _int
lib.gw_server_poll.argtypes = [_p, ctypes.POINTER(GwResponse), _int, _int]
lib.gw_server_poll.restype = _int
lib.gw_server_stats.argtypes = [_p, ctypes.POINTER(_int), ctypes.POINTER(_int)]
lib.gw_server_stats.restype = _int
lib.gw_server_request_bytes.argtypes = [ctypes.POINTER(GwRequest)]
lib.gw_server_request_bytes.restype = _sz
lib.gw_server_set_slice.argtypes = [_p, _int]
lib.gw_server_set_slice.restype = _int
lib.gw_server_set_batching.argtypes = [_p, _int]
lib.gw_server_set_batching.restype = _int
lib.gw_server_cancel.argtypes = [_p, ctypes.c_uint64]
lib.gw_server_cancel.restype = _int
lib.gw_server_set_deadline.argtypes = [_p, ctypes.c_double]
lib.gw_server_set_deadline.restype = _int
lib.gw_server_destroy.argtypes = [_p]
lib.gw_server_destroy.restype = None
lib.gw_workspace_size.argtypes = [_int, _i64, _i64, _int, _int, _int]
lib.gw_workspace_size.restype = _sz
lib.gw_last_error.restype = ctypes.c_char_p
lib.gw_version.restype = _int
lib.gw_kernel_launches.argtypes = [_int]
lib.gw_kernel_launches.restype = ctypes.c_ulonglong
lib.gw_set_wait_limit_ns.argtypes = [ctypes.c_ulonglong]
lib.gw_set_wait_limit_ns.restype = _int
lib.gw_wait_limit_ns.argtypes = []
lib.gw_wait_limit_ns.restype = ctypes.c_ulonglong
lib.gw_wait_status.argtypes = [_int]
lib.gw_wait_status.restype = _int
lib.gw_probe_ex2.argtypes = [_int, _int, _p, ctypes.POINTER(ctypes.c_ulonglong), _p]
lib.gw_probe_ex2.restype = _int
for _name in ("gw_sinkhorn_softmin", "gw_cross_cov", "gw_energy", "gw_solve", "gw_lift", "gw_grad_x",
              "gw_coarsen", "gw_multiscale", "gw_sgw", "gw_kernel_gw", "gw_transfer", "gw_sinkhorn_iteration", "gw_transfer"):
    getattr(lib, _name).restype = _int


def gw_last_error() -> str:
    return lib.gw_last_error().decode()


def gw_version() -> int:
    return lib.gw_version()


def gw_kernel_launches(reset: bool = False) -> int:
    """Kernels libgw has enqueued in this process (graph captures count once)."""
    return int(lib.gw_kernel_launches(int(bool(reset))))


def gw_set_wait_limit_ns(ns: int) -> int:
    """Set the bounded-wait limit of the tensor-core kernels enqueued from now
    on; returns the previous limit."""
    prev = int(lib.gw_wait_limit_ns())
    _check(lib.gw_set_wait_limit_ns(int(ns)))
    return prev


def gw_wait_limit_ns() -> int:
    return int(lib.gw_wait_limit_ns())


def gw_wait_status(reset: bool = False) -> int:
    """GW_OK, or GW_ETIMEOUT (5) when a bounded wait of this device gave up
    since the last reset.  Synchronizes the device; does not raise for a
    timeout (other errors raise)."""
    rc = int(lib.gw_wait_status(int(bool(reset))))
    if rc not in (GW_OK, 5):
        raise GWError(rc, gw_last_error())
    return rc


def gw_probe_ex2(blocks: int, iters: int, out=None, stream=None) -> int:
    """Enqueue the exponential-throughput probe (measurement aid); returns
    the number of exponentials the launch evaluates."""
    if out is None:
        out = torch.empty(blocks * 512, dtype=torch.float32, device="cuda")
    ops = ctypes.c_ulonglong(0)
    _check(lib.gw_probe_ex2(int(blocks), int(iters), _ptr(out), ctypes.byref(ops), _stream(stream)))
    return int(ops.value)


def gw_workspace_size(op: int, n: int, m: int, D: int, E: int, prec: int = PREC_FP32) -> int:
    return int(lib.gw_workspace_size(op, n, m, D, E, prec))


def _check(rc: int):
    if rc != GW_OK:
        raise GWError(rc, gw_last_error())


def _ptr(t):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch tensor")
    if not t.is_cuda:
        raise ValueError("tensors must live on the GPU")
    if not t.is_contiguous():
        raise ValueError("tensors must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _f32(t, name):
    if t is None:
        return None
    if t.dtype != torch.float32:
        raise TypeError(f"{name} must be float32")
    return t


def _f64(t, name):
    if t is None:
        return None
    if t.dtype != torch.float64:
        raise TypeError(f"{name} must be float64")
    return t


def _stream(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def workspace(nbytes: int, device=None) -> torch.Tensor:
    """Caller-owned scratch buffer (256-byte aligned by the caching allocator)."""
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device or "cuda")


def gw_sinkhorn_softmin(A, B, sA, sB, h, logw, eps, prec=PREC_FP32, avg_with=None, out=None,
                        ws=None, stream=None):
    """out_i = -eps LSE_j[logw_j + (h_j + 16<A_i,B_j> + 4 sA_i sB_j)/eps]
    (optionally averaged with avg_with); see gw.h."""
    n, K = A.shape
    m = B.shape[0]
    if out is None:
        out = torch.empty(n, dtype=torch.float32, device=A.device)
    if ws is None:
        ws = workspace(gw_workspace_size(OP_SOFTMIN, n, m, K, 1, prec), A.device)
    _check(lib.gw_sinkhorn_softmin(
        _ptr(_f32(A, "A")), _ptr(_f32(B, "B")), _ptr(_f32(sA, "sA")), _ptr(_f32(sB, "sB")),
        _ptr(_f32(h, "h")), _ptr(_f32(logw, "logw")), float(eps), n, m, K, prec,
        _ptr(_f32(avg_with, "avg_with")), _ptr(_f32(out, "out")), _ptr(ws), ws.numel(),
        _stream(stream)))
    return out


def gw_sinkhorn_softmin_noalloc(A, B, sA, sB, h, logw, eps, prec=PREC_FP32, avg_with=None,
                                out=None, stream=None):
    """gw_sinkhorn_softmin without a workspace, for callers that cannot
    allocate: the library keeps the scratch in a 2 MiB static device array
    (see gw.h for the limits, the first-call set-up and why overlapping calls
    race).  `out` must be preallocated by a caller that cannot allocate."""
    n, K = A.shape
    m = B.shape[0]
    if out is None:
        out = torch.empty(n, dtype=torch.float32, device=A.device)
    _check(lib.gw_sinkhorn_softmin_noalloc(
        _ptr(_f32(A, "A")), _ptr(_f32(B, "B")), _ptr(_f32(sA, "sA")), _ptr(_f32(sB, "sB")),
        _ptr(_f32(h, "h")), _ptr(_f32(logw, "logw")), float(eps), n, m, K, prec,
        _ptr(_f32(avg_with, "avg_with")), _ptr(_f32(out, "out")), _stream(stream)))
    return out


def gw_cross_cov(X, Y, s, t, a, b, f, g, Gamma_t, eps, prec=PREC_FP32, want_W=False, ws=None,
                 stream=None):
    """Gamma_{t+1} = sum pi X Y^T and column statistics (see gw.h).
    Returns (Gamma, stats[8], W or None)."""
    n, D = X.shape
    m, E = Y.shape
    G = torch.empty(D, E, dtype=torch.float64, device=X.device)
    stats = torch.empty(8, dtype=torch.float64, device=X.device)
    W = torch.empty(m, D + 2, dtype=torch.float64, device=X.device) if want_W else None
    if ws is None:
        ws = workspace(gw_workspace_size(OP_CROSS_COV, n, m, D, E, prec), X.device)
    _check(lib.gw_cross_cov(
        _ptr(_f32(X, "X")), _ptr(_f32(Y, "Y")), _ptr(_f32(s, "s")), _ptr(_f32(t, "t")),
        _ptr(_f32(a, "a")), _ptr(_f32(b, "b")), _ptr(_f32(f, "f")), _ptr(_f32(g, "g")),
        _ptr(_f64(Gamma_t, "Gamma_t")), float(eps), n, m, D, E, prec, _ptr(G), _ptr(stats), _ptr(W),
        _ptr(ws), ws.numel(), _stream(stream)))
    return G, stats, W


def gw_energy(X, Y, s, t, a, b, f, g, Gamma_t, eps, prec=PREC_FP32, ws=None, stream=None):
    """Energy record (float64[16], layout EN) and Gamma_{t+1}."""
    n, D = X.shape
    m, E = Y.shape
    en = torch.empty(EN_LEN, dtype=torch.float64, device=X.device)
    G = torch.empty(D, E, dtype=torch.float64, device=X.device)
    if ws is None:
        ws = workspace(gw_workspace_size(OP_ENERGY, n, m, D, E, prec), X.device)
    _check(lib.gw_energy(
        _ptr(_f32(X, "X")), _ptr(_f32(Y, "Y")), _ptr(_f32(s, "s")), _ptr(_f32(t, "t")),
        _ptr(_f32(a, "a")), _ptr(_f32(b, "b")), _ptr(_f32(f, "f")), _ptr(_f32(g, "g")),
        _ptr(_f64(Gamma_t, "Gamma_t")), float(eps), n, m, D, E, prec, _ptr(en), _ptr(G),
        _ptr(ws), ws.numel(), _stream(stream)))
    return en, G


def gw_solve(X, Y, s, t, a, b, eps, n_outer, n_inner, eps_final=0.0, symmetric=True,
             prec=PREC_FP32, record=True, use_graph=True, Gamma0=None, f0=None, g0=None, ws=None,
             out=None, stream=None, adaptive=False, n_inner_max=0, adapt_rtol=0.0, stop_tol=0.0,
             stop_every=1, outer_offset=0, outer_total=0):
    """CNT-GW (Algorithm 1) on device.  Returns dict(Gamma, Gamma_plan, f, g,
    energy, history) of device tensors; nothing is synchronised unless
    adaptive (Algorithm 6) or stop_tol > 0 (hybrid stop) asks for host
    decisions."""
    n, D = X.shape
    m, E = Y.shape
    dev = X.device
    if out is None:
        out = {"Gamma": torch.empty(D, E, dtype=torch.float64, device=dev),
               "Gamma_plan": torch.empty(D, E, dtype=torch.float64, device=dev),
               "f": torch.empty(n, dtype=torch.float32, device=dev),
               "g": torch.empty(m, dtype=torch.float32, device=dev),
               "energy": torch.empty(EN_LEN, dtype=torch.float64, device=dev),
               "history": torch.empty(n_outer, EN_LEN, dtype=torch.float64, device=dev)
               if record else None}
    if ws is None:
        ws = workspace(gw_workspace_size(OP_SOLVE, n, m, D, E, prec), dev)
    P = GwProblem(_ptr(_f32(X, "X")), _ptr(_f32(Y, "Y")), _ptr(_f32(s, "s")), _ptr(_f32(t, "t")),
                  _ptr(_f32(a, "a")), _ptr(_f32(b, "b")), n, m, D, E)
    O = GwOptions(float(eps), float(eps_final), int(n_outer), int(n_inner), int(bool(symmetric)),
                  int(prec), int(bool(record)), _graph_mode(use_graph),
                  _ptr(_f64(Gamma0, "Gamma0")), _ptr(_f32(f0, "f0")), _ptr(_f32(g0, "g0")),
                  int(bool(adaptive)), int(n_inner_max), float(adapt_rtol), float(stop_tol),
                  int(stop_every), int(outer_offset), int(outer_total))
    R = GwResult(_ptr(out["Gamma"]), _ptr(out.get("Gamma_plan")), _ptr(out["f"]), _ptr(out["g"]), _ptr(out["energy"]),
                 _ptr(out["history"]))
    _check(lib.gw_solve(ctypes.byref(P), ctypes.byref(O), ctypes.byref(R), _ptr(ws), ws.numel(),
                        _stream(stream)))
    return out


def _idx64(t, name):
    if t.dtype != torch.int64:
        raise TypeError(f"{name} must be int64")
    return t


def gw_coarsen(X, init_idx, n_iter, a=None, ws=None, stream=None):
    """K-Means coarsening (gw.h: gw_coarsen).  Returns (Xc, ac, sc, assign)
    of the non-empty clusters; synchronises with the stream (the cluster
    count is read back)."""
    n, D = X.shape
    k = int(init_idx.numel())
    dev = X.device
    Xc = torch.empty(k, D, dtype=torch.float32, device=dev)
    ac = torch.empty(k, dtype=torch.float32, device=dev)
    sc = torch.empty(k, dtype=torch.float32, device=dev)
    assign = torch.empty(n, dtype=torch.int32, device=dev)
    if ws is None:
        ws = workspace(gw_workspace_size(OP_COARSEN, n, k, D, 1, PREC_FP32), dev)
    kout = _i64(0)
    _check(lib.gw_coarsen(_ptr(_f32(X, "X")), _ptr(_f32(a, "a")), n, D,
                          _ptr(_idx64(init_idx, "init_idx")), k, int(n_iter), _ptr(Xc), _ptr(ac),
                          _ptr(sc), _ptr(assign), ctypes.byref(kout), _ptr(ws), ws.numel(),
                          _stream(stream)))
    k2 = int(kout.value)
    return Xc[:k2], ac[:k2], sc[:k2], assign


def gw_multiscale(X, Y, s, t, a, b, eps, init_x, init_y, km_iter, coarse_outer, coarse_inner,
                  fine_outer, fine_inner, eps_final=0.0, symmetric=True, prec=PREC_FP32,
                  record=True, use_graph=True, Gamma0=None, ws=None, stream=None):
    """Multiscale-GW (Algorithm 7; gw.h: gw_multiscale).  The coarse solve
    runs at the fine solve's first temperature.  Returns the gw_solve dict
    plus "coarse_energy"."""
    n, D = X.shape
    m, E = Y.shape
    dev = X.device
    kx, ky = int(init_x.numel()), int(init_y.numel())
    out = {"Gamma": torch.empty(D, E, dtype=torch.float64, device=dev),
           "Gamma_plan": torch.empty(D, E, dtype=torch.float64, device=dev),
           "f": torch.empty(n, dtype=torch.float32, device=dev),
           "g": torch.empty(m, dtype=torch.float32, device=dev),
           "energy": torch.empty(EN_LEN, dtype=torch.float64, device=dev),
           "history": torch.empty(fine_outer, EN_LEN, dtype=torch.float64, device=dev)
           if record else None,
           "coarse_energy": torch.empty(EN_LEN, dtype=torch.float64, device=dev)}
    if ws is None:
        ws = workspace(lib.gw_multiscale_workspace_size(n, m, D, E, kx, ky, int(prec)), dev)
    P = GwProblem(_ptr(_f32(X, "X")), _ptr(_f32(Y, "Y")), _ptr(_f32(s, "s")), _ptr(_f32(t, "t")),
                  _ptr(_f32(a, "a")), _ptr(_f32(b, "b")), n, m, D, E)
    Oc = GwOptions(float(eps), 0.0, int(coarse_outer), int(coarse_inner), int(bool(symmetric)),
                   int(prec), 0, _graph_mode(use_graph), _ptr(_f64(Gamma0, "Gamma0")), None, None)
    Of = GwOptions(float(eps), float(eps_final), int(fine_outer), int(fine_inner),
                   int(bool(symmetric)), int(prec), int(bool(record)), _graph_mode(use_graph),
                   None, None, None)
    R = GwResult(_ptr(out["Gamma"]), _ptr(out["Gamma_plan"]), _ptr(out["f"]), _ptr(out["g"]),
                 _ptr(out["energy"]), _ptr(out["history"]))
    _check(lib.gw_multiscale(ctypes.byref(P), ctypes.byref(Oc), ctypes.byref(Of),
                             _ptr(_idx64(init_x, "init_x")), kx, _ptr(_idx64(init_y, "init_y")), ky,
                             int(km_iter), ctypes.byref(R), _ptr(out["coarse_energy"]), _ptr(ws),
                             ws.numel(), _stream(stream)))
    return out


def gw_sinkhorn_iteration(X, V, s, t, loga, logb, f, g, eps, prec=PREC_FP32, symmetric=True,
                          reuse=False, f_out=None, g_out=None, ws=None, stream=None):
    """One Sinkhorn iteration on c_Gamma, both halves in one launch (gw.h:
    gw_sinkhorn_iteration).  reuse=True keeps the 16-bit operands already in
    `ws` (same X, V, s, t, eps, prec as the previous call).  Returns (f', g')."""
    n, K = X.shape
    m = V.shape[0]
    dev = X.device
    f_out = torch.empty(n, dtype=torch.float32, device=dev) if f_out is None else f_out
    g_out = torch.empty(m, dtype=torch.float32, device=dev) if g_out is None else g_out
    if ws is None:
        ws = workspace(gw_workspace_size(OP_ITERATION, n, m, K, 1, prec), dev)
    _check(lib.gw_sinkhorn_iteration(_ptr(_f32(X, "X")), _ptr(_f32(V, "V")), _ptr(_f32(s, "s")),
                                     _ptr(_f32(t, "t")), _ptr(_f32(loga, "loga")),
                                     _ptr(_f32(logb, "logb")), _ptr(_f32(f, "f")),
                                     _ptr(_f32(g, "g")), _ptr(f_out), _ptr(g_out), float(eps), n,
                                     m, K, int(prec), int(bool(symmetric)), int(bool(reuse)),
                                     _ptr(ws), ws.numel(), _stream(stream)))
    return f_out, g_out


def gw_transfer(X, Y, s, t, a, b, f, g, Gamma_t, eps, U, ws=None, stream=None):
    """Color / UV transfer (Appendix E; gw.h: gw_transfer).  Returns (out, mass):
    out_j = sum_i pi_ij U_i / b_j and the plan's column sums."""
    n, D = X.shape
    m, E = Y.shape
    k = int(U.shape[1])
    dev = X.device
    out = torch.empty(m, k, dtype=torch.float32, device=dev)
    mass = torch.empty(m, dtype=torch.float32, device=dev)
    if ws is None:
        ws = workspace(lib.gw_transfer_workspace_size(n, m, D, k), dev)
    P = GwProblem(_ptr(_f32(X, "X")), _ptr(_f32(Y, "Y")), _ptr(_f32(s, "s")), _ptr(_f32(t, "t")),
                  _ptr(_f32(a, "a")), _ptr(_f32(b, "b")), n, m, D, E)
    _check(lib.gw_transfer(ctypes.byref(P), _ptr(_f32(f, "f")), _ptr(_f32(g, "g")),
                           _ptr(_f64(Gamma_t, "Gamma_t")), float(eps), _ptr(_f32(U, "U")), k,
                           _ptr(out), _ptr(mass), _ptr(ws), ws.numel(), _stream(stream)))
    return out, mass


def gw_kernel_gw(CX, CY, a, b, eps, n_outer, n_inner, eps_final=0.0, symmetric=True, record=True,
                 f0=None, g0=None, ws=None, stream=None):
    """Kernel-GW exact mode (Algorithm 5; gw.h: gw_kernel_gw) on dense cost
    matrices.  Returns dict(pi, f, g, energy, history) of device tensors."""
    n, m = CX.shape[0], CY.shape[0]
    dev = CX.device
    out = {"pi": torch.empty(n, m, dtype=torch.float32, device=dev),
           "f": torch.empty(n, dtype=torch.float32, device=dev),
           "g": torch.empty(m, dtype=torch.float32, device=dev),
           "energy": torch.empty(EN_LEN, dtype=torch.float64, device=dev),
           "history": torch.empty(n_outer, EN_LEN, dtype=torch.float64, device=dev)
           if record else None}
    if ws is None:
        ws = workspace(lib.gw_kernel_gw_workspace_size(n, m), dev)
    O = GwOptions(float(eps), float(eps_final), int(n_outer), int(n_inner), int(bool(symmetric)),
                  PREC_FP32, int(bool(record)), 0, None, _ptr(_f32(f0, "f0")), _ptr(_f32(g0, "g0")),
                  0, 0, 0.0, 0.0, 1)
    _check(lib.gw_kernel_gw(_ptr(_f32(CX, "CX")), _ptr(_f32(CY, "CY")), _ptr(_f32(a, "a")),
                            _ptr(_f32(b, "b")), n, m, ctypes.byref(O), _ptr(out["pi"]),
                            _ptr(out["f"]), _ptr(out["g"]), _ptr(out["energy"]),
                            _ptr(out["history"]), _ptr(ws), ws.numel(), _stream(stream)))
    return out


def gw_sgw(X, Y, s, t, a, b, eps, n_outer, n_inner, eps_final=0.0, symmetric=True,
           prec=PREC_FP32, use_graph=True, grad=False, x=None, kind=PEN_SQEUCLID, param=2.0,
           basis=None, eigvals=None, ws=None, stream=None, **solve_kw):
    """Sinkhorn GW divergence (gw.h: gw_sgw).  Returns dict(sgw (4: SGW and
    the three GW values), records (3 x EN_LEN), dX, dx) of device tensors."""
    n, D = X.shape
    m, E = Y.shape
    dev = X.device
    out = {"sgw": torch.empty(4, dtype=torch.float64, device=dev),
           "records": torch.empty(3, EN_LEN, dtype=torch.float64, device=dev),
           "dX": torch.empty(n, D, dtype=torch.float32, device=dev) if grad else None,
           "dx": torch.empty(n, x.shape[1], dtype=torch.float32, device=dev)
           if (grad and x is not None) else None}
    dxd = int(x.shape[1]) if (grad and x is not None) else 0
    if ws is None:
        ws = workspace(lib.gw_sgw_workspace_size(n, m, D, E, int(prec), int(bool(grad)), dxd), dev)
    P = GwProblem(_ptr(_f32(X, "X")), _ptr(_f32(Y, "Y")), _ptr(_f32(s, "s")), _ptr(_f32(t, "t")),
                  _ptr(_f32(a, "a")), _ptr(_f32(b, "b")), n, m, D, E)
    O = GwOptions(float(eps), float(eps_final), int(n_outer), int(n_inner), int(bool(symmetric)),
                  int(prec), 0, _graph_mode(use_graph), None, None, None,
                  int(bool(solve_kw.get("adaptive", False))), int(solve_kw.get("n_inner_max", 0)),
                  float(solve_kw.get("adapt_rtol", 0.0)), float(solve_kw.get("stop_tol", 0.0)),
                  int(solve_kw.get("stop_every", 1)))
    _check(lib.gw_sgw(ctypes.byref(P), ctypes.byref(O), _ptr(out["sgw"]), _ptr(out["records"]),
                      _ptr(out["dX"]), _ptr(_f32(x, "x")) if grad else None, dxd, int(kind),
                      float(param), _ptr(_f32(basis, "basis")), _ptr(_f32(eigvals, "eigvals")),
                      _ptr(out["dx"]), _ptr(ws), ws.numel(), _stream(stream)))
    return out


def pack_problems(problems, device=None):
    """Packs a list of problems, each dict(X, Y, s, t, a, b) of host or device
    arrays, into the layout of gw_solve_batch: concatenated float32 device
    tensors and int64 offsets xo, yo (nprob + 1).  Returns a dict with those
    and n_max, m_max."""
    import numpy as np
    dev = device or "cuda"

    def dev32(v):
        v = v if torch.is_tensor(v) else torch.as_tensor(np.asarray(v, np.float32))
        return v.to(device=dev, dtype=torch.float32)

    cat = {k: torch.cat([dev32(p[k]) for p in problems]).contiguous()
           for k in ("X", "Y", "s", "t", "a", "b")}
    ns = [len(p["s"]) for p in problems]
    ms = [len(p["t"]) for p in problems]
    cat["xo"] = torch.tensor([0] + list(np.cumsum(ns)), dtype=torch.int64, device=dev)
    cat["yo"] = torch.tensor([0] + list(np.cumsum(ms)), dtype=torch.int64, device=dev)
    cat["n_max"], cat["m_max"] = max(ns), max(ms)
    return cat


def gw_solve_batch(packed, eps, n_outer, n_inner, eps_final=None, symmetric=True, record=False,
                   ws=None, stream=None):
    """Persistent batched solver (gw.h: gw_solve_batch) over the problems of
    pack_problems().  eps, eps_final: one value per problem (float tensors or
    sequences) or a scalar for all.  Returns dict(f, g packed like s, t;
    Gamma, Gamma_plan (nprob, D, E) float64; energy (nprob, GW_EN_LEN);
    history (nprob, n_outer, GW_EN_LEN) when record)."""
    X, Y = packed["X"], packed["Y"]
    dev = X.device
    nprob = packed["xo"].numel() - 1
    D, E = X.shape[1], Y.shape[1]

    def per_problem(v):
        if v is None:
            return None
        if torch.is_tensor(v) and v.numel() == nprob:
            return v.to(device=dev, dtype=torch.float32).contiguous()
        if not torch.is_tensor(v) and hasattr(v, "__len__"):
            return torch.tensor([float(e) for e in v], dtype=torch.float32, device=dev)
        return torch.full((nprob,), float(v), dtype=torch.float32, device=dev)

    e0, e1 = per_problem(eps), per_problem(eps_final)
    out = {"f": torch.empty(packed["s"].numel(), dtype=torch.float32, device=dev),
           "g": torch.empty(packed["t"].numel(), dtype=torch.float32, device=dev),
           "Gamma": torch.empty(nprob, D, E, dtype=torch.float64, device=dev),
           "Gamma_plan": torch.empty(nprob, D, E, dtype=torch.float64, device=dev),
           "energy": torch.zeros(nprob, 16, dtype=torch.float64, device=dev),
           "history": torch.zeros(nprob, int(n_outer), 16, dtype=torch.float64, device=dev)
           if record else None}
    if ws is None:
        ws = workspace(lib.gw_solve_batch_workspace_size(), dev)
    _check(lib.gw_solve_batch(nprob, _ptr(packed["xo"]), _ptr(packed["yo"]), int(packed["n_max"]),
                              int(packed["m_max"]), D, E, _ptr(_f32(X, "X")), _ptr(_f32(Y, "Y")),
                              _ptr(_f32(packed["s"], "s")), _ptr(_f32(packed["t"], "t")),
                              _ptr(_f32(packed["a"], "a")), _ptr(_f32(packed["b"], "b")),
                              _ptr(e0), _ptr(e1), int(n_outer), int(n_inner), int(bool(symmetric)),
                              _ptr(out["f"]), _ptr(out["g"]), _ptr(out["Gamma"]),
                              _ptr(out["Gamma_plan"]), _ptr(out["energy"]), _ptr(out["history"]),
                              _ptr(ws), ws.numel(), _stream(stream)))
    return out


def gw_lift(x, D, kind=PEN_SQEUCLID, param=2.0, w=None, n_iter=0, seed=0, want_basis=False,
            ws=None, stream=None):
    """Embedding step (see gw.h).  Returns dict(X, s, V, lam)."""
    n, d = x.shape
    dev = x.device
    X = torch.empty(n, D, dtype=torch.float32, device=dev)
    s = torch.empty(n, dtype=torch.float32, device=dev)
    V = torch.empty(n, D, dtype=torch.float32, device=dev) if want_basis else None
    lam = torch.empty(D, dtype=torch.float32, device=dev) if want_basis else None
    if ws is None:
        ws = workspace(gw_workspace_size(OP_LIFT, n, n, D, d, PREC_FP32), dev)
    _check(lib.gw_lift(_ptr(_f32(x, "x")), n, d, _ptr(_f32(w, "w")), int(kind), float(param),
                       int(D), int(n_iter), int(seed), _ptr(X), _ptr(s), _ptr(V), _ptr(lam),
                       _ptr(ws), ws.numel(), _stream(stream)))
    return {"X": X, "s": s, "V": V, "lam": lam}


def gw_grad_x(X, Y, s, t, a, b, f, g, Gamma_t, Gamma_pi, eps, prec=PREC_FP32, x=None, kind=0,
              param=2.0, basis=None, eigvals=None, ws=None, stream=None):
    """Adjoint: gradient of the EGW energy w.r.t. the features (dX) and, for
    lifted features, w.r.t. the raw points x (dx)."""
    n, D = X.shape
    m, E = Y.shape
    dev = X.device
    dX = torch.empty(n, D, dtype=torch.float32, device=dev)
    dx = torch.empty(n, x.shape[1], dtype=torch.float32, device=dev) if x is not None else None
    if ws is None:
        ws = workspace(gw_workspace_size(OP_GRAD, n, m, D, E, prec), dev)
    P = GwProblem(_ptr(_f32(X, "X")), _ptr(_f32(Y, "Y")), _ptr(_f32(s, "s")), _ptr(_f32(t, "t")),
                  _ptr(_f32(a, "a")), _ptr(_f32(b, "b")), n, m, D, E)
    _check(lib.gw_grad_x(ctypes.byref(P), _ptr(_f32(f, "f")), _ptr(_f32(g, "g")),
                         _ptr(_f64(Gamma_t, "Gamma_t")), _ptr(_f64(Gamma_pi, "Gamma_pi")),
                         float(eps), int(prec), _ptr(_f32(x, "x")),
                         int(x.shape[1]) if x is not None else 0, int(kind), float(param),
                         _ptr(_f32(basis, "basis")), _ptr(_f32(eigvals, "eigvals")), _ptr(dX),
                         _ptr(dx), _ptr(ws), ws.numel(), _stream(stream)))
    return dX, dx


class Server:
    """Continuous-batching request server (gw_server_* in gw.h).  The device
    pool is one caller-owned buffer; admission is by memory and slots."""

    def __init__(self, pool_bytes: int, max_active: int = 4, device: int = 0):
        import numpy as _np  # noqa: F401
        self.pool = torch.empty(int(pool_bytes), dtype=torch.uint8, device=f"cuda:{device}")
        self.h = lib.gw_server_create(ctypes.c_void_p(self.pool.data_ptr()), int(pool_bytes),
                                      int(max_active), int(device))
        if not self.h:
            raise GWError(GW_EINVAL_CODE, gw_last_error())

    def submit(self, x, y, id, kind=PEN_SQEUCLID, param=2.0, D=0, eps=0.05, n_outer=10,
               n_inner=50, prec=PREC_FP32, eps_final=0.0):
        import numpy as np
        x = np.ascontiguousarray(x, dtype=np.float32)
        y = np.ascontiguousarray(y, dtype=np.float32)
        r = GwRequest(int(id), x.shape[0], y.shape[0], x.shape[1], int(kind), float(param), int(D),
                      float(eps), float(eps_final), int(n_outer), int(n_inner), int(prec))
        _check(lib.gw_server_submit(self.h, ctypes.byref(r), x.ctypes.data_as(ctypes.c_void_p),
                                    y.ctypes.data_as(ctypes.c_void_p)))

    def poll(self, max_out: int = 64, wait_ms: int = 0):
        buf = (GwResponse * max_out)()
        k = lib.gw_server_poll(self.h, buf, max_out, int(wait_ms))
        return [{"id": int(buf[i].id), "status": int(buf[i].status),
                 "energy": list(buf[i].energy), "t_submit": buf[i].t_submit,
                 "t_admit": buf[i].t_admit, "t_done": buf[i].t_done,
                 "preempted": int(buf[i].preempted)} for i in range(k)]

    def set_slice(self, outer_steps: int):
        """Time slicing with checkpoint / resume (gw.h: gw_server_set_slice)."""
        _check(lib.gw_server_set_slice(self.h, int(outer_steps)))

    def set_batching(self, on: bool):
        """Batch lane for small squared requests (gw.h: gw_server_set_batching)."""
        _check(lib.gw_server_set_batching(self.h, int(bool(on))))

    def cancel(self, id):
        """Cancel request `id` (gw.h: gw_server_cancel); answered with GW_ECANCELED."""
        _check(lib.gw_server_cancel(self.h, int(id)))

    def set_deadline(self, seconds: float):
        """Host watchdog deadline per request (gw.h: gw_server_set_deadline)."""
        _check(lib.gw_server_set_deadline(self.h, float(seconds)))

    @staticmethod
    def request_bytes(n, m, d=3, kind=PEN_SQEUCLID, D=0, prec=PREC_FP32, param=2.0):
        r = GwRequest(0, int(n), int(m), int(d), int(kind), float(param), int(D), 0.1, 0.0, 1, 1,
                      int(prec))
        return int(lib.gw_server_request_bytes(ctypes.byref(r)))

    def stats(self):
        p, a = _int(0), _int(0)
        lib.gw_server_stats(self.h, ctypes.byref(p), ctypes.byref(a))
        return {"pending": p.value, "active": a.value}

    def close(self):
        if self.h:
            lib.gw_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


GW_EINVAL_CODE = 1
