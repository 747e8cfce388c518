"""Python binding of libbnb.so, the B300 (sm_103a) l0-l2 branch-and-bound library.

Argument marshalling only: every step of the computation runs in the CUDA
kernels behind the C ABI declared in include/bnb.h.  The function names are
those of the C ABI.  Host arrays are numpy; the *_device entry points accept
torch CUDA tensors (their data pointers are passed through).

The library must have been built (``python -m paper_2602_04551_b300.build`` or
``__graft_entry__.build()``); importing the binding without it raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbnb.so")

BNB_OK = 0
BNB_EINVAL, BNB_ENOMEM, BNB_ECUDA, BNB_ETIMEOUT, BNB_EQUEUE, BNB_ENODEV = -1, -2, -3, -4, -5, -6
BNB_PREC_FP64, BNB_PREC_FP32, BNB_PREC_BF16, BNB_PREC_TC3, BNB_PREC_BF16X2 = 0, 1, 2, 3, 4
STATUS_NAMES = {0: "optimal", 1: "gap", 2: "time_limit", 3: "queue_full", 4: "node_limit",
                5: "depth_limit", 6: "support_limit"}

# exported symbols (kept in step with include/bnb.h)
SYMBOLS = ("bnb_options_default", "bnb_footprint", "bnb_create", "bnb_create_device", "bnb_relax_batch",
           "bnb_relax_batch_device", "bnb_dual_bound", "bnb_upper_batch", "bnb_solve",
           "bnb_solve_start", "bnb_solve_launch", "bnb_solve_poll", "bnb_solve_finish",
           "bnb_stream", "bnb_root_heuristic", "bnb_profile_round", "bnb_dual_bound_static",
           "bnb_get_stats", "bnb_get_histograms", "bnb_get_node_log",
           "bnb_last_error", "bnb_destroy")
LOG_FIELDS = ("lb", "exact", "width", "node_lb", "parent_lb", "threshold", "depth", "iters",
              "est_dual", "est_primal")
# exported by libbnb_diag.so (kept in step with include/bnb_diag.h)
DIAG_SYMBOLS = ("bnb_tc_gemm_check", "bnb_tc_gemm_check_cluster", "bnb_tc_gemm_check_pair",
                "bnb_diag_wait_expiry", "bnb_diag_tma_stream")
DIAG_LIB_PATH = os.path.join(_HERE, "libbnb_diag.so")
STAGES = ("select_refill", "gemm_xw", "reduce_t_or_make_w", "gemm_ginv_t", "finalize_u", "gemm_xtu_prox",
          "check_xbeta", "stop_test", "certificate", "branch", "upper_bound", "push", "status",
          "cert_screen", "cert_exact")


class bnb_options(ctypes.Structure):
    _fields_ = [("M", ctypes.c_double), ("rho", ctypes.c_double), ("node_tol", ctypes.c_double),
                ("max_admm_iter", ctypes.c_int), ("check_every", ctypes.c_int),
                ("batch_K", ctypes.c_int), ("precision", ctypes.c_int),
                ("use_graphs", ctypes.c_int), ("time_limit_s", ctypes.c_double),
                ("max_nodes", ctypes.c_longlong), ("queue_capacity", ctypes.c_longlong),
                ("warm_capacity", ctypes.c_longlong), ("support_max", ctypes.c_int),
                ("ub_max_iter", ctypes.c_int), ("device", ctypes.c_int),
                ("stream", ctypes.c_void_p), ("relax_alpha", ctypes.c_double),
                ("root_heuristic", ctypes.c_int), ("max_depth", ctypes.c_int),
                ("lockstep", ctypes.c_int), ("mv_crossover", ctypes.c_int),
                ("fused_shape", ctypes.c_int), ("u_shape", ctypes.c_int),
                ("ub_polish", ctypes.c_int), ("fused_width", ctypes.c_int),
                ("fused_select", ctypes.c_int), ("exact_bounds", ctypes.c_int),
                ("log_nodes", ctypes.c_int), ("early_branch", ctypes.c_int)]


class bnb_stats(ctypes.Structure):
    _fields_ = [("nodes", ctypes.c_longlong), ("rounds", ctypes.c_longlong),
                ("admm_iters", ctypes.c_longlong), ("slot_iters", ctypes.c_longlong),
                ("pruned", ctypes.c_longlong), ("ub_polished", ctypes.c_longlong),
                ("pool_peak", ctypes.c_longlong), ("max_depth", ctypes.c_int),
                ("solve_seconds", ctypes.c_double), ("setup_seconds", ctypes.c_double),
                ("final_ub", ctypes.c_double), ("final_lb", ctypes.c_double),
                ("round_kernels", ctypes.c_int), ("xw_tile_width", ctypes.c_int),
                ("xw_cluster", ctypes.c_int), ("fused_tile_width", ctypes.c_int),
                ("fused_clusters", ctypes.c_int), ("fused_pairs", ctypes.c_int),
                ("fused_transposed", ctypes.c_int), ("u_split", ctypes.c_int),
                ("u_cluster_pairs", ctypes.c_int)]


class bnb_progress(ctypes.Structure):
    _fields_ = [("ub", ctypes.c_double), ("lb", ctypes.c_double), ("nodes", ctypes.c_longlong),
                ("open_nodes", ctypes.c_longlong), ("active_slots", ctypes.c_longlong),
                ("rounds", ctypes.c_longlong),
                ("seconds", ctypes.c_double), ("done", ctypes.c_int), ("status", ctypes.c_int)]


class BnbError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"bnb error {code}: {msg}")
        self.code = code


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libbnb.so (raises if it is missing: there is no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} not built; run python -m paper_2602_04551_b300.build")
    lib = ctypes.CDLL(path)
    P, D, I, LL = ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_longlong
    sig = {
        "bnb_options_default": ([P], I),
        "bnb_create": ([P, P, I, I, D, D, P, P], I),
        "bnb_footprint": ([I, I, P, P], I),
        "bnb_create_device": ([P, P, I, I, D, D, P, P], I),
        "bnb_relax_batch": ([P, I, P, P, P, I, P, P, P, P, P, P, P], I),
        "bnb_relax_batch_device": ([P, I, P, P, P, I, P, P, P, P, P, P, P], I),
        "bnb_dual_bound": ([P, I, P, P, P], I),
        "bnb_upper_batch": ([P, I, P, P, P], I),
        "bnb_solve": ([P, D, P, P, P, P, P], I),
        "bnb_solve_start": ([P, D], I),
        "bnb_solve_launch": ([P, I], I),
        "bnb_solve_poll": ([P, P], I),
        "bnb_solve_finish": ([P, P, P, P, P, P], I),
        "bnb_stream": ([P], P),
        "bnb_root_heuristic": ([P, P, P], I),
        "bnb_profile_round": ([P, P, P, I], I),
        "bnb_get_histograms": ([P, P, I, P, I], I),
        "bnb_get_node_log": ([P, I, P, P, P, P], I),
        "bnb_dual_bound_static": ([P, P, I, I, D, D, D, I, P, P, P, P], I),
        "bnb_get_stats": ([P, P], I),
        "bnb_last_error": ([P], ctypes.c_char_p),
        "bnb_destroy": ([P], None),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


_diag = None


def load_diag_library(path: str = DIAG_LIB_PATH):
    """Load libbnb_diag.so, the diagnostics of include/bnb_diag.h (raises if missing)."""
    global _diag
    if _diag is not None:
        return _diag
    load_library()
    if not os.path.exists(path):
        raise ImportError(f"{path} not built; run python -m paper_2602_04551_b300.build")
    lib = ctypes.CDLL(path)
    P, D, I, LL = ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_longlong
    sig = {
        "bnb_tc_gemm_check": ([P, P, I, I, I, I, I, I, P, P], I),
        "bnb_tc_gemm_check_cluster": ([P, P, I, I, I, I, I, P, P], I),
        "bnb_tc_gemm_check_pair": ([P, P, I, I, I, I, I, P, P], I),
        "bnb_diag_wait_expiry": ([LL, D, P, P], I),
        "bnb_diag_tma_stream": ([I, I, I, I, I, P, P, P], I),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _diag = lib
    return lib


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(rc, h=None):
    if rc != BNB_OK:
        msg = load_library().bnb_last_error(h)
        raise BnbError(rc, msg.decode() if msg else "")


def bnb_options_default(**overrides) -> bnb_options:
    """bnb_options with the library's defaults, then the given fields (an unknown field
    name is an error: ctypes would otherwise keep it as a plain Python attribute that the
    library never sees)."""
    lib = load_library()
    o = bnb_options()
    _check(lib.bnb_options_default(ctypes.byref(o)))
    fields = {name for name, _ in bnb_options._fields_}
    for k, v in overrides.items():
        if k not in fields:
            raise TypeError(f"bnb_options has no field {k!r}")
        setattr(o, k, v)
    return o


class Handle:
    """Owns a bnb_handle*; destroyed with bnb_destroy."""

    def __init__(self, ptr, n, p, options):
        self.ptr = ptr
        self.n, self.p = n, p
        self.options = options

    def close(self):
        if self.ptr:
            load_library().bnb_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def bnb_footprint(n: int, p: int, options: bnb_options) -> int:
    b = ctypes.c_size_t(0)
    _check(load_library().bnb_footprint(int(n), int(p), ctypes.byref(options), ctypes.byref(b)))
    return int(b.value)


def bnb_create(X, y, lambda0: float, lambda2: float, options: bnb_options) -> Handle:
    lib = load_library()
    X = np.asfortranarray(X, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    n, p = X.shape
    h = ctypes.c_void_p()
    _check(lib.bnb_create(_ptr(X), _ptr(y), n, p, float(lambda0), float(lambda2),
                          ctypes.byref(options), ctypes.byref(h)))
    return Handle(h, n, p, options)


def bnb_create_device(dX, dy, n: int, p: int, lambda0: float, lambda2: float,
                      options: bnb_options) -> Handle:
    lib = load_library()
    h = ctypes.c_void_p()
    _check(lib.bnb_create_device(_ptr(dX), _ptr(dy), n, p, float(lambda0), float(lambda2),
                                 ctypes.byref(options), ctypes.byref(h)))
    return Handle(h, n, p, options)


def bnb_relax_batch(h: Handle, fix, warm_beta=None, warm_v=None, max_iter: int = 0,
                    want_beta=True, want_v=False, want_z=True):
    lib = load_library()
    fix = np.ascontiguousarray(fix, dtype=np.int8)
    K, p = fix.shape
    wb = None if warm_beta is None else np.ascontiguousarray(warm_beta, dtype=np.float32)
    wv = None if warm_v is None else np.ascontiguousarray(warm_v, dtype=np.float32)
    lb = np.empty(K, np.float64)
    beta = np.empty((K, p), np.float32) if want_beta else None
    v = np.empty((K, p), np.float32) if want_v else None
    z = np.empty((K, p), np.float32) if want_z else None
    br = np.empty(K, np.int32)
    gap = np.empty(K, np.float64)
    iters = np.empty(K, np.int32)
    _check(lib.bnb_relax_batch(h.ptr, K, _ptr(fix), _ptr(wb), _ptr(wv), int(max_iter), _ptr(lb),
                               _ptr(beta), _ptr(v), _ptr(z), _ptr(br), _ptr(gap), _ptr(iters)), h.ptr)
    return dict(lb=lb, beta=beta, v=v, z=z, branch=br, gap=gap, iters=iters)


def bnb_relax_batch_device(h: Handle, K: int, dfix, dwarm_beta, dwarm_v, max_iter, dlb,
                           dbeta=None, dv=None, dz=None, dbr=None, dgap=None, diters=None):
    lib = load_library()
    _check(lib.bnb_relax_batch_device(h.ptr, K, _ptr(dfix), _ptr(dwarm_beta), _ptr(dwarm_v),
                                      int(max_iter), _ptr(dlb), _ptr(dbeta), _ptr(dv), _ptr(dz),
                                      _ptr(dbr), _ptr(dgap), _ptr(diters)), h.ptr)


def bnb_dual_bound(h: Handle, fix, r):
    lib = load_library()
    fix = np.ascontiguousarray(fix, dtype=np.int8)
    r = np.ascontiguousarray(r, dtype=np.float64)
    K = fix.shape[0]
    lb = np.empty(K, np.float64)
    _check(lib.bnb_dual_bound(h.ptr, K, _ptr(fix), _ptr(r), _ptr(lb)), h.ptr)
    return lb


def _check_device_tensor(name, t, dtype, numel, device):
    if not hasattr(t, "is_cuda") or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.numel() != numel:
        raise ValueError(f"{name} has {t.numel()} elements, expected {numel}")
    if t.device != device:
        raise ValueError(f"{name} is on {t.device}, expected {device}")


def bnb_dual_bound_static(dX, dy, n, p, lambda0, lambda2, M, dfix, dr, dlb, stream=0):
    """Allocation-free dual bound on device tensors (see include/bnb.h).

    dX (n*p float64, column-major), dy (n float64), dfix (K x p int8), dr (K x n float64)
    and dlb (K float64) must be contiguous CUDA tensors on one device; a size, dtype or
    device mismatch raises ValueError before the library is called, so no kernel ever
    reads or writes past a caller's buffer.  Sizes beyond the library's fixed scratch
    come back as BnbError(BNB_EINVAL)."""
    import torch
    n, p = int(n), int(p)
    if dfix.dim() != 2:
        raise ValueError("dfix must be a K x p tensor")
    K = int(dfix.shape[0])
    dev = dX.device if hasattr(dX, "device") else None
    _check_device_tensor("dX", dX, torch.float64, n * p, dev)
    _check_device_tensor("dy", dy, torch.float64, n, dev)
    _check_device_tensor("dfix", dfix, torch.int8, K * p, dev)
    _check_device_tensor("dr", dr, torch.float64, K * n, dev)
    _check_device_tensor("dlb", dlb, torch.float64, K, dev)
    _check(load_library().bnb_dual_bound_static(_ptr(dX), _ptr(dy), int(n), int(p), float(lambda0),
                                                float(lambda2), float(M), K, _ptr(dfix), _ptr(dr),
                                                _ptr(dlb), ctypes.c_void_p(stream or 0)))


def bnb_upper_batch(h: Handle, support):
    lib = load_library()
    support = np.ascontiguousarray(support, dtype=np.uint8)
    K, p = support.shape
    ub = np.empty(K, np.float64)
    beta = np.empty((K, p), np.float64)
    _check(lib.bnb_upper_batch(h.ptr, K, _ptr(support), _ptr(ub), _ptr(beta)), h.ptr)
    return ub, beta


def bnb_solve(h: Handle, rel_gap: float):
    lib = load_library()
    beta = np.empty(h.p, np.float64)
    ub, lb = ctypes.c_double(), ctypes.c_double()
    nodes, status = ctypes.c_longlong(), ctypes.c_int()
    _check(lib.bnb_solve(h.ptr, float(rel_gap), _ptr(beta), ctypes.byref(ub), ctypes.byref(lb),
                         ctypes.byref(nodes), ctypes.byref(status)), h.ptr)
    return dict(beta=beta, ub=ub.value, lb=lb.value, nodes=nodes.value,
                status=STATUS_NAMES.get(status.value, status.value))


def bnb_solve_start(h: Handle, rel_gap: float):
    _check(load_library().bnb_solve_start(h.ptr, float(rel_gap)), h.ptr)


def bnb_solve_launch(h: Handle, rounds: int = 1):
    _check(load_library().bnb_solve_launch(h.ptr, int(rounds)), h.ptr)


def bnb_solve_poll(h: Handle) -> dict:
    pr = bnb_progress()
    _check(load_library().bnb_solve_poll(h.ptr, ctypes.byref(pr)), h.ptr)
    d = {k: getattr(pr, k) for k, _ in bnb_progress._fields_}
    d["done"] = bool(d["done"])
    d["status"] = STATUS_NAMES.get(d["status"], d["status"])
    return d


def bnb_solve_finish(h: Handle):
    lib = load_library()
    beta = np.empty(h.p, np.float64)
    ub, lb = ctypes.c_double(), ctypes.c_double()
    nodes, status = ctypes.c_longlong(), ctypes.c_int()
    _check(lib.bnb_solve_finish(h.ptr, _ptr(beta), ctypes.byref(ub), ctypes.byref(lb),
                                ctypes.byref(nodes), ctypes.byref(status)), h.ptr)
    return dict(beta=beta, ub=ub.value, lb=lb.value, nodes=nodes.value,
                status=STATUS_NAMES.get(status.value, status.value))


def bnb_profile_round(h: Handle) -> dict:
    ms = np.zeros(len(STAGES), np.float64)
    cnt = np.zeros(len(STAGES), np.int32)
    _check(load_library().bnb_profile_round(h.ptr, _ptr(ms), _ptr(cnt), len(STAGES)), h.ptr)
    return {name: (float(ms[i]), int(cnt[i])) for i, name in enumerate(STAGES)}


def bnb_tc_gemm_check(dA, dB, M, N, Kd, nsplit=1, bn=128, splits=1, dC=None):
    """Tensor-core contraction C = A B^T on torch CUDA tensors (FP64 in, FP32 out)."""
    err = ctypes.c_int(0)
    _check(load_diag_library().bnb_tc_gemm_check(_ptr(dA), _ptr(dB), M, N, Kd, nsplit, bn, splits,
                                            _ptr(dC), ctypes.byref(err)))
    return err.value


def bnb_get_histograms(h: Handle, ndepth: int = 257, nsupport: int = 258):
    """Solved-node histograms: (depth counts, rounded-support-size counts)."""
    d = np.zeros(ndepth, np.int64)
    s = np.zeros(nsupport, np.int64)
    _check(load_library().bnb_get_histograms(h.ptr, _ptr(d), ndepth, _ptr(s), nsupport), h.ptr)
    return d, s


def bnb_get_node_log(h: Handle, max_entries: int | None = None) -> dict:
    """The node log of the last solve (options.log_nodes > 0): fixings, FP64 residuals and
    one record per certified node (fields LOG_FIELDS), in retirement order."""
    lib = load_library()
    cnt = ctypes.c_int(0)
    _check(lib.bnb_get_node_log(h.ptr, 0, None, None, None, ctypes.byref(cnt)), h.ptr)
    m = cnt.value if max_entries is None else min(cnt.value, int(max_entries))
    fix = np.empty((m, h.p), np.int8)
    r = np.empty((m, h.n), np.float64)
    rec = np.empty((m, len(LOG_FIELDS)), np.float64)
    if m:
        _check(lib.bnb_get_node_log(h.ptr, m, _ptr(fix), _ptr(r), _ptr(rec), ctypes.byref(cnt)),
               h.ptr)
    out = {"count": cnt.value, "fix": fix, "r": r}
    for i, name in enumerate(LOG_FIELDS):
        out[name] = rec[:, i]
    return out


def bnb_tc_gemm_check_pair(dA, dB, M, N, Kd, nsplit=3, bn=144, dC=None):
    """C = A B^T through the CTA-pair tensor-core kernel (FP64 in, FP32 out)."""
    err = ctypes.c_int(0)
    _check(load_diag_library().bnb_tc_gemm_check_pair(_ptr(dA), _ptr(dB), M, N, Kd, nsplit, bn,
                                                 _ptr(dC), ctypes.byref(err)))
    return err.value


def bnb_tc_gemm_check_cluster(dA, dB, M, N, Kd, nsplit=3, cluster=8, dC=None):
    """C = A B^T through the cluster-reduced tensor-core kernel (FP64 in, FP32 out)."""
    err = ctypes.c_int(0)
    _check(load_diag_library().bnb_tc_gemm_check_cluster(_ptr(dA), _ptr(dB), M, N, Kd, nsplit, cluster,
                                                    _ptr(dC), ctypes.byref(err)))
    return err.value


def bnb_diag_wait_expiry(max_polls: int, max_seconds: float):
    """The kernels' bounded mbarrier wait on a barrier nothing arrives on, with short limits
    (include/bnb_diag.h); returns (error word, seconds spent waiting)."""
    err = ctypes.c_int(-1)
    sec = ctypes.c_double(-1.0)
    _check(load_diag_library().bnb_diag_wait_expiry(int(max_polls), float(max_seconds),
                                                    ctypes.byref(err), ctypes.byref(sec)))
    return err.value, sec.value


def bnb_diag_tma_stream(ctas: int, stages: int = 3, b_rows: int = 88, reps: int = 8,
                        launches: int = 5):
    """The TMA operand ring alone (include/bnb_diag.h): dict with the best launch time
    (us), the bytes one launch delivers, GB/s per CTA (one CTA per SM) and in total, and
    the kernel's error word."""
    us, nbytes, err = ctypes.c_double(-1.0), ctypes.c_double(-1.0), ctypes.c_int(-1)
    _check(load_diag_library().bnb_diag_tma_stream(int(ctas), int(stages), int(b_rows), int(reps),
                                                   int(launches), ctypes.byref(us),
                                                   ctypes.byref(nbytes), ctypes.byref(err)))
    t = us.value * 1e-6
    return {"us": us.value, "bytes": nbytes.value, "err": err.value,
            "gbs_per_sm": nbytes.value / ctas / t / 1e9 if t > 0 else 0.0,
            "tbs_total": nbytes.value / t / 1e12 if t > 0 else 0.0}


def bnb_root_heuristic(h: Handle):
    beta = np.empty(h.p, np.float64)
    ub = ctypes.c_double()
    _check(load_library().bnb_root_heuristic(h.ptr, _ptr(beta), ctypes.byref(ub)), h.ptr)
    return beta, ub.value


def bnb_stream(h: Handle) -> int:
    return load_library().bnb_stream(h.ptr) or 0


def bnb_get_stats(h: Handle) -> dict:
    lib = load_library()
    s = bnb_stats()
    _check(lib.bnb_get_stats(h.ptr, ctypes.byref(s)), h.ptr)
    return {k: getattr(s, k) for k, _ in bnb_stats._fields_}


def bnb_last_error(h: Handle | None = None) -> str:
    m = load_library().bnb_last_error(h.ptr if h else None)
    return m.decode() if m else ""


def bnb_destroy(h: Handle):
    h.close()
