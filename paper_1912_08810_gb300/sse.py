"""ctypes binding of libsse_gb300.so -- argument marshalling only.

The functions here carry the C ABI's names (include/sse.h) and do no arithmetic: every
step of the self-energy runs in the CUDA library.  If the library is missing the import
of a function fails loudly; there is no CPU fallback.

``Plan`` is a convenience wrapper that takes torch tensors (PyTorch supplies device
memory and streams only) and passes their device pointers to the same entry points.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsse_gb300.so")

SSE_OK = 0
SSE_NOT_READY = 1
SSE_E_INVALID_ARG = -1
SSE_E_OUT_OF_MEMORY = -2
SSE_E_CUDA = -3
SSE_E_OVER_BUDGET = -4
SSE_E_TIMEOUT = -5
SSE_E_UNKNOWN_TICKET = -6
SSE_E_SHUTDOWN = -7
SSE_E_CANCELLED = -9
SSE_E_BOUNDS = -10

SSE_C128 = 0
SSE_C64 = 1
SSE_MODE_FP64 = 0
SSE_MODE_MIXED = 1

SSE_INJECT_NONE = 0
SSE_INJECT_STALL = 1
SSE_INJECT_ALLOC_FAIL = 2

# Every function include/sse.h declares (checked by the CPU test suite).
EXPORTED = (
    "sse_plan", "sse_plan_destroy", "sse_plan_query", "sse_execute", "sse_execute_host",
    "sse_plan_status", "sse_status_string", "sse_last_error", "sse_abi_version",
    "sse_execute_noalloc", "sse_execute_batch", "sse_batch_tuning",
    "sse_server_create", "sse_submit", "sse_poll", "sse_server_shutdown", "sse_server_destroy",
    "sse_server_stats", "sse_plan_set_timing", "sse_plan_timing", "sse_debug_inject",
    "sse_dtilde", "sse_retarded", "sse_execute_full", "sse_pi",
)


class sse_geometry(ctypes.Structure):
    _fields_ = [("nkz", ctypes.c_int32), ("nqz", ctypes.c_int32), ("ne", ctypes.c_int32),
                ("nw", ctypes.c_int32), ("na", ctypes.c_int32), ("nb_max", ctypes.c_int32),
                ("norb", ctypes.c_int32), ("omega_first", ctypes.c_int32),
                ("neigh", ctypes.c_void_p), ("dH", ctypes.c_void_p),
                ("dtype", ctypes.c_int32), ("mode", ctypes.c_int32)]


class sse_io(ctypes.Structure):
    _fields_ = [("G_gt", ctypes.c_void_p), ("G_lt", ctypes.c_void_p),
                ("D_gt", ctypes.c_void_p), ("D_lt", ctypes.c_void_p),
                ("S_gt", ctypes.c_void_p), ("S_lt", ctypes.c_void_p)]


class sse_plan_info(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("dtype", ctypes.c_int32), ("points", ctypes.c_int64),
                ("flops_per_sign", ctypes.c_double), ("bytes_per_sign", ctypes.c_double),
                ("workspace_bytes", ctypes.c_int64), ("tile_e", ctypes.c_int32),
                ("kernel_id", ctypes.c_int32)]


class sse_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("t_submit_ms", ctypes.c_double), ("t_start_ms", ctypes.c_double),
                ("t_end_ms", ctypes.c_double), ("round_size", ctypes.c_int32)]


class SSEError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: {status_name(status)} ({status}): {message}")
        self.status = status


_lock = threading.Lock()
_lib = None


def load(path: Optional[str] = None):
    """Load the CUDA library once; raises if it has not been built.  SSE_GB300_LIB may name
    another build of it (the bounds-checked libsse_gb300_bc.so)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or os.environ.get("SSE_GB300_LIB") or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"CUDA library not built: {p} is missing (run __graft_entry__.build())")
        lib = ctypes.CDLL(p)
        vp, st = ctypes.c_void_p, ctypes.c_int32
        sig = {
            "sse_plan": ([ctypes.POINTER(sse_geometry), ctypes.POINTER(vp)], st),
            "sse_plan_destroy": ([vp], st),
            "sse_plan_query": ([vp, ctypes.POINTER(sse_plan_info)], st),
            "sse_execute": ([vp, ctypes.POINTER(sse_io), vp], st),
            "sse_execute_host": ([vp, ctypes.POINTER(sse_io), vp], st),
            "sse_plan_status": ([vp], st),
            "sse_status_string": ([st], ctypes.c_char_p),
            "sse_last_error": ([], ctypes.c_char_p),
            "sse_abi_version": ([], st),
            "sse_execute_noalloc": ([ctypes.POINTER(sse_geometry), ctypes.POINTER(sse_io), vp], st),
            "sse_execute_batch": ([ctypes.POINTER(vp), ctypes.POINTER(sse_io), ctypes.c_int32, vp], st),
            "sse_batch_tuning": ([ctypes.POINTER(vp), ctypes.POINTER(sse_io), ctypes.c_int32,
                                  ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)], st),
            "sse_server_create": ([ctypes.c_uint64, ctypes.c_int32, ctypes.c_uint32, ctypes.POINTER(vp)], st),
            "sse_submit": ([vp, vp, ctypes.POINTER(sse_io), ctypes.POINTER(ctypes.c_uint64)], st),
            "sse_poll": ([vp, ctypes.c_uint64, ctypes.POINTER(sse_result)], st),
            "sse_server_shutdown": ([vp], st),
            "sse_server_destroy": ([vp], st),
            "sse_debug_inject": ([st], st),
            "sse_dtilde": ([vp, vp, vp, vp], st),
            "sse_retarded": ([vp, vp, vp, vp, vp], st),
            "sse_execute_full": ([vp, ctypes.POINTER(sse_io), vp, vp], st),
            "sse_pi": ([vp, vp, vp, vp, vp, vp], st),
            "sse_server_stats": ([vp, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64),
                                  ctypes.POINTER(ctypes.c_int32)], st),
            "sse_plan_set_timing": ([vp, ctypes.c_int32], st),
            "sse_plan_timing": ([vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                 ctypes.POINTER(ctypes.c_int64)], st),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes, fn.restype = args, res
        _lib = lib
        return lib


def status_name(status: int) -> str:
    try:
        return load().sse_status_string(status).decode()
    except Exception:  # library missing: still format the error
        return str(status)


def sse_last_error() -> str:
    return load().sse_last_error().decode()


def _check(status: int, where: str) -> int:
    if status < 0:
        raise SSEError(status, where, sse_last_error())
    return status


def sse_plan(geo: sse_geometry) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(load().sse_plan(ctypes.byref(geo), ctypes.byref(h)), "sse_plan")
    return h


def sse_plan_destroy(plan) -> None:
    _check(load().sse_plan_destroy(plan), "sse_plan_destroy")


def sse_plan_query(plan) -> sse_plan_info:
    info = sse_plan_info()
    _check(load().sse_plan_query(plan, ctypes.byref(info)), "sse_plan_query")
    return info


def sse_execute(plan, io: sse_io, stream: int = 0) -> None:
    _check(load().sse_execute(plan, ctypes.byref(io), ctypes.c_void_p(stream)), "sse_execute")


def sse_execute_host(plan, io: sse_io, stream: int = 0) -> None:
    _check(load().sse_execute_host(plan, ctypes.byref(io), ctypes.c_void_p(stream)), "sse_execute_host")


def sse_plan_status(plan) -> None:
    _check(load().sse_plan_status(plan), "sse_plan_status")


def sse_plan_set_timing(plan, enable: bool) -> None:
    _check(load().sse_plan_set_timing(plan, ctypes.c_int32(1 if enable else 0)), "sse_plan_set_timing")


def sse_plan_timing(plan):
    """(workspace-pass ms, main-kernel ms, timed calls) since timing was enabled."""
    a, b, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
    _check(load().sse_plan_timing(plan, ctypes.byref(a), ctypes.byref(b), ctypes.byref(n)), "sse_plan_timing")
    return a.value, b.value, n.value


def sse_dtilde(plan, D: int, Dt: int, stream: int = 0) -> None:
    """Pre-combined phonon term of Eq. 3 (device pointers; see include/sse.h)."""
    _check(load().sse_dtilde(plan, ctypes.c_void_p(D), ctypes.c_void_p(Dt), ctypes.c_void_p(stream)), "sse_dtilde")


def sse_retarded(plan, S_gt: int, S_lt: int, S_r: int, stream: int = 0) -> None:
    """Sigma^R = (Sigma^> - Sigma^<) / 2 (device pointers)."""
    _check(load().sse_retarded(plan, ctypes.c_void_p(S_gt), ctypes.c_void_p(S_lt), ctypes.c_void_p(S_r),
                               ctypes.c_void_p(stream)), "sse_retarded")


def sse_execute_full(plan, io: sse_io, S_r: Optional[int] = None, stream: int = 0) -> None:
    """Full phonon tensors in io.D_gt / io.D_lt; Sigma^> / Sigma^< and optionally Sigma^R out."""
    _check(load().sse_execute_full(plan, ctypes.byref(io), ctypes.c_void_p(S_r), ctypes.c_void_p(stream)),
           "sse_execute_full")


def sse_pi(plan, G_gt: int, G_lt: int, Pi_gt: Optional[int], Pi_lt: Optional[int], stream: int = 0) -> None:
    """Phonon self-energy of Eqs. 4-5 (device pointers; see include/sse.h)."""
    _check(load().sse_pi(plan, ctypes.c_void_p(G_gt), ctypes.c_void_p(G_lt), ctypes.c_void_p(Pi_gt),
                         ctypes.c_void_p(Pi_lt), ctypes.c_void_p(stream)), "sse_pi")


def sse_execute_noalloc(geo: sse_geometry, io: sse_io, stream: int = 0) -> None:
    """Mixed-mode evaluation that allocates nothing (see include/sse.h); synchronous."""
    _check(load().sse_execute_noalloc(ctypes.byref(geo), ctypes.byref(io), ctypes.c_void_p(stream)),
           "sse_execute_noalloc")


def _batch_args(plans, ios):
    n = len(plans)
    parr = (ctypes.c_void_p * max(n, 1))(*[p.value if hasattr(p, "value") else p for p in plans])
    iarr = (sse_io * max(n, 1))(*ios)
    return parr, iarr, n


def sse_execute_batch(plans, ios, stream: int = 0) -> None:
    """Many instances in one persistent launch (plan handles and sse_io structs)."""
    parr, iarr, n = _batch_args(plans, ios)
    _check(load().sse_execute_batch(parr, iarr, n, ctypes.c_void_p(stream)), "sse_execute_batch")


def sse_batch_tuning(plans, ios):
    """(tiles_per_unit, longest_first) chosen by the autotuner, or None if not tuned yet."""
    parr, iarr, n = _batch_args(plans, ios)
    tpc, lpt = ctypes.c_int32(), ctypes.c_int32()
    rc = _check(load().sse_batch_tuning(parr, iarr, n, ctypes.byref(tpc), ctypes.byref(lpt)), "sse_batch_tuning")
    return None if rc == SSE_NOT_READY else (tpc.value, lpt.value)


def sse_server_create(mem_budget_bytes: int, max_inflight: int, wait_limit_ms: int = 0):
    h = ctypes.c_void_p()
    _check(load().sse_server_create(mem_budget_bytes, max_inflight, wait_limit_ms, ctypes.byref(h)),
           "sse_server_create")
    return h


def sse_submit(server, plan, io: sse_io) -> int:
    t = ctypes.c_uint64()
    _check(load().sse_submit(server, plan, ctypes.byref(io), ctypes.byref(t)), "sse_submit")
    return t.value


def sse_poll(server, ticket: int):
    """(status, sse_result); status is SSE_NOT_READY, SSE_OK or a negative error code
    (returned, not raised, so callers can inspect failed requests)."""
    r = sse_result()
    rc = load().sse_poll(server, ticket, ctypes.byref(r))
    return rc, r


def sse_server_shutdown(server) -> None:
    """Cancel what has not started (pollable as SSE_E_CANCELLED), wait for running rounds."""
    _check(load().sse_server_shutdown(server), "sse_server_shutdown")


def sse_debug_inject(kind: int) -> None:
    """Arm a one-shot test fault (SSE_INJECT_STALL or SSE_INJECT_ALLOC_FAIL; see include/sse.h)."""
    _check(load().sse_debug_inject(kind), "sse_debug_inject")


def sse_server_destroy(server) -> None:
    _check(load().sse_server_destroy(server), "sse_server_destroy")


def sse_server_stats(server):
    rounds, nbytes, n = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_int32()
    _check(load().sse_server_stats(server, ctypes.byref(rounds), ctypes.byref(nbytes), ctypes.byref(n)),
           "sse_server_stats")
    return rounds.value, nbytes.value, n.value


def sse_status_string(status: int) -> str:
    return load().sse_status_string(status).decode()


def sse_abi_version() -> int:
    return int(load().sse_abi_version())


# --- torch convenience wrapper (pointers and streams only) ----------------------------

def _ptr(t) -> Optional[int]:
    return None if t is None else int(t.data_ptr())


class Plan:
    """A plan over device tensors: neigh int32 [na, nb], dH complex [na, nb, 3, 12, 12].

    ``mode`` is "fp64" or "mixed"; the dtype follows dH (complex128 or complex64).
    """

    def __init__(self, neigh, dH, *, nkz: int, nqz: int, ne: int, nw: int,
                 omega_first: int = 1, mode: str = "fp64"):
        import torch
        if not (neigh.is_cuda and dH.is_cuda):
            raise ValueError("neigh and dH must be CUDA tensors")
        if not (neigh.is_contiguous() and dH.is_contiguous()):
            raise ValueError("neigh and dH must be contiguous")
        if neigh.dtype != torch.int32:
            raise ValueError("neigh must be int32")
        dtype = {torch.complex128: SSE_C128, torch.complex64: SSE_C64}.get(dH.dtype)
        if dtype is None:
            raise ValueError("dH must be complex128 or complex64")
        na, nb = neigh.shape
        if tuple(dH.shape) != (na, nb, 3, 12, 12):
            raise ValueError(f"dH shape {tuple(dH.shape)} != {(na, nb, 3, 12, 12)}")
        self.neigh, self.dH = neigh, dH  # kept alive: the plan borrows them
        self.torch_dtype = dH.dtype
        self.shape_g = (nkz, ne, na, 12, 12)
        self.shape_d = (nqz, nw, na, nb, 3, 3)
        self.geo = sse_geometry(nkz, nqz, ne, nw, na, nb, 12, omega_first, _ptr(neigh), _ptr(dH),
                                dtype, SSE_MODE_MIXED if mode == "mixed" else SSE_MODE_FP64)
        self.handle = sse_plan(self.geo)

    def info(self) -> sse_plan_info:
        return sse_plan_query(self.handle)

    def _io(self, G_gt, G_lt, D_gt, D_lt, S_gt, S_lt) -> sse_io:
        for t, shp in ((G_gt, self.shape_g), (G_lt, self.shape_g), (S_gt, self.shape_g),
                       (S_lt, self.shape_g), (D_gt, self.shape_d), (D_lt, self.shape_d)):
            if t is None:
                continue
            if tuple(t.shape) != shp or t.dtype != self.torch_dtype or not t.is_contiguous():
                raise ValueError(f"tensor mismatch: shape {tuple(t.shape)} dtype {t.dtype} contiguous {t.is_contiguous()}; want shape {shp} dtype {self.torch_dtype}, contiguous")
        return sse_io(_ptr(G_gt), _ptr(G_lt), _ptr(D_gt), _ptr(D_lt), _ptr(S_gt), _ptr(S_lt))

    def execute(self, G_gt=None, G_lt=None, D_gt=None, D_lt=None, S_gt=None, S_lt=None,
                stream=None) -> None:
        import torch
        for t in (G_gt, G_lt, D_gt, D_lt, S_gt, S_lt):
            if t is not None and not t.is_cuda:
                raise ValueError("execute() takes CUDA tensors; use execute_host() for host arrays")
        s = stream if stream is not None else torch.cuda.current_stream()
        sse_execute(self.handle, self._io(G_gt, G_lt, D_gt, D_lt, S_gt, S_lt), s.cuda_stream)

    def execute_host(self, G_gt=None, G_lt=None, D_gt=None, D_lt=None, S_gt=None, S_lt=None,
                     stream=None) -> None:
        """Host tensors in and out (pinned or pageable); synchronous."""
        import torch
        for t in (G_gt, G_lt, D_gt, D_lt, S_gt, S_lt):
            if t is not None and t.is_cuda:
                raise ValueError("execute_host() takes host tensors")
        s = stream if stream is not None else torch.cuda.current_stream()
        sse_execute_host(self.handle, self._io(G_gt, G_lt, D_gt, D_lt, S_gt, S_lt), s.cuda_stream)

    def dtilde(self, D, Dt, stream=None) -> None:
        """Dt [nqz, nw, na, nb, 3, 3] from the full phonon tensor D [nqz, nw, na, nb + 1, 3, 3]."""
        import torch
        nqz, nw, na, nb = self.shape_d[:4]
        self._check_tensor(D, (nqz, nw, na, nb + 1, 3, 3))
        self._check_tensor(Dt, self.shape_d)
        s = stream if stream is not None else torch.cuda.current_stream()
        sse_dtilde(self.handle, _ptr(D), _ptr(Dt), s.cuda_stream)

    def retarded(self, S_gt, S_lt, S_r, stream=None) -> None:
        import torch
        for t in (S_gt, S_lt, S_r):
            self._check_tensor(t, self.shape_g)
        s = stream if stream is not None else torch.cuda.current_stream()
        sse_retarded(self.handle, _ptr(S_gt), _ptr(S_lt), _ptr(S_r), s.cuda_stream)

    def execute_full(self, G_gt=None, G_lt=None, D_gt=None, D_lt=None, S_gt=None, S_lt=None, S_r=None,
                     stream=None) -> None:
        """As execute(), with the FULL phonon tensors [nqz, nw, na, nb + 1, 3, 3] in D_gt / D_lt;
        also writes Sigma^R into S_r when given."""
        import torch
        nqz, nw, na, nb = self.shape_d[:4]
        full = (nqz, nw, na, nb + 1, 3, 3)
        for t, shp in ((G_gt, self.shape_g), (G_lt, self.shape_g), (S_gt, self.shape_g), (S_lt, self.shape_g),
                       (S_r, self.shape_g), (D_gt, full), (D_lt, full)):
            if t is not None:
                self._check_tensor(t, shp)
        io = sse_io(_ptr(G_gt), _ptr(G_lt), _ptr(D_gt), _ptr(D_lt), _ptr(S_gt), _ptr(S_lt))
        s = stream if stream is not None else torch.cuda.current_stream()
        sse_execute_full(self.handle, io, _ptr(S_r), s.cuda_stream)

    def pi(self, G_gt, G_lt, Pi_gt=None, Pi_lt=None, stream=None) -> None:
        """Pi^> / Pi^< [nqz, nw, na, nb + 1, 3, 3] from G^> and G^< (both needed for either sign)."""
        import torch
        nqz, nw, na, nb = self.shape_d[:4]
        for t, shp in ((G_gt, self.shape_g), (G_lt, self.shape_g), (Pi_gt, (nqz, nw, na, nb + 1, 3, 3)),
                       (Pi_lt, (nqz, nw, na, nb + 1, 3, 3))):
            if t is not None:
                self._check_tensor(t, shp)
        s = stream if stream is not None else torch.cuda.current_stream()
        sse_pi(self.handle, _ptr(G_gt), _ptr(G_lt), _ptr(Pi_gt), _ptr(Pi_lt), s.cuda_stream)

    def _check_tensor(self, t, shp) -> None:
        if not t.is_cuda or tuple(t.shape) != tuple(shp) or t.dtype != self.torch_dtype or not t.is_contiguous():
            raise ValueError(f"tensor mismatch: shape {tuple(t.shape)} dtype {t.dtype}; want {tuple(shp)} "
                             f"{self.torch_dtype}, contiguous, on the GPU")

    def status(self) -> None:
        sse_plan_status(self.handle)

    def close(self) -> None:
        if getattr(self, "handle", None) is not None and self.handle.value:
            sse_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
