"""CPU FP64 oracle for Sigma^{<>} (Eq. 3) -- TEST INFRASTRUCTURE ONLY.

Only the test suite, the smoke check and the CPU-baseline leg of the benchmark may
import this package.  The product path (the CUDA library and its binding) never
imports, links or calls it, and it imports nothing from the product package.

``build()`` compiles ``sse_oracle.c`` with gcc (-O2, OpenMP) into ``libsse_oracle.so``
beside it.  The wrappers below only marshal numpy arrays; every arithmetic step is in
the C file.  Inputs stored as complex64 are widened to complex128 here, so the oracle
always computes in FP64.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sse_oracle.c")
_LIB = os.path.join(_HERE, "libsse_oracle.so")
_lock = threading.Lock()
_lib = None


class _Geometry(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in
                ("nkz", "nqz", "ne", "nw", "na", "nb", "norb", "omega_first")]


def build(force: bool = False) -> str:
    """Compile the oracle shared library (plain C, no CUDA)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-std=c11", "-O2", "-fopenmp", "-fcx-limited-range", "-fPIC", "-shared",
               "-o", _LIB + ".tmp", _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            p = ctypes.c_void_p
            lib.oracle_sigma_points.argtypes = [ctypes.POINTER(_Geometry), p, p, p, p,
                                                ctypes.c_int64, p, p]
            lib.oracle_sigma_points.restype = ctypes.c_int
            lib.oracle_sigma_atoms.argtypes = [ctypes.POINTER(_Geometry), p, p, p, p,
                                               ctypes.c_int32, ctypes.c_int32, p]
            lib.oracle_sigma_atoms.restype = ctypes.c_int
            lib.oracle_num_threads.restype = ctypes.c_int
            lib.oracle_dtilde.argtypes = [ctypes.POINTER(_Geometry), p, p, p]
            lib.oracle_dtilde.restype = ctypes.c_int
            lib.oracle_pi.argtypes = [ctypes.POINTER(_Geometry), p, p, p, p, p]
            lib.oracle_pi.restype = ctypes.c_int
            lib.oracle_retarded.argtypes = [ctypes.c_int64, p, p, p]
            lib.oracle_retarded.restype = ctypes.c_int
            _lib = lib
    return _lib


def _geometry(G, Dt, dH, neigh, omega_first):
    nkz, ne, na, norb, norb2 = G.shape
    nqz, nw, na2, nb, d1, d2 = Dt.shape
    if norb != norb2 or na2 != na or (d1, d2) != (3, 3):
        raise ValueError("inconsistent G / Dt shapes")
    if dH.shape != (na, nb, 3, norb, norb) or neigh.shape != (na, nb):
        raise ValueError("inconsistent dH / neigh shapes")
    return _Geometry(nkz, nqz, ne, nw, na, nb, norb, omega_first)


def _c128(x):
    return np.ascontiguousarray(x, dtype=np.complex128)


def sigma_points(G, Dt, dH, neigh, points, omega_first: int = 1) -> np.ndarray:
    """Eq. 3 term by term at the given (k, E, a) points; returns [npts, norb, norb]."""
    G, Dt, dH = _c128(G), _c128(Dt), _c128(dH)
    neigh = np.ascontiguousarray(neigh, dtype=np.int32)
    pts = np.ascontiguousarray(np.asarray(points, dtype=np.int32).reshape(-1, 3))
    geo = _geometry(G, Dt, dH, neigh, omega_first)
    out = np.zeros((pts.shape[0], geo.norb, geo.norb), dtype=np.complex128)
    rc = _load().oracle_sigma_points(ctypes.byref(geo), neigh.ctypes.data, dH.ctypes.data,
                                     G.ctypes.data, Dt.ctypes.data, pts.shape[0],
                                     pts.ctypes.data, out.ctypes.data)
    if rc != 0:
        raise ValueError("oracle_sigma_points rejected its arguments")
    return out


def sigma_atoms(G, Dt, dH, neigh, a_begin: int = 0, a_end=None, omega_first: int = 1) -> np.ndarray:
    """All (k, E) points of atoms [a_begin, a_end) via the redundancy-removed sum;
    returns [nkz, ne, a_end - a_begin, norb, norb]."""
    G, Dt, dH = _c128(G), _c128(Dt), _c128(dH)
    neigh = np.ascontiguousarray(neigh, dtype=np.int32)
    geo = _geometry(G, Dt, dH, neigh, omega_first)
    a_end = geo.na if a_end is None else int(a_end)
    out = np.zeros((geo.nkz, geo.ne, a_end - a_begin, geo.norb, geo.norb), dtype=np.complex128)
    rc = _load().oracle_sigma_atoms(ctypes.byref(geo), neigh.ctypes.data, dH.ctypes.data,
                                    G.ctypes.data, Dt.ctypes.data, int(a_begin), a_end,
                                    out.ctypes.data)
    if rc != 0:
        raise ValueError("oracle_sigma_atoms rejected its arguments")
    return out


def dtilde(D, neigh) -> np.ndarray:
    """Pre-combined phonon term of Eq. 3 from the full tensor D [nqz, nw, na, nb+1, 3, 3]
    (block nb = the diagonal D_aa); returns Dt [nqz, nw, na, nb, 3, 3]."""
    D = _c128(D)
    neigh = np.ascontiguousarray(neigh, dtype=np.int32)
    nqz, nw, na, nb1, d1, d2 = D.shape
    na2, nb = neigh.shape
    if na2 != na or nb1 != nb + 1 or (d1, d2) != (3, 3):
        raise ValueError("inconsistent D / neigh shapes")
    geo = _Geometry(1, nqz, 1, nw, na, nb, 1, 0)
    out = np.zeros((nqz, nw, na, nb, 3, 3), dtype=np.complex128)
    rc = _load().oracle_dtilde(ctypes.byref(geo), neigh.ctypes.data, D.ctypes.data, out.ctypes.data)
    if rc != 0:
        raise ValueError("oracle_dtilde rejected its arguments (neighbour out of range or a bond without its reverse)")
    return out


def retarded(S_gt, S_lt) -> np.ndarray:
    """Sigma^R = (Sigma^> - Sigma^<) / 2 (Section 2)."""
    S_gt, S_lt = _c128(S_gt), _c128(S_lt)
    if S_gt.shape != S_lt.shape:
        raise ValueError("shape mismatch")
    out = np.empty_like(S_gt)
    rc = _load().oracle_retarded(S_gt.size, S_gt.ctypes.data, S_lt.ctypes.data, out.ctypes.data)
    if rc != 0:
        raise ValueError("oracle_retarded rejected its arguments")
    return out


def pi(Ga, Gb, dH, neigh, nqz: int, nw: int, omega_first: int = 1) -> np.ndarray:
    """Phonon self-energy of Eqs. 4-5 with Ga paired at atom a (energy E + omega, momentum
    k + q) and Gb at the neighbour (E, k): Pi^> = pi(G^>, G^<, ...), Pi^< = pi(G^<, G^>, ...).
    Returns [nqz, nw, na, nb + 1, 3, 3] (block nb = the diagonal block)."""
    Ga, Gb, dH = _c128(Ga), _c128(Gb), _c128(dH)
    neigh = np.ascontiguousarray(neigh, dtype=np.int32)
    nkz, ne, na, norb, _ = Ga.shape
    nb = neigh.shape[1]
    if Gb.shape != Ga.shape or dH.shape != (na, nb, 3, norb, norb) or neigh.shape[0] != na:
        raise ValueError("inconsistent shapes")
    geo = _Geometry(nkz, nqz, ne, nw, na, nb, norb, omega_first)
    out = np.zeros((nqz, nw, na, nb + 1, 3, 3), dtype=np.complex128)
    rc = _load().oracle_pi(ctypes.byref(geo), neigh.ctypes.data, dH.ctypes.data, Ga.ctypes.data,
                           Gb.ctypes.data, out.ctypes.data)
    if rc != 0:
        raise ValueError("oracle_pi rejected its arguments")
    return out


def num_threads() -> int:
    """OpenMP threads the oracle uses."""
    return int(_load().oracle_num_threads())
