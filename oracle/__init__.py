"""ctypes wrapper of the FP64 CPU oracle (oracle/pcc_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg, never by the library.  It shares no code with
the CUDA path.  Inputs are converted to float64 (exactly, from float32)
before the oracle sees them.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_lib = None
_P = ctypes.c_void_p
_I64 = ctypes.c_int64


def lib(path: str | None = None):
    """Load (building first if needed) the oracle shared library."""
    global _lib
    if path is not None:
        return _load(path)
    if _lib is None:
        _lib = _load(_build.build())
    return _lib


def _load(path):
    L = ctypes.CDLL(path)
    L.oracle_pcc_pair.restype = ctypes.c_double
    L.oracle_pcc_pair.argtypes = [_P, _P, _I64]
    L.oracle_row_stats.argtypes = [_P, _I64, _I64, _I64, _P, _P]
    L.oracle_num_pairs.restype = _I64
    L.oracle_num_pairs.argtypes = [_I64]
    L.oracle_pair_index.restype = _I64
    L.oracle_pair_index.argtypes = [_I64, _I64, _I64]
    L.oracle_pair_coords.restype = ctypes.c_int
    L.oracle_pair_coords.argtypes = [_I64, _I64, _P, _P]
    L.oracle_job_index_diag.restype = _I64
    L.oracle_job_index_diag.argtypes = [_I64, _I64, _I64]
    L.oracle_job_coords_diag.restype = ctypes.c_int
    L.oracle_job_coords_diag.argtypes = [_I64, _I64, _P, _P]
    L.oracle_pcc_pairs.argtypes = [_P, _I64, _I64, _I64, _I64, _P, _P, _P]
    L.oracle_pcc_rows.argtypes = [_P, _I64, _I64, _I64, _I64, _I64, _P]
    L.oracle_standardize.argtypes = [_P, _I64, _I64, _I64, _P, _I64, _P]
    L.oracle_edges.restype = _I64
    L.oracle_edges.argtypes = [_P, _I64, _I64, _I64, ctypes.c_double, _I64,
                               _I64, _I64, _P, _P, _P]
    L.oracle_perm_counts.argtypes = [_P, _I64, _I64, _I64, _I64, _P, _I64,
                                     _P, _P, ctypes.c_double, _P, _P, _P]
    L.oracle_cross_job_index.restype = _I64
    L.oracle_cross_job_index.argtypes = [_I64, _I64, _I64, _I64]
    L.oracle_cross_job_coords.restype = ctypes.c_int
    L.oracle_cross_job_coords.argtypes = [_I64, _I64, _I64, _P, _P]
    L.oracle_cross_rows.argtypes = [_P, _I64, _I64, _P, _I64, _I64, _I64,
                                    _I64, _I64, _P]
    L.oracle_cross_pairs.argtypes = [_P, _I64, _I64, _P, _I64, _I64, _I64,
                                     _I64, _P, _P, _P]
    L.oracle_num_threads.restype = ctypes.c_int
    return L


def _f64(X):
    X = np.ascontiguousarray(np.asarray(X, dtype=np.float64))
    if X.ndim == 1:
        X = X[None, :]
    return X


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def num_threads() -> int:
    return int(lib().oracle_num_threads())


def pcc_pair(u, v, L=None) -> float:
    """Eq. (1) for two vectors."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    v = np.ascontiguousarray(v, dtype=np.float64)
    assert u.shape == v.shape
    return float((L or lib()).oracle_pcc_pair(_ptr(u), _ptr(v), u.size))


def row_stats(X, L=None):
    X = _f64(X)
    n, l = X.shape
    mean = np.empty(n)
    ssq = np.empty(n)
    (L or lib()).oracle_row_stats(_ptr(X), n, l, l, _ptr(mean), _ptr(ssq))
    return mean, ssq


def num_pairs(n: int, L=None) -> int:
    return int((L or lib()).oracle_num_pairs(n))


def pair_index(n: int, i: int, j: int, L=None) -> int:
    return int((L or lib()).oracle_pair_index(n, i, j))


def pair_coords(n: int, J: int, L=None):
    i = ctypes.c_int64()
    j = ctypes.c_int64()
    rc = (L or lib()).oracle_pair_coords(n, J, ctypes.byref(i),
                                         ctypes.byref(j))
    if rc != 0:
        raise ValueError(f"pair id {J} out of range for n={n}")
    return int(i.value), int(j.value)


def job_index_diag(n: int, y: int, x: int, L=None) -> int:
    """Eq. (9)-(10) with the diagonal counted in."""
    return int((L or lib()).oracle_job_index_diag(n, y, x))


def job_coords_diag(n: int, J: int, L=None):
    y = ctypes.c_int64()
    x = ctypes.c_int64()
    rc = (L or lib()).oracle_job_coords_diag(n, J, ctypes.byref(y),
                                             ctypes.byref(x))
    if rc != 0:
        raise ValueError(f"job id {J} out of range for n={n}")
    return int(y.value), int(x.value)


def pcc_pairs(X, I, J, L=None) -> np.ndarray:
    """Eq. (1) for pairs (I[p], J[p])."""
    X = _f64(X)
    n, l = X.shape
    I = np.ascontiguousarray(I, dtype=np.int64)
    J = np.ascontiguousarray(J, dtype=np.int64)
    r = np.empty(I.size)
    (L or lib()).oracle_pcc_pairs(_ptr(X), n, l, l, I.size, _ptr(I), _ptr(J),
                                  _ptr(r))
    return r


def pcc_rows(X, i0: int, i1: int, L=None) -> np.ndarray:
    """Packed strict-upper r for rows [i0, i1)."""
    X = _f64(X)
    n, l = X.shape
    first = i0 * (2 * n - i0 - 1) // 2
    last = i1 * (2 * n - i1 - 1) // 2
    out = np.empty(last - first)
    (L or lib()).oracle_pcc_rows(_ptr(X), n, l, l, i0, i1, _ptr(out))
    return out


def pcc_upper(X, L=None) -> np.ndarray:
    """Whole packed strict upper triangle, pair (i,j) at pair_index(i,j)."""
    X = _f64(X)
    return pcc_rows(X, 0, X.shape[0], L)


def standardize(X, L=None):
    """Eq. (5): returns (Z float64 n x l, flags uint8 n)."""
    X = _f64(X)
    n, l = X.shape
    Z = np.empty((n, l))
    flag = np.empty(n, dtype=np.uint8)
    (L or lib()).oracle_standardize(_ptr(X), n, l, l, _ptr(Z), l, _ptr(flag))
    return Z, flag


def edges(X, tau: float, i0: int = 0, i1: int | None = None, L=None):
    """(I, J, r) of pairs with |r| >= tau among rows [i0, i1)."""
    X = _f64(X)
    n, l = X.shape
    i1 = n if i1 is None else i1
    Lb = L or lib()
    cnt = Lb.oracle_edges(_ptr(X), n, l, l, float(tau), i0, i1, 0, None,
                          None, None)
    ei = np.empty(max(cnt, 1), dtype=np.int64)
    ej = np.empty(max(cnt, 1), dtype=np.int64)
    er = np.empty(max(cnt, 1))
    cnt2 = Lb.oracle_edges(_ptr(X), n, l, l, float(tau), i0, i1, cnt,
                           _ptr(ei), _ptr(ej), _ptr(er))
    assert cnt2 == cnt
    return ei[:cnt], ej[:cnt], er[:cnt]


def perm_counts(X, perms, I, J, delta: float = 0.0, L=None):
    """(cnt, cnt_lo, cnt_hi) for pairs (I[p], J[p]); see pcc_oracle.c."""
    X = _f64(X)
    n, l = X.shape
    perms = np.ascontiguousarray(perms, dtype=np.int32)
    P = perms.shape[0]
    assert perms.shape[1] == l
    I = np.ascontiguousarray(I, dtype=np.int64)
    J = np.ascontiguousarray(J, dtype=np.int64)
    c = np.empty(I.size, dtype=np.uint32)
    clo = np.empty(I.size, dtype=np.uint32)
    chi = np.empty(I.size, dtype=np.uint32)
    (L or lib()).oracle_perm_counts(_ptr(X), n, l, l, P, _ptr(perms), I.size,
                                    _ptr(I), _ptr(J), float(delta), _ptr(c),
                                    _ptr(clo), _ptr(chi))
    return c, clo, chi


def cross_job_index(nrow: int, ncol: int, y: int, x: int, L=None) -> int:
    """Eq. (7): J = y * ncol + x on an nrow x ncol job matrix."""
    return int((L or lib()).oracle_cross_job_index(nrow, ncol, y, x))


def cross_job_coords(nrow: int, ncol: int, J: int, L=None):
    """Eq. (8): (y, x) of job J (by search)."""
    y = ctypes.c_int64()
    x = ctypes.c_int64()
    rc = (L or lib()).oracle_cross_job_coords(nrow, ncol, J, ctypes.byref(y),
                                              ctypes.byref(x))
    if rc != 0:
        raise ValueError(f"job id {J} out of range for {nrow} x {ncol}")
    return int(y.value), int(x.value)


def cross_rows(X, Y, i0: int = 0, i1: int | None = None, L=None):
    """Eq. (1) for (x_i, y_j), i in [i0, i1), all j: (i1 - i0) x ny."""
    X = _f64(X)
    Y = _f64(Y)
    nx, l = X.shape
    ny, ly = Y.shape
    assert ly == l
    i1 = nx if i1 is None else i1
    out = np.empty((i1 - i0, ny))
    (L or lib()).oracle_cross_rows(_ptr(X), nx, l, _ptr(Y), ny, l, l, i0, i1,
                                   _ptr(out))
    return out


def cross_pairs(X, Y, I, J, L=None) -> np.ndarray:
    """Eq. (1) for (x_{I[p]}, y_{J[p]})."""
    X = _f64(X)
    Y = _f64(Y)
    nx, l = X.shape
    ny, ly = Y.shape
    assert ly == l
    I = np.ascontiguousarray(I, dtype=np.int64)
    J = np.ascontiguousarray(J, dtype=np.int64)
    r = np.empty(I.size)
    (L or lib()).oracle_cross_pairs(_ptr(X), nx, l, _ptr(Y), ny, l, l, I.size,
                                    _ptr(I), _ptr(J), _ptr(r))
    return r
