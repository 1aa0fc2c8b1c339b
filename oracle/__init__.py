"""ctypes front end of the plain FP64 CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY.  Only tests/, the package smoke check and the
benchmark's CPU-baseline leg may import this module; the CUDA product path never
touches it.  It shares no code with the CUDA library: it has its own Morton
code, HEALPix table, octree validation and walk.

Parity status: every function is pinned by tests/test_oracle_*.py against
closed forms, invariants and brute force on tiny grids; the paper prints no
column or path values to compare against.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import build, lib_path

OK, ERR_ARG, ERR_UNSORTED, ERR_MISALIGNED, ERR_OVERLAP_OR_GAP = 0, 1, 2, 3, 4
ERR_SOURCE_OUTSIDE, ERR_STEP_LIMIT, ERR_NONFINITE, ERR_MISS = 5, 6, 7, 10

_lib = None


def use_library(path):
    """Swap in another build of oracle.c (tests load planted-mistake copies);
    returns the previously loaded library handle (None = default)."""
    global _lib
    prev = _lib
    _lib = None if path is None else _bind(C.CDLL(path))
    return prev


def restore_library(prev):
    global _lib
    _lib = prev


def _load():
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        build()
    _lib = _bind(C.CDLL(path))
    return _lib


def _bind(lib):
    P = C.c_void_p
    i64, i32 = C.c_int64, C.c_int
    lib.or_morton_encode.restype = C.c_uint64
    lib.or_morton_encode.argtypes = [C.c_uint32] * 3
    lib.or_morton_encode_many.argtypes = [P, i64, P]
    lib.or_morton_decode_many.argtypes = [P, i64, P]
    lib.or_healpix.argtypes = [i32, P]
    lib.or_validate.argtypes = [P, P, i64, P]
    lib.or_trace.argtypes = [P, P, i64, P, P, i32, P, i64, P, i32, P, P, P, i32]
    lib.or_adjoint.argtypes = [P, P, i64, P, i32, P, i64, P, i32, P, P, i32]
    lib.or_trace_path.restype = C.c_int64
    lib.or_trace_path.argtypes = [P, P, i64, P, P, P, P, P, i64]
    return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _ext(extent):
    if extent is None:
        return None
    return np.ascontiguousarray(np.asarray(extent, dtype=np.int32))


class OracleError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"oracle {what} failed with status {code}")
        self.code = code


def nthreads_default() -> int:
    return int(os.environ.get("RT_ORACLE_THREADS", os.cpu_count() or 1))


def morton_encode(xyz) -> np.ndarray:
    xyz = np.ascontiguousarray(np.asarray(xyz, dtype=np.uint32).reshape(-1, 3))
    out = np.empty(xyz.shape[0], dtype=np.uint64)
    _load().or_morton_encode_many(_ptr(xyz), xyz.shape[0], _ptr(out))
    return out


def morton_decode(keys) -> np.ndarray:
    keys = np.ascontiguousarray(np.asarray(keys, dtype=np.uint64).ravel())
    out = np.empty((keys.shape[0], 3), dtype=np.uint32)
    _load().or_morton_decode_many(_ptr(keys), keys.shape[0], _ptr(out))
    return out


def healpix(nside: int) -> np.ndarray:
    out = np.zeros((12 * nside * nside, 3), dtype=np.float64)
    st = _load().or_healpix(int(nside), _ptr(out))
    if st != OK:
        raise OracleError(st, "healpix")
    return out


def validate(keys, levels, extent=None) -> int:
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    levels = np.ascontiguousarray(levels, dtype=np.uint8)
    return int(_load().or_validate(_ptr(keys), _ptr(levels), keys.shape[0], _ptr(_ext(extent))))


def _tree(keys, levels, extent):
    return (np.ascontiguousarray(keys, dtype=np.uint64),
            np.ascontiguousarray(levels, dtype=np.uint8), _ext(extent))


def trace(keys, levels, dens, src, dirs, extent=None, want_cols=True, want_paths=True,
          nthreads=None):
    """Columns [n_src][nd][S] (FP64), path hashes and segment counts [n_src][nd]."""
    keys, levels, ext = _tree(keys, levels, extent)
    dens = np.ascontiguousarray(np.asarray(dens, dtype=np.float64).reshape(keys.shape[0], -1))
    src = np.ascontiguousarray(np.asarray(src, dtype=np.float64).reshape(-1, 3))
    dirs = np.ascontiguousarray(np.asarray(dirs, dtype=np.float64).reshape(-1, 3))
    S, ns, nd = dens.shape[1], src.shape[0], dirs.shape[0]
    cols = np.zeros((ns, nd, S), dtype=np.float64) if want_cols else None
    hsh = np.zeros((ns, nd), dtype=np.uint64) if want_paths else None
    nseg = np.zeros((ns, nd), dtype=np.uint64) if want_paths else None
    st = _load().or_trace(_ptr(keys), _ptr(levels), keys.shape[0], _ptr(ext), _ptr(dens), S,
                          _ptr(src), ns, _ptr(dirs), nd, _ptr(cols), _ptr(hsh), _ptr(nseg),
                          nthreads or nthreads_default())
    if st != OK:
        raise OracleError(st, "trace")
    return cols, hsh, nseg


def adjoint(keys, levels, S, src, dirs, g, extent=None, nthreads=None) -> np.ndarray:
    """grad[j,k] = sum over rays of g[s,q,k] * ds(s,q,j) (FP64)."""
    keys, levels, ext = _tree(keys, levels, extent)
    src = np.ascontiguousarray(np.asarray(src, dtype=np.float64).reshape(-1, 3))
    dirs = np.ascontiguousarray(np.asarray(dirs, dtype=np.float64).reshape(-1, 3))
    g = np.ascontiguousarray(np.asarray(g, dtype=np.float64).reshape(src.shape[0], dirs.shape[0], S))
    grad = np.zeros((keys.shape[0], S), dtype=np.float64)
    st = _load().or_adjoint(_ptr(keys), _ptr(levels), keys.shape[0], _ptr(ext), S, _ptr(src),
                            src.shape[0], _ptr(dirs), dirs.shape[0], _ptr(g), _ptr(grad),
                            nthreads or nthreads_default())
    if st != OK:
        raise OracleError(st, "adjoint")
    return grad


def trace_path(keys, levels, src, direction, extent=None, max_out=1 << 16):
    """(leaf indices, ds) of one ray in walk order."""
    keys, levels, ext = _tree(keys, levels, extent)
    src = np.ascontiguousarray(np.asarray(src, dtype=np.float64).reshape(3))
    d = np.ascontiguousarray(np.asarray(direction, dtype=np.float64).reshape(3))
    leaf = np.zeros(max_out, dtype=np.int64)
    ds = np.zeros(max_out, dtype=np.float64)
    n = _load().or_trace_path(_ptr(keys), _ptr(levels), keys.shape[0], _ptr(ext), _ptr(src),
                              _ptr(d), _ptr(leaf), _ptr(ds), max_out)
    if n < 0:
        raise OracleError(-n, "trace_path")
    if n > max_out:
        raise OracleError(ERR_ARG, f"trace_path (path of {n} segments exceeds {max_out})")
    return leaf[:n].copy(), ds[:n].copy()
