"""FP64 CPU oracle for the gamma index -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The product path (``paper_1012_1900_gb300``)
never imports it, and it never imports the product path.

The arithmetic lives in ``gamma_oracle.c`` (paper Section 2.1, Eq. 1 and
Algorithm A1, with Ju's simplex recursion); this module only builds the
shared library with gcc and marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gamma_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libgamma_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, no fast-math)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                               "-Wall", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64p = ctypes.POINTER(ctypes.c_int64)
            f64p = ctypes.POINTER(ctypes.c_double)
            f32p = ctypes.POINTER(ctypes.c_float)
            lib.oracle_gamma.restype = ctypes.c_int
            lib.oracle_gamma.argtypes = [f32p, f32p, ctypes.c_int, i64p, f64p, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                         ctypes.c_double, i64p, ctypes.c_int64, f64p, i64p,
                                         ctypes.c_int64, ctypes.c_int, f64p]
            lib.oracle_simplex_distance.restype = ctypes.c_double
            lib.oracle_simplex_distance.argtypes = [ctypes.c_int, ctypes.c_int, f64p, f64p]
            lib.oracle_cell_table.restype = ctypes.c_int64
            lib.oracle_cell_table.argtypes = [ctypes.c_int, i64p, f64p, ctypes.c_double,
                                              ctypes.c_double, ctypes.POINTER(ctypes.c_int32),
                                              f64p, ctypes.c_int64]
            lib.oracle_max_threads.restype = ctypes.c_int
            lib.oracle_gamma_grids.restype = ctypes.c_int
            lib.oracle_gamma_grids.argtypes = [f32p, i64p, f64p, f64p, f32p, i64p, f64p, f64p,
                                               ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                               ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                               i64p, ctypes.c_int64, f64p, ctypes.c_int]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _geometry(ref: np.ndarray, spacing: Sequence[float]):
    if ref.ndim == 2:
        shape = np.array([1, ref.shape[0], ref.shape[1]], dtype=np.int64)
        sp = np.array([1.0, spacing[0], spacing[1]], dtype=np.float64)
        return 2, shape, sp
    if ref.ndim == 3:
        return 3, np.array(ref.shape, dtype=np.int64), np.array(spacing, dtype=np.float64)
    raise ValueError("dose arrays must be 2D (y, x) or 3D (z, y, x)")


_ERRORS = {-1: "invalid argument", -2: "bad shape (every axis needs >= 2 voxels)",
           -3: "non-finite dose", -4: "out of memory"}


def gamma(ref: np.ndarray, ev: np.ndarray, spacing: Sequence[float], dd_frac: float,
          dta_mm: float, local: bool = False, cutoff_frac: float = 0.0,
          dose_norm: float = 0.0, idx: Optional[np.ndarray] = None,
          table_cap: int = 1 << 22, threads: int = 0, return_cells: bool = False):
    """Gamma of every voxel (or of the flat voxel indices ``idx``), FP64.

    ref, ev: float32 arrays (y, x) or (z, y, x); spacing in mm, same order.
    Returns float64 gamma (NaN where not evaluated), shaped like ref when idx
    is None, else like idx.  With return_cells, also the number of grid cubes
    each voxel's walk processed, and R_max = max over voxels of DD/dD."""
    lib = _load()
    ref = np.ascontiguousarray(ref, dtype=np.float32)
    ev = np.ascontiguousarray(ev, dtype=np.float32)
    if ref.shape != ev.shape:
        raise ValueError("reference and evaluation grids differ")
    ndim, shape, sp = _geometry(ref, spacing)
    if idx is None:
        n = ref.size
        idx_arr = None
        out_shape = ref.shape
    else:
        idx_arr = np.ascontiguousarray(idx, dtype=np.int64).ravel()
        n = idx_arr.size
        out_shape = np.shape(idx)
    out = np.empty(n, dtype=np.float64)
    cells = np.zeros(n, dtype=np.int64)
    rmax = ctypes.c_double(0.0)
    rc = lib.oracle_gamma(_ptr(ref, ctypes.c_float), _ptr(ev, ctypes.c_float), ndim,
                          _ptr(shape, ctypes.c_int64), _ptr(sp, ctypes.c_double),
                          float(dd_frac), float(dta_mm), int(bool(local)), float(cutoff_frac),
                          float(dose_norm),
                          _ptr(idx_arr, ctypes.c_int64) if idx_arr is not None else None,
                          int(n), _ptr(out, ctypes.c_double), _ptr(cells, ctypes.c_int64),
                          int(table_cap), int(threads), ctypes.byref(rmax))
    if rc != 0:
        raise ValueError(f"oracle_gamma failed: {_ERRORS.get(rc, rc)}")
    out = out.reshape(out_shape)
    if return_cells:
        return out, cells.reshape(out_shape), rmax.value
    return out


def _grid3(a: np.ndarray, spacing: Sequence[float], origin: Sequence[float]):
    if a.ndim == 2:
        return (np.array([1, a.shape[0], a.shape[1]], dtype=np.int64),
                np.array([1.0, spacing[0], spacing[1]], dtype=np.float64),
                np.array([0.0, origin[0], origin[1]], dtype=np.float64))
    return (np.array(a.shape, dtype=np.int64), np.array(spacing, dtype=np.float64),
            np.array(origin, dtype=np.float64))


def gamma_grids(ref: np.ndarray, ref_spacing: Sequence[float], ref_origin: Sequence[float],
                ev: np.ndarray, ev_spacing: Sequence[float], ev_origin: Sequence[float],
                dd_frac: float, dta_mm: float, local: bool = False, cutoff_frac: float = 0.0,
                dose_norm: float = 0.0, idx: Optional[np.ndarray] = None, threads: int = 0):
    """Gamma of every reference voxel (or of the flat indices ``idx``) when the
    reference and evaluation doses sit on different grids: each grid with its
    own shape, spacing and origin (mm, array order).  FP64; NaN where not
    evaluated; shaped like ref (or idx)."""
    lib = _load()
    ref = np.ascontiguousarray(ref, dtype=np.float32)
    ev = np.ascontiguousarray(ev, dtype=np.float32)
    if ref.ndim != ev.ndim or ref.ndim not in (2, 3):
        raise ValueError("both grids must be 2D or both 3D")
    rs, rsp, ro = _grid3(ref, ref_spacing, ref_origin)
    es, esp, eo = _grid3(ev, ev_spacing, ev_origin)
    if idx is None:
        n, idx_arr, out_shape = ref.size, None, ref.shape
    else:
        idx_arr = np.ascontiguousarray(idx, dtype=np.int64).ravel()
        n, out_shape = idx_arr.size, np.shape(idx)
    out = np.empty(n, dtype=np.float64)
    rc = lib.oracle_gamma_grids(_ptr(ref, ctypes.c_float), _ptr(rs, ctypes.c_int64),
                                _ptr(rsp, ctypes.c_double), _ptr(ro, ctypes.c_double),
                                _ptr(ev, ctypes.c_float), _ptr(es, ctypes.c_int64),
                                _ptr(esp, ctypes.c_double), _ptr(eo, ctypes.c_double),
                                ref.ndim, float(dd_frac), float(dta_mm), int(bool(local)),
                                float(cutoff_frac), float(dose_norm),
                                _ptr(idx_arr, ctypes.c_int64) if idx_arr is not None else None,
                                int(n), _ptr(out, ctypes.c_double), int(threads))
    if rc != 0:
        raise ValueError(f"oracle_gamma_grids failed: {_ERRORS.get(rc, rc)}")
    return out.reshape(out_shape)


def gamma_pair(pair, idx=None, **kw):
    """gamma() for a synth.Pair with its own criteria."""
    c = pair.criteria
    return gamma(pair.ref, pair.eval, pair.spacing, c.dd_frac, c.dta_mm, local=c.local,
                 cutoff_frac=c.cutoff_frac, dose_norm=c.dose_norm, idx=idx, **kw)


def simplex_distance(W: np.ndarray, P: np.ndarray) -> float:
    """Distance from P to the closed simplex whose vertices are the rows of W
    (Ju recursion on the normal equations)."""
    lib = _load()
    W = np.ascontiguousarray(W, dtype=np.float64)
    P = np.ascontiguousarray(P, dtype=np.float64)
    nv, K = W.shape
    if P.shape != (K,) or not (1 <= nv <= K + 1) or K > 4:
        raise ValueError("bad simplex shape")
    return lib.oracle_simplex_distance(K, nv, _ptr(W, ctypes.c_double), _ptr(P, ctypes.c_double))


def cell_table(ndim: int, shape: Sequence[int], spacing: Sequence[float], dta_mm: float,
               radius: float) -> Tuple[np.ndarray, np.ndarray]:
    """The oracle's sorted cube table: (offsets (n, 3) as x, y, z; keys)."""
    lib = _load()
    if ndim == 2:
        shp = np.array([1, shape[0], shape[1]], dtype=np.int64)
        sp = np.array([1.0, spacing[0], spacing[1]], dtype=np.float64)
    else:
        shp = np.array(shape, dtype=np.int64)
        sp = np.array(spacing, dtype=np.float64)
    n = lib.oracle_cell_table(ndim, _ptr(shp, ctypes.c_int64), _ptr(sp, ctypes.c_double),
                              float(dta_mm), float(radius), None, None, 0)
    if n < 0:
        raise MemoryError("oracle_cell_table")
    offs = np.zeros((max(n, 1), 3), dtype=np.int32)
    keys = np.zeros(max(n, 1), dtype=np.float64)
    lib.oracle_cell_table(ndim, _ptr(shp, ctypes.c_int64), _ptr(sp, ctypes.c_double),
                          float(dta_mm), float(radius), _ptr(offs, ctypes.c_int32),
                          _ptr(keys, ctypes.c_double), n)
    return offs[:n], keys[:n]


def max_threads() -> int:
    return int(_load().oracle_max_threads())
