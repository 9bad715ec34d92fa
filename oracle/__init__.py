"""FP64 CPU oracle for the SPIDER stencil path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product package
(``paper_2506_22035_gb300``) never imports it, and this package imports
nothing from the product: the two share no code, headers or constants.

Contents
--------
``stencil``          the direct FP64 stencil sweep (C, OpenMP), i.e. the
                     definition of the operation (Sec. 1 / Sec. 2.2):
                     ``u_{t+1}[i] = sum_o w[o] u_t[i+o]`` with zero Dirichlet
                     (or periodic) boundaries.
``stencil_points``   the same definition evaluated at a few sampled points of
                     a large grid through each point's dependency cone.
``lowered``          the paper's transform written out step by step
                     (Sec. 3.1): banded kernel matrices, padding, the strided
                     column swap, 2:4 / 1:2 compression with 2-bit metadata,
                     and the brute-force lowered products used as secondary
                     checkers on tiny grids.
``cost_model``       the per-point work/access model of Sec. 3.1.2 and
                     Table 2.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "stencil_ref.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (OpenMP, no FP contraction) and return the .so path."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
           _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_stencil_fp64.restype = ctypes.c_int
            lib.oracle_stencil_fp64.argtypes = [
                ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.c_int,
                ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                ctypes.POINTER(ctypes.c_double), ctypes.c_int64, ctypes.c_int, ctypes.c_int]
            lib.oracle_max_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def _radius_of(coeffs: np.ndarray) -> int:
    side = coeffs.shape[0]
    if side % 2 != 1 or any(s != side for s in coeffs.shape):
        raise ValueError("coefficients must be a (2r+1)^d cube")
    return (side - 1) // 2


def stencil(u0, coeffs, steps: int, periodic: bool = False, threads: int | None = None) -> np.ndarray:
    """Direct FP64 stencil sweep of ``steps`` time steps (Sec. 1, Sec. 2.2).

    ``u0``: 1-, 2- or 3-D array (x fastest); converted exactly to float64.
    ``coeffs``: (2r+1)^d array indexed [dz][dy][dx], offsets -r..r; converted
    exactly to float64 (float32 coefficients keep their value).
    Returns a new float64 array of the same shape.
    """
    u = np.ascontiguousarray(np.asarray(u0, dtype=np.float64))
    w = np.ascontiguousarray(np.asarray(coeffs, dtype=np.float64))
    if w.ndim != u.ndim:
        raise ValueError("coefficient cube and grid must have the same number of dimensions")
    r = _radius_of(w)
    ext = (ctypes.c_int64 * u.ndim)(*u.shape)
    out = np.empty_like(u)
    lib = _load()
    nt = threads if threads is not None else lib.oracle_max_threads()
    rc = lib.oracle_stencil_fp64(
        u.ndim, ext, r, w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
        u.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
        out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(steps), int(bool(periodic)), int(nt))
    if rc != 0:
        raise RuntimeError(f"oracle_stencil_fp64 failed with code {rc}")
    return out


def stencil_points(u0, coeffs, steps: int, points, threads: int | None = None) -> np.ndarray:
    """Exact zero-Dirichlet FP64 values of the stepped grid at the given points.

    The value at point p after ``steps`` steps depends only on the initial
    values within ``steps * r`` of p along every axis (the dependency cone).
    Each point is computed on the crop of that cone, clipped to the grid:
    clipping at the true boundary keeps the zero-outside rule exactly, and a
    crop edge inside the grid is ``steps * r`` away from p, so its spurious
    zeros cannot reach p within ``steps`` steps.
    """
    u = np.asarray(u0)
    w = np.asarray(coeffs, dtype=np.float64)
    r = _radius_of(w)
    reach = int(steps) * r
    vals = []
    for p in points:
        p = tuple(int(c) for c in p)
        lo = [max(0, c - reach) for c in p]
        hi = [min(n, c + reach + 1) for c, n in zip(p, u.shape)]
        crop = u[tuple(slice(a, b) for a, b in zip(lo, hi))]
        res = stencil(crop, w, steps, periodic=False, threads=threads)
        vals.append(res[tuple(c - a for c, a in zip(p, lo))])
    return np.asarray(vals, dtype=np.float64)
