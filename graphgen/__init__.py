"""Seeded synthetic digraph generators (R-MAT, Chung-Lu) shared by the oracle and the
GPU library's tests and benchmark.

The generators only produce inputs: distinct, loop-free directed arcs sorted by
(src, dst).  They contain none of the triad-census arithmetic.  The C source
(``graphgen.c``) documents the exact recipes and the counter-based random generator.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB = os.path.join(_HERE, "libgraphgen.so")
_lib = None

# R-MAT quadrant probabilities used by every R-MAT workload here (a, b, c; d = 1-a-b-c)
RMAT_ABC = (0.57, 0.19, 0.19)


def build(force: bool = False) -> str:
    """Compile libgraphgen.so in place with gcc (OpenMP when available)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O3", "-std=c11", "-shared", "-fPIC", _SRC, "-o", _LIB + ".tmp", "-lm"]
    try:
        subprocess.run(base[:3] + ["-fopenmp"] + base[3:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P32 = ctypes.POINTER(ctypes.POINTER(ctypes.c_uint32))
        lib.gg_rmat.restype = ctypes.c_int64
        lib.gg_rmat.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_double, ctypes.c_double,
                                ctypes.c_double, ctypes.c_double, ctypes.c_uint64, ctypes.c_int, P32, P32]
        lib.gg_chung_lu.restype = ctypes.c_int64
        lib.gg_chung_lu.argtypes = [ctypes.c_uint32, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_uint64, ctypes.c_uint64, P32, P32]
        lib.gg_loguniform_sizes.restype = None
        lib.gg_loguniform_sizes.argtypes = [ctypes.c_uint32, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint32)]
        lib.gg_chung_lu_batch.restype = ctypes.c_int64
        lib.gg_chung_lu_batch.argtypes = [ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint32), ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_uint64, P32, P32,
                                          ctypes.POINTER(ctypes.POINTER(ctypes.c_uint64))]
        lib.gg_free.argtypes = [ctypes.c_void_p]
        _lib = lib
    return _lib


def _take(lib, cnt, ps, pd):
    if cnt < 0:
        raise MemoryError("graphgen: generation failed (bad arguments or out of memory)")
    src = np.ctypeslib.as_array(ps, shape=(max(cnt, 1),))[:cnt].copy()
    dst = np.ctypeslib.as_array(pd, shape=(max(cnt, 1),))[:cnt].copy()
    lib.gg_free(ps)
    lib.gg_free(pd)
    return src, dst


def rmat(scale: int, edge_factor: int = 16, recip: float = 0.2, seed: int = 1,
         abc=RMAT_ABC, permute: bool = True):
    """Directed R-MAT graph: returns (n, src, dst) with uint32 arrays of distinct arcs."""
    lib = _load()
    ps, pd = ctypes.POINTER(ctypes.c_uint32)(), ctypes.POINTER(ctypes.c_uint32)()
    cnt = lib.gg_rmat(scale, edge_factor, abc[0], abc[1], abc[2], recip, seed, int(permute),
                      ctypes.byref(ps), ctypes.byref(pd))
    src, dst = _take(lib, cnt, ps, pd)
    return 1 << scale, src, dst


def chung_lu(n: int, mean_deg: float = 8.0, gamma: float = 2.1, recip: float = 0.1,
             seed: int = 4, graph_index: int = 0):
    """Directed Chung-Lu graph: returns (n, src, dst) with uint32 arrays of distinct arcs."""
    lib = _load()
    ps, pd = ctypes.POINTER(ctypes.c_uint32)(), ctypes.POINTER(ctypes.c_uint32)()
    cnt = lib.gg_chung_lu(n, mean_deg, gamma, recip, seed, graph_index, ctypes.byref(ps), ctypes.byref(pd))
    src, dst = _take(lib, cnt, ps, pd)
    return n, src, dst


def loguniform_sizes(k: int, lo: float, hi: float, seed: int) -> np.ndarray:
    """k vertex counts floor(exp(U(ln lo, ln hi)))."""
    lib = _load()
    out = np.zeros(k, dtype=np.uint32)
    lib.gg_loguniform_sizes(k, lo, hi, seed, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
    return out


def batch_chung_lu(k: int = 4096, lo: float = 32, hi: float = 65536, mean_deg: float = 8.0,
                   gamma: float = 2.1, recip: float = 0.1, seed: int = 4):
    """k Chung-Lu graphs with log-uniform sizes (graph i = chung_lu(n_i, ..., graph_index=i)),
    generated in parallel: list of (n, src, dst)."""
    sizes = loguniform_sizes(k, lo, hi, seed)
    lib = _load()
    ps, pd = ctypes.POINTER(ctypes.c_uint32)(), ctypes.POINTER(ctypes.c_uint32)()
    po = ctypes.POINTER(ctypes.c_uint64)()
    tot = lib.gg_chung_lu_batch(k, sizes.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), mean_deg, gamma, recip,
                                seed, ctypes.byref(ps), ctypes.byref(pd), ctypes.byref(po))
    src, dst = _take(lib, tot, ps, pd)
    off = np.ctypeslib.as_array(po, shape=(k + 1,)).copy()
    lib.gg_free(po)
    return [(int(sizes[i]), src[off[i]:off[i + 1]], dst[off[i]:off[i + 1]]) for i in range(k)]


def gnp(n: int, p: float, seed: int):
    """Directed G(n, p) (each ordered pair x != y independently) for small test graphs."""
    rng = np.random.default_rng(seed)
    a = rng.random((n, n)) < p
    np.fill_diagonal(a, False)
    s, d = np.nonzero(a)
    return n, s.astype(np.uint32), d.astype(np.uint32)
