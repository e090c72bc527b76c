"""CPU oracle for the directed triad census - TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may
import this package.  The GPU library never imports, links or runs it, and the two share
no code.  ``census_oracle.cpp`` documents the method (Batagelj-Mrvar census of Fig. 5,
O(n^3) brute force, and two independent derivations of the tricode table) and every
reading of the paper it relies on.

Counts are returned as Python ints (the 003 count can exceed 2^64).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "census_oracle.cpp")
_LIB = os.path.join(_HERE, "libcensus_oracle.so")
_lib = None

CLASS_NAMES = ("003", "012", "102", "021D", "021U", "021C", "111D", "111U",
               "030T", "030C", "201", "120D", "120U", "120C", "210", "300")


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (-O3, OpenMP when available) into libcensus_oracle.so."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["g++", "-O3", "-std=c++17", "-shared", "-fPIC", _SRC, "-o", _LIB + ".tmp"]
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
        u8p = ctypes.POINTER(ctypes.c_uint8)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        lib.or_table_rules.argtypes = [u8p]
        lib.or_table_canonical.argtypes = [u8p]
        lib.or_census_bm.argtypes = [ctypes.c_uint32, ctypes.c_uint64, u32p, u32p, u64p, u64p]
        lib.or_census_bm_parallel.argtypes = [ctypes.c_uint32, ctypes.c_uint64, u32p, u32p, u64p, ctypes.c_int]
        lib.or_census_brute.argtypes = [ctypes.c_uint32, ctypes.c_uint64, u32p, u32p, u64p]
        lib.or_invariants.argtypes = [ctypes.c_uint32, ctypes.c_uint64, u32p, u32p, u64p]
        lib.or_invariants_opt.argtypes = [ctypes.c_uint32, ctypes.c_uint64, u32p, u32p, u64p, ctypes.c_int]
        lib.or_census64_brute.argtypes = [ctypes.c_uint32, ctypes.c_uint64, u32p, u32p, u64p]
        lib.or_census64.argtypes = [ctypes.c_uint32, ctypes.c_uint64, u32p, u32p, u64p]
        lib.or_graph_new.restype = ctypes.c_void_p
        lib.or_graph_new.argtypes = [ctypes.c_uint32, ctypes.c_uint64, u32p, u32p]
        lib.or_graph_free.argtypes = [ctypes.c_void_p]
        lib.or_census_bm_sample.restype = ctypes.c_double
        lib.or_census_bm_sample.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32, u64p, u64p, u64p]
        lib.or_census_bm_sample_parallel.restype = ctypes.c_double
        lib.or_census_bm_sample_parallel.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int,
                                                     u64p, u64p, u64p, ctypes.POINTER(ctypes.c_int)]
        _lib = lib
    return _lib


def _arcs(src, dst):
    s = np.ascontiguousarray(src, dtype=np.uint32)
    d = np.ascontiguousarray(dst, dtype=np.uint32)
    if s.shape != d.shape:
        raise ValueError("src and dst differ in length")
    return s, d, s.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), d.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def _u128(buf, k):
    return [int(buf[2 * i]) | (int(buf[2 * i + 1]) << 64) for i in range(k)]


def _p64(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def table_rules() -> np.ndarray:
    t = np.zeros(64, dtype=np.uint8)
    if _load().or_table_rules(t.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))) != 0:
        raise RuntimeError("rule table left a code unclassified")
    return t


def table_canonical() -> np.ndarray:
    t = np.zeros(64, dtype=np.uint8)
    if _load().or_table_canonical(t.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))) != 0:
        raise RuntimeError("canonical table is not a function onto 16 classes")
    return t


def census_bm(n: int, src, dst, with_stats: bool = False):
    """Fig. 5 census: list of 16 ints (and optionally (arcs, loops, dups))."""
    s, d, ps, pd = _arcs(src, dst)
    out = np.zeros(32, dtype=np.uint64)
    st = np.zeros(3, dtype=np.uint64)
    rc = _load().or_census_bm(n, len(s), ps, pd, _p64(out), _p64(st))
    if rc != 0:
        raise ValueError("vertex id out of range")
    res = _u128(out, 16)
    return (res, tuple(int(x) for x in st)) if with_stats else res


def census_bm_parallel(n: int, src, dst, threads: int = 0):
    """The paper's OpenMP form of Fig. 5 (flattened loops, dynamic schedule, private vectors)."""
    s, d, ps, pd = _arcs(src, dst)
    out = np.zeros(32, dtype=np.uint64)
    if _load().or_census_bm_parallel(n, len(s), ps, pd, _p64(out), threads) != 0:
        raise ValueError("vertex id out of range")
    return _u128(out, 16)


def census_brute(n: int, src, dst):
    """O(n^3) census by canonical form (n <= 4096)."""
    s, d, ps, pd = _arcs(src, dst)
    out = np.zeros(32, dtype=np.uint64)
    rc = _load().or_census_brute(n, len(s), ps, pd, _p64(out))
    if rc != 0:
        raise ValueError(f"brute-force census refused (code {rc})")
    return _u128(out, 16)


def census64_brute(n: int, src, dst):
    """64-state census by definition (n <= 4096): the state of every a<b<c over the roles
    (u, v, w) = (a, b, c), tricode bits 1 v->u, 2 u->v, 4 v->w, 8 w->v, 16 u->w, 32 w->u."""
    s, d, ps, pd = _arcs(src, dst)
    out = np.zeros(128, dtype=np.uint64)
    rc = _load().or_census64_brute(n, len(s), ps, pd, _p64(out))
    if rc != 0:
        raise ValueError(f"brute-force 64-state census refused (code {rc})")
    return _u128(out, 64)


def census64(n: int, src, dst):
    """64-state census per linked pair (first-linked-pair rule, range counts, null by
    subtraction): the same states as census64_brute, for any n."""
    s, d, ps, pd = _arcs(src, dst)
    out = np.zeros(128, dtype=np.uint64)
    if _load().or_census64(n, len(s), ps, pd, _p64(out)) != 0:
        raise ValueError("vertex id out of range")
    return _u128(out, 64)


def fold64(c64) -> list:
    """The 16-class census of a 64-state census (Sec. 3: isomorphic states merged)."""
    t = table_rules()
    out = [0] * 16
    for code, k in enumerate(c64):
        out[int(t[code])] += int(k)
    return out


def invariants(n: int, src, dst, triangles: bool = True) -> dict:
    """O(m) statistics of the digraph; triangles=False skips the triangle count (reported 0)."""
    s, d, ps, pd = _arcs(src, dst)
    out = np.zeros(16, dtype=np.uint64)
    if _load().or_invariants_opt(n, len(s), ps, pd, _p64(out), int(triangles)) != 0:
        raise ValueError("vertex id out of range")
    v = _u128(out, 8)
    return dict(zip(("M", "A", "N", "out2", "in2", "paths", "triangles", "arcs"), v))


class SampledGraph:
    """The oracle's graph built once, for repeated timing samples of the Fig. 5 loop."""

    def __init__(self, n: int, src, dst):
        s, d, ps, pd = _arcs(src, dst)
        self._h = _load().or_graph_new(n, len(s), ps, pd)
        if not self._h:
            raise ValueError("vertex id out of range")

    def sample(self, stride: int, offset: int = 0):
        """Time the loop over vertices u = offset (mod stride): (seconds, partial counts,
        merge work of the sample, total merge work)."""
        out = np.zeros(32, dtype=np.uint64)
        ws = np.zeros(1, dtype=np.uint64)
        wt = np.zeros(1, dtype=np.uint64)
        sec = _load().or_census_bm_sample(self._h, stride, offset, _p64(out), _p64(ws), _p64(wt))
        return sec, _u128(out, 16), int(ws[0]), int(wt[0])

    def sample_parallel(self, stride: int, offset: int = 0, threads: int = 0):
        """The same sample with the sampled vertices shared by OpenMP threads (the paper's CPU
        form): (wall seconds, partial counts, merge work of the sample, total merge work,
        threads used)."""
        out = np.zeros(32, dtype=np.uint64)
        ws = np.zeros(1, dtype=np.uint64)
        wt = np.zeros(1, dtype=np.uint64)
        used = ctypes.c_int(0)
        sec = _load().or_census_bm_sample_parallel(self._h, stride, offset, threads, _p64(out), _p64(ws), _p64(wt),
                                                   ctypes.byref(used))
        return sec, _u128(out, 16), int(ws[0]), int(wt[0]), int(used.value)

    def close(self):
        if self._h:
            _load().or_graph_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def census_bm_sample(n: int, src, dst, stride: int, offset: int = 0):
    """One timing sample (builds and frees the graph): see SampledGraph.sample."""
    g = SampledGraph(n, src, dst)
    try:
        return g.sample(stride, offset)
    finally:
        g.close()


def choose3(n: int) -> int:
    return n * (n - 1) * (n - 2) // 6 if n >= 3 else 0
