"""The oracle's pins must catch plausible mistakes.  Each case plants one mistake in a copy
of the oracle source (a dropped term, a wrong index, a transposed operand, a wrong
comparison), compiles it on the CPU, and checks that at least one pin fails."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import graphgen
from census_facts import check_invariants, choose3

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "census_oracle.cpp")

MUTANTS = {
    "canonical rule drops the not-neighbour-of-u test": ("(u < w && w < v && !s.in_u)", "(u < w && w < v)"),
    "dyadic count off by one": ("(u128)(n - S.size() - 2)", "(u128)(n - S.size() - 1)"),
    "tricode operands u,v transposed": ("int code = (g.arc(v, u) ? 1 : 0) | (g.arc(u, v) ? 2 : 0) | (g.arc(v, w) ? 4 : 0)",
                                        "int code = (g.arc(u, v) ? 1 : 0) | (g.arc(v, u) ? 2 : 0) | (g.arc(v, w) ? 4 : 0)"),
    "111D and 111U swapped in the rule table": ("(outd[z] == 1) ? T111D : T111U", "(outd[z] == 0) ? T111D : T111U"),
    "null count misses the 012 term": ("for (int t = 1; t < 16; ++t) sum += census[t];", "for (int t = 2; t < 16; ++t) sum += census[t];"),
    "two-pointer walk misorders equal ids": ("(i < Nu.size() && Nu[i].id < Nv[j].id)", "(i < Nu.size() && Nu[i].id <= Nv[j].id)"),
    "canonical rule admits w below u": ("(u < w && w < v && !s.in_u)", "(w < v && !s.in_u)"),
}


def _compile(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, name
    path = tmp_path / "mut.cpp"
    path.write_text(src.replace(old, new))
    so = tmp_path / "libmut.so"
    subprocess.run(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", str(path), "-o", str(so)], check=True)
    lib = ctypes.CDLL(str(so))
    u32p, u64p = ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint64)
    lib.or_census_bm.argtypes = [ctypes.c_uint32, ctypes.c_uint64, u32p, u32p, u64p, u64p]
    lib.or_census_brute.argtypes = [ctypes.c_uint32, ctypes.c_uint64, u32p, u32p, u64p]
    lib.or_invariants.argtypes = [ctypes.c_uint32, ctypes.c_uint64, u32p, u32p, u64p]
    return lib


def _call(fn, n, s, d, k, *extra):
    s = np.ascontiguousarray(s, np.uint32)
    d = np.ascontiguousarray(d, np.uint32)
    out = np.zeros(2 * k, np.uint64)
    fn(n, len(s), s.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), d.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
       out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), *extra)
    return [int(out[2 * i]) | (int(out[2 * i + 1]) << 64) for i in range(k)]


def _pins_hold(lib):
    """Run a cheap subset of the oracle's pins against a (possibly mutated) build."""
    bm = lambda n, s, d: _call(lib.or_census_bm, n, s, d, 16, None)  # noqa: E731
    brute = lambda n, s, d: _call(lib.or_census_brute, n, s, d, 16)  # noqa: E731
    try:
        ordered = [(a, b) for a in range(4) for b in range(4) if a != b]
        rng = np.random.default_rng(0)
        for mask in rng.choice(1 << 12, 300, replace=False):
            pairs = np.array([ordered[i] for i in range(12) if mask >> i & 1] or [(0, 0)], np.uint32)
            if bm(4, pairs[:, 0], pairs[:, 1]) != brute(4, pairs[:, 0], pairs[:, 1]):
                return False
        n, s, d = graphgen.rmat(8, 16, 0.2, 2)
        c = bm(n, s, d)
        inv = dict(zip(("M", "A", "N", "out2", "in2", "paths", "triangles", "arcs"), _call(lib.or_invariants, n, s, d, 8)))
        check_invariants(n, c, inv)
        assert sum(c) == choose3(n)
    except AssertionError:
        return False
    return True


def test_unmutated_copy_passes(tmp_path):
    if shutil.which("g++") is None:
        pytest.skip("no g++")
    assert _pins_hold(_compile_same(tmp_path))


def _compile_same(tmp_path):
    src = open(SRC).read()
    path = tmp_path / "same.cpp"
    path.write_text(src)
    so = tmp_path / "libsame.so"
    subprocess.run(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", str(path), "-o", str(so)], check=True)
    lib = ctypes.CDLL(str(so))
    u32p, u64p = ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint64)
    lib.or_census_bm.argtypes = [ctypes.c_uint32, ctypes.c_uint64, u32p, u32p, u64p, u64p]
    lib.or_census_brute.argtypes = [ctypes.c_uint32, ctypes.c_uint64, u32p, u32p, u64p]
    lib.or_invariants.argtypes = [ctypes.c_uint32, ctypes.c_uint64, u32p, u32p, u64p]
    return lib


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(tmp_path, name):
    if shutil.which("g++") is None:
        pytest.skip("no g++")
    old, new = MUTANTS[name]
    assert not _pins_hold(_compile(tmp_path, name, old, new)), f"pins missed: {name}"
