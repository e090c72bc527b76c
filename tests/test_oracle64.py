"""Pins of the oracle's 64-state census (Sec. 3, Fig. 2: the labelled triad states before the
fold to 16 classes).  Reading: a triad's three actors take the roles (u, v, w) in increasing
vertex id; the state has the tricode's bits 1 v->u, 2 u->v, 4 v->w, 8 w->v, 16 u->w, 32 w->u.
The oracle computes it two ways (by definition, and per linked pair); the pins below fix it
independently: each labelled 3-vertex digraph is one state, closed forms whose state depends
on the role order, the fold to the 16-class census of Fig. 5, and the relabelings that permute
the states.  The last test plants mistakes in a copy of the oracle and checks that the pins
catch each one."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import graphgen
import oracle
from census_facts import choose3

# the arc each state bit stands for, over the roles u = 0, v = 1, w = 2
BIT_ARC = {1: (1, 0), 2: (0, 1), 4: (1, 2), 8: (2, 1), 16: (0, 2), 32: (2, 0)}


def arcs_of_state(state, ids):
    pairs = [(ids[a], ids[b]) for bit, (a, b) in BIT_ARC.items() if state & bit]
    s = np.array([p[0] for p in pairs], np.uint32)
    d = np.array([p[1] for p in pairs], np.uint32)
    return s, d


def swap_directions(state):
    """The state after every arc is reversed: bits 1<->2, 4<->8, 16<->32."""
    out = 0
    for lo, hi in ((1, 2), (4, 8), (16, 32)):
        out |= (hi if state & lo else 0) | (lo if state & hi else 0)
    return out


def reverse_order(state):
    """The state after ids are relabelled i -> n-1-i: the roles u and w trade places, so
    y->x (1) becomes v'->w' (4), x->y (2) w'->v' (8), y->z (4) v'->u' (1), z->y (8) u'->v' (2),
    x->z (16) w'->u' (32), z->x (32) u'->w' (16)."""
    perm = {1: 4, 2: 8, 4: 1, 8: 2, 16: 32, 32: 16}
    return sum(perm[b] for b in perm if state & b)


@pytest.mark.parametrize("route", ["brute", "pairs"])
def test_every_labelled_3_vertex_digraph_is_one_state(route):
    f = oracle.census64_brute if route == "brute" else oracle.census64
    for state in range(64):
        for ids, n in (((0, 1, 2), 3), ((2, 5, 9), 12)):
            s, d = arcs_of_state(state, ids)
            c = f(n, s, d)
            assert c[state] >= 1, (state, ids)
            # the three actors form exactly one triad; every other triad has at most one link
            # to them, so it is the null state or a one-link state
            if n == 3:
                assert c == [1 if k == state else 0 for k in range(64)], state
            assert sum(c) == choose3(n)


def test_exhaustive_4_vertices_routes_agree_and_fold_to_fig5():
    ordered = [(a, b) for a in range(4) for b in range(4) if a != b]
    for mask in range(1 << 12):
        pairs = [ordered[i] for i in range(12) if mask >> i & 1]
        s = np.array([p[0] for p in pairs], np.uint32)
        d = np.array([p[1] for p in pairs], np.uint32)
        c = oracle.census64_brute(4, s, d)
        assert oracle.census64(4, s, d) == c, mask
        assert oracle.fold64(c) == oracle.census_bm(4, s, d), mask


@pytest.mark.parametrize("spec", [("gnp", 60, 0.1, 1), ("gnp", 80, 0.35, 2), ("chung_lu", 300, 6.0, 3), ("rmat", 10, 15, 1)])
def test_random_graphs_match_brute(spec):
    if spec[0] == "gnp":
        n, s, d = graphgen.gnp(spec[1], spec[2], spec[3])
    elif spec[0] == "chung_lu":
        n, s, d = graphgen.chung_lu(spec[1], spec[2], 2.1, 0.1, 4, spec[3])
    else:
        n, s, d = graphgen.rmat(spec[1], 16, spec[2] / 100.0, spec[3])
    c = oracle.census64(n, s, d)
    assert c == oracle.census64_brute(n, s, d)
    assert oracle.fold64(c) == oracle.census_bm(n, s, d)
    assert sum(c) == choose3(n)


@pytest.mark.parametrize("n", [3, 7, 30])
def test_closed_forms_that_fix_the_role_order(n):
    ids = np.arange(n, dtype=np.uint32)
    lo, hi = np.triu_indices(n, 1)
    lo, hi = lo.astype(np.uint32), hi.astype(np.uint32)
    total = choose3(n)
    # transitive tournament from low to high ids: x->y, y->z, x->z = 2 + 4 + 16
    c = oracle.census64(n, lo, hi)
    assert c[22] == total and sum(c) == total
    # the reverse tournament: y->x, z->y, z->x = 1 + 8 + 32
    c = oracle.census64(n, hi, lo)
    assert c[41] == total
    # complete mutual graph and empty graph
    assert oracle.census64(n, np.concatenate([lo, hi]), np.concatenate([hi, lo]))[63] == total
    assert oracle.census64(n, np.zeros(0, np.uint32), np.zeros(0, np.uint32))[0] == total
    # out-star from the smallest id: u->v, u->w = 18; from the largest: w->u, w->v = 40
    others = ids[1:]
    c = oracle.census64(n, np.zeros(n - 1, np.uint32), others)
    assert c[18] == (n - 1) * (n - 2) // 2 and c[0] == choose3(n - 1)
    c = oracle.census64(n, np.full(n - 1, n - 1, np.uint32), ids[:-1])
    assert c[40] == (n - 1) * (n - 2) // 2 and c[0] == choose3(n - 1)
    # in-star into a middle vertex m: below and above (u->v, w->v = 10), m smallest
    # (v->u, w->u = 33), m largest (u->w, v->w = 20)
    m = n // 2
    leaves = np.array([i for i in range(n) if i != m], np.uint32)
    c = oracle.census64(n, leaves, np.full(len(leaves), m, np.uint32))
    assert c[10] == m * (n - 1 - m)
    assert c[33] == (n - 1 - m) * (n - 2 - m) // 2
    assert c[20] == m * (m - 1) // 2


def test_reversal_and_reordering_permute_the_states():
    n, s, d = graphgen.chung_lu(1500, 8.0, 2.1, 0.2, 4, 7)
    c = oracle.census64(n, s, d)
    rev = oracle.census64(n, d, s)
    assert all(rev[swap_directions(k)] == c[k] for k in range(64))
    flip = oracle.census64(n, (n - 1 - s.astype(np.int64)).astype(np.uint32), (n - 1 - d.astype(np.int64)).astype(np.uint32))
    assert all(flip[reverse_order(k)] == c[k] for k in range(64))
    # both maps are involutions
    assert all(swap_directions(swap_directions(k)) == k and reverse_order(reverse_order(k)) == k for k in range(64))


def test_the_16_class_census_is_the_fold():
    for spec in (graphgen.rmat(9, 16, 0.2, 5), graphgen.chung_lu(2000, 10.0, 2.1, 0.1, 4, 9)):
        n, s, d = spec
        assert oracle.fold64(oracle.census64(n, s, d)) == oracle.census_bm(n, s, d)


# ---------------------------------------------------------------- planted mistakes
SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "census_oracle.cpp")

MUTANTS = {
    "state bits u,v transposed (both routes)": ("return (ba ? 1 : 0) | (ab ? 2 : 0)", "return (ab ? 1 : 0) | (ba ? 2 : 0)"),
    "between-range size off by one": ("n_between = b - a - 1", "n_between = b - a"),
    "below-range dyad in the wrong roles": ("census[state_of(false, false, ab, ba, false, false)] += n_below - below;",
                                            "census[state_of(false, false, ba, ab, false, false)] += n_below - below;"),
    "above-range dyad in the wrong roles": ("census[state_of(ab, ba, false, false, false, false)] += n_above - above;",
                                            "census[state_of(ba, ab, false, false, false, false)] += n_above - above;"),
    "merged vertices above b not counted": ("if (c < a) ++below; else if (c < b) ++between; else ++above;",
                                            "if (c < a) ++below; else ++between;"),
    "connected triads counted at every linked pair": ("if (!(p0 == a && q0 == b)) continue;", "if (false) continue;"),
    "null state misses state 1": ("for (int t = 1; t < 64; ++t) rest += census[t];", "for (int t = 2; t < 64; ++t) rest += census[t];"),
    "a-c arc read backwards": ("if (p == a && q == c) return la.out;", "if (p == a && q == c) return la.in;"),
}


def _build(tmp_path, text, tag):
    path = tmp_path / f"{tag}.cpp"
    path.write_text(text)
    so = tmp_path / f"lib{tag}.so"
    subprocess.run(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", str(path), "-o", str(so)], check=True)
    lib = ctypes.CDLL(str(so))
    u32p, u64p = ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint64)
    for f in (lib.or_census64, lib.or_census64_brute):
        f.argtypes = [ctypes.c_uint32, ctypes.c_uint64, u32p, u32p, u64p]
    lib.or_census_bm.argtypes = [ctypes.c_uint32, ctypes.c_uint64, u32p, u32p, u64p, u64p]
    return lib


def _call(fn, n, s, d, k, *extra):
    s = np.ascontiguousarray(s, np.uint32)
    d = np.ascontiguousarray(d, np.uint32)
    out = np.zeros(2 * k, np.uint64)
    fn(n, len(s), s.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), d.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
       out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), *extra)
    return [int(out[2 * i]) | (int(out[2 * i + 1]) << 64) for i in range(k)]


def _pins64_hold(lib):
    """A cheap subset of the pins above, against a (possibly mutated) build."""
    fast = lambda n, s, d: _call(lib.or_census64, n, s, d, 64)  # noqa: E731
    brute = lambda n, s, d: _call(lib.or_census64_brute, n, s, d, 64)  # noqa: E731
    table = oracle.table_rules()
    try:
        for state in range(64):
            s, d = arcs_of_state(state, (2, 5, 9))
            for f in (fast, brute):
                c = f(12, s, d)
                assert c[state] >= 1 and sum(c) == choose3(12)
        rng = np.random.default_rng(3)
        ordered = [(a, b) for a in range(5) for b in range(5) if a != b]
        for mask in rng.choice(1 << 20, 200, replace=False):
            pairs = np.array([ordered[i] for i in range(20) if mask >> i & 1] or [(0, 0)], np.uint32)
            assert fast(5, pairs[:, 0], pairs[:, 1]) == brute(5, pairs[:, 0], pairs[:, 1])
        n, s, d = graphgen.rmat(8, 16, 0.2, 2)
        c = fast(n, s, d)
        assert c == brute(n, s, d)
        fold = [0] * 16
        for k, v in enumerate(c):
            fold[int(table[k])] += v
        assert fold == _call(lib.or_census_bm, n, s, d, 16, None)
        lo, hi = np.triu_indices(7, 1)
        assert fast(7, lo, hi)[22] == choose3(7)
    except AssertionError:
        return False
    return True


def test_unmutated_64_state_copy_passes(tmp_path):
    if shutil.which("g++") is None:
        pytest.skip("no g++")
    assert _pins64_hold(_build(tmp_path, open(SRC).read(), "same"))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_64_state_mistake_is_caught(tmp_path, name):
    if shutil.which("g++") is None:
        pytest.skip("no g++")
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, name
    assert not _pins64_hold(_build(tmp_path, src.replace(old, new), "mut")), f"pins missed: {name}"
