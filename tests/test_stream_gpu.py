"""Interval census over a timestamped arc stream: each window's census equals the oracle's
census of exactly the arcs in that window (loops and repeats dropped); pushes interleaved with
censuses, buffer growth and eviction keep it so.  Counts are exact: tolerance zero."""
import numpy as np
import pytest

import graphgen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1209_6308_gb300 import _build
    _build.build()
    import paper_1209_6308_gb300 as m
    m.load()
    return m


def _timeline(seed=3):
    """R-MAT scale-11 arcs plus repeats and self-loops, at sorted random times in [0, 1000)."""
    n, s, d = graphgen.rmat(11, 16, 0.2, seed)
    rng = np.random.default_rng(seed)
    rep = rng.integers(0, len(s), len(s) // 10)
    loops = rng.integers(0, n, 50).astype(np.uint32)
    src = np.concatenate([s, s[rep], loops]).astype(np.uint32)
    dst = np.concatenate([d, d[rep], loops]).astype(np.uint32)
    perm = rng.permutation(len(src))
    src, dst = src[perm], dst[perm]
    t = np.sort(rng.integers(0, 1000, len(src))).astype(np.uint64)
    return n, src, dst, t


def _want(n, src, dst, t, t_now, window):
    lo = t_now - window
    sel = (t <= t_now) & ((t > lo) if t_now >= window else np.ones(len(t), bool))
    return oracle.census_bm(n, src[sel], dst[sel]), int(sel.sum())


@pytest.mark.parametrize("window", [1, 150, 400, 5000])
def test_windows_equal_the_oracle(tc, window):
    n, src, dst, t = _timeline()
    with tc.Stream(n, window, options={"algo": 1}) as st:
        st.push(src, dst, t)
        for t_now in (0, 99, 100, 350, 351, 720, 999, 1500):
            got, m = st.census(t_now)
            want, wm = _want(n, src, dst, t, t_now, window)
            assert m == wm
            assert got == want, (window, t_now)


def test_pushes_interleaved_with_censuses_grow_and_evict(tc):
    n, src, dst, t = _timeline(5)
    window = 200
    with tc.Stream(n, window) as st:
        pos = 0
        caps = set()
        for t_now in range(50, 1100, 50):
            end = int(np.searchsorted(t, t_now, side="right"))
            # push in a few uneven pieces
            for cut in np.linspace(pos, end, 4).astype(int)[1:]:
                if cut > pos:
                    st.push(src[pos:cut], dst[pos:cut], t[pos:cut])
                    pos = cut
            got, m = st.census(t_now)
            want, wm = _want(n, src, dst, t, t_now, window)
            assert (got, m) == (want, wm), t_now
            info = st.stats()
            caps.add(info["capacity"])
            # arcs older than this window were freed
            assert info["live_arcs"] == int(np.sum(t[:pos].astype(np.int64) > t_now - window))
        assert len(caps) > 1                                  # the buffer grew


def test_empty_window_and_time_order_errors(tc):
    n = 100
    with tc.Stream(n, 10) as st:
        got, m = st.census(5)
        assert m == 0 and got[0] == n * (n - 1) * (n - 2) // 6 and sum(got[1:]) == 0
        st.push([1, 2], [2, 3], [7, 9])
        got, m = st.census(12)
        assert m == 2 and got[1] == 2 * (n - 3) and got[4] == 0 and got[5] == 1   # 012 and one 021C
        with pytest.raises(tc.TcError) as e:
            st.census(11)                                     # census times must not decrease
        assert e.value.status == tc.TC_ERR_ARG
        with pytest.raises(tc.TcError) as e:
            st.push([1], [2], [8])                            # arc times must not decrease
        assert e.value.status == tc.TC_ERR_ARG


def _distinct(src, dst, sel):
    """Distinct non-loop arcs among the selected ones."""
    s, d = src[sel].astype(np.int64), dst[sel].astype(np.int64)
    keep = s != d
    return len(np.unique(s[keep] * (1 << 32) + d[keep]))


def test_arc_set_is_updated_incrementally(tc):
    """Small steps: after the first census every window is reached by merging the arcs that
    entered and left into the kept set (no rebuild, no repair), the set holds exactly the
    window's distinct arcs, and every census equals the oracle's."""
    n, src, dst, t = _timeline(7)
    window = 300
    with tc.Stream(n, window, options={"algo": 2}) as st:
        st.push(src, dst, t)
        prev_a, prev_b = 0, 0
        for k, t_now in enumerate(range(100, 1000, 37)):
            got, m = st.census(t_now)
            want, wm = _want(n, src, dst, t, t_now, window)
            assert (got, m) == (want, wm), t_now
            sel = (t <= t_now) & ((t > t_now - window) if t_now >= window else True)
            a = int(np.searchsorted(t, t_now - window, side="right")) if t_now >= window else 0
            b = int(np.searchsorted(t, t_now, side="right"))
            info = st.stats()
            assert info["distinct_arcs"] == _distinct(src, dst, sel)
            assert info["repairs"] == 0
            if k == 0:
                assert info["rebuilds"] == 1 and info["last_added"] == b
            else:
                assert info["rebuilds"] == 1, t_now                  # merged, not rebuilt
                assert info["last_added"] == b - prev_b and info["last_evicted"] == a - prev_a
            prev_a, prev_b = a, b


def test_a_jump_past_the_window_rebuilds_the_set(tc):
    n, src, dst, t = _timeline(8)
    window = 100
    with tc.Stream(n, window) as st:
        st.push(src, dst, t)
        for t_now, rebuilt in ((150, 1), (180, 1), (600, 2), (610, 2), (999, 3)):
            got, m = st.census(t_now)
            assert (got, m) == _want(n, src, dst, t, t_now, window)
            info = st.stats()
            assert (info["rebuilds"], info["repairs"]) == (rebuilt, 0), t_now


def test_a_repeated_arc_stays_until_its_last_copy_leaves(tc):
    n = 10
    c3 = n * (n - 1) * (n - 2) // 6
    one_arc = [c3 - (n - 2), n - 2] + [0] * 14          # one arc: n - 2 triads 012, the rest 003
    empty = [c3] + [0] * 15
    with tc.Stream(n, 5) as st:
        st.push([1, 1, 4], [2, 2, 4], [1, 5, 6])         # 1 -> 2 twice, and a self-loop
        assert st.census(5) == (one_arc, 2)
        assert st.stats()["distinct_arcs"] == 1
        assert st.census(7) == (one_arc, 2)              # the copy at time 1 left, the one at 5 stays
        assert st.stats()["distinct_arcs"] == 1
        assert st.census(9) == (one_arc, 2)
        assert st.census(10) == (empty, 1)               # (5, 10]: only the self-loop is left
        info = st.stats()
        assert info["distinct_arcs"] == 0 and info["repairs"] == 0
        st.push([2], [1], [12])                          # the reverse arc: 102 if both were in
        assert st.census(12) == (one_arc, 1)
        assert st.census(16) == (one_arc, 1)
        assert st.stats()["repairs"] == 0
