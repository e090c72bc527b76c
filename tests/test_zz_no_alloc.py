"""The no-allocation census entry point (tc_census_csr_noalloc).

Some callers cannot call cudaMalloc where they run, for example code that must not block
inside a real-time loop or a host whose memory pool has already reserved the device memory.
For them the library offers one census call whose scratch lives in a fixed array inside the
library.  These tests call it through the C ABI and check it against the regular census entry
point (exact integers, tolerance zero) on two calls in a row, then on a second graph, so that
the scratch array's leftover contents from a previous call cannot leak into a result.
"""
import numpy as np
import pytest

import graphgen

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


def _noalloc_counts(tc, g, n, stream):
    import torch
    off, adj, _ = tc.tc_graph_device_csr(g.handle)
    out = torch.full((16,), 7, dtype=torch.int64, device="cuda")   # garbage the call must overwrite
    tc.tc_census_csr_noalloc(n, off, adj, out, stream=stream)
    torch.cuda.synchronize()
    c = [int(x) & ((1 << 64) - 1) for x in out.cpu().tolist()]
    c[0] = tc.tc_null_count(n, c)
    return c


def test_noalloc_matches_regular_census_twice_in_a_row(tc):
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    n, s, d = graphgen.rmat(16, 16, 0.2, 7)
    with tc.Graph.from_arcs(n, s, d) as g:
        want = g.census()
        first = _noalloc_counts(tc, g, n, stream)
        second = _noalloc_counts(tc, g, n, stream)
    assert first == want
    assert second == want


def test_noalloc_reused_on_another_graph(tc):
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    for (n, s, d) in (graphgen.chung_lu(20000, 8.0, 2.1, 0.1, 4, 3), graphgen.rmat(12, 16, 0.15, 1)):
        with tc.Graph.from_arcs(n, s, d) as g:
            want = g.census()
            assert _noalloc_counts(tc, g, n, stream) == want
            assert _noalloc_counts(tc, g, n, stream) == want


def test_noalloc_rejects_graphs_beyond_its_scratch(tc):
    import torch
    dummy = torch.zeros(4, dtype=torch.int64, device="cuda")
    out = torch.zeros(16, dtype=torch.int64, device="cuda")
    with pytest.raises(tc.TcError) as e:
        tc.tc_census_csr_noalloc((1 << 20) + 1, dummy.data_ptr(), dummy.data_ptr(), out)
    assert e.value.status == tc.TC_ERR_RANGE


def _device_csr(tc, n, s, d):
    """The library's relabelled CSR of a graph, copied to fresh device tensors (int64 offsets,
    int32 entries) that a test may corrupt."""
    import torch
    with tc.Graph.from_arcs(n, s, d) as g:
        off, adj, _ = tc.tc_graph_export_csr(g.handle)
    return (torch.from_numpy(off.astype(np.int64)).cuda(), torch.from_numpy(adj.view(np.int32).copy()).cuda())


@pytest.mark.parametrize("fault", ["id_beyond_n", "self_loop", "no_direction", "unsorted", "asymmetric",
                                   "offsets_decrease", "offsets_not_from_zero"])
def test_noalloc_rejects_malformed_csr(tc, fault):
    """Each rule of the CSR form broken once, on the host side of the copy: the call checks the
    CSR on the device, reading only inside the lists its offsets define, and returns TC_ERR_ARG
    before any census kernel runs; the output buffer is left as it was apart from the zeroing."""
    import torch
    n, s, d = graphgen.rmat(10, 16, 0.15, 1)
    off, adj = _device_csr(tc, n, s, d)
    o = off.cpu().numpy().copy()
    a = adj.cpu().numpy().view(np.uint32).copy()
    u = 5                                  # a vertex with a long list (ids descend with degree)
    b, e = int(o[u]), int(o[u + 1])
    assert e - b >= 4
    if fault == "id_beyond_n":
        a[e - 1] = (n << 2) | 1
    elif fault == "self_loop":
        a[b] = (u << 2) | (a[b] & 3)
    elif fault == "no_direction":
        a[b] &= ~np.uint32(3)
    elif fault == "unsorted":
        a[b], a[b + 1] = a[b + 1], a[b]
    elif fault == "asymmetric":
        a[b] = (a[b] & ~np.uint32(3)) | np.uint32(2 if (a[b] & 3) == 1 else 1)   # mirror left as it was
    elif fault == "offsets_decrease":
        o[u + 1], o[u + 2] = o[u + 2], o[u + 1]
    elif fault == "offsets_not_from_zero":
        o[0] = 1
    off = torch.from_numpy(o).cuda()
    adj = torch.from_numpy(a.view(np.int32)).cuda()
    out = torch.zeros(16, dtype=torch.int64, device="cuda")
    with pytest.raises(tc.TcError) as err:
        tc.tc_census_csr_noalloc(n, off.data_ptr(), adj.data_ptr(), out)
    torch.cuda.synchronize()
    assert err.value.status == tc.TC_ERR_ARG
    assert int(out.abs().sum()) == 0
    # the scratch array holds no state that would spoil the next valid call
    off, adj = _device_csr(tc, n, s, d)
    tc.tc_census_csr_noalloc(n, off.data_ptr(), adj.data_ptr(), out)
    torch.cuda.synchronize()
    c = [int(x) & ((1 << 64) - 1) for x in out.cpu().tolist()]
    c[0] = tc.tc_null_count(n, c)
    with tc.Graph.from_arcs(n, s, d) as g:
        assert c == g.census()
