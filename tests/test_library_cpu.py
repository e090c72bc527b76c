"""Host-side checks of the C-ABI library that need no GPU: it builds, loads, exports every
function include/tc.h declares, and its host-only helpers are right."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tc.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tc_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1209_6308_gb300 import _build
    _build.build()
    import paper_1209_6308_gb300 as tc
    return tc.load()


def test_header_declares_the_census_entry_points():
    names = _declared_functions()
    for must in ("tc_graph_create_arcs", "tc_graph_create_csr", "tc_census", "tc_census_batch",
                 "tc_graph_stats", "tc_graph_destroy", "tc_status_str"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", os.path.join(ROOT, "paper_1209_6308_gb300", "libtc.so")],
                         capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (tc_[a-z0-9_]+)", out))
    assert set(_declared_functions()) <= exported


def test_binding_covers_every_declared_symbol():
    import paper_1209_6308_gb300 as tc
    assert set(_declared_functions()) <= set(tc.SIGNATURES)


def test_library_table_matches_oracle_tables(lib):
    import oracle
    import paper_1209_6308_gb300 as tc
    t = tc.tc_tricode_table()
    assert (t == oracle.table_rules()).all()
    assert (t == oracle.table_canonical()).all()


@pytest.mark.parametrize("n", [0, 1, 2, 3, 10, 1 << 20, (1 << 30)])
def test_null_count_closed_form(lib, n):
    import paper_1209_6308_gb300 as tc
    c3 = n * (n - 1) * (n - 2) // 6 if n >= 3 else 0
    assert tc.tc_null_count(n, [0] * 16) == c3
    if c3 > 100:
        counts = [0, 7, 5, 3] + [1] * 12
        assert tc.tc_null_count(n, counts) == c3 - sum(counts[1:])


def test_null_count_exceeds_64_bits(lib):
    import paper_1209_6308_gb300 as tc
    n = 1 << 26                       # C(2^26, 3) ~ 5e22 > 2^64
    assert tc.tc_null_count(n, [0] * 16) == n * (n - 1) * (n - 2) // 6 > (1 << 64)


def test_status_strings(lib):
    import paper_1209_6308_gb300 as tc
    for s, name in enumerate(["TC_OK", "TC_ERR_ARG", "TC_ERR_RANGE", "TC_ERR_OOM", "TC_ERR_CUDA",
                              "TC_ERR_TIMEOUT", "TC_ERR_BUSY"]):
        assert lib.tc_status_str(s).decode() == name


def test_null_arguments_are_rejected_without_a_gpu(lib):
    import paper_1209_6308_gb300 as tc
    assert lib.tc_graph_create_arcs(4, 0, None, None, 0, None, None, None) == tc.TC_ERR_ARG
    assert lib.tc_graph_stats(None, None) == tc.TC_ERR_ARG
    out = ctypes.c_void_p()
    assert lib.tc_graph_create_arcs(1 << 30 + 1, 0, None, None, 0, None, None, ctypes.byref(out)) == tc.TC_ERR_RANGE


def test_struct_layouts_match_header(lib, tmp_path):
    """Every struct the binding mirrors has the header's size and field offsets (the header
    compiled by the host C compiler)."""
    import paper_1209_6308_gb300 as tc
    structs = [tc.tc_u128, tc.tc_options, tc.tc_graph_info, tc.tc_server_options, tc.tc_serve_result,
               tc.tc_server_info, tc.tc_wave_record]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "tc.h"', 'int main(void) {']
    for st in structs:
        name = st.__name__
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for f, _ in st._fields_:
            lines.append(f'printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        name, field, val = line.split()
        got[(name, field)] = int(val)
    for st in structs:
        name = st.__name__
        assert got[(name, "size")] == ctypes.sizeof(st), name
        for f, _ in st._fields_:
            assert got[(name, f)] == getattr(st, f).offset, (name, f)


def test_stream_arguments_are_checked_without_a_gpu(lib):
    import paper_1209_6308_gb300 as tc
    out = ctypes.c_void_p()
    assert lib.tc_stream_create((1 << 30) + 1, 10, None, None, ctypes.byref(out)) == tc.TC_ERR_RANGE
    assert lib.tc_stream_create(10, 0, None, None, ctypes.byref(out)) == tc.TC_ERR_ARG
    assert lib.tc_stream_create(10, 5, None, None, ctypes.byref(out)) == tc.TC_OK
    s = np.array([1, 2], np.uint32)
    d = np.array([2, 3], np.uint32)
    t = np.array([5, 4], np.uint64)                            # decreasing
    assert lib.tc_stream_push(out, 2, s.ctypes.data, d.ctypes.data, t.ctypes.data) == tc.TC_ERR_ARG
    bad = np.array([1, 99], np.uint32)                         # id >= n
    t2 = np.array([4, 5], np.uint64)
    assert lib.tc_stream_push(out, 2, bad.ctypes.data, d.ctypes.data, t2.ctypes.data) == tc.TC_ERR_RANGE
    lib.tc_stream_destroy(out)
