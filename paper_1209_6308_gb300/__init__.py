"""Python binding of libtc.so, the GB300 triad-census library (include/tc.h).

Argument marshalling only: every step of the census runs in the library's CUDA kernels.
The functions keep the C names (tc_graph_create_arcs, tc_census, ...).  Buffers may be
numpy arrays (host) or CUDA tensors (device); a CUDA stream may be passed as an int handle,
a torch.cuda.Stream, or None for torch's current stream.  Counts come back as Python ints.

If libtc.so cannot be loaded this module raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtc.so")

CLASS_NAMES = ("003", "012", "102", "021D", "021U", "021C", "111D", "111U",
               "030T", "030C", "201", "120D", "120U", "120C", "210", "300")

TC_OK, TC_ERR_ARG, TC_ERR_RANGE, TC_ERR_OOM, TC_ERR_CUDA, TC_ERR_TIMEOUT, TC_ERR_BUSY = range(7)
TC_ALGO_UNION, TC_ALGO_SUFFIX, TC_ALGO_TRIANGLE = 0, 1, 2
TC_SCHED_PLAIN, TC_SCHED_LEARNED = 0, 1


class TcError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {_status_name(status)}: {msg}")
        self.status = status


class tc_u128(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_uint64), ("hi", ctypes.c_uint64)]

    def value(self) -> int:
        return int(self.lo) | (int(self.hi) << 64)


class tc_options(ctypes.Structure):
    _fields_ = [("algo", ctypes.c_uint32), ("schedule", ctypes.c_uint32), ("warp_max_deg", ctypes.c_uint32),
                ("chunk_entries", ctypes.c_uint32), ("item_work", ctypes.c_uint32), ("ctas_per_sm", ctypes.c_uint32),
                ("map_mode", ctypes.c_uint32), ("reserved", ctypes.c_uint32 * 9)]


class tc_autotune_trial(ctypes.Structure):
    _fields_ = [("opts", tc_options), ("ms", ctypes.c_float)]


class tc_graph_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint32), ("max_deg", ctypes.c_uint32), ("arcs", ctypes.c_uint64),
                ("e_sym", ctypes.c_uint64), ("mutual", ctypes.c_uint64), ("loops_dropped", ctypes.c_uint64),
                ("dups_dropped", ctypes.c_uint64), ("sum_d2", ctypes.c_uint64), ("sum_dv_upper", ctypes.c_uint64),
                ("bytes_alg", ctypes.c_uint64), ("sum_walk", ctypes.c_uint64), ("sum_walk_map", ctypes.c_uint64),
                ("sum_tri_walk", ctypes.c_uint64), ("bytes_alg_tri", ctypes.c_uint64)]

    def as_dict(self) -> dict:
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class tc_server_options(ctypes.Structure):
    _fields_ = [("census", tc_options), ("budget_bytes", ctypes.c_uint64), ("max_active", ctypes.c_uint32),
                ("max_pending", ctypes.c_uint32), ("quantum_us", ctypes.c_uint32), ("lanes", ctypes.c_uint32),
                ("starve_ms", ctypes.c_uint32), ("max_item_units", ctypes.c_uint32), ("reserved", ctypes.c_uint32 * 8)]


class tc_serve_result(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("graph", ctypes.c_uint32), ("status", ctypes.c_int32),
                ("counts", ctypes.c_uint64 * 16), ("c003", tc_u128), ("submit_ns", ctypes.c_uint64),
                ("start_ns", ctypes.c_uint64), ("done_ns", ctypes.c_uint64), ("waves", ctypes.c_uint32),
                ("lane", ctypes.c_uint32)]

    def census(self) -> list:
        return [self.c003.value()] + [int(self.counts[t]) for t in range(1, 16)]


class tc_server_info(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("refused", ctypes.c_uint64),
                ("waves", ctypes.c_uint64), ("slices", ctypes.c_uint64), ("resident_bytes", ctypes.c_uint64),
                ("budget_bytes", ctypes.c_uint64), ("graphs", ctypes.c_uint32), ("active", ctypes.c_uint32),
                ("pending", ctypes.c_uint32), ("inflight_waves", ctypes.c_uint32), ("gpu_ms", ctypes.c_double),
                ("ns_per_unit", ctypes.c_double), ("error", ctypes.c_int32), ("reserved", ctypes.c_uint32 * 7)]

    def as_dict(self) -> dict:
        return {k: (float(getattr(self, k)) if k in ("gpu_ms", "ns_per_unit") else int(getattr(self, k)))
                for k, _ in self._fields_ if k != "reserved"}


class tc_wave_record(ctypes.Structure):
    _fields_ = [("launch_ns", ctypes.c_uint64), ("done_ns", ctypes.c_uint64), ("units", ctypes.c_uint64),
                ("budget", ctypes.c_uint64), ("gpu_ms", ctypes.c_float), ("lane", ctypes.c_uint32),
                ("slices", ctypes.c_uint32), ("finished", ctypes.c_uint32), ("items", ctypes.c_uint32),
                ("blocks", ctypes.c_uint32)]

    def as_dict(self) -> dict:
        return {k: (float(getattr(self, k)) if k == "gpu_ms" else int(getattr(self, k))) for k, _ in self._fields_}


class tc_stream_info(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in ("live_arcs", "capacity", "censuses", "distinct_arcs", "rebuilds",
                                               "repairs", "last_added", "last_evicted")]


_lib = None
_VP, _U32, _U64 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64

# name -> (restype, argtypes); every symbol include/tc.h declares
SIGNATURES = {
    "tc_graph_create_arcs": (ctypes.c_int, [_U32, _U64, _VP, _VP, ctypes.c_int, _VP, _VP, ctypes.POINTER(_VP)]),
    "tc_graph_create_csr": (ctypes.c_int, [_U32, _VP, _VP, ctypes.c_int, _VP, _VP, ctypes.POINTER(_VP)]),
    "tc_census": (ctypes.c_int, [_VP, _VP, ctypes.POINTER(tc_u128)]),
    "tc_census_opts": (ctypes.c_int, [_VP, _VP, _VP, ctypes.POINTER(tc_u128)]),
    "tc_census_async": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "tc_census_profile": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "tc_census_grid": (ctypes.c_uint32, [_VP]),
    "tc_census_shard": (ctypes.c_int, [_VP, _VP, _VP, _U32, _U32, _VP]),
    "tc_census_shard_bounds": (ctypes.c_int, [_VP, _VP, _VP, _U32, _VP]),
    "tc_census_csr_noalloc": (ctypes.c_int, [_U32, _VP, _VP, _VP, _VP]),
    "tc_null_count": (tc_u128, [_U32, ctypes.POINTER(_U64)]),
    "tc_census64": (ctypes.c_int, [_VP, _VP, ctypes.POINTER(tc_u128)]),
    "tc_census_matrix": (ctypes.c_int, [_VP, _VP, ctypes.POINTER(tc_u128)]),
    "tc_census_batch": (ctypes.c_int, [_VP, _U32, _VP, ctypes.POINTER(_U64), ctypes.POINTER(tc_u128)]),
    "tc_batch_create": (ctypes.c_int, [_VP, _U32, _VP, _VP, ctypes.POINTER(_VP)]),
    "tc_batch_census_async": (ctypes.c_int, [_VP, _VP, _VP]),
    "tc_batch_census": (ctypes.c_int, [_VP, _VP, ctypes.POINTER(_U64), ctypes.POINTER(tc_u128)]),
    "tc_batch_autotune": (ctypes.c_int, [_VP, _VP, _U32, _VP, ctypes.POINTER(ctypes.c_float)]),
    "tc_batch_stats": (ctypes.c_int, [_VP, ctypes.POINTER(_U32), ctypes.POINTER(_U32)]),
    "tc_batch_autotune_history": (ctypes.c_int, [_VP, _VP, _U32, ctypes.POINTER(_U32)]),
    "tc_batch_destroy": (None, [_VP]),
    "tc_costmodel_num_params": (ctypes.c_uint32, []),
    "tc_costmodel_create": (ctypes.c_int, [_U64, ctypes.POINTER(_VP)]),
    "tc_costmodel_destroy": (None, [_VP]),
    "tc_costmodel_set_params": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_float)]),
    "tc_costmodel_get_params": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_float)]),
    "tc_costmodel_set_norm": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float),
                                             ctypes.c_float, ctypes.c_float]),
    "tc_costmodel_get_norm": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float),
                                             ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)]),
    "tc_costmodel_fit_norm": (ctypes.c_int, [_VP, _VP, _VP, _U32, ctypes.c_float, _VP]),
    "tc_graph_features": (ctypes.c_int, [_VP, _VP, _VP]),
    "tc_costmodel_samples": (ctypes.c_int, [_VP, _VP, _VP, _U32, _VP, _VP, _VP, ctypes.POINTER(_U32),
                                            ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "tc_costmodel_grad": (ctypes.c_int, [_VP, _VP, _VP, _U32, _VP, ctypes.POINTER(ctypes.c_float),
                                         ctypes.POINTER(ctypes.c_float)]),
    "tc_costmodel_train": (ctypes.c_int, [_VP, _VP, _VP, _U32, _U32, ctypes.c_float, _VP, ctypes.POINTER(ctypes.c_float)]),
    "tc_costmodel_predict": (ctypes.c_int, [_VP, _VP, _U32, _VP, _VP]),
    "tc_graph_attach_costmodel": (ctypes.c_int, [_VP, _VP, _VP]),
    "tc_graph_stats": (ctypes.c_int, [_VP, ctypes.POINTER(tc_graph_info)]),
    "tc_graph_device_csr": (ctypes.c_int, [_VP, ctypes.POINTER(_VP), ctypes.POINTER(_VP), ctypes.POINTER(_VP)]),
    "tc_graph_export_csr": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "tc_graph_destroy": (None, [_VP]),
    "tc_status_str": (ctypes.c_char_p, [ctypes.c_int]),
    "tc_last_error": (ctypes.c_char_p, []),
    "tc_server_now_ns": (_U64, []),
    "tc_server_create": (ctypes.c_int, [ctypes.POINTER(tc_server_options), ctypes.POINTER(_VP)]),
    "tc_server_add_graph": (ctypes.c_int, [_VP, _VP, _VP, ctypes.POINTER(_U32)]),
    "tc_server_remove_graph": (ctypes.c_int, [_VP, _U32]),
    "tc_server_submit": (ctypes.c_int, [_VP, _U32, ctypes.POINTER(_U64)]),
    "tc_server_poll": (ctypes.c_int, [_VP, ctypes.POINTER(tc_serve_result), _U32, _U32, ctypes.POINTER(_U32)]),
    "tc_server_drain": (ctypes.c_int, [_VP, _U32]),
    "tc_server_stats": (ctypes.c_int, [_VP, ctypes.POINTER(tc_server_info)]),
    "tc_server_graph_units": (ctypes.c_int, [_VP, _U32, ctypes.POINTER(_U64), ctypes.POINTER(_U32),
                                             ctypes.POINTER(_U32)]),
    "tc_server_trace": (ctypes.c_int, [_VP, ctypes.POINTER(tc_wave_record), _U32, ctypes.POINTER(_U32)]),
    "tc_server_destroy": (None, [_VP]),
    "tc_stream_create": (ctypes.c_int, [_U32, _U64, _VP, _VP, ctypes.POINTER(_VP)]),
    "tc_stream_push": (ctypes.c_int, [_VP, _U64, _VP, _VP, _VP]),
    "tc_stream_census": (ctypes.c_int, [_VP, _U64, ctypes.POINTER(tc_u128), ctypes.POINTER(_U64)]),
    "tc_stream_stats": (ctypes.c_int, [_VP, _VP]),
    "tc_stream_destroy": (None, [_VP]),
    "tc_tricode_table": (None, [ctypes.POINTER(ctypes.c_uint8)]),
}


def load():
    """Load libtc.so (built by _build.build() / __graft_entry__.build()); raises if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1209_6308_gb300._build.build() "
                               "(there is no CPU fallback)")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _status_name(s: int) -> str:
    names = ["TC_OK", "TC_ERR_ARG", "TC_ERR_RANGE", "TC_ERR_OOM", "TC_ERR_CUDA", "TC_ERR_TIMEOUT", "TC_ERR_BUSY"]
    return names[s] if 0 <= s < len(names) else f"status {s}"


def _check(status: int, where: str):
    if status != TC_OK:
        raise TcError(status, where, load().tc_last_error().decode(errors="replace"))


def _stream_handle(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return 0
    if isinstance(stream, int):
        return stream
    return int(getattr(stream, "cuda_stream"))


def _buffer(x, dtype):
    """(pointer, is_device, keepalive) for a numpy array or a CUDA tensor."""
    if hasattr(x, "data_ptr") and hasattr(x, "is_cuda"):
        if x.element_size() != np.dtype(dtype).itemsize or not x.is_contiguous():
            raise ValueError(f"tensor must be contiguous with {np.dtype(dtype).itemsize}-byte elements")
        return x.data_ptr(), bool(x.is_cuda), x
    a = np.ascontiguousarray(x, dtype=dtype)
    return a.ctypes.data, False, a


def _options(opts):
    if opts is None:
        return None, None
    o = tc_options()
    for k, v in dict(opts).items():
        setattr(o, k, int(v))
    return ctypes.addressof(o), o


def tc_graph_create_arcs(n: int, src, dst, stream=None, options=None) -> int:
    """Build a graph from arcs src[i] -> dst[i]; returns an opaque handle (int)."""
    ps, ds, ka = _buffer(src, np.uint32)
    pd, dd, kb = _buffer(dst, np.uint32)
    m = len(ka) if hasattr(ka, "__len__") else ka.numel()
    if (len(kb) if hasattr(kb, "__len__") else kb.numel()) != m:
        raise ValueError("src and dst differ in length")
    if ds != dd:
        raise ValueError("src and dst must both be host or both be device buffers")
    po, keep = _options(options)
    out = _VP()
    _check(load().tc_graph_create_arcs(n, m, ps, pd, int(ds), _stream_handle(stream), po, ctypes.byref(out)),
           "tc_graph_create_arcs")
    return out.value


def tc_graph_create_csr(n: int, off, adj_flagged, stream=None, options=None) -> int:
    """Build a graph from a canonical flagged CSR (off: uint64[n+1], adj: uint32)."""
    po_, dev_o, ko = _buffer(off, np.uint64)
    pa, dev_a, ka = _buffer(adj_flagged, np.uint32)
    if dev_o != dev_a:
        raise ValueError("off and adj must both be host or both be device buffers")
    po, keep = _options(options)
    out = _VP()
    _check(load().tc_graph_create_csr(n, po_, pa, int(dev_o), _stream_handle(stream), po, ctypes.byref(out)),
           "tc_graph_create_csr")
    return out.value


def tc_census64(g: int, stream=None) -> list:
    """64-state census (Sec. 3, Fig. 2): triads per labelled state, the actors in increasing
    vertex id taking the roles u, v, w (synchronises the stream)."""
    out = (tc_u128 * 64)()
    _check(load().tc_census64(g, _stream_handle(stream), out), "tc_census64")
    return [out[i].value() for i in range(64)]


def tc_census_matrix(g: int, stream=None) -> list:
    """The census by its matrix form (Sec. 4): 16 class counts from masked sums of products of
    the bit-packed one-way, mutual and null dyad matrices (n <= 2^14; synchronises the stream)."""
    out = (tc_u128 * 16)()
    _check(load().tc_census_matrix(g, _stream_handle(stream), out), "tc_census_matrix")
    return [out[i].value() for i in range(16)]


def tc_census(g: int, stream=None, options=None) -> list:
    """Full 16-class census of a graph (synchronises the stream)."""
    out = (tc_u128 * 16)()
    po, keep = _options(options)
    _check(load().tc_census_opts(g, _stream_handle(stream), po, out), "tc_census")
    return [out[i].value() for i in range(16)]


def tc_census_async(g: int, d_out16, stream=None, options=None) -> None:
    """Enqueue a census writing counts 1..15 into a 16-element uint64 device buffer."""
    p, dev, keep = _buffer(d_out16, np.uint64)
    if not dev:
        raise ValueError("d_out16 must be device memory")
    po, keepo = _options(options)
    _check(load().tc_census_async(g, _stream_handle(stream), po, p), "tc_census_async")


def tc_census_profile(g: int, d_out16, d_vcost, d_phase=None, stream=None, options=None) -> None:
    """Instrumented census: counts into d_out16, per-vertex SM cycles added into d_vcost[n]
    (relabelled ids), optional per-CTA timestamps into d_phase[3 * tc_census_grid()]."""
    p, dev, k1 = _buffer(d_out16, np.uint64)
    pv, devv, k2 = _buffer(d_vcost, np.uint64)
    pp = 0
    if d_phase is not None:
        pp, devp, k3 = _buffer(d_phase, np.uint64)
    if not (dev and devv):
        raise ValueError("d_out16 and d_vcost must be device memory")
    po, keepo = _options(options)
    _check(load().tc_census_profile(g, _stream_handle(stream), po, p, pv, pp or None), "tc_census_profile")


def tc_census_csr_noalloc(n: int, d_off: int, d_adj: int, d_out16, stream=None) -> None:
    """Census of a device CSR in the library's form using only the library's fixed scratch
    array (no device allocation); d_off/d_adj are device pointers (ints), d_out16 a 16-element
    uint64 device buffer."""
    p, dev, keep = _buffer(d_out16, np.uint64)
    if not dev:
        raise ValueError("d_out16 must be device memory")
    _check(load().tc_census_csr_noalloc(n, d_off, d_adj, _stream_handle(stream), p), "tc_census_csr_noalloc")


def tc_census_shard(g: int, d_out16, rank: int, world: int, stream=None, options=None) -> None:
    """Shard `rank` of `world` of the census of g (Sec. 6-7: independent pairs): its counts of
    classes 1..15 into d_out16 (16 uint64 on the device); the shards' sum is the census."""
    p, dev, keep = _buffer(d_out16, np.uint64)
    if not dev:
        raise ValueError("d_out16 must be device memory")
    po, keepo = _options(options)
    _check(load().tc_census_shard(g, _stream_handle(stream), po, rank, world, p), "tc_census_shard")


def tc_census_shard_bounds(g: int, world: int, stream=None, options=None) -> np.ndarray:
    """[(first item, first warp-tier vertex) for r = 0..world] as a (world + 1, 2) uint32 array."""
    b = np.zeros(2 * (world + 1), np.uint32)
    po, keepo = _options(options)
    _check(load().tc_census_shard_bounds(g, _stream_handle(stream), po, world, b.ctypes.data), "tc_census_shard_bounds")
    return b.reshape(world + 1, 2)


def tc_census_grid(options=None) -> int:
    po, keepo = _options(options)
    return int(load().tc_census_grid(po))


def tc_null_count(n: int, counts16) -> int:
    c = (ctypes.c_uint64 * 16)(*[int(x) & 0xFFFFFFFFFFFFFFFF for x in counts16])
    return load().tc_null_count(n, c).value()


def tc_census_batch(graphs, stream=None) -> list:
    """Census of many graphs: list of 16-int lists (index 0 is the full 128-bit null count)."""
    k = len(graphs)
    arr = (_VP * k)(*graphs)
    out = (ctypes.c_uint64 * (16 * k))()
    z = (tc_u128 * k)()
    _check(load().tc_census_batch(ctypes.cast(arr, _VP), k, _stream_handle(stream), out, z), "tc_census_batch")
    res = []
    for i in range(k):
        row = [int(out[16 * i + t]) for t in range(16)]
        row[0] = z[i].value()
        res.append(row)
    return res


def tc_batch_create(graphs, stream=None, options=None) -> int:
    """Reusable batched census over graph handles (one persistent, graph-captured launch)."""
    k = len(graphs)
    arr = (_VP * max(k, 1))(*graphs)
    po, keep = _options(options)
    out = _VP()
    _check(load().tc_batch_create(ctypes.cast(arr, _VP), k, po, _stream_handle(stream), ctypes.byref(out)),
           "tc_batch_create")
    return out.value


def tc_batch_census_async(b: int, d_out16xk=None, stream=None) -> None:
    p = 0
    if d_out16xk is not None:
        p, dev, keep = _buffer(d_out16xk, np.uint64)
        if not dev:
            raise ValueError("d_out16xk must be device memory")
    _check(load().tc_batch_census_async(b, _stream_handle(stream), p or None), "tc_batch_census_async")


def tc_batch_census(b: int, k: int, stream=None) -> list:
    out = (ctypes.c_uint64 * (16 * max(k, 1)))()
    z = (tc_u128 * max(k, 1))()
    _check(load().tc_batch_census(b, _stream_handle(stream), out, z), "tc_batch_census")
    res = []
    for i in range(k):
        row = [int(out[16 * i + t]) for t in range(16)]
        row[0] = z[i].value()
        res.append(row)
    return res


def tc_batch_autotune(b: int, max_trials: int = 0, stream=None):
    """Returns (best options dict, median ms per launch); the batch keeps the best plan."""
    o = tc_options()
    ms = ctypes.c_float()
    _check(load().tc_batch_autotune(b, _stream_handle(stream), max_trials, ctypes.addressof(o), ctypes.byref(ms)),
           "tc_batch_autotune")
    best = {k: int(getattr(o, k)) for k in ("algo", "schedule", "warp_max_deg", "chunk_entries", "item_work",
                                             "ctas_per_sm")}
    return best, float(ms.value)


def tc_batch_autotune_history(b: int, max_trials: int = 1024) -> list:
    """The last autotune's trials in order: [(options dict, median ms)]."""
    arr = (tc_autotune_trial * max(max_trials, 1))()
    cnt = _U32()
    _check(load().tc_batch_autotune_history(b, ctypes.addressof(arr), max_trials, ctypes.byref(cnt)),
           "tc_batch_autotune_history")
    keys = ("algo", "schedule", "warp_max_deg", "chunk_entries", "item_work", "ctas_per_sm")
    return [({k: int(getattr(arr[i].opts, k)) for k in keys}, float(arr[i].ms)) for i in range(cnt.value)]


def tc_batch_stats(b: int):
    ni, nw = _U32(), _U32()
    _check(load().tc_batch_stats(b, ctypes.byref(ni), ctypes.byref(nw)), "tc_batch_stats")
    return int(ni.value), int(nw.value)


def tc_batch_destroy(b: int) -> None:
    if b:
        load().tc_batch_destroy(b)


def _fptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def tc_costmodel_num_params() -> int:
    return int(load().tc_costmodel_num_params())


def tc_costmodel_create(seed: int = 0) -> int:
    out = _VP()
    _check(load().tc_costmodel_create(seed, ctypes.byref(out)), "tc_costmodel_create")
    return out.value


def tc_costmodel_destroy(c: int) -> None:
    if c:
        load().tc_costmodel_destroy(c)


def tc_costmodel_set_params(c: int, params) -> None:
    a = np.ascontiguousarray(params, dtype=np.float32)
    if a.size != tc_costmodel_num_params():
        raise ValueError("wrong parameter count")
    _check(load().tc_costmodel_set_params(c, _fptr(a)), "tc_costmodel_set_params")


def tc_costmodel_get_params(c: int) -> np.ndarray:
    a = np.zeros(tc_costmodel_num_params(), np.float32)
    _check(load().tc_costmodel_get_params(c, _fptr(a)), "tc_costmodel_get_params")
    return a


def tc_costmodel_set_norm(c: int, mean, std, target_mean: float, kappa: float) -> None:
    m = np.ascontiguousarray(mean, np.float32)
    sd = np.ascontiguousarray(std, np.float32)
    _check(load().tc_costmodel_set_norm(c, _fptr(m), _fptr(sd), float(target_mean), float(kappa)),
           "tc_costmodel_set_norm")


def tc_costmodel_get_norm(c: int):
    m = np.zeros(4, np.float32)
    sd = np.zeros(4, np.float32)
    tm, kp = ctypes.c_float(), ctypes.c_float()
    _check(load().tc_costmodel_get_norm(c, _fptr(m), _fptr(sd), ctypes.byref(tm), ctypes.byref(kp)),
           "tc_costmodel_get_norm")
    return m, sd, float(tm.value), float(kp.value)


def tc_costmodel_fit_norm(c: int, d_x4, d_y, count: int, kappa: float, stream=None) -> None:
    px, _, k1 = _buffer(d_x4, np.float32)
    py, _, k2 = _buffer(d_y, np.float32)
    _check(load().tc_costmodel_fit_norm(c, px, py, count, float(kappa), _stream_handle(stream)), "tc_costmodel_fit_norm")


def tc_graph_features(g: int, d_feat4, stream=None) -> None:
    p, dev, keep = _buffer(d_feat4, np.float32)
    _check(load().tc_graph_features(g, _stream_handle(stream), p), "tc_graph_features")


def tc_costmodel_samples(g: int, d_vcost, d_feat4, d_x4, d_y, capacity: int, stream=None):
    """-> (count, plain estimate sum, measured cycle sum)"""
    pv, _, k1 = _buffer(d_vcost, np.uint64)
    pf, _, k2 = _buffer(d_feat4, np.float32)
    px, _, k3 = _buffer(d_x4, np.float32)
    py, _, k4 = _buffer(d_y, np.float32)
    cnt = _U32()
    es, cs = ctypes.c_double(), ctypes.c_double()
    _check(load().tc_costmodel_samples(g, pv, pf, capacity, _stream_handle(stream), px, py, ctypes.byref(cnt),
                                       ctypes.byref(es), ctypes.byref(cs)), "tc_costmodel_samples")
    return int(cnt.value), float(es.value), float(cs.value)


def tc_costmodel_grad(c: int, d_x4, d_y, count: int, stream=None):
    px, _, k1 = _buffer(d_x4, np.float32)
    py, _, k2 = _buffer(d_y, np.float32)
    g = np.zeros(tc_costmodel_num_params(), np.float32)
    loss = ctypes.c_float()
    _check(load().tc_costmodel_grad(c, px, py, count, _stream_handle(stream), _fptr(g), ctypes.byref(loss)),
           "tc_costmodel_grad")
    return g, float(loss.value)


def tc_costmodel_train(c: int, d_x4, d_y, count: int, steps: int, lr: float, stream=None) -> float:
    px, _, k1 = _buffer(d_x4, np.float32)
    py, _, k2 = _buffer(d_y, np.float32)
    loss = ctypes.c_float()
    _check(load().tc_costmodel_train(c, px, py, count, steps, float(lr), _stream_handle(stream), ctypes.byref(loss)),
           "tc_costmodel_train")
    return float(loss.value)


def tc_costmodel_predict(c: int, d_x4, count: int, d_out, stream=None) -> None:
    px, _, k1 = _buffer(d_x4, np.float32)
    po, _, k2 = _buffer(d_out, np.float32)
    _check(load().tc_costmodel_predict(c, px, count, _stream_handle(stream), po), "tc_costmodel_predict")


def tc_graph_attach_costmodel(g: int, c: int, stream=None) -> None:
    _check(load().tc_graph_attach_costmodel(g, c, _stream_handle(stream)), "tc_graph_attach_costmodel")


def tc_graph_stats(g: int) -> dict:
    info = tc_graph_info()
    _check(load().tc_graph_stats(g, ctypes.byref(info)), "tc_graph_stats")
    return info.as_dict()


def tc_graph_device_csr(g: int):
    """(off, adj, new_of_old) device pointers as ints."""
    o, a, p = _VP(), _VP(), _VP()
    _check(load().tc_graph_device_csr(g, ctypes.byref(o), ctypes.byref(a), ctypes.byref(p)), "tc_graph_device_csr")
    return o.value, a.value, p.value


def tc_graph_export_csr(g: int):
    """(off uint64[n+1], adj uint32[2 e_sym], new_of_old uint32[n]) copied to host numpy arrays."""
    st = tc_graph_stats(g)
    n = st["n"]
    off = np.zeros(n + 1, np.uint64)
    adj = np.zeros(2 * st["e_sym"], np.uint32)
    perm = np.zeros(n, np.uint32)
    _check(load().tc_graph_export_csr(g, off.ctypes.data, adj.ctypes.data, perm.ctypes.data), "tc_graph_export_csr")
    return off, adj, perm


def tc_graph_destroy(g: int) -> None:
    if g:
        load().tc_graph_destroy(g)


def tc_tricode_table() -> np.ndarray:
    t = np.zeros(64, dtype=np.uint8)
    load().tc_tricode_table(t.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
    return t


def tc_server_now_ns() -> int:
    return int(load().tc_server_now_ns())


def tc_server_create(options=None, census=None) -> int:
    """Start a census server; `options` sets tc_server_options fields, `census` its tc_options."""
    o = tc_server_options()
    for k, v in dict(options or {}).items():
        setattr(o, k, int(v))
    for k, v in dict(census or {}).items():
        setattr(o.census, k, int(v))
    out = _VP()
    _check(load().tc_server_create(ctypes.byref(o), ctypes.byref(out)), "tc_server_create")
    return out.value


def tc_server_add_graph(s: int, g: int, stream=None) -> int:
    gid = _U32()
    _check(load().tc_server_add_graph(s, g, _stream_handle(stream), ctypes.byref(gid)), "tc_server_add_graph")
    return int(gid.value)


def tc_server_remove_graph(s: int, graph_id: int) -> None:
    _check(load().tc_server_remove_graph(s, graph_id), "tc_server_remove_graph")


def tc_server_submit(s: int, graph_id: int) -> int:
    rid = _U64()
    _check(load().tc_server_submit(s, graph_id, ctypes.byref(rid)), "tc_server_submit")
    return int(rid.value)


def tc_server_poll(s: int, max_results: int = 256, timeout_ms: int = 0) -> list:
    buf = (tc_serve_result * max(max_results, 1))()
    cnt = _U32()
    _check(load().tc_server_poll(s, buf, max_results, timeout_ms, ctypes.byref(cnt)), "tc_server_poll")
    return [buf[i] for i in range(cnt.value)]


def tc_server_drain(s: int, timeout_ms: int = 60000) -> None:
    _check(load().tc_server_drain(s, timeout_ms), "tc_server_drain")


def tc_server_stats(s: int) -> dict:
    info = tc_server_info()
    _check(load().tc_server_stats(s, ctypes.byref(info)), "tc_server_stats")
    return info.as_dict()


def tc_server_graph_units(s: int, graph_id: int):
    u, ni, nb = _U64(), _U32(), _U32()
    _check(load().tc_server_graph_units(s, graph_id, ctypes.byref(u), ctypes.byref(ni), ctypes.byref(nb)),
           "tc_server_graph_units")
    return int(u.value), int(ni.value), int(nb.value)


def tc_server_trace(s: int, max_records: int = 8192) -> list:
    """The last waves of the engine (oldest first) as dicts."""
    buf = (tc_wave_record * max(max_records, 1))()
    cnt = _U32()
    _check(load().tc_server_trace(s, buf, max_records, ctypes.byref(cnt)), "tc_server_trace")
    return [buf[i].as_dict() for i in range(cnt.value)]


def tc_server_destroy(s: int) -> None:
    if s:
        load().tc_server_destroy(s)


class Server:
    """Owning wrapper around a tc_server handle (continuous-batching census serving)."""

    def __init__(self, options=None, census=None):
        self.handle = tc_server_create(options, census)

    def add(self, g, stream=None) -> int:
        return tc_server_add_graph(self.handle, g.handle if isinstance(g, Graph) else g, stream)

    def remove(self, graph_id: int) -> None:
        tc_server_remove_graph(self.handle, graph_id)

    def submit(self, graph_id: int) -> int:
        return tc_server_submit(self.handle, graph_id)

    def poll(self, max_results: int = 256, timeout_ms: int = 0) -> list:
        return tc_server_poll(self.handle, max_results, timeout_ms)

    def drain(self, timeout_ms: int = 60000) -> None:
        tc_server_drain(self.handle, timeout_ms)

    def stats(self) -> dict:
        return tc_server_stats(self.handle)

    def trace(self, max_records: int = 8192) -> list:
        return tc_server_trace(self.handle, max_records)

    def close(self):
        tc_server_destroy(self.handle)
        self.handle = 0

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            if self.handle:
                self.close()
        except Exception:
            pass


class Stream:
    """Interval census over a stream of timestamped arcs (owning wrapper around tc_stream)."""

    def __init__(self, n: int, window: int, options=None, stream=None):
        po, self._keep = _options(options)
        out = _VP()
        _check(load().tc_stream_create(n, window, po, _stream_handle(stream), ctypes.byref(out)), "tc_stream_create")
        self.handle, self.n = out.value, n

    def push(self, src, dst, t) -> None:
        s = np.ascontiguousarray(src, dtype=np.uint32)
        d = np.ascontiguousarray(dst, dtype=np.uint32)
        tt = np.ascontiguousarray(t, dtype=np.uint64)
        if not (len(s) == len(d) == len(tt)):
            raise ValueError("src, dst and t must have the same length")
        _check(load().tc_stream_push(self.handle, len(s), s.ctypes.data, d.ctypes.data, tt.ctypes.data),
               "tc_stream_push")

    def census(self, t_now: int):
        """(16 counts, arcs pushed into the window) for the window ending at t_now."""
        out = (tc_u128 * 16)()
        m = _U64()
        _check(load().tc_stream_census(self.handle, t_now, out, ctypes.byref(m)), "tc_stream_census")
        return [out[i].value() for i in range(16)], int(m.value)

    def stats(self) -> dict:
        info = tc_stream_info()
        _check(load().tc_stream_stats(self.handle, ctypes.byref(info)), "tc_stream_stats")
        return {f: int(getattr(info, f)) for f, _ in tc_stream_info._fields_}

    def close(self):
        if self.handle:
            load().tc_stream_destroy(self.handle)
        self.handle = 0

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Graph:
    """Owning wrapper around a tc_graph handle."""

    def __init__(self, handle: int, n: int):
        self.handle, self.n = handle, n

    @classmethod
    def from_arcs(cls, n, src, dst, stream=None, options=None):
        return cls(tc_graph_create_arcs(n, src, dst, stream, options), n)

    @classmethod
    def from_csr(cls, n, off, adj, stream=None, options=None):
        return cls(tc_graph_create_csr(n, off, adj, stream, options), n)

    def census(self, stream=None, options=None):
        return tc_census(self.handle, stream, options)

    def census64(self, stream=None):
        return tc_census64(self.handle, stream)

    def census_matrix(self, stream=None):
        return tc_census_matrix(self.handle, stream)

    def stats(self):
        return tc_graph_stats(self.handle)

    def close(self):
        tc_graph_destroy(self.handle)
        self.handle = 0

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            if self.handle:
                self.close()
        except Exception:
            pass
