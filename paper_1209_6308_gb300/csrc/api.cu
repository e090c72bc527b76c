// api.cu - the C ABI declared in include/tc.h: graph lifecycle, census entry points and
// the 128-bit null count of Fig. 5 steps 3-5.
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "graph.cuh"


namespace tc {

namespace {
thread_local std::string t_err;
}

void set_error(const std::string& msg) { t_err = msg; }

tc_status fail(tc_status s, const std::string& msg) {
    t_err = msg;
    return s;
}

tc_status cuda_fail(cudaError_t e, const char* what) {
    t_err = std::string(what) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return TC_ERR_OOM;
    }
    return TC_ERR_CUDA;
}

namespace {

// The library's own stream-ordered memory pool on each device.  Freed blocks stay in it, up to
// a quarter of the device's memory, for the next graph or call: CUDA's default pool gives
// them back at every synchronisation, so each build paid again for mapping its temporaries.
// Persistent buffers come from the same pool on a stream of their own that is synchronised
// at once, so they are valid on every stream when alloc_persistent returns.
struct DevicePool {
    cudaMemPool_t pool = nullptr;
    cudaStream_t st = nullptr;
};
std::mutex g_pool_mu;
DevicePool g_pools[64];

tc_status device_pool(DevicePool* out) {
    int dev = 0;
    TC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(TC_ERR_CUDA, "device index out of range");
    std::lock_guard<std::mutex> lk(g_pool_mu);
    DevicePool& d = g_pools[dev];
    if (!d.pool) {
        cudaMemPoolProps props;
        std::memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        size_t fr = 0, total = 0;
        TC_CUDA(cudaMemGetInfo(&fr, &total));
        cudaMemPool_t pool = nullptr;
        TC_CUDA(cudaMemPoolCreate(&pool, &props));
        uint64_t keep = total / 4;
        TC_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
        cudaStream_t st = nullptr;
        TC_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        d.pool = pool;
        d.st = st;
    }
    *out = d;
    return TC_OK;
}

tc_status pool_alloc(void** p, size_t b, cudaStream_t s, const DevicePool& d) {
    cudaError_t e = cudaMallocFromPoolAsync(p, b, d.pool, s);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? TC_ERR_OOM : TC_ERR_CUDA,
                    std::string("device allocation of ") + std::to_string(b) + " bytes: " + cudaGetErrorString(e));
    }
    return TC_OK;
}

}  // namespace

tc_status DevBuf::alloc(size_t b, cudaStream_t s) {
    release();
    if (b == 0) b = 16;
    DevicePool d;
    TC_TRY(device_pool(&d));
    TC_TRY(pool_alloc(&p, b, s, d));
    bytes = b;
    st = s;
    async = true;
    return TC_OK;
}

tc_status DevBuf::alloc_persistent(size_t b) {
    release();
    if (b == 0) b = 16;
    DevicePool d;
    TC_TRY(device_pool(&d));
    TC_TRY(pool_alloc(&p, b, d.st, d));
    const cudaError_t e = cudaStreamSynchronize(d.st);
    if (e != cudaSuccess) {
        cudaFreeAsync(p, d.st);
        p = nullptr;
        return cuda_fail(e, "device allocation");
    }
    bytes = b;
    st = d.st;
    async = false;
    return TC_OK;
}

void DevBuf::release() {
    if (p) {
        // a persistent buffer may be in use on any stream: like cudaFree, wait for the device
        if (!async) cudaDeviceSynchronize();
        cudaFreeAsync(p, st);
    }
    p = nullptr;
    bytes = 0;
}

int sm_count() {
    int dev = 0, c = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev);
    return c > 0 ? c : 1;
}

Opts merge_opts(const tc_options* in, const Opts* base) {
    Opts o = base ? *base : Opts();
    if (in) {
        if (in->algo) o.algo = in->algo;
        if (in->schedule) o.schedule = in->schedule;
        if (in->warp_max_deg) o.warp_max_deg = in->warp_max_deg;
        if (in->chunk_entries) o.chunk = in->chunk_entries;
        if (in->item_work) o.item_work = in->item_work;
        if (in->ctas_per_sm) o.ctas_per_sm = in->ctas_per_sm;
        if (in->map_mode) o.map_mode = in->map_mode;
    }
    return o;
}

tc_status resolve_opts(const tc_options* in, const Opts* base, Opts* out) {
    Opts o = merge_opts(in, base);
    if (o.algo > TC_ALGO_TRIANGLE) return fail(TC_ERR_ARG, "unknown algo");
    if (o.schedule > TC_SCHED_LEARNED) return fail(TC_ERR_ARG, "unknown schedule");
    // the suffix form's hash takes 4 slots per entry, the union walk's 2 plus the sorted copy:
    // both fill about 70 KB of shared memory, three CTAs per SM
    // the triangle form's CTAs hold a small hash (2 slots per staged entry) and few registers:
    // eight per SM keep the most loads in flight
    if (!o.chunk) {
        o.chunk = o.algo == TC_ALGO_UNION ? 4096u : 2048u;
        o.chunk_auto = true;
    }
    if (!o.ctas_per_sm) o.ctas_per_sm = o.algo == TC_ALGO_TRIANGLE ? 8 : 3;
    const uint32_t max_chunk = o.algo == TC_ALGO_UNION ? 16384u : 8192u;   // shared-memory hash sizes
    // the triangle form stages a warp-tier vertex's lower neighbours in a 256-slot warp hash
    if (o.algo == TC_ALGO_TRIANGLE && o.warp_max_deg > 128)
        return fail(TC_ERR_ARG, "warp_max_deg must be <= 128 for the triangle form");
    if (o.chunk < 512 || o.chunk > max_chunk || (o.chunk & (o.chunk - 1)))
        return fail(TC_ERR_ARG, "chunk_entries must be a power of two in [512, 16384] (8192 for the suffix form)");
    if (o.warp_max_deg > o.chunk / 8) return fail(TC_ERR_ARG, "warp_max_deg must be <= chunk_entries / 8");
    if (o.ctas_per_sm < 1 || o.ctas_per_sm > 8) return fail(TC_ERR_ARG, "ctas_per_sm must be in [1, 8]");
    if (o.map_mode > 2) return fail(TC_ERR_ARG, "map_mode must be 0, 1 or 2");
    if (o.item_work && o.item_work < 256) return fail(TC_ERR_ARG, "item_work must be 0 (sized to the graph) or >= 256");
    *out = o;
    return TC_OK;
}

namespace {

tc_status init_graph(tc_graph* g, uint32_t n, const tc_options* opt) {
    g->s.n = n;
    Opts check;
    TC_TRY(resolve_opts(opt, nullptr, &check));
    g->s.opts = merge_opts(opt, nullptr);
    TC_TRY(g->s.ctr.alloc_persistent(sizeof(uint32_t) * 4));
    TC_TRY(g->s.acc.alloc_persistent(sizeof(unsigned long long) * 16));
    TC_CUDA(cudaMallocHost(&g->s.h_counts, sizeof(unsigned long long) * 16));
    return TC_OK;
}

void destroy(tc_graph* g) {
    if (!g) return;
    cudaDeviceSynchronize();
    if (g->s.h_counts) cudaFreeHost(g->s.h_counts);
    delete g;
}

// Host -> device copy of `count` elements into a stream-ordered buffer
template <typename T>
tc_status upload(const T* h, uint64_t count, DevBuf& b, cudaStream_t st) {
    TC_TRY(b.alloc(sizeof(T) * (count ? count : 1), st));
    if (count) TC_CUDA(cudaMemcpyAsync(b.p, h, sizeof(T) * count, cudaMemcpyHostToDevice, st));
    return TC_OK;
}

// The device's address of page-locked host memory (cudaHostAlloc / cudaHostRegister), which a
// kernel can read directly over the host link, or null for any other pointer.
template <typename T>
const T* mapped_host(const T* h) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, h) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost && a.devicePointer ? static_cast<const T*>(a.devicePointer) : nullptr;
}

}  // namespace
}  // namespace tc

using namespace tc;

extern "C" {

const char* tc_last_error(void) { return t_err.c_str(); }

const char* tc_status_str(tc_status s) {
    switch (s) {
        case TC_OK: return "TC_OK";
        case TC_ERR_ARG: return "TC_ERR_ARG";
        case TC_ERR_RANGE: return "TC_ERR_RANGE";
        case TC_ERR_OOM: return "TC_ERR_OOM";
        case TC_ERR_CUDA: return "TC_ERR_CUDA";
        case TC_ERR_TIMEOUT: return "TC_ERR_TIMEOUT";
        case TC_ERR_BUSY: return "TC_ERR_BUSY";
    }
    return "TC_ERR_UNKNOWN";
}

void tc_tricode_table(uint8_t out[64]) {
    const uint8_t* t = host_tricode_table();
    if (t) std::memcpy(out, t, 64);
    else std::memset(out, 0xff, 64);
}

tc_status tc_graph_create_arcs(uint32_t n, uint64_t m, const uint32_t* src, const uint32_t* dst, int ptr_is_device,
                               void* stream, const tc_options* opt, tc_graph** out) {
    if (!out) return fail(TC_ERR_ARG, "out is null");
    *out = nullptr;
    if (m && (!src || !dst)) return fail(TC_ERR_ARG, "src/dst is null");
    if (n > (1u << 30)) return fail(TC_ERR_RANGE, "n > 2^30 (ids carry two direction bits)");
    cudaStream_t st = (cudaStream_t)stream;
    tc_graph* g = new tc_graph();
    tc_status s = init_graph(g, n, opt);
    if (s == TC_OK) {
        if (ptr_is_device) {
            s = build_from_arcs(g->s, m, src, dst, st);
        } else if (const uint32_t* ms = m ? mapped_host(src) : nullptr) {
            // page-locked arcs: the key kernel, which reads each arc once, reads them over the
            // host link, so there is no device copy to write and read back
            const uint32_t* md = mapped_host(dst);
            if (md) {
                s = build_from_arcs(g->s, m, ms, md, st);
            } else {
                DevBuf dd;
                s = upload(dst, m, dd, st);
                if (s == TC_OK) s = build_from_arcs(g->s, m, ms, dd.as<uint32_t>(), st);
            }
        } else {
            DevBuf ds, dd;
            s = upload(src, m, ds, st);
            if (s == TC_OK) s = upload(dst, m, dd, st);
            if (s == TC_OK) s = build_from_arcs(g->s, m, ds.as<uint32_t>(), dd.as<uint32_t>(), st);
        }
    }
    if (s == TC_OK) {
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) s = cuda_fail(e, "graph build");
    }
    if (s != TC_OK) {
        std::string keep = t_err;
        destroy(g);
        t_err = keep;
        return s;
    }
    *out = g;
    return TC_OK;
}

}  // extern "C"

namespace tc {

tc_status graph_create_sorted(uint32_t n, const uint64_t* d_keys, uint64_t m, cudaStream_t st, const tc_options* opt,
                              tc_graph** out) {
    if (!out) return fail(TC_ERR_ARG, "out is null");
    *out = nullptr;
    if (m && !d_keys) return fail(TC_ERR_ARG, "keys are null");
    tc_graph* g = new tc_graph();
    tc_status s = init_graph(g, n, opt);
    if (s == TC_OK) s = build_from_sorted_arcs(g->s, d_keys, m, st);
    if (s == TC_OK) {
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) s = cuda_fail(e, "graph build");
    }
    if (s != TC_OK) {
        std::string keep = t_err;
        destroy(g);
        t_err = keep;
        return s;
    }
    *out = g;
    return TC_OK;
}

}  // namespace tc

extern "C" {

tc_status tc_graph_create_csr(uint32_t n, const uint64_t* off, const uint32_t* adj_flagged, int ptr_is_device,
                              void* stream, const tc_options* opt, tc_graph** out) {
    if (!out) return fail(TC_ERR_ARG, "out is null");
    *out = nullptr;
    if (!off) return fail(TC_ERR_ARG, "off is null");
    if (n > (1u << 30)) return fail(TC_ERR_RANGE, "n > 2^30 (ids carry two direction bits)");
    cudaStream_t st = (cudaStream_t)stream;
    tc_graph* g = new tc_graph();
    tc_status s = init_graph(g, n, opt);
    if (s == TC_OK) {
        if (ptr_is_device) {
            s = build_from_csr(g->s, off, adj_flagged, st);
        } else {
            uint64_t total = off[n];
            if (off[0] != 0 || (total && !adj_flagged)) s = fail(TC_ERR_ARG, "malformed CSR offsets");
            for (uint32_t x = 0; s == TC_OK && x < n; ++x)
                if (off[x + 1] < off[x]) s = fail(TC_ERR_ARG, "CSR offsets decrease");
            DevBuf doff, dadj;
            if (s == TC_OK) s = upload(off, (uint64_t)n + 1, doff, st);
            if (s == TC_OK) s = upload(adj_flagged, total, dadj, st);
            if (s == TC_OK) s = build_from_csr(g->s, doff.as<uint64_t>(), dadj.as<uint32_t>(), st);
        }
    }
    if (s == TC_OK) {
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) s = cuda_fail(e, "graph build");
    }
    if (s != TC_OK) {
        std::string keep = t_err;
        destroy(g);
        t_err = keep;
        return s;
    }
    *out = g;
    return TC_OK;
}

void tc_graph_destroy(tc_graph* g) { destroy(g); }

tc_status tc_graph_stats(const tc_graph* g, tc_graph_info* info) {
    if (!g || !info) return fail(TC_ERR_ARG, "null argument");
    const GraphStore& s = g->s;
    info->n = s.n;
    info->max_deg = s.max_deg;
    info->arcs = s.arcs;
    info->e_sym = s.e_sym;
    info->mutual = s.mutual;
    info->loops_dropped = s.loops;
    info->dups_dropped = s.dups;
    info->sum_d2 = s.sum_d2;
    info->sum_dv_upper = s.sum_dv_upper;
    info->sum_walk = s.sum_walk;
    info->sum_walk_map = s.sum_walk_map;
    info->sum_tri_walk = s.sum_tri_walk;
    info->bytes_alg_tri = 32ull * (s.n + 1ull) + 60ull * s.e_sym + 4ull * s.sum_tri_walk + 1280ull;
    info->bytes_alg = 16ull * (s.n + 1ull) + 44ull * s.e_sym + 4ull * s.sum_walk + 128ull;
    return TC_OK;
}

tc_status tc_graph_device_csr(const tc_graph* g, const uint64_t** off, const uint32_t** adj,
                              const uint32_t** new_of_old) {
    if (!g) return fail(TC_ERR_ARG, "null graph");
    if (off) *off = g->s.off.as<uint64_t>();
    if (adj) *adj = g->s.adj.as<uint32_t>();
    if (new_of_old) *new_of_old = g->s.new_of_old.as<uint32_t>();
    return TC_OK;
}

tc_status tc_graph_export_csr(const tc_graph* g, uint64_t* off_host, uint32_t* adj_host, uint32_t* new_of_old_host) {
    if (!g) return fail(TC_ERR_ARG, "null graph");
    const GraphStore& s = g->s;
    TC_CUDA(cudaDeviceSynchronize());
    if (off_host) TC_CUDA(cudaMemcpy(off_host, s.off.p, sizeof(uint64_t) * (s.n + 1ull), cudaMemcpyDeviceToHost));
    if (adj_host && s.e_sym) TC_CUDA(cudaMemcpy(adj_host, s.adj.p, sizeof(uint32_t) * 2ull * s.e_sym, cudaMemcpyDeviceToHost));
    if (new_of_old_host && s.n) TC_CUDA(cudaMemcpy(new_of_old_host, s.new_of_old.p, sizeof(uint32_t) * s.n, cudaMemcpyDeviceToHost));
    return TC_OK;
}

tc_u128 tc_null_count(uint32_t n, const uint64_t counts16[16]) {
    unsigned __int128 sum = 0;
    for (int t = 1; t < 16; ++t) sum += counts16[t];
    return to_u128(choose3(n) - sum);
}

tc_status tc_census_async(tc_graph* g, void* stream, const tc_options* opt, uint64_t* d_out16) {
    if (!g || !d_out16) return fail(TC_ERR_ARG, "null argument");
    cudaStream_t st = (cudaStream_t)stream;
    Opts o;
    TC_TRY(resolve_opts(opt, &g->s.opts, &o));
    std::unique_lock<std::mutex> lk(g->s.busy, std::try_to_lock);
    if (!lk.owns_lock()) return fail(TC_ERR_BUSY, "graph is in use by another call");
    census_fit_chunk(g->s, o);
    Plan* p = nullptr;
    TC_TRY(get_plan(g->s, o, st, &p));
    TC_CUDA(cudaMemsetAsync(d_out16, 0, sizeof(uint64_t) * 16, st));
    return census_enqueue(g->s, o, *p, st, reinterpret_cast<unsigned long long*>(d_out16));
}

tc_status tc_census_profile(tc_graph* g, void* stream, const tc_options* opt, uint64_t* d_out16, uint64_t* d_vcost,
                            uint64_t* d_phase) {
    if (!g || !d_out16 || !d_vcost) return fail(TC_ERR_ARG, "null argument");
    cudaStream_t st = (cudaStream_t)stream;
    Opts o;
    TC_TRY(resolve_opts(opt, &g->s.opts, &o));
    std::unique_lock<std::mutex> lk(g->s.busy, std::try_to_lock);
    if (!lk.owns_lock()) return fail(TC_ERR_BUSY, "graph is in use by another call");
    census_fit_chunk(g->s, o);
    Plan* p = nullptr;
    TC_TRY(get_plan(g->s, o, st, &p));
    TC_CUDA(cudaMemsetAsync(d_out16, 0, sizeof(uint64_t) * 16, st));
    return census_enqueue(g->s, o, *p, st, reinterpret_cast<unsigned long long*>(d_out16),
                          reinterpret_cast<unsigned long long*>(d_vcost), reinterpret_cast<unsigned long long*>(d_phase));
}

tc_status tc_census_shard(tc_graph* g, void* stream, const tc_options* opt, uint32_t rank, uint32_t world,
                          uint64_t* d_out16) {
    if (!g || !d_out16) return fail(TC_ERR_ARG, "null argument");
    if (world == 0 || rank >= world) return fail(TC_ERR_ARG, "tc_census_shard: need 0 <= rank < world");
    if (world > (1u << 20)) return fail(TC_ERR_RANGE, "tc_census_shard: world above 2^20");
    cudaStream_t st = (cudaStream_t)stream;
    Opts o;
    TC_TRY(resolve_opts(opt, &g->s.opts, &o));
    std::unique_lock<std::mutex> lk(g->s.busy, std::try_to_lock);
    if (!lk.owns_lock()) return fail(TC_ERR_BUSY, "graph is in use by another call");
    census_fit_chunk(g->s, o);
    Plan* p = nullptr;
    TC_TRY(get_plan(g->s, o, st, &p));
    TC_TRY(plan_shards(g->s, o, *p, world, st));
    const uint32_t* b = p->shard_bounds.data();
    const uint32_t i0 = b[2 * rank], i1 = b[2 * rank + 2];
    const uint32_t v0 = b[2 * rank + 1], v1 = b[2 * rank + 3];
    TC_CUDA(cudaMemsetAsync(d_out16, 0, sizeof(uint64_t) * 16, st));
    return census_enqueue_range(g->s, o, p->items.as<Item>() + i0, i1 - i0, p->warp_begin + v0, p->warp_begin + v1, st,
                                reinterpret_cast<unsigned long long*>(d_out16));
}

tc_status tc_census_shard_bounds(tc_graph* g, void* stream, const tc_options* opt, uint32_t world, uint32_t* bounds) {
    if (!g || !bounds) return fail(TC_ERR_ARG, "null argument");
    if (world == 0) return fail(TC_ERR_ARG, "tc_census_shard_bounds: world must be >= 1");
    if (world > (1u << 20)) return fail(TC_ERR_RANGE, "tc_census_shard_bounds: world above 2^20");
    cudaStream_t st = (cudaStream_t)stream;
    Opts o;
    TC_TRY(resolve_opts(opt, &g->s.opts, &o));
    std::unique_lock<std::mutex> lk(g->s.busy, std::try_to_lock);
    if (!lk.owns_lock()) return fail(TC_ERR_BUSY, "graph is in use by another call");
    census_fit_chunk(g->s, o);
    Plan* p = nullptr;
    TC_TRY(get_plan(g->s, o, st, &p));
    TC_TRY(plan_shards(g->s, o, *p, world, st));
    for (uint32_t r = 0; r <= world; ++r) {
        bounds[2 * r] = p->shard_bounds[2 * r];
        bounds[2 * r + 1] = p->warp_begin + p->shard_bounds[2 * r + 1];
    }
    return TC_OK;
}

uint32_t tc_census_grid(const tc_options* opt) {
    Opts o;
    if (resolve_opts(opt, nullptr, &o) != TC_OK) return 0;
    return (uint32_t)census_grid(o);
}

tc_status tc_census_opts(tc_graph* g, void* stream, const tc_options* opt, tc_u128 out[16]) {
    if (!g || !out) return fail(TC_ERR_ARG, "null argument");
    cudaStream_t st = (cudaStream_t)stream;
    Opts o;
    TC_TRY(resolve_opts(opt, &g->s.opts, &o));
    std::unique_lock<std::mutex> lk(g->s.busy, std::try_to_lock);
    if (!lk.owns_lock()) return fail(TC_ERR_BUSY, "graph is in use by another call");
    census_fit_chunk(g->s, o);
    Plan* p = nullptr;
    TC_TRY(get_plan(g->s, o, st, &p));
    TC_CUDA(cudaMemsetAsync(g->s.acc.p, 0, sizeof(unsigned long long) * 16, st));
    TC_TRY(census_enqueue(g->s, o, *p, st, g->s.acc.as<unsigned long long>()));
    TC_CUDA(cudaMemcpyAsync(g->s.h_counts, g->s.acc.p, sizeof(unsigned long long) * 16, cudaMemcpyDeviceToHost, st));
    TC_CUDA(cudaStreamSynchronize(st));
    uint64_t c[16];
    for (int t = 0; t < 16; ++t) c[t] = g->s.h_counts[t];
    c[0] = 0;
    out[0] = tc_null_count(g->s.n, c);
    for (int t = 1; t < 16; ++t) { out[t].lo = c[t]; out[t].hi = 0; }
    return TC_OK;
}

tc_status tc_census(tc_graph* g, void* stream, tc_u128 out[16]) { return tc_census_opts(g, stream, nullptr, out); }

}  // extern "C"
