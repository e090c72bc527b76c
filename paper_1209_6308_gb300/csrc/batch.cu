// batch.cu - census of many graphs in one persistent launch (the batched form of the Fig. 5
// census), with its combined work plan built on the device, the launch captured once in a
// CUDA graph and replayed, and an autotuner for the tile and tier thresholds.
//
// Plan: the graphs are ordered by size (largest first, so the longest items start first);
// each graph's vertices with degree above the warp-tier threshold become CTA items exactly as
// in the single-graph plan, tagged with the graph index, and its remaining active vertices
// become (u0, u1, graph) blocks of 32 for the one-warp-per-vertex tier.  One launch runs
// every item of every graph, then every block, from two device-side work counters.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <numeric>
#include <vector>

#include "graph.cuh"
#include "plan.cuh"

namespace tc {
namespace {

__device__ __forceinline__ uint32_t graph_of(const uint64_t* __restrict__ pre, uint32_t k, uint64_t i) {
    uint32_t lo = 0, hi = k;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (pre[mid] <= i) lo = mid; else hi = mid;
    }
    return lo;
}

// wide[g] = vertices of graph g with degree > warp_max (a prefix of its ids)
__global__ void k_batch_wide(const GraphDev* __restrict__ gs, const uint64_t* __restrict__ voff, uint32_t k,
                             uint64_t total, uint32_t warp_max, uint32_t* wide) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < total; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t g = graph_of(voff, k, i);
        const uint64_t x = i - voff[g];
        const uint64_t* off = gs[g].off;
        if (off[x + 1] - off[x] > warp_max) atomicAdd(&wide[g], 1u);
    }
}

// Items of every wide vertex of every graph (plan.cuh), one warp per vertex, tagged with the
// graph index; the same splitting as the single-graph plain plan.
__global__ void k_batch_work(const GraphDev* __restrict__ gs, const uint64_t* __restrict__ woff, uint32_t k,
                             uint64_t total, uint32_t chunk, int algo, unsigned long long* W, unsigned long long* sum) {
    const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long acc = 0;
    for (uint64_t i = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; i < total; i += warps) {
        const uint32_t g = graph_of(woff, k, i);
        const GraphDev G = gs[g];
        const unsigned long long w = vertex_units(G, (uint32_t)(i - woff[g]), chunk, algo);
        acc += w;
        if ((threadIdx.x & 31) == 0) W[i] = w;
    }
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(sum, acc);
}

__global__ void k_batch_count(const GraphDev* __restrict__ gs, const uint64_t* __restrict__ woff, uint32_t k,
                              uint64_t total, uint32_t chunk, uint32_t item_work, int algo,
                              const unsigned long long* __restrict__ W, uint32_t* cnt) {
    const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t i = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; i < total; i += warps) {
        const uint32_t g = graph_of(woff, k, i);
        const GraphDev G = gs[g];
        const uint32_t x = (uint32_t)(i - woff[g]);
        const uint64_t ubase = G.off[x];
        const uint32_t du = (uint32_t)(G.off[x + 1] - ubase), upx = G.up[x], chunks = (du + chunk - 1) / chunk;
        const uint32_t c = plan_vertex(G, x, item_work, 0.0, W[i],
                                       [&](uint32_t j) { return pair_units(G, x, ubase, du, upx, j, chunks, algo); },
                                       [](uint32_t, uint32_t) {});
        if ((threadIdx.x & 31) == 0) cnt[i] = c;
    }
}

__global__ void k_batch_emit(const GraphDev* __restrict__ gs, const uint64_t* __restrict__ woff, uint32_t k,
                             uint64_t total, uint32_t chunk, uint32_t item_work, int algo,
                             const unsigned long long* __restrict__ W, const uint32_t* __restrict__ pos, Item* items) {
    const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t i = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; i < total; i += warps) {
        const uint32_t g = graph_of(woff, k, i);
        const GraphDev G = gs[g];
        const uint32_t x = (uint32_t)(i - woff[g]);
        Item* out = items + pos[i];
        const uint64_t ubase = G.off[x];
        const uint32_t du = (uint32_t)(G.off[x + 1] - ubase), upx = G.up[x], chunks = (du + chunk - 1) / chunk;
        const uint32_t c = plan_vertex(G, x, item_work, 0.0, W[i],
                                       [&](uint32_t j) { return pair_units(G, x, ubase, du, upx, j, chunks, algo); },
                                       [&](uint32_t j, uint32_t rank) { out[rank] = Item{x, j, 0u, g}; });
        plan_ends(out, c, (uint32_t)(G.off[x + 1] - G.off[x]));
    }
}

__global__ void k_batch_scatter(const unsigned long long* __restrict__ src, const uint32_t* __restrict__ order,
                                uint32_t k, unsigned long long* dst) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < 16ull * k; i += (uint64_t)gridDim.x * blockDim.x)
        dst[16ull * order[i / 16] + (i % 16)] = src[i];
}

}  // namespace

struct BatchStore {
    uint32_t k = 0;
    std::vector<tc_graph*> graphs;      // in launch order (largest first)
    std::vector<uint32_t> order;        // launch position -> caller's index
    Opts opts;
    cudaStream_t cap = nullptr;         // stream used only to capture the launch
    DevBuf d_graphs, d_voff, d_woff, d_wide, d_order, items, wblocks, ctr, out;
    DevBuf tri;                         // triangle form: 96 uint64 of scratch per graph
    uint32_t n_items = 0, n_wblocks = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    unsigned long long* h_out = nullptr;
    std::vector<uint64_t> woff_h;
    std::vector<tc_autotune_trial> history;   // the last autotune's trials, in order

    ~BatchStore() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (h_out) cudaFreeHost(h_out);
        if (cap) cudaStreamDestroy(cap);
    }
};

namespace {

// (Re)build the combined plan for b.opts and capture its launch.
tc_status batch_plan(BatchStore& b, cudaStream_t st) {
    const Opts& o = b.opts;
    const uint32_t k = b.k;
    if (b.exec) { cudaGraphExecDestroy(b.exec); b.exec = nullptr; }
    if (b.graph) { cudaGraphDestroy(b.graph); b.graph = nullptr; }
    // per-graph vertex prefix and wide counts
    std::vector<uint64_t> voff(k + 1, 0);
    for (uint32_t i = 0; i < k; ++i) voff[i + 1] = voff[i] + b.graphs[i]->s.n;
    TC_TRY(b.d_voff.alloc_persistent(sizeof(uint64_t) * (k + 1)));
    TC_CUDA(cudaMemcpyAsync(b.d_voff.p, voff.data(), sizeof(uint64_t) * (k + 1), cudaMemcpyHostToDevice, st));
    TC_TRY(b.d_wide.alloc_persistent(sizeof(uint32_t) * k));
    TC_CUDA(cudaMemsetAsync(b.d_wide.p, 0, sizeof(uint32_t) * k, st));
    if (voff[k]) {
        k_batch_wide<<<grid_for(voff[k], 256, 1u << 16), 256, 0, st>>>(b.d_graphs.as<GraphDev>(), b.d_voff.as<uint64_t>(),
                                                                      k, voff[k], o.warp_max_deg, b.d_wide.as<uint32_t>());
        TC_LAUNCH("k_batch_wide");
    }
    std::vector<uint32_t> wide(k);
    TC_CUDA(cudaMemcpyAsync(wide.data(), b.d_wide.p, sizeof(uint32_t) * k, cudaMemcpyDeviceToHost, st));
    TC_CUDA(cudaStreamSynchronize(st));
    // CTA items of the wide vertices of every graph
    b.woff_h.assign(k + 1, 0);
    for (uint32_t i = 0; i < k; ++i) b.woff_h[i + 1] = b.woff_h[i] + wide[i];
    const uint64_t total_w = b.woff_h[k];
    TC_TRY(b.d_woff.alloc_persistent(sizeof(uint64_t) * (k + 1)));
    TC_CUDA(cudaMemcpyAsync(b.d_woff.p, b.woff_h.data(), sizeof(uint64_t) * (k + 1), cudaMemcpyHostToDevice, st));
    b.n_items = 0;
    if (total_w) {
        if (total_w >= (1ull << 32)) return fail(TC_ERR_RANGE, "batch has too many wide vertices");
        DevBuf cnt, pos, tot, wv, wt;
        TC_TRY(cnt.alloc(sizeof(uint32_t) * total_w, st));
        TC_TRY(pos.alloc(sizeof(uint32_t) * total_w, st));
        TC_TRY(tot.alloc(sizeof(uint32_t), st));
        TC_TRY(wv.alloc(sizeof(unsigned long long) * total_w, st));
        TC_TRY(wt.alloc(sizeof(unsigned long long), st));
        TC_CUDA(cudaMemsetAsync(wt.p, 0, sizeof(unsigned long long), st));
        const unsigned pgrid = grid_for(total_w * 32, 256, 1u << 16);
        k_batch_work<<<pgrid, 256, 0, st>>>(b.d_graphs.as<GraphDev>(), b.d_woff.as<uint64_t>(), k, total_w, o.chunk,
                                            (int)o.algo, wv.as<unsigned long long>(), wt.as<unsigned long long>());
        TC_LAUNCH("k_batch_work");
        unsigned long long total_units = 0;
        TC_CUDA(cudaMemcpyAsync(&total_units, wt.p, sizeof(total_units), cudaMemcpyDeviceToHost, st));
        TC_CUDA(cudaStreamSynchronize(st));
        const uint32_t iw = o.item_work ? o.item_work : adaptive_item_work(total_units, (unsigned)census_grid(o));
        k_batch_count<<<pgrid, 256, 0, st>>>(b.d_graphs.as<GraphDev>(), b.d_woff.as<uint64_t>(), k, total_w, o.chunk,
                                             iw, (int)o.algo, wv.as<unsigned long long>(), cnt.as<uint32_t>());
        TC_LAUNCH("k_batch_count");
        TC_TRY(scan_u32(cnt.as<uint32_t>(), pos.as<uint32_t>(), total_w, tot.as<uint32_t>(), st));
        TC_CUDA(cudaMemcpyAsync(&b.n_items, tot.p, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
        TC_CUDA(cudaStreamSynchronize(st));
        TC_TRY(b.items.alloc_persistent(sizeof(Item) * (b.n_items ? b.n_items : 1)));
        if (b.n_items) {
            k_batch_emit<<<pgrid, 256, 0, st>>>(b.d_graphs.as<GraphDev>(), b.d_woff.as<uint64_t>(), k, total_w, o.chunk,
                                                iw, (int)o.algo, wv.as<unsigned long long>(), pos.as<uint32_t>(),
                                                b.items.as<Item>());
            TC_LAUNCH("k_batch_emit");
        }
        TC_CUDA(cudaStreamSynchronize(st));
    } else {
        TC_TRY(b.items.alloc_persistent(sizeof(Item)));
    }
    // warp-tier blocks (32 vertices each) of every graph
    std::vector<uint4> wb;
    for (uint32_t i = 0; i < k; ++i) {
        const uint32_t act = b.graphs[i]->s.n_active;
        for (uint32_t u = wide[i]; u < act; u += 32) wb.push_back(make_uint4(u, std::min(u + 32u, act), i, 0u));
    }
    b.n_wblocks = (uint32_t)wb.size();
    TC_TRY(b.wblocks.alloc_persistent(sizeof(uint4) * (wb.empty() ? 1 : wb.size())));
    if (!wb.empty())
        TC_CUDA(cudaMemcpyAsync(b.wblocks.p, wb.data(), sizeof(uint4) * wb.size(), cudaMemcpyHostToDevice, st));
    TC_CUDA(cudaStreamSynchronize(st));
    // capture: zero counters and outputs, launch
    if (o.algo == TC_ALGO_TRIANGLE) {
        if (!b.tri.p) TC_TRY(b.tri.alloc_persistent(sizeof(unsigned long long) * 96ull * (k ? k : 1)));
    } else {
        TC_TRY(census_prepare(st, o));
    }
    TC_CUDA(cudaStreamBeginCapture(b.cap, cudaStreamCaptureModeThreadLocal));
    tc_status s = TC_OK;
    if (cudaMemsetAsync(b.ctr.p, 0, sizeof(uint32_t) * 4, b.cap) != cudaSuccess ||
        cudaMemsetAsync(b.out.p, 0, sizeof(unsigned long long) * 16ull * k, b.cap) != cudaSuccess)
        s = fail(TC_ERR_CUDA, "batch capture: memset failed");
    if (s == TC_OK && o.algo == TC_ALGO_TRIANGLE)
        s = triangle_census_batch(b.d_graphs.as<GraphDev>(), k, b.items.as<Item>(), b.n_items, b.wblocks.as<uint4>(),
                                  b.n_wblocks, o, b.ctr.as<uint32_t>(), b.tri.as<unsigned long long>(),
                                  b.out.as<unsigned long long>(), b.cap);
    else if (s == TC_OK)
        s = census_launch_batch(b.d_graphs.as<GraphDev>(), b.items.as<Item>(), b.n_items, b.wblocks.as<uint4>(),
                                b.n_wblocks, o, b.ctr.as<uint32_t>(), b.out.as<unsigned long long>(), b.cap);
    cudaGraph_t gph = nullptr;
    cudaError_t e = cudaStreamEndCapture(b.cap, &gph);
    if (s != TC_OK) {
        if (gph) cudaGraphDestroy(gph);
        return s;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    b.graph = gph;
    TC_CUDA(cudaGraphInstantiate(&b.exec, b.graph, 0));
    return TC_OK;
}

tc_status batch_run(BatchStore& b, cudaStream_t st) {
    if (b.k == 0) return TC_OK;
    TC_CUDA(cudaGraphLaunch(b.exec, st));
    return TC_OK;
}

}  // namespace
}  // namespace tc

struct tc_batch {
    tc::BatchStore s;
};

using namespace tc;

extern "C" {

tc_status tc_batch_create(tc_graph* const* gs, uint32_t k, const tc_options* opt, void* stream, tc_batch** out) {
    if (!out || (k && !gs)) return fail(TC_ERR_ARG, "null argument");
    *out = nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    tc_batch* b = new tc_batch();
    BatchStore& B = b->s;
    B.k = k;
    tc_status s = resolve_opts(opt, nullptr, &B.opts);
    for (uint32_t i = 0; s == TC_OK && i < k; ++i)
        if (!gs[i]) s = fail(TC_ERR_ARG, "null graph in batch");
    if (s == TC_OK) {
        B.order.resize(k);
        std::iota(B.order.begin(), B.order.end(), 0u);
        std::stable_sort(B.order.begin(), B.order.end(),
                         [&](uint32_t a, uint32_t c) { return gs[a]->s.e_sym > gs[c]->s.e_sym; });
        for (uint32_t i = 0; i < k; ++i) B.graphs.push_back(gs[B.order[i]]);
        std::vector<GraphDev> gd(k);
        for (uint32_t i = 0; i < k; ++i) gd[i] = B.graphs[i]->s.dev();
        s = B.d_graphs.alloc_persistent(sizeof(GraphDev) * (k ? k : 1));
        if (s == TC_OK && k && cudaMemcpy(B.d_graphs.p, gd.data(), sizeof(GraphDev) * k, cudaMemcpyHostToDevice) != cudaSuccess)
            s = fail(TC_ERR_CUDA, "batch: upload of graph table failed");
        if (s == TC_OK) s = B.d_order.alloc_persistent(sizeof(uint32_t) * (k ? k : 1));
        if (s == TC_OK && k &&
            cudaMemcpy(B.d_order.p, B.order.data(), sizeof(uint32_t) * k, cudaMemcpyHostToDevice) != cudaSuccess)
            s = fail(TC_ERR_CUDA, "batch: upload of graph order failed");
        if (s == TC_OK) s = B.ctr.alloc_persistent(sizeof(uint32_t) * 4);
        if (s == TC_OK) s = B.out.alloc_persistent(sizeof(unsigned long long) * 16ull * (k ? k : 1));
        if (s == TC_OK && cudaMallocHost(&B.h_out, sizeof(unsigned long long) * 16ull * (k ? k : 1)) != cudaSuccess)
            s = fail(TC_ERR_OOM, "batch: pinned host buffer");
        if (s == TC_OK && cudaStreamCreateWithFlags(&B.cap, cudaStreamNonBlocking) != cudaSuccess)
            s = fail(TC_ERR_CUDA, "batch: capture stream");
        if (s == TC_OK && k) s = batch_plan(B, st);
    }
    if (s != TC_OK) {
        std::string keep = tc_last_error();
        delete b;
        set_error(keep);
        return s;
    }
    *out = b;
    return TC_OK;
}

tc_status tc_batch_census_async(tc_batch* b, void* stream, uint64_t* d_out16xk) {
    if (!b) return fail(TC_ERR_ARG, "null batch");
    cudaStream_t st = (cudaStream_t)stream;
    TC_TRY(batch_run(b->s, st));
    if (d_out16xk && b->s.k) {
        // the launch writes in size order; scatter back to the caller's order
        k_batch_scatter<<<grid_for(16ull * b->s.k, 256, 4096), 256, 0, st>>>(
            b->s.out.as<unsigned long long>(), b->s.d_order.as<uint32_t>(), b->s.k,
            reinterpret_cast<unsigned long long*>(d_out16xk));
        TC_LAUNCH("k_batch_scatter");
    }
    return TC_OK;
}

tc_status tc_batch_census(tc_batch* b, void* stream, uint64_t* out16xk, tc_u128* out003_k) {
    if (!b || !out16xk) return fail(TC_ERR_ARG, "null argument");
    BatchStore& B = b->s;
    cudaStream_t st = (cudaStream_t)stream;
    if (B.k == 0) return TC_OK;
    TC_TRY(batch_run(B, st));
    TC_CUDA(cudaMemcpyAsync(B.h_out, B.out.p, sizeof(unsigned long long) * 16ull * B.k, cudaMemcpyDeviceToHost, st));
    TC_CUDA(cudaStreamSynchronize(st));
    for (uint32_t i = 0; i < B.k; ++i) {
        uint64_t* c = out16xk + 16ull * B.order[i];
        for (int t = 0; t < 16; ++t) c[t] = B.h_out[16ull * i + t];
        c[0] = 0;
        tc_u128 z = tc_null_count(B.graphs[i]->s.n, c);
        c[0] = z.lo;
        if (out003_k) out003_k[B.order[i]] = z;
    }
    return TC_OK;
}

namespace {

tc_options to_options(const Opts& o) {
    tc_options t;
    std::memset(&t, 0, sizeof(t));
    t.algo = o.algo;
    t.schedule = o.schedule;
    t.warp_max_deg = o.warp_max_deg;
    t.chunk_entries = o.chunk;
    t.item_work = o.item_work;
    t.ctas_per_sm = o.ctas_per_sm;
    return t;
}

bool valid_batch_opts(const Opts& o) {
    const uint32_t max_chunk = o.algo == TC_ALGO_UNION ? 16384u : 8192u;
    if (o.algo == TC_ALGO_TRIANGLE && o.warp_max_deg > 128) return false;
    return o.chunk >= 512 && o.chunk <= max_chunk && o.warp_max_deg <= o.chunk / 8 && o.ctas_per_sm >= 1 &&
           o.ctas_per_sm <= 8;
}

}  // namespace

tc_status tc_batch_autotune(tc_batch* b, void* stream, uint32_t max_trials, tc_options* best_out, float* best_ms) {
    if (!b) return fail(TC_ERR_ARG, "null batch");
    BatchStore& B = b->s;
    cudaStream_t st = (cudaStream_t)stream;
    B.history.clear();
    if (B.k == 0) return TC_OK;
    const Opts base = B.opts;
    cudaEvent_t e0, e1;
    TC_CUDA(cudaEventCreate(&e0));
    TC_CUDA(cudaEventCreate(&e1));
    tc_status s = TC_OK;
    // median of three timed replays after one untimed one; +inf when the plan cannot be made
    auto measure = [&](const Opts& o, float* ms) -> tc_status {
        *ms = 1e30f;
        if (!valid_batch_opts(o)) return TC_OK;
        B.opts = o;
        tc_status r = batch_plan(B, st);
        if (r == TC_ERR_ARG) return TC_OK;   // e.g. shared memory beyond this GPU's limit
        if (r != TC_OK) return r;
        float ts[3];
        for (int k = 0; k < 4; ++k) {
            if (cudaEventRecord(e0, st) != cudaSuccess) return fail(TC_ERR_CUDA, "event");
            TC_TRY(batch_run(B, st));
            if (cudaEventRecord(e1, st) != cudaSuccess) return fail(TC_ERR_CUDA, "event");
            if (cudaEventSynchronize(e1) != cudaSuccess) return fail(TC_ERR_CUDA, "event sync");
            if (k > 0) cudaEventElapsedTime(&ts[k - 1], e0, e1);
        }
        std::sort(ts, ts + 3);
        *ms = ts[1];
        B.history.push_back({to_options(o), ts[1]});
        return TC_OK;
    };
    // coordinate descent from the current options: each pass varies one threshold at a time
    // over its range, keeping the best value found, until a pass improves nothing by 1% or the
    // trial budget (0 = none) is spent
    Opts best_o = base;
    float best = 1e30f;
    s = measure(base, &best);
    uint32_t trials = 1;
    for (int pass = 0; s == TC_OK && pass < 3; ++pass) {
        const float pass_start = best;
        for (int dim = 0; dim < 5 && s == TC_OK; ++dim) {
            std::vector<uint32_t> vals;
            if (dim == 0) vals = {TC_ALGO_UNION, TC_ALGO_SUFFIX, TC_ALGO_TRIANGLE};
            if (dim == 1) vals = {16u, 32u, 64u, 128u, 256u};
            if (dim == 2) vals = {1024u, 2048u, 4096u, 8192u};
            if (dim == 3) vals = {2u, 3u, 4u, 6u, 8u};
            if (dim == 4) vals = {0u, 1u << 14, 1u << 16, 1u << 18, 1u << 20, 1u << 22};
            for (uint32_t v : vals) {
                if (max_trials && trials >= max_trials) break;
                Opts o = best_o;
                if (dim == 0) o.algo = v;
                if (dim == 1) o.warp_max_deg = v;
                if (dim == 2) o.chunk = v;
                if (dim == 3) o.ctas_per_sm = v;
                if (dim == 4) o.item_work = v;
                if (o == best_o) continue;
                bool seen = false;
                for (const auto& h : B.history) {
                    const tc_options t = to_options(o);
                    seen |= std::memcmp(&h.opts, &t, sizeof(t)) == 0;
                }
                if (seen) continue;
                float ms;
                s = measure(o, &ms);
                ++trials;
                if (s != TC_OK) break;
                if (ms < best) {
                    best = ms;
                    best_o = o;
                }
            }
        }
        if (best > 0.99f * pass_start) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    B.opts = best_o;
    TC_TRY(batch_plan(B, st));
    if (s != TC_OK) return s;
    if (best_out) *best_out = to_options(best_o);
    if (best_ms) *best_ms = best;
    return TC_OK;
}

tc_status tc_batch_autotune_history(const tc_batch* b, tc_autotune_trial* out, uint32_t max, uint32_t* count) {
    if (!b || !count || (max && !out)) return fail(TC_ERR_ARG, "null argument");
    const auto& h = b->s.history;
    const uint32_t c = (uint32_t)std::min<size_t>(h.size(), max);
    for (uint32_t i = 0; i < c; ++i) out[i] = h[i];
    *count = c;
    return TC_OK;
}

tc_status tc_batch_stats(const tc_batch* b, uint32_t* n_items, uint32_t* n_warp_blocks) {
    if (!b) return fail(TC_ERR_ARG, "null batch");
    if (n_items) *n_items = b->s.n_items;
    if (n_warp_blocks) *n_warp_blocks = b->s.n_wblocks;
    return TC_OK;
}

void tc_batch_destroy(tc_batch* b) {
    if (!b) return;
    cudaDeviceSynchronize();
    delete b;
}

// One-shot batched census: build the batch, run it once, destroy it.
tc_status tc_census_batch(tc_graph* const* gs, uint32_t k, void* stream, uint64_t* out16xk, tc_u128* out003_k) {
    if (!gs || !out16xk) return fail(TC_ERR_ARG, "null argument");
    if (k == 0) return TC_OK;
    tc_batch* b = nullptr;
    TC_TRY(tc_batch_create(gs, k, nullptr, stream, &b));
    tc_status s = tc_batch_census(b, stream, out16xk, out003_k);
    tc_batch_destroy(b);
    return s;
}

}  // extern "C"
