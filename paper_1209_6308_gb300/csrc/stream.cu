// stream.cu - interval census over a stream of timestamped arcs: the census of the network
// formed by the arcs of a sliding time window, taken at chosen times (the paper's monitoring
// application, Sec. 3, runs the census at fixed intervals to watch how the triad mix moves).
//
// The arcs of the window live in device memory in arrival order (src and dst arrays); their
// times stay on the host, where they only serve to find the window's bounds.  A push copies the
// new arcs to the device once; a census takes the window's contiguous range, builds the graph
// from it on the device (loops and repeated arcs dropped, Sec. 6 CSR, per-pair tables) and
// runs the Fig. 5 census on it; afterwards arcs older than the window are dropped by moving the
// start of the live range.  The buffer grows by doubling and is compacted when its free tail
// runs out, so pushes cost O(1) amortised device copies.
#include <algorithm>
#include <cstring>
#include <vector>

#include "graph.cuh"

struct tc_stream {
    uint32_t n = 0;
    uint64_t window = 0;
    tc_options opt;
    bool has_opt = false;
    cudaStream_t st = nullptr;
    tc::DevBuf src, dst;             // capacity cap; live arcs at [lo, hi)
    uint64_t cap = 0, lo = 0, hi = 0;
    std::vector<uint64_t> t;         // times of positions [lo, hi), t[i - lo]
    uint64_t last_t = 0, last_census = 0;
    bool any_push = false, any_census = false;
    uint64_t censuses = 0;
};

namespace tc {
namespace {

// Make room for `extra` more arcs after hi: compact the live range to the front of a buffer
// at least twice its new size.
tc_status reserve(tc_stream* s, uint64_t extra) {
    const uint64_t live = s->hi - s->lo;
    if (s->hi + extra <= s->cap) return TC_OK;
    uint64_t ncap = std::max<uint64_t>(1024, 2 * (live + extra));
    DevBuf ns, nd;
    TC_TRY(ns.alloc_persistent(sizeof(uint32_t) * ncap));
    TC_TRY(nd.alloc_persistent(sizeof(uint32_t) * ncap));
    if (live) {
        TC_CUDA(cudaMemcpyAsync(ns.p, s->src.as<uint32_t>() + s->lo, sizeof(uint32_t) * live, cudaMemcpyDeviceToDevice, s->st));
        TC_CUDA(cudaMemcpyAsync(nd.p, s->dst.as<uint32_t>() + s->lo, sizeof(uint32_t) * live, cudaMemcpyDeviceToDevice, s->st));
    }
    TC_CUDA(cudaStreamSynchronize(s->st));
    std::swap(s->src.p, ns.p);
    std::swap(s->src.bytes, ns.bytes);
    std::swap(s->dst.p, nd.p);
    std::swap(s->dst.bytes, nd.bytes);
    s->cap = ncap;
    s->lo = 0;
    s->hi = live;
    return TC_OK;
}

}  // namespace
}  // namespace tc

using namespace tc;

extern "C" {

tc_status tc_stream_create(uint32_t n, uint64_t window, const tc_options* opt, void* stream, tc_stream** out) {
    if (!out) return fail(TC_ERR_ARG, "null argument");
    *out = nullptr;
    if (n > (1u << 30)) return fail(TC_ERR_RANGE, "n > 2^30 (ids carry two direction bits)");
    if (window == 0) return fail(TC_ERR_ARG, "window must be positive");
    Opts check;
    TC_TRY(resolve_opts(opt, nullptr, &check));
    tc_stream* s = new tc_stream();
    s->n = n;
    s->window = window;
    s->st = (cudaStream_t)stream;
    if (opt) {
        s->opt = *opt;
        s->has_opt = true;
    }
    *out = s;
    return TC_OK;
}

tc_status tc_stream_push(tc_stream* s, uint64_t m, const uint32_t* src, const uint32_t* dst, const uint64_t* t) {
    if (!s) return fail(TC_ERR_ARG, "null argument");
    if (m == 0) return TC_OK;
    if (!src || !dst || !t) return fail(TC_ERR_ARG, "src/dst/t is null");
    uint64_t prev = s->any_push ? s->last_t : 0;
    for (uint64_t i = 0; i < m; ++i) {
        if (t[i] < prev) return fail(TC_ERR_ARG, "arc times must not decrease");
        if (src[i] >= s->n || dst[i] >= s->n) return fail(TC_ERR_RANGE, "vertex id >= n");
        prev = t[i];
    }
    TC_TRY(reserve(s, m));
    TC_CUDA(cudaMemcpyAsync(s->src.as<uint32_t>() + s->hi, src, sizeof(uint32_t) * m, cudaMemcpyHostToDevice, s->st));
    TC_CUDA(cudaMemcpyAsync(s->dst.as<uint32_t>() + s->hi, dst, sizeof(uint32_t) * m, cudaMemcpyHostToDevice, s->st));
    TC_CUDA(cudaStreamSynchronize(s->st));   // the caller's host arrays may be reused at return
    s->t.insert(s->t.end(), t, t + m);
    s->hi += m;
    s->last_t = prev;
    s->any_push = true;
    return TC_OK;
}

tc_status tc_stream_census(tc_stream* s, uint64_t t_now, tc_u128 out[16], uint64_t* arcs_in_window) {
    if (!s || !out) return fail(TC_ERR_ARG, "null argument");
    if (s->any_census && t_now < s->last_census) return fail(TC_ERR_ARG, "census times must not decrease");
    // window (t_now - window, t_now]: positions [a, b) of the live range
    const uint64_t t0 = t_now >= s->window ? t_now - s->window : 0;
    const bool from_zero = t_now < s->window;   // the window reaches back past time 0
    auto first_after = [&](uint64_t x) {
        return (uint64_t)(std::upper_bound(s->t.begin(), s->t.end(), x) - s->t.begin());
    };
    const uint64_t a = from_zero ? 0 : first_after(t0), b = first_after(t_now);
    const uint64_t m = b > a ? b - a : 0;
    tc_graph* g = nullptr;
    TC_TRY(tc_graph_create_arcs(s->n, m, m ? s->src.as<uint32_t>() + s->lo + a : nullptr,
                                m ? s->dst.as<uint32_t>() + s->lo + a : nullptr, 1, s->st,
                                s->has_opt ? &s->opt : nullptr, &g));
    const tc_status cs = tc_census_opts(g, s->st, s->has_opt ? &s->opt : nullptr, out);
    tc_graph_destroy(g);
    TC_TRY(cs);
    if (arcs_in_window) *arcs_in_window = m;
    // later censuses start no earlier than this window: drop the arcs before it
    if (a) {
        s->t.erase(s->t.begin(), s->t.begin() + a);
        s->lo += a;
        if (s->lo == s->hi) s->lo = s->hi = 0;
    }
    s->last_census = t_now;
    s->any_census = true;
    s->censuses++;
    return TC_OK;
}

tc_status tc_stream_stats(const tc_stream* s, uint64_t* live_arcs, uint64_t* capacity, uint64_t* censuses) {
    if (!s) return fail(TC_ERR_ARG, "null argument");
    if (live_arcs) *live_arcs = s->hi - s->lo;
    if (capacity) *capacity = s->cap;
    if (censuses) *censuses = s->censuses;
    return TC_OK;
}

void tc_stream_destroy(tc_stream* s) {
    if (!s) return;
    if (s->st) cudaStreamSynchronize(s->st);
    delete s;
}

}  // extern "C"
