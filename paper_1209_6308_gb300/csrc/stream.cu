// stream.cu - interval census over a stream of timestamped arcs: the census of the network
// formed by the arcs of a sliding time window, taken at chosen times (the paper's monitoring
// application, Sec. 3, runs the census at fixed intervals to watch how the triad mix moves).
//
// The arcs of the window live in device memory in arrival order (src and dst arrays); their
// times stay on the host, where they only serve to find the window's bounds.  A push copies the
// new arcs to the device once.  Between censuses the window's arc set is kept up to date on the
// device: the distinct directed arcs of the last window, sorted by key, each with the number of
// times it occurs there.  A census keys only the arcs that entered the window since the last
// one (+1 each) and those that left it (-1 each), sorts those few, nets each key's changes, and
// merges them into the sorted set by binary searches (counts updated in place, new keys placed
// by their ranks, keys whose count fell to zero dropped) - no sort over the whole window.  The
// window's graph is then built from the sorted set (its pairs, degrees, the degree relabel, the
// Sec. 6 CSR and the per-pair tables, which depend on every degree and so are derived afresh)
// and counted by Fig. 5.  When the change is as large as the window itself (the first census,
// or a jump past the whole last window) the set is made from the window's arcs instead.
// Arcs older than the window are then dropped by moving the start of the live range; the
// buffer grows by doubling and is compacted when its free tail runs out, so pushes cost O(1)
// amortised device copies.
#include <algorithm>
#include <cstring>
#include <vector>

#include "graph.cuh"

struct tc_stream {
    uint32_t n = 0;
    int B = 1;                       // id bits of the arc keys
    uint64_t window = 0;
    tc_options opt;
    bool has_opt = false;
    cudaStream_t st = nullptr;
    tc::DevBuf src, dst;             // capacity cap; live arcs at [lo, hi)
    uint64_t cap = 0, lo = 0, hi = 0;
    std::vector<uint64_t> t;         // times of positions [lo, hi) at t[t0 + i - lo]; the dropped
    uint64_t t0 = 0;                 // front t[0, t0) is erased once it is half the vector
    uint64_t last_t = 0, last_census = 0;
    bool any_push = false, any_census = false;
    uint64_t censuses = 0;
    // the arc set of the last window: live positions [lo, lo + nb) as set_len distinct directed
    // arc keys, ascending, with their multiplicities; set_ok is false until a census made it (or
    // after a census failed part way)
    tc::DevBuf set_key, set_cnt;
    uint64_t nb = 0, set_len = 0;
    bool set_ok = false;
    uint64_t rebuilds = 0, repairs = 0, last_added = 0, last_evicted = 0;
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

constexpr int kT = 256;

// Signed keys of the arcs at live positions [add0, add0 + n_add) (entering the window, sign
// bit 0) and [del0, del0 + n_del) (leaving it, sign bit 1): the build's arc key
// (lo << (B+2)) | (hi << 2) | dir shifted up by one over the sign.  Self-loops give all-ones
// keys (counted in *loops), which sort past every arc.
__global__ void k_delta_keys(const uint32_t* src, const uint32_t* dst, uint64_t add0, uint64_t n_add, uint64_t del0,
                             uint64_t n_del, int B, uint64_t* keys, unsigned long long* loops) {
    uint32_t nl = 0;
    const uint64_t total = n_add + n_del;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < total; i += (uint64_t)gridDim.x * blockDim.x) {
        const bool del = i >= n_add;
        const uint64_t p = del ? del0 + (i - n_add) : add0 + i;
        const uint32_t a = src[p], b = dst[p];
        uint64_t key = ~0ull;
        if (a == b) {
            ++nl;
        } else {
            const uint64_t lo = a < b ? a : b, hi = a < b ? b : a;
            key = ((((lo << (B + 2)) | (hi << 2) | (a < b ? 1u : 2u))) << 1) | (del ? 1u : 0u);
        }
        keys[i] = key;
    }
    for (int o = 16; o; o >>= 1) nl += __shfl_xor_sync(0xffffffffu, nl, o);
    if ((threadIdx.x & 31) == 0 && nl) atomicAdd(loops, (unsigned long long)nl);
}

// flag[i] = 1 where the arc key (the signed key without its sign) differs from the one before.
__global__ void k_run_heads(const uint64_t* keys, uint64_t cnt, uint32_t* flag) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < cnt; i += (uint64_t)gridDim.x * blockDim.x)
        flag[i] = (i == 0 || (keys[i] >> 1) != (keys[i - 1] >> 1)) ? 1u : 0u;
}

// Each run -> one arc key and its net change (+1 per entering copy, -1 per leaving one).
__global__ void k_run_net(const uint64_t* keys, uint64_t cnt, const uint32_t* flag, const uint32_t* pos,
                          uint64_t* dkey, int* dnet) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < cnt; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t r = pos[i] + flag[i] - 1u;
        if (flag[i]) dkey[r] = keys[i] >> 1;
        atomicAdd(&dnet[r], (keys[i] & 1u) ? -1 : 1);
    }
}

__device__ __forceinline__ uint64_t lower_bound_key(const uint64_t* a, uint64_t len, uint64_t x) {
    uint64_t lo = 0, hi = len;
    while (lo < hi) {
        const uint64_t mid = (lo + hi) >> 1;
        if (a[mid] < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Apply the net changes of the D changed keys: a key already in the set has its count moved in
// place; a new key is marked (fresh[j] = 1) when its change is positive.  A count that would go
// negative, or a leaving arc that is not in the set, means the set and the window disagree
// (bad[0] is raised and the caller rebuilds the set).
__global__ void k_apply_net(const uint64_t* dkey, const int* dnet, uint64_t D, const uint64_t* skey, uint32_t* scnt,
                            uint64_t S, uint32_t* fresh, unsigned int* bad) {
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < D; j += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t k = dkey[j];
        const int d = dnet[j];
        const uint64_t at = lower_bound_key(skey, S, k);
        uint32_t f = 0;
        if (at < S && skey[at] == k) {
            const long long c = (long long)scnt[at] + d;
            if (c < 0) atomicOr(bad, 1u);
            scnt[at] = c < 0 ? 0u : (uint32_t)c;
        } else if (d > 0) {
            f = 1;
        } else if (d < 0) {
            atomicOr(bad, 1u);
        }
        fresh[j] = f;
    }
}

__global__ void k_kept(const uint32_t* scnt, uint64_t S, uint32_t* kept) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < S; i += (uint64_t)gridDim.x * blockDim.x)
        kept[i] = scnt[i] ? 1u : 0u;
}

// The merged set: kept old keys and fresh keys in one ascending array.  An old key i lands at
// (kept keys before it) + (fresh keys below it); a fresh key j at (fresh keys before it) +
// (kept old keys below it).  kpos / fpos are the exclusive scans of kept / fresh, K / F their
// totals.
__global__ void k_merge_old(const uint64_t* skey, const uint32_t* scnt, uint64_t S, const uint32_t* kpos,
                            const uint64_t* dkey, uint64_t D, const uint32_t* fpos, uint64_t F, uint64_t* okey,
                            uint32_t* ocnt) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < S; i += (uint64_t)gridDim.x * blockDim.x) {
        if (!scnt[i]) continue;
        const uint64_t t = lower_bound_key(dkey, D, skey[i]);
        const uint64_t o = kpos[i] + (t < D ? fpos[t] : F);
        okey[o] = skey[i];
        ocnt[o] = scnt[i];
    }
}

__global__ void k_merge_fresh(const uint64_t* dkey, const int* dnet, const uint32_t* fresh, const uint32_t* fpos,
                              uint64_t D, const uint64_t* skey, uint64_t S, const uint32_t* kpos, uint64_t K,
                              uint64_t* okey, uint32_t* ocnt) {
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < D; j += (uint64_t)gridDim.x * blockDim.x) {
        if (!fresh[j]) continue;
        const uint64_t b = lower_bound_key(skey, S, dkey[j]);
        const uint64_t o = fpos[j] + (b < S ? kpos[b] : K);
        okey[o] = dkey[j];
        ocnt[o] = (uint32_t)dnet[j];
    }
}

// Exclusive scan of `flag` into `pos`; returns the total on the host.
tc_status scan_total(const uint32_t* flag, uint32_t* pos, uint64_t cnt, DevBuf& tot, uint64_t* total, cudaStream_t st) {
    uint32_t h = 0;
    if (cnt) {
        TC_TRY(scan_u32(flag, pos, cnt, tot.as<uint32_t>(), st));
        TC_CUDA(cudaMemcpyAsync(&h, tot.p, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
        TC_CUDA(cudaStreamSynchronize(st));
    }
    *total = h;
    return TC_OK;
}

// Bring the arc set from live positions [0, nb) to [a, b) (relative to lo): key the arcs that
// entered and left, net them per key, merge into the set.
tc_status update_set(tc_stream* s, uint64_t a, uint64_t b) {
    cudaStream_t st = s->st;
    if (!s->set_ok) {
        s->nb = 0;
        s->set_len = 0;
    }
    uint64_t del0 = 0, n_del = std::min(a, s->nb);
    uint64_t add0 = std::max(a, s->nb), n_add = b > add0 ? b - add0 : 0;
    if (n_del == s->nb || n_del + n_add >= b - a) {
        // nothing of the old set survives, or the change is the size of the window: make the
        // set from the window's arcs
        s->set_len = 0;
        n_del = 0;
        add0 = a;
        n_add = b - a;
        s->rebuilds++;
    }
    s->last_added = n_add;
    s->last_evicted = n_del;
    const uint64_t m = n_add + n_del;
    if (m == 0) return TC_OK;
    if (m >= (1ull << 32)) return fail(TC_ERR_RANGE, "more than 2^32-1 arcs entering and leaving the window");
    DevBuf keys, tmp, loops;
    TC_TRY(keys.alloc(sizeof(uint64_t) * m, st));
    TC_TRY(tmp.alloc(sizeof(uint64_t) * m, st));
    TC_TRY(loops.alloc(sizeof(unsigned long long), st));
    TC_CUDA(cudaMemsetAsync(loops.p, 0, sizeof(unsigned long long), st));
    const uint32_t* src = s->src.as<uint32_t>() + s->lo;
    const uint32_t* dst = s->dst.as<uint32_t>() + s->lo;
    k_delta_keys<<<grid_for(m, kT, 1u << 16), kT, 0, st>>>(src, dst, add0, n_add, del0, n_del, s->B,
                                                           keys.as<uint64_t>(), loops.as<unsigned long long>());
    TC_LAUNCH("k_delta_keys");
    uint64_t* kp = keys.as<uint64_t>();
    uint64_t* tp = tmp.as<uint64_t>();
    // sort by the arc key (bits 1 .. 2B+2); the sign bit stays unsorted within a run
    TC_TRY(radix_sort_u64(&kp, &tp, m, 1, 2 * s->B + 3, st));
    unsigned long long nloops = 0;
    TC_CUDA(cudaMemcpyAsync(&nloops, loops.p, sizeof(nloops), cudaMemcpyDeviceToHost, st));
    TC_CUDA(cudaStreamSynchronize(st));
    const uint64_t mv = m - nloops;
    DevBuf flag, pos, tot;
    TC_TRY(flag.alloc(sizeof(uint32_t) * (mv ? mv : 1), st));
    TC_TRY(pos.alloc(sizeof(uint32_t) * (mv ? mv : 1), st));
    TC_TRY(tot.alloc(sizeof(uint32_t), st));
    uint64_t D = 0;
    if (mv) {
        k_run_heads<<<grid_for(mv, kT, 1u << 16), kT, 0, st>>>(kp, mv, flag.as<uint32_t>());
        TC_LAUNCH("k_run_heads");
    }
    TC_TRY(scan_total(flag.as<uint32_t>(), pos.as<uint32_t>(), mv, tot, &D, st));
    if (D == 0) return TC_OK;
    DevBuf dkey, dnet, fresh, fpos, kept, kpos, bad;
    TC_TRY(dkey.alloc(sizeof(uint64_t) * D, st));
    TC_TRY(dnet.alloc(sizeof(int) * D, st));
    TC_CUDA(cudaMemsetAsync(dnet.p, 0, sizeof(int) * D, st));
    k_run_net<<<grid_for(mv, kT, 1u << 16), kT, 0, st>>>(kp, mv, flag.as<uint32_t>(), pos.as<uint32_t>(),
                                                         dkey.as<uint64_t>(), dnet.as<int>());
    TC_LAUNCH("k_run_net");
    keys.release();
    tmp.release();
    flag.release();
    pos.release();
    const uint64_t S = s->set_len;
    TC_TRY(fresh.alloc(sizeof(uint32_t) * D, st));
    TC_TRY(fpos.alloc(sizeof(uint32_t) * D, st));
    TC_TRY(kept.alloc(sizeof(uint32_t) * (S ? S : 1), st));
    TC_TRY(kpos.alloc(sizeof(uint32_t) * (S ? S : 1), st));
    TC_TRY(bad.alloc(sizeof(unsigned int), st));
    TC_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(unsigned int), st));
    uint64_t* skey = S ? s->set_key.as<uint64_t>() : nullptr;
    uint32_t* scnt = S ? s->set_cnt.as<uint32_t>() : nullptr;
    k_apply_net<<<grid_for(D, kT, 1u << 16), kT, 0, st>>>(dkey.as<uint64_t>(), dnet.as<int>(), D, skey, scnt, S,
                                                          fresh.as<uint32_t>(), bad.as<unsigned int>());
    TC_LAUNCH("k_apply_net");
    if (S) {
        k_kept<<<grid_for(S, kT, 1u << 16), kT, 0, st>>>(scnt, S, kept.as<uint32_t>());
        TC_LAUNCH("k_kept");
    }
    uint64_t F = 0, K = 0;
    TC_TRY(scan_total(fresh.as<uint32_t>(), fpos.as<uint32_t>(), D, tot, &F, st));
    TC_TRY(scan_total(kept.as<uint32_t>(), kpos.as<uint32_t>(), S, tot, &K, st));
    unsigned int hbad = 0;
    TC_CUDA(cudaMemcpyAsync(&hbad, bad.p, sizeof(hbad), cudaMemcpyDeviceToHost, st));
    TC_CUDA(cudaStreamSynchronize(st));
    if (hbad) {
        // cannot happen while the set follows the window; should it, make the set afresh
        s->repairs++;
        s->set_ok = false;
        return update_set(s, a, b);
    }
    DevBuf okey, ocnt;
    const uint64_t N = K + F;
    TC_TRY(okey.alloc(sizeof(uint64_t) * (N ? N : 1), st));   // stream-ordered: the set lives on st
    TC_TRY(ocnt.alloc(sizeof(uint32_t) * (N ? N : 1), st));
    if (S) {
        k_merge_old<<<grid_for(S, kT, 1u << 16), kT, 0, st>>>(skey, scnt, S, kpos.as<uint32_t>(), dkey.as<uint64_t>(), D,
                                                              fpos.as<uint32_t>(), F, okey.as<uint64_t>(),
                                                              ocnt.as<uint32_t>());
        TC_LAUNCH("k_merge_old");
    }
    k_merge_fresh<<<grid_for(D, kT, 1u << 16), kT, 0, st>>>(dkey.as<uint64_t>(), dnet.as<int>(), fresh.as<uint32_t>(),
                                                            fpos.as<uint32_t>(), D, skey, S, kpos.as<uint32_t>(), K,
                                                            okey.as<uint64_t>(), ocnt.as<uint32_t>());
    TC_LAUNCH("k_merge_fresh");
    std::swap(s->set_key.p, okey.p);
    std::swap(s->set_key.bytes, okey.bytes);
    std::swap(s->set_key.st, okey.st);
    std::swap(s->set_key.async, okey.async);
    std::swap(s->set_cnt.p, ocnt.p);
    std::swap(s->set_cnt.bytes, ocnt.bytes);
    std::swap(s->set_cnt.st, ocnt.st);
    std::swap(s->set_cnt.async, ocnt.async);
    s->set_len = N;
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
    s->B = bits_for(n);
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
        const auto first = s->t.begin() + (std::ptrdiff_t)s->t0;
        return (uint64_t)(std::upper_bound(first, s->t.end(), x) - first);
    };
    const uint64_t a = from_zero ? 0 : first_after(t0), b = first_after(t_now);
    const uint64_t m = b > a ? b - a : 0;
    tc_status us = update_set(s, a, b);
    s->set_ok = us == TC_OK;
    TC_TRY(us);
    // the set now follows this window: drop the arcs before it (later censuses start no earlier)
    if (a) {
        s->t0 += a;
        if (2 * s->t0 >= s->t.size()) {   // amortised O(1) per arc
            s->t.erase(s->t.begin(), s->t.begin() + (std::ptrdiff_t)s->t0);
            s->t0 = 0;
        }
        s->lo += a;
        if (s->lo == s->hi) s->lo = s->hi = 0;
    }
    s->nb = b - a;
    s->last_census = t_now;
    s->any_census = true;
    tc_graph* g = nullptr;
    TC_TRY(graph_create_sorted(s->n, s->set_len ? s->set_key.as<uint64_t>() : nullptr, s->set_len, s->st,
                               s->has_opt ? &s->opt : nullptr, &g));
    const tc_status cs = tc_census_opts(g, s->st, s->has_opt ? &s->opt : nullptr, out);
    tc_graph_destroy(g);
    TC_TRY(cs);
    if (arcs_in_window) *arcs_in_window = m;
    s->censuses++;
    return TC_OK;
}

tc_status tc_stream_stats(const tc_stream* s, tc_stream_info* info) {
    if (!s || !info) return fail(TC_ERR_ARG, "null argument");
    info->live_arcs = s->hi - s->lo;
    info->capacity = s->cap;
    info->censuses = s->censuses;
    info->distinct_arcs = s->set_ok ? s->set_len : 0;
    info->rebuilds = s->rebuilds;
    info->repairs = s->repairs;
    info->last_added = s->last_added;
    info->last_evicted = s->last_evicted;
    return TC_OK;
}

void tc_stream_destroy(tc_stream* s) {
    if (!s) return;
    if (s->st) cudaStreamSynchronize(s->st);
    delete s;
}

}  // extern "C"
