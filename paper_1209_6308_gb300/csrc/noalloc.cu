// noalloc.cu - a census entry point that allocates nothing, for callers that cannot call
// cudaMalloc: code running where allocation is forbidden or must not block, such as inside
// a memory-pool budget owned by someone else, a real-time loop, or a host that has already
// reserved all device memory for its own use.  The paper has no counterpart to this.
//
// Its scratch (the upper-neighbour index of every vertex, the CTA work items and the work
// counters) lives in one file-scope device array of fixed size, held by every GPU that loads
// the library until the process exits.  Every call shares that array and it keeps the last
// call's contents; calls that overlap on the GPU race, so the caller must serialise them.
#include <atomic>
#include <cstring>

#include "graph.cuh"

namespace tc {
namespace {

constexpr uint32_t kNoAllocMaxN = 1u << 20;        // vertices
constexpr uint32_t kNoAllocMaxItems = 1u << 18;    // CTA work items
constexpr uint32_t kCounters = 64;                 // uint32 counters at the start of the array

// [0, 256): counters; then up[kNoAllocMaxN] uint32; then items[kNoAllocMaxItems]
constexpr size_t kUpOffset = 256;
constexpr size_t kItemsOffset = kUpOffset + sizeof(uint32_t) * kNoAllocMaxN;
constexpr size_t kScratchBytes = kItemsOffset + sizeof(Item) * kNoAllocMaxItems;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// counter slots
enum {
    kCntItems = 0, kCntWideVerts = 1, kCntActive = 2, kCntBadOrder = 3, kCntOverflow = 4,
    kCntBadOff = 5, kCntBadAdj = 6, kCntBadSym = 7, kCntCensus = 8
};

// The offsets: off[x] <= off[x+1] for every x (with off[0] = 0, checked on the host, every list
// then lies inside adj[0, off[n])).  Counts vertices with deg > warp_max and with deg > 0, and
// flags lists whose degrees increase with the id (the census tiers rely on descending degrees).
// Reads off[] only, so it is safe on any offsets.
__global__ void k_noalloc_check_off(uint32_t n, const uint64_t* __restrict__ off, uint32_t warp_max, uint32_t* cnt) {
    uint32_t wide = 0, act = 0, bad = 0, badoff = 0;
    for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < n; x += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t b = off[x], e = off[x + 1];
        if (e < b) { ++badoff; continue; }
        const uint64_t d = e - b;
        wide += d > warp_max;
        act += d > 0;
        if (x + 1 < n && off[x + 2] >= e && off[x + 2] - e > d) ++bad;
    }
    wide = __reduce_add_sync(0xffffffffu, wide);
    act = __reduce_add_sync(0xffffffffu, act);
    bad = __reduce_add_sync(0xffffffffu, bad);
    badoff = __reduce_add_sync(0xffffffffu, badoff);
    if ((threadIdx.x & 31) == 0) {
        if (wide) atomicAdd(&cnt[kCntWideVerts], wide);
        if (act) atomicAdd(&cnt[kCntActive], act);
        if (bad) atomicAdd(&cnt[kCntBadOrder], bad);
        if (badoff) atomicAdd(&cnt[kCntBadOff], badoff);
    }
}

// The lists, one warp per vertex x (run only once the offsets passed k_noalloc_check_off, so
// every read lies inside adj[0, off[n])): each entry has an id below n other than x and a
// non-zero direction, the ids ascend strictly, and x appears in the neighbour's list with the
// mirrored direction bits (found by binary search, which reads only inside that list).  Also
// writes up[x], the number of neighbours with a smaller id (the index of the first v > x).
__global__ void k_noalloc_check_adj(uint32_t n, const uint64_t* __restrict__ off, const uint32_t* __restrict__ adj,
                                    uint32_t* cnt, uint32_t* up) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    uint32_t badadj = 0, badsym = 0;
    for (uint64_t x = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; x < n; x += warps) {
        const uint64_t b = off[x], e = off[x + 1];
        uint32_t below = 0;
        for (uint64_t k = b + lane; k < e; k += 32) {
            const uint32_t w = adj[k], id = w >> 2, dir = w & 3u;
            below += id < x;
            if (id >= n || id == x || dir == 0u || (k > b && (adj[k - 1] >> 2) >= id)) {
                ++badadj;
                continue;
            }
            const uint32_t mirror = ((dir & 1u) << 1) | (dir >> 1);
            uint64_t lo = off[id], hi = off[id + 1];
            const uint64_t end = hi;
            while (lo < hi) {
                const uint64_t mid = (lo + hi) >> 1;
                if ((adj[mid] >> 2) < (uint32_t)x) lo = mid + 1; else hi = mid;
            }
            if (lo >= end || adj[lo] != (((uint32_t)x << 2) | mirror)) ++badsym;
        }
        below = __reduce_add_sync(0xffffffffu, below);
        if (lane == 0) up[x] = below;
    }
    badadj = __reduce_add_sync(0xffffffffu, badadj);
    badsym = __reduce_add_sync(0xffffffffu, badsym);
    if (lane == 0) {
        if (badadj) atomicAdd(&cnt[kCntBadAdj], badadj);
        if (badsym) atomicAdd(&cnt[kCntBadSym], badsym);
    }
}

// Items for the vertices u < u_end (deg > warp_max): the pairs of u in ranges of at most
// kMaxItemPairs, sized by the plain estimate like the regular plan; appended in any order.
__global__ void k_noalloc_items(uint32_t u_end, const uint64_t* __restrict__ off, const uint32_t* __restrict__ up,
                                uint32_t chunk, uint32_t item_work, float dbar, uint32_t* cnt, Item* items) {
    for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < u_end; x += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t du = (uint32_t)(off[x + 1] - off[x]);
        const uint32_t P = du - up[x];
        if (P == 0) continue;
        const uint32_t C = (du + chunk - 1) / chunk;
        double s = ceil((double)P * ((double)dbar + 16.0 + 16.0 * (double)C) / (double)item_work);
        const double smin = ceil((double)P / (double)kMaxItemPairs);
        if (s < smin) s = smin;
        if (s < 1.0) s = 1.0;
        if (s > (double)P) s = (double)P;
        const uint32_t S = (uint32_t)s;
        const uint32_t o = atomicAdd(&cnt[kCntItems], S);
        if (o + S > kNoAllocMaxItems || o + S < o) {
            atomicAdd(&cnt[kCntOverflow], 1u);
            continue;
        }
        for (uint32_t k = 0; k < S; ++k) {
            Item it;
            it.u = (uint32_t)x;
            it.j0 = up[x] + (uint32_t)((uint64_t)P * k / S);
            it.j1 = up[x] + (uint32_t)((uint64_t)P * (k + 1) / S);
            it.pad = 0;
            items[o + k] = it;
        }
    }
}

// Device address of the scratch array, looked up once per device (with that device current);
// atomics, since several host threads may make their first call at once.
std::atomic<unsigned char*> g_scratch_ptr[64];

tc_status scratch_for_current_device(unsigned char** out) {
    int dev = 0;
    TC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(TC_ERR_ARG, "device index beyond 63");
    unsigned char* p = g_scratch_ptr[dev].load();
    if (!p) {
        void* q = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&q, g_scratch);
        if (e != cudaSuccess || !q) return cuda_fail(e != cudaSuccess ? e : cudaErrorInvalidSymbol, "cudaGetSymbolAddress(scratch)");
        p = static_cast<unsigned char*>(q);
        g_scratch_ptr[dev].store(p);
    }
    *out = p;
    return TC_OK;
}

}  // namespace
}  // namespace tc

using namespace tc;

extern "C" tc_status tc_census_csr_noalloc(uint32_t n, const uint64_t* d_off, const uint32_t* d_adj, void* stream,
                                           uint64_t* d_out16) {
    if (!d_off || !d_adj || !d_out16) return fail(TC_ERR_ARG, "null argument");
    if (n > kNoAllocMaxN)
        return fail(TC_ERR_RANGE, "tc_census_csr_noalloc: n = " + std::to_string(n) + " exceeds its scratch limit of " +
                                      std::to_string(kNoAllocMaxN) + " vertices");
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char* base = nullptr;
    TC_TRY(scratch_for_current_device(&base));
    uint32_t* cnt = reinterpret_cast<uint32_t*>(base);
    uint32_t* up = reinterpret_cast<uint32_t*>(base + kUpOffset);
    Item* items = reinterpret_cast<Item*>(base + kItemsOffset);
    Opts o;
    tc_options opt;
    std::memset(&opt, 0, sizeof(opt));
    opt.algo = TC_ALGO_SUFFIX;
    TC_TRY(resolve_opts(&opt, nullptr, &o));

    TC_CUDA(cudaMemsetAsync(d_out16, 0, sizeof(uint64_t) * 16, st));
    TC_CUDA(cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * kCounters, st));
    uint64_t first = 0, total = 0;
    TC_CUDA(cudaMemcpyAsync(&first, d_off, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    TC_CUDA(cudaMemcpyAsync(&total, d_off + n, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    if (n) {
        k_noalloc_check_off<<<grid_for(n, 256, 4096), 256, 0, st>>>(n, d_off, o.warp_max_deg, cnt);
        TC_LAUNCH("k_noalloc_check_off");
    }
    uint32_t h[kCounters];
    TC_CUDA(cudaMemcpyAsync(h, cnt, sizeof(h), cudaMemcpyDeviceToHost, st));
    TC_CUDA(cudaStreamSynchronize(st));
    if (first != 0 || h[kCntBadOff])
        return fail(TC_ERR_ARG, "tc_census_csr_noalloc: offsets must start at 0 and never decrease");
    if (h[kCntBadOrder]) return fail(TC_ERR_ARG, "tc_census_csr_noalloc: vertex degrees must not increase with the id");
    if (total == 0) return TC_OK;
    // the offsets are sound: every list lies inside d_adj[0, total)
    k_noalloc_check_adj<<<grid_for((uint64_t)n * 32, 256, 8192), 256, 0, st>>>(n, d_off, d_adj, cnt, up);
    TC_LAUNCH("k_noalloc_check_adj");
    TC_CUDA(cudaMemcpyAsync(h, cnt, sizeof(h), cudaMemcpyDeviceToHost, st));
    TC_CUDA(cudaStreamSynchronize(st));
    if (h[kCntBadAdj])
        return fail(TC_ERR_ARG, "tc_census_csr_noalloc: a list entry has an id >= n, a self-loop, no direction bits, "
                                "or breaks the ascending order");
    if (h[kCntBadSym])
        return fail(TC_ERR_ARG, "tc_census_csr_noalloc: the lists are not symmetric with mirrored direction bits");
    const uint32_t u_end = h[kCntWideVerts], n_active = h[kCntActive];
    const float dbar = n_active ? (float)((double)total / (double)n_active) : 0.f;
    if (u_end) {
        k_noalloc_items<<<grid_for(u_end, 256, 4096), 256, 0, st>>>(u_end, d_off, up, o.chunk,
                                                                    o.item_work ? o.item_work : (1u << 18), dbar, cnt,
                                                                     items);
        TC_LAUNCH("k_noalloc_items");
        TC_CUDA(cudaMemcpyAsync(h, cnt, sizeof(h), cudaMemcpyDeviceToHost, st));
        TC_CUDA(cudaStreamSynchronize(st));
        if (h[kCntOverflow])
            return fail(TC_ERR_RANGE, "tc_census_csr_noalloc: the graph needs more than " +
                                          std::to_string(kNoAllocMaxItems) + " work items");
    }
    GraphDev gd;
    gd.n = n;
    gd.n_active = n_active;
    gd.off = d_off;
    gd.adj = d_adj;
    gd.up = up;
    gd.ub = nullptr;   // no per-pair tables: the census walks whole lists
    gd.rp = nullptr;
    gd.vs = nullptr;
    gd.us = nullptr;
    return census_launch_raw(gd, o, items, u_end ? h[kCntItems] : 0u, u_end, n_active, cnt + kCntCensus,
                             reinterpret_cast<unsigned long long*>(d_out16), st);
}
