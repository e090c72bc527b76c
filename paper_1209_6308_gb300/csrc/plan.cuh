// plan.cuh - census work items from the exact work of each pair.
//
// A vertex u of the CTA tier becomes items: ranges of its upper pairs (u, N[u][j]), j >= up[u]
// (Fig. 5 step 2.1's pairs).  A pair's work is the part of N[v] the census walks (the entries
// past u, known from the per-pair tables; all of N[v] without them) plus fixed overheads per
// pair and per chunk of N[u], in the units of the plan's degree estimate.  With W the vertex's
// total and S items wanted (from W and the item size, or from the learned cost), pair j goes to
// item floor((its prefix of the work + half its own work) * S / W) plus one more item every
// kMaxItemPairs pairs: contiguous ranges of about W / S work each - a hub's pairs with other
// hubs, at the front of its list, no longer share one heavy item - and never more than
// kMaxItemPairs pairs.  Counting and emitting run the same arithmetic, so they agree.
#pragma once

#include "tc_internal.cuh"

namespace tc {

__device__ __forceinline__ uint64_t pair_units(const GraphDev& g, uint32_t u, uint64_t ubase, uint32_t du, uint32_t upu,
                                               uint32_t j, uint32_t chunks, int algo) {
    const uint32_t v = g.adj[ubase + j] >> 2;
    const uint64_t dv = g.off[v + 1] - g.off[v];
    const uint64_t walk = g.rp ? dv - 1 - g.rp[g.ub[u] + (j - upu)] : dv;
    return walk + 16ull + 16ull * chunks + (algo == TC_ALGO_UNION ? du / 2 : 0ull);
}

// One warp: the total work W of vertex u's upper pairs (all lanes get it).
__device__ __forceinline__ unsigned long long vertex_units(const GraphDev& g, uint32_t u, uint32_t chunk, int algo) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t ubase = g.off[u];
    const uint32_t du = (uint32_t)(g.off[u + 1] - ubase), upu = g.up[u];
    const uint32_t chunks = (du + chunk - 1) / chunk;
    unsigned long long W = 0;
    for (uint32_t j = upu + lane; j < du; j += 32) W += pair_units(g, u, ubase, du, upu, j, chunks, algo);
    for (int o = 16; o; o >>= 1) W += __shfl_xor_sync(0xffffffffu, W, o);
    return W;
}

// One warp per vertex (all lanes call it with the same u and W = vertex_units(u)).  s_hint > 0
// fixes S (the learned schedule), else S = ceil(W / item_work).  units(j) gives pair j's work
// (stored by a first pass, or pair_units); emit(j, rank) runs on the lane of each pair that
// starts an item, rank = the item's index within the vertex.  Returns the vertex's item count.
// The cuts are computed in single precision: both passes run the same arithmetic on the same
// values, so they agree, and items are at least 2^14 units, far above the rounding.
template <typename Units, typename Emit>
__device__ uint32_t plan_vertex(const GraphDev& g, uint32_t u, uint32_t item_work, double s_hint,
                                unsigned long long W, Units units, Emit emit) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t ubase = g.off[u];
    const uint32_t du = (uint32_t)(g.off[u + 1] - ubase), upu = g.up[u];
    if (du <= upu) return 0;
    float S = s_hint > 0.0 ? ceilf((float)s_hint) : ceilf((float)W / (float)item_work);
    if (S < 1.f) S = 1.f;
    const float inv_per = S / (float)(W ? W : 1ull);
    unsigned long long carry = 0;
    uint32_t prev = 0xffffffffu, count = 0;
    for (uint32_t jb = upu; jb < du; jb += 32) {
        const uint32_t j = jb + lane;
        const bool ok = j < du;
        const unsigned long long c = ok ? units(j) : 0ull;
        unsigned long long incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= (uint32_t)o) incl += y;
        }
        const float mid = (float)(carry + incl - c) + 0.5f * (float)c;
        uint32_t id = ok ? (uint32_t)floorf(mid * inv_per) + (j - upu) / kMaxItemPairs : 0xffffffffu;
        uint32_t before = __shfl_up_sync(0xffffffffu, id, 1);
        if (lane == 0) before = prev;
        const bool start = ok && id != before;
        const uint32_t bm = __ballot_sync(0xffffffffu, start);
        if (start) emit(j, count + __popc(bm & ((1u << lane) - 1u)));
        count += __popc(bm);
        carry += __shfl_sync(0xffffffffu, incl, 31);
        const uint32_t last = 31u - __clz(__ballot_sync(0xffffffffu, ok));
        prev = __shfl_sync(0xffffffffu, id, last);
    }
    return count;
}

// Item starts of a vertex are written in order by plan_vertex's emit; each item ends where the
// next one starts, the last at du.  One warp, after its emits (a __syncwarp orders them).
__device__ __forceinline__ void plan_vertex_ends(Item* items, uint32_t count, uint32_t du) {
    __syncwarp();
    const uint32_t lane = threadIdx.x & 31;
    for (uint32_t k = lane; k < count; k += 32) items[k].j1 = k + 1 < count ? items[k + 1].j0 : du;
    __syncwarp();
}

}  // namespace tc
