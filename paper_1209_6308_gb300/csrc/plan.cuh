// plan.cuh - census work items from the exact work of each pair.
//
// A vertex u of the CTA tier becomes items: ranges of its upper pairs (u, N[u][j]), j >= up[u]
// (Fig. 5 step 2.1's pairs).  A pair's work is the part of N[v] the census walks (the entries
// past u, known from the per-pair tables; all of N[v] without them) plus fixed overheads per
// pair and per chunk of N[u], in the units of the plan's degree estimate.  With W the vertex's
// total and S items wanted (from W and the item size, or from the learned cost), pair j goes to
// item floor((its prefix of the work + half its own work) * S / W), and a new item starts at
// every block of kMaxItemPairs pairs: contiguous ranges of about W / S work each - a hub's
// pairs with other hubs, at the front of its list, no longer share one heavy item - and never
// more than kMaxItemPairs pairs.  Each block can be planned by its own warp from the work
// before it, so a hub's thousands of pairs are no serial chain.  Counting and emitting run the
// same arithmetic, so they agree.
#pragma once

#include "tc_internal.cuh"

namespace tc {

__device__ __forceinline__ uint64_t pair_units(const GraphDev& g, uint32_t u, uint64_t ubase, uint32_t du, uint32_t upu,
                                               uint32_t j, uint32_t chunks, int algo) {
    const uint32_t v = g.adj[ubase + j] >> 2;
    // the triangle form walks the entries of N[v] below u (rp = u's position in N[v]) and a pair overhead
    if (algo == TC_ALGO_TRIANGLE) return (uint64_t)g.rp[g.ub[u] + (j - upu)] + 32ull;
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

// Items wanted for a vertex of work W: the learned count when s_hint > 0, else W / item_work.
__device__ __forceinline__ float plan_items(unsigned long long W, uint32_t item_work, double s_hint) {
    const float S = s_hint > 0.0 ? ceilf((float)s_hint) : ceilf((float)W / (float)item_work);
    return S < 1.f ? 1.f : S;
}

// One warp (all lanes call it with the same arguments): the items of pairs [j0, j1) of one
// vertex, a block of at most kMaxItemPairs pairs that starts a multiple of kMaxItemPairs past
// up[u].  carry holds the work of the vertex's pairs before j0 and comes back with the block's
// own added; W is the vertex's total and S its item count.  Pair j (work c, prefix p) gets the
// item id floor((p + c/2) * S / W); j0 and each pair whose id differs from its predecessor's
// start an item.  units(j) gives pair j's work; emit(j, rank) runs on the lane of each pair that
// starts an item, rank = the item's index within the block.  Returns the block's item count.
// The ids are computed in single precision: every pass runs the same arithmetic on the same
// integers, so counting and emitting agree, and items are at least 2^14 units, far above the
// rounding.
template <typename Units, typename Emit>
__device__ uint32_t plan_block(uint32_t j0, uint32_t j1, unsigned long long& carry, unsigned long long W, float S,
                               Units units, Emit emit) {
    const uint32_t lane = threadIdx.x & 31;
    const float inv_per = S / (float)(W ? W : 1ull);
    uint32_t prev = 0xffffffffu, count = 0;
    for (uint32_t jb = j0; jb < j1; jb += 32) {
        const uint32_t j = jb + lane;
        const bool ok = j < j1;
        const unsigned long long c = ok ? units(j) : 0ull;
        unsigned long long incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= (uint32_t)o) incl += y;
        }
        const float mid = (float)(carry + incl - c) + 0.5f * (float)c;
        const uint32_t id = ok ? (uint32_t)floorf(mid * inv_per) : 0xffffffffu;
        uint32_t before = __shfl_up_sync(0xffffffffu, id, 1);
        if (lane == 0) before = prev;
        const bool start = ok && (id != before || j == j0);
        const uint32_t bm = __ballot_sync(0xffffffffu, start);
        if (start) emit(j, count + __popc(bm & ((1u << lane) - 1u)));
        count += __popc(bm);
        carry += __shfl_sync(0xffffffffu, incl, 31);
        const uint32_t last = 31u - __clz(__ballot_sync(0xffffffffu, ok));
        prev = __shfl_sync(0xffffffffu, id, last);
    }
    return count;
}

// One warp per vertex (all lanes call it with the same u and W = vertex_units(u)): the vertex's
// blocks in order, the same items as a warp per block gives.  s_hint > 0 fixes S (the learned
// schedule), else S = ceil(W / item_work).  units(j) gives pair j's work (stored by a first
// pass, or pair_units); emit(j, rank) runs on the lane of each pair that starts an item, rank =
// the item's index within the vertex.  Returns the vertex's item count.
template <typename Units, typename Emit>
__device__ uint32_t plan_vertex(const GraphDev& g, uint32_t u, uint32_t item_work, double s_hint,
                                unsigned long long W, Units units, Emit emit) {
    const uint64_t ubase = g.off[u];
    const uint32_t du = (uint32_t)(g.off[u + 1] - ubase), upu = g.up[u];
    if (du <= upu) return 0;
    const float S = plan_items(W, item_work, s_hint);
    unsigned long long carry = 0;
    uint32_t count = 0;
    for (uint32_t j0 = upu; j0 < du; j0 += kMaxItemPairs) {
        const uint32_t j1 = du - j0 > kMaxItemPairs ? j0 + kMaxItemPairs : du;
        count += plan_block(j0, j1, carry, W, S, units, [&](uint32_t j, uint32_t r) { emit(j, count + r); });
    }
    return count;
}

// Items are written in order by the emits of plan_vertex or plan_block; each ends where the next
// one starts, the last at `end` (du for a vertex, j1 for a block).  One warp, after its emits (a
// __syncwarp orders them).
__device__ __forceinline__ void plan_ends(Item* items, uint32_t count, uint32_t end) {
    __syncwarp();
    const uint32_t lane = threadIdx.x & 31;
    for (uint32_t k = lane; k < count; k += 32) items[k].j1 = k + 1 < count ? items[k + 1].j0 : end;
    __syncwarp();
}

}  // namespace tc
