// triangles.cu - the census with the common neighbours enumerated once per triangle.
//
// For a connected pair (u, v), u < v (Fig. 5 step 2.1), every third vertex w of
// S = N[u] u N[v] \ {u, v} that only one endpoint reaches has a class fixed by two direction
// bits (dir(u,v) and the link of w to that endpoint), so those triads are counted in bulk
// from the per upper pair tables' direction-class suffix counts; only the common neighbours
// need their full tricode (the union-free rewrite of step 2.1.4).  The suffix kernel finds
// each pair's common neighbours by walking N[v] past u.  Here each common neighbour is found
// once, as a triangle: with ids in descending degree, L(x) = the neighbours of x with smaller
// ids (a prefix of N[x]) is short for every x, and the triangle a < b < c is met exactly
// once, when the walk of the entries of N[c] below b (a prefix of L(c), its length the pair
// table's position of b in N[c]) for the pair (b, c) finds a in L(b), staged in shared memory
// (a hash, or a direct map of two direction bits per id when b's id is small).
// Its tricode (roles (a, b, c)) then gives every correction it makes to the pairs' bulk
// counts (Fig. 5 steps 2.1.2 - 2.1.4):
//   + the triad itself, counted once at the pair (a, b) with w = c > b (step 2.1.4's rule);
//   - c among the u-only third vertices of (a, b) and among its v-only ones, b among the
//     v-only ones of (a, c): common neighbours, not one-sided;
//   + one common neighbour in the dyadic count n - |S| - 2 of each of its three pairs.
// So the kernel only histograms the 64 tricodes of the triangles; a small fold kernel turns
// them and the bulk sums into the 16 classes on the device.
//
// The same walk in the caller's id order (the triangle's state with its actors ordered by
// their original ids) serves the 64-state census (census64.cu).
//
// Work: a vertex b with degree above the warp tier becomes CTA items (b, range of its upper
// pairs (b, c)), cut by the plan (plan.cuh) with pair work |L(c)|; the CTA stages L(b) in a
// shared-memory hash, and its warps walk the lists L(c) of 32 pairs at a time as one
// flattened range, so short and long lists share the lanes.  The other vertices run one warp
// each, with L(b) in the warp's own hash.
#include <atomic>
#include <cstring>

#include "graph.cuh"

namespace tc {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
// Prefixes of at least kLongPrefix entries are walked one pair at a time by the whole warp
// (walk_pairs<..., LONGW = true>), kLongRounds loads of 32 entries in flight per lane; shorter
// ones share flattened ranges.
// (Swept at scales 20 and 26: thresholds 64-512, 2-8 rounds.)
constexpr uint32_t kLongPrefix = 128;
constexpr int kLongRounds = 8;
constexpr uint32_t kWarpSlots = 256;     // per-warp hash slots: |L(b)| <= warp_max_deg <= 128
constexpr uint32_t kFlushElems = 1u << 30;

__device__ __forceinline__ unsigned long long tri_clock_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t tri_hash(uint32_t x, int hb) { return (x * 2654435761u) >> (32 - hb); }

// Tricode of the triangle (a, b, c) from the direction bits of three stored entries: a in N[b]
// (seen from b: 1 b->a, 2 a->b), c in N[b] (1 b->c, 2 c->b) and a in N[c] (1 c->a, 2 a->c).
// Tricode bits: 1 b->a, 2 a->b, 4 b->c, 8 c->b, 16 a->c, 32 c->a.  The walk keeps the second
// term pre-shifted per pair (bc_bits = (dir(b,c)) << 2) and maps the third through a four-entry
// byte table: dir(c,a) 1 -> 32, 2 -> 16, 3 -> 48.
__device__ __forceinline__ uint32_t tri_code(uint32_t dir_ba, uint32_t bc_bits, uint32_t e_ca) {
    return dir_ba | bc_bits | __byte_perm(0x30102000u, 0u, e_ca & 3u);
}

struct TriParams {
    GraphDev g;
    const Item* items;
    uint32_t n_items;
    uint32_t warp_begin, warp_end;
    uint32_t wshift;              // warp tier: 2^wshift consecutive vertices per grab
    uint32_t chunk;               // entries of L(b) staged per pass of a CTA item (hash: 2 x chunk slots)
    uint32_t* ctr;                // [0] next item, [1] next warp-tier vertex
    const uint32_t* old;          // OLD: the caller's id of each vertex
    const uint8_t* perm_state;    // OLD: [9][64] state of a tricode under the rank pattern 3 ra + rb
    unsigned long long* hist;     // 64 bins (triangle tricodes, or states with OLD); batched: graph g's at
                                  // hist + kBatchStride g
    unsigned long long* vcost;    // optional [n]: SM cycles per CTA-tier vertex b
    unsigned long long* phase;    // optional [3 * gridDim]: globaltimer at start, end of items, end
    // batched launch: item.pad is the graph index, warp-tier blocks are (u0, u1, graph)
    const GraphDev* graphs;
    const uint4* wblocks;
    uint32_t n_wblocks;
    // serving wave: n_items / n_wblocks are the wave's totals over its request slices
    const WaveReq* reqs;
    uint32_t n_reqs;
};

// batched triangle form: per graph 96 uint64 of scratch, the 21 bulk sums at [0, 21) and the 64
// triangle tricodes at [32, 96); a serving wave's requests have the same scratch at WaveReq.out
constexpr uint32_t kBatchStride = 96;

// launch modes: one graph; a batch of graphs (items tagged with the graph, blocks (u0, u1, g));
// a serving wave (slices of several requests, descriptors in global memory)
enum { kTriSingle = 0, kTriBatch = 1, kTriWave = 2 };

// index r of the last request whose prefix is <= i (prefixes ascend from 0)
template <typename F>
__device__ __forceinline__ uint32_t find_req(uint32_t count, uint32_t i, F pre) {
    uint32_t lo = 0, hi = count;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (pre(mid) <= i) lo = mid; else hi = mid;
    }
    return lo;
}

// Walk, for the pairs (b, c = N[b][j]), j in [j0, j1), 32 pairs per batch, the entries of N[c]
// below b (rp = b's position in N[c], from the pair tables; pb + j indexes the pair) and count
// each a found in the staged L(b).  MAP: L(b) is a direct map of two direction bits per id (every
// a < b is in its range); else a hash.  One warp: a batch's pairs with long prefixes are walked
// one after another by all lanes, and the lanes share the flattened (pair, position) range of
// the others.  Returns the entries walked (warp-uniform).
template <bool OLD, bool MAP, bool LONGW>
__device__ __forceinline__ uint32_t walk_pairs(const TriParams& P, const GraphDev& G, uint64_t bbase, uint64_t pb,
                                               uint32_t j0, uint32_t j1, const uint32_t* sH, const uint32_t* sO,
                                               int hb, uint32_t hmask, uint32_t ob, const uint8_t* sPerm,
                                               uint32_t* myHist, int lane) {
    const uint64_t* __restrict__ off = G.off;
    const uint32_t* __restrict__ adj = G.adj;
    const uint32_t* __restrict__ rp = G.rp;
    const uint32_t le_mask = (2u << lane) - 1u;
    uint32_t walked = 0;
    // one walked entry e_ca = a in N[c] of the pair whose b-c tricode bits are bcb (and whose c has
    // the caller id oc2): look a up in L(b), count the triangle's tricode (or state) if found
    auto count = [&](uint32_t e_ca, uint32_t bcb, uint32_t oc2) {
        if (!e_ca) return;
        const uint32_t a = e_ca >> 2;
        uint32_t dir, oa = 0;
        if (MAP) {   // word a / 16, bits 2 (a mod 16), read straight from the entry
            dir = (sH[e_ca >> 6] >> ((e_ca >> 1) & 30u)) & 3u;
            if (OLD && dir) oa = P.old[a];
        } else {
            uint32_t h = tri_hash(a, hb);
            uint32_t e = sH[h];
            while (e != 0u && (e >> 2) != a) {
                h = (h + 1u) & hmask;
                e = sH[h];
            }
            dir = e & 3u;
            if (OLD && e) oa = sO[h];
        }
        if (dir != 0u) {
            uint32_t t = tri_code(dir, bcb, e_ca);
            if (OLD) {
                const uint32_t ra = (oa > ob) + (oa > oc2), rb = (ob > oa) + (ob > oc2);
                t = sPerm[(3u * ra + rb) * 64u + t];
            }
            atomicAdd(&myHist[t], 1u);
        }
    };
    for (uint32_t jb = j0; jb < j1; jb += 32) {
        const uint32_t j = jb + lane;
        const bool ok = j < j1;
        uint32_t e_bc = ok ? adj[bbase + j] : 0u;
        const uint32_t c = e_bc >> 2;
        uint64_t cb = ok ? off[c] : 0ull;
        uint32_t len = ok ? rp[pb + j] : 0u;
        uint32_t oc = (OLD && ok) ? P.old[c] : 0u;
        if (LONGW) {
            // pairs with long prefixes, one at a time over the whole warp: consecutive entries,
            // no search for the pair that holds an entry
            uint32_t lm = __ballot_sync(0xffffffffu, len >= kLongPrefix);
            while (lm) {
                const int q = __ffs(lm) - 1;
                lm &= lm - 1u;
                const uint64_t B = __shfl_sync(0xffffffffu, cb, q);
                const uint32_t L = __shfl_sync(0xffffffffu, len, q);
                const uint32_t bcb = (__shfl_sync(0xffffffffu, e_bc, q) & 3u) << 2;
                const uint32_t oq = OLD ? __shfl_sync(0xffffffffu, oc, q) : 0u;
                walked += L;
                for (uint32_t i = lane; i < L; i += 32u * kLongRounds) {
                    uint32_t x[kLongRounds];
#pragma unroll
                    for (int r = 0; r < kLongRounds; ++r)
                        x[r] = i + 32u * r < L ? __ldg(adj + (B + i + 32u * r)) : 0u;
#pragma unroll
                    for (int r = 0; r < kLongRounds; ++r) count(x[r], bcb, oq);
                }
            }
            if (len >= kLongPrefix) len = 0u;
        }
        // compact the pairs with a non-empty L(c) into lanes 0 .. cnt-1
        const uint32_t nz = __ballot_sync(0xffffffffu, len != 0u);
        if (!nz) continue;
        const uint32_t cnt = __popc(nz);
        const uint32_t src = __fns(nz, 0, lane + 1) & 31u;
        e_bc = __shfl_sync(0xffffffffu, e_bc, src);
        cb = __shfl_sync(0xffffffffu, cb, src);
        len = __shfl_sync(0xffffffffu, len, src);
        if (OLD) oc = __shfl_sync(0xffffffffu, oc, src);
        if ((uint32_t)lane >= cnt) len = 0u;
        uint32_t incl = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const uint32_t excl = incl - len;
        const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
        walked += total;
        // entry i of the flattened range lies at adj[cbx + i] for the pair that holds it (modular
        // arithmetic: i >= excl), and its tricode's b-c bits are bcb
        const uint64_t cbx = cb - excl;
        const uint32_t bcb = (e_bc & 3u) << 2;
        int seg_prev = -1;
        // two rounds of 32 entries per iteration, so each lane has two loads in flight
        for (uint32_t base = 0; base < total; base += 64) {
            // the pairs whose range starts in a round mark their start; lane i's pair is the
            // last one started at or before the round's entry i
            const bool stA = (uint32_t)lane < cnt && excl >= base && excl < base + 32u;
            const bool stB = (uint32_t)lane < cnt && excl >= base + 32u && excl < base + 64u;
            const uint32_t MA = __reduce_or_sync(0xffffffffu, stA ? (1u << (excl - base)) : 0u);
            const uint32_t MB = __reduce_or_sync(0xffffffffu, stB ? (1u << (excl - base - 32u)) : 0u);
            // (lane 31's count covers the whole round: the last pair of a round needs no shuffle)
            const int segA = seg_prev + __popc(MA & le_mask);
            const int lastA = seg_prev + __popc(MA);
            const int segB = lastA + __popc(MB & le_mask);
            seg_prev = lastA + __popc(MB);
            const uint32_t sa = (uint32_t)segA & 31u, sb = (uint32_t)segB & 31u;
            const uint64_t BA = __shfl_sync(0xffffffffu, cbx, sa), BB = __shfl_sync(0xffffffffu, cbx, sb);
            const uint32_t EA = __shfl_sync(0xffffffffu, bcb, sa), EB = __shfl_sync(0xffffffffu, bcb, sb);
            uint32_t OA = 0, OB = 0;
            if (OLD) {
                OA = __shfl_sync(0xffffffffu, oc, sa);
                OB = __shfl_sync(0xffffffffu, oc, sb);
            }
            const uint32_t iA = base + lane, iB = base + 32u + lane;
            const uint32_t xA = iA < total ? __ldg(adj + (BA + iA)) : 0u;
            const uint32_t xB = iB < total ? __ldg(adj + (BB + iB)) : 0u;
            count(xA, EA, OA);
            count(xB, EB, OB);
        }
    }
    return walked;
}

// A warp's next pairs of the CTA's item: guided sizes, 32 pairs while many remain, then fewer
// (down to 4) as the item runs out, so that the warps reach the item's end barrier together.
__device__ __forceinline__ void grab_pairs(uint32_t* s_next, uint32_t j1, int lane, uint32_t& jb, uint32_t& g) {
    jb = 0;
    g = 32;
    if (lane == 0) {
        const uint32_t cur = *(volatile uint32_t*)s_next;
        const uint32_t rem = cur < j1 ? j1 - cur : 0u;
        g = max(4u, min(32u, rem / (2u * kWarps)));
        jb = atomicAdd(s_next, g);
    }
    jb = __shfl_sync(0xffffffffu, jb, 0);
    g = __shfl_sync(0xffffffffu, g, 0);
}

// Add a warp's 64 bins to the graph's histogram and clear them (one warp).
__device__ __forceinline__ void flush_warp_hist(uint32_t* myHist, unsigned long long* hist, int lane) {
    __syncwarp();
    for (int t = lane; t < 64; t += 32) {
        const uint32_t v = myHist[t];
        if (v) atomicAdd(&hist[t], (unsigned long long)v);
        myHist[t] = 0u;
    }
    __syncwarp();
}

template <bool OLD, int MODE>
__global__ void __launch_bounds__(kThreads, 8) k_triangles(TriParams P) {
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t slots = 2u * P.chunk;
    uint32_t* sH = reinterpret_cast<uint32_t*>(smem);                 // [slots] CTA hash of L(b)
    uint32_t* sO = sH + slots;                                         // [slots] OLD: caller ids
    uint32_t* sWH = sO + (OLD ? slots : 0u);                           // [kWarps][kWarpSlots]
    uint32_t* sWO = sWH + kWarps * kWarpSlots;                         // [kWarps][kWarpSlots] OLD
    uint32_t* sHist = sWO + (OLD ? kWarps * kWarpSlots : 0u);         // [kWarps][64]
    uint8_t* sPerm = reinterpret_cast<uint8_t*>(sHist + kWarps * 64);  // [9][64] OLD
    __shared__ uint32_t s_item, s_next;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // the whole-warp walk of long prefixes, except in a batch of graphs (small graphs, short
    // prefixes: the path would only cost the kernel registers); the one-warp tier's prefixes
    // are below its degree bound, never long
    constexpr bool kLongWalk = MODE != kTriBatch;
    if (P.phase && tid == 0) P.phase[3 * blockIdx.x] = tri_clock_ns();
    for (int k = tid; k < kWarps * 64; k += kThreads) sHist[k] = 0u;
    if (OLD)
        for (int k = tid; k < 9 * 64; k += kThreads) sPerm[k] = P.perm_state[k];
    __syncthreads();
    uint32_t* myHist = sHist + warp * 64;
    GraphDev G = P.g;
    unsigned long long* ghist = P.hist;
    uint32_t cur_graph = 0xffffffffu;   // batched: the graph whose counts the warp's bins hold
    // batched: move to graph gi, flushing this warp's bins to the graph they belong to
    auto use_graph = [&](uint32_t gi) {
        if (cur_graph != 0xffffffffu) flush_warp_hist(myHist, ghist, lane);
        cur_graph = gi;
        if (MODE == kTriWave) {
            G = P.reqs[gi].g;
            ghist = P.reqs[gi].out + 32;
        } else {
            G = P.graphs[gi];
            ghist = P.hist + (uint64_t)kBatchStride * gi;
        }
    };
    uint32_t since_flush = 0;   // warp-uniform: entries walked since this warp's bins were flushed
    // the hash region (2 x chunk words) holds a direct map of 32 x chunk ids at two bits each
    const uint32_t map_ids = 32u * P.chunk;

    // ---------------------------------------------------------------- CTA items
    for (;;) {
        if (tid == 0) s_item = atomicAdd(&P.ctr[0], 1u);
        __syncthreads();
        const uint32_t it = s_item;
        if (it >= P.n_items) break;
        Item w;
        if (MODE == kTriWave) {
            const uint32_t r = find_req(P.n_reqs, it, [&](uint32_t q) { return P.reqs[q].item_pre; });
            w = P.reqs[r].items[it - P.reqs[r].item_pre];
            if (r != cur_graph) use_graph(r);
        } else {
            w = P.items[it];
            if (MODE == kTriBatch && w.pad != cur_graph) use_graph(w.pad);
        }
        const long long t0 = clock64();
        const uint32_t b = w.u;
        const uint64_t bbase = G.off[b];
        const uint32_t lb = G.up[b];
        const uint32_t ob = OLD ? P.old[b] : 0u;
        const uint64_t pb = G.ub[b] - lb;   // table index of the pair (b, N[b][j]) is pb + j
        if (b <= map_ids) {
            // L(b) as a direct map of two direction bits per id below b: one pass, no probing
            for (uint32_t k = tid; k < map_ids / 16u; k += kThreads) sH[k] = 0u;
            if (tid == 0) s_next = w.j0;
            __syncthreads();
            for (uint32_t k = tid; k < lb; k += kThreads) {
                const uint32_t e = G.adj[bbase + k], a = e >> 2;
                atomicOr(&sH[a >> 4], (e & 3u) << ((a & 15u) << 1));
            }
            __syncthreads();
            for (;;) {
                uint32_t jb, g;
                grab_pairs(&s_next, w.j1, lane, jb, g);
                if (jb >= w.j1) break;
                since_flush += walk_pairs<OLD, true, kLongWalk>(P, G, bbase, pb, jb, min(jb + g, w.j1), sH, nullptr, 0, 0u, ob,
                                                     sPerm, myHist, lane);
                if (since_flush >= kFlushElems) {
                    flush_warp_hist(myHist, ghist, lane);
                    since_flush = 0;
                }
            }
            __syncthreads();
        }
        // L(b) = N[b][0, lb), staged `chunk` entries per pass in a hash; every pass walks the item's pairs
        for (uint32_t c0 = 0; b > map_ids && c0 < lb; c0 += P.chunk) {
            const uint32_t LA = min(P.chunk, lb - c0);
            int hb = 6;
            while ((1u << hb) < 2u * LA) ++hb;
            const uint32_t H = 1u << hb, hmask = H - 1u;
            for (uint32_t k = tid; k < H; k += kThreads) sH[k] = 0u;
            if (tid == 0) s_next = w.j0;
            __syncthreads();
            for (uint32_t k = tid; k < LA; k += kThreads) {
                const uint32_t e = G.adj[bbase + c0 + k];
                uint32_t h = tri_hash(e >> 2, hb);
                while (atomicCAS(&sH[h], 0u, e) != 0u) h = (h + 1u) & hmask;
                if (OLD) sO[h] = P.old[e >> 2];
            }
            __syncthreads();
            for (;;) {
                uint32_t jb, g;
                grab_pairs(&s_next, w.j1, lane, jb, g);
                if (jb >= w.j1) break;
                since_flush += walk_pairs<OLD, false, kLongWalk>(P, G, bbase, pb, jb, min(jb + g, w.j1), sH, sO, hb, hmask, ob,
                                                      sPerm, myHist, lane);
                if (since_flush >= kFlushElems) {
                    flush_warp_hist(myHist, ghist, lane);
                    since_flush = 0;
                }
            }
            __syncthreads();   // every warp is done with this pass before the hash is replaced
        }
        if (P.vcost && tid == 0) atomicAdd(&P.vcost[b], (unsigned long long)(clock64() - t0));
        __syncthreads();   // every thread has read s_item before thread 0 takes the next item
    }

    if (P.phase && tid == 0) P.phase[3 * blockIdx.x + 1] = tri_clock_ns();

    // ---------------------------------------------------------------- one warp per vertex
    uint32_t* wH = sWH + warp * kWarpSlots;
    uint32_t* wO = sWO + (OLD ? warp * kWarpSlots : 0u);
    for (;;) {
        uint32_t b0, b1;
        if (MODE == kTriWave) {
            uint32_t bk = 0;
            if (lane == 0) bk = atomicAdd(&P.ctr[1], 1u);
            bk = __shfl_sync(0xffffffffu, bk, 0);
            if (bk >= P.n_wblocks) break;
            const uint32_t r = find_req(P.n_reqs, bk, [&](uint32_t q) { return P.reqs[q].block_pre; });
            if (r != cur_graph) use_graph(r);
            const WaveReq& q = P.reqs[r];
            b0 = q.warp_begin + ((bk - q.block_pre) << q.pad);
            b1 = min(b0 + (1u << q.pad), q.warp_end);
        } else if (MODE == kTriBatch) {
            uint32_t bk = 0;
            if (lane == 0) bk = atomicAdd(&P.ctr[1], 1u);
            bk = __shfl_sync(0xffffffffu, bk, 0);
            if (bk >= P.n_wblocks) break;
            const uint4 wb = P.wblocks[bk];
            if (wb.z != cur_graph) use_graph(wb.z);
            b0 = wb.x;
            b1 = wb.y;
        } else {
            uint32_t vb = 0;
            if (lane == 0) vb = atomicAdd(&P.ctr[1], 1u << P.wshift);
            vb = __shfl_sync(0xffffffffu, vb, 0);
            if (vb >= P.warp_end - P.warp_begin) break;
            b0 = P.warp_begin + vb;
            b1 = min(b0 + (1u << P.wshift), P.warp_end);
        }
        for (uint32_t b = b0; b < b1; ++b) {
            const uint64_t bbase = G.off[b];
            const uint32_t db = (uint32_t)(G.off[b + 1] - bbase), lb = G.up[b];
            if (lb == 0u || lb >= db) continue;   // no lower or no upper neighbour: no triangle has b in the middle
            int hb = 6;
            while ((1u << hb) < 2u * lb) ++hb;
            const uint32_t hmask = (1u << hb) - 1u;
            __syncwarp();
            for (uint32_t k = lane; k < (1u << hb); k += 32) wH[k] = 0u;
            __syncwarp();
            for (uint32_t k = lane; k < lb; k += 32) {
                const uint32_t e = G.adj[bbase + k];
                uint32_t h = tri_hash(e >> 2, hb);
                while (atomicCAS(&wH[h], 0u, e) != 0u) h = (h + 1u) & hmask;
                if (OLD) wO[h] = P.old[e >> 2];
            }
            __syncwarp();
            since_flush += walk_pairs<OLD, false, false>(P, G, bbase, G.ub[b] - lb, lb, db, wH, wO, hb, hmask,
                                                  OLD ? P.old[b] : 0u, sPerm, myHist, lane);
            if (since_flush >= kFlushElems) {
                flush_warp_hist(myHist, ghist, lane);
                since_flush = 0;
            }
        }
    }
    if (MODE == kTriSingle || cur_graph != 0xffffffffu) flush_warp_hist(myHist, ghist, lane);
    if (P.phase) {   // uniform over the CTA
        __syncthreads();
        if (tid == 0) P.phase[3 * blockIdx.x + 2] = tri_clock_ns();
    }
}

// One pair's bulk sums into acc (see k_pair_bulk): u of degree du, the pair's entry e = N[u][j]
// and its table index p.
__device__ __forceinline__ void bulk_pair(const GraphDev& g, unsigned long long n, uint32_t du, uint32_t j, uint32_t e,
                                          uint64_t p, unsigned long long (&acc)[3][7]) {
    const uint32_t v = e >> 2, duv = e & 3u;
    const uint32_t cuv = ((duv & 1u) << 1) | (duv >> 1);
    const uint2 vs = g.vs[p], us = g.us[p];
    const uint32_t rpv = g.rp[p];
    const uint32_t dv = (uint32_t)(g.off[v + 1] - g.off[v]);
    const uint32_t vlen = dv - 1u - rpv, ulen = du - 1u - j;
    const unsigned long long val[7] = {vs.x, vs.y, (unsigned long long)(vlen - vs.x - vs.y),
                                       us.x, us.y, (unsigned long long)(ulen - us.x - us.y), n - du - dv};
#pragma unroll
    for (int c = 0; c < 3; ++c)
        if (cuv == (uint32_t)(c + 1))
#pragma unroll
            for (int k = 0; k < 7; ++k) acc[c][k] += val[k];
}

// Bulk counts of the census's pairs: per dir(u,v) code c (tricode bits 1|2, 1..3),
// raw[7(c-1) + d - 1] += the entries of N[v] past u with direction class d (v-only third
// vertices before the common ones come off), raw[7(c-1) + 3 + d - 1] += those of N[u] past v
// (u-only), raw[7(c-1) + 6] += the dyadic base n - d_u - d_v (steps 2.1.2 - 2.1.3 before the
// common neighbours).  The pairs are the plan's: its CTA items (at most kMaxItemPairs pairs of
// one vertex each, a warp per item), then the one-warp vertices in blocks of 32 consecutive
// ones, whose upper pairs are consecutive in the table order and are walked as one flattened
// range.  Work comes from the counters ctr[2] (items) and ctr[3] (blocks), zeroed by the caller.
// Batched: item.pad and the blocks' third field name the graph (graphs[g], sums at raw +
// kBatchStride g); serving wave: request slices as in the census kernel's wave mode (sums at
// the request's scratch, WaveReq.out).
struct BulkParams {
    GraphDev g;
    const Item* items;
    uint32_t n_items;
    uint32_t wb, we;              // single graph: the one-warp vertices
    const GraphDev* graphs;       // batched
    const uint4* wblocks;
    uint32_t n_wblocks;
    const WaveReq* reqs;          // serving wave (n_items, n_wblocks: the wave's totals)
    uint32_t n_reqs;
    uint32_t* ctr;
    unsigned long long* raw;
};

__device__ __forceinline__ void flush_bulk(unsigned long long (&acc)[3][7], unsigned long long* raw, uint32_t lane) {
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int k = 0; k < 7; ++k) {
            unsigned long long s = acc[c][k];
            for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0 && s) atomicAdd(&raw[7 * c + k], s);
            acc[c][k] = 0ull;
        }
}

template <int MODE>
__global__ void __launch_bounds__(256, 4) k_pair_bulk(BulkParams P) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t le_mask = (2u << lane) - 1u;
    unsigned long long acc[3][7];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int k = 0; k < 7; ++k) acc[c][k] = 0ull;
    GraphDev G = P.g;
    unsigned long long* raw = P.raw;
    uint32_t cur_graph = 0xffffffffu;
    auto use_graph = [&](uint32_t gi) {
        if (cur_graph != 0xffffffffu) flush_bulk(acc, raw, lane);
        cur_graph = gi;
        if (MODE == kTriWave) {
            G = P.reqs[gi].g;
            raw = P.reqs[gi].out;
        } else {
            G = P.graphs[gi];
            raw = P.raw + (uint64_t)kBatchStride * gi;
        }
    };
    // the CTA items, a warp each
    for (;;) {
        uint32_t it = 0;
        if (lane == 0) it = atomicAdd(&P.ctr[2], 1u);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= P.n_items) break;
        Item w;
        if (MODE == kTriWave) {
            const uint32_t r = find_req(P.n_reqs, it, [&](uint32_t q) { return P.reqs[q].item_pre; });
            w = P.reqs[r].items[it - P.reqs[r].item_pre];
            if (r != cur_graph) use_graph(r);
        } else {
            w = P.items[it];
            if (MODE == kTriBatch && w.pad != cur_graph) use_graph(w.pad);
        }
        const unsigned long long n = G.n;
        const uint64_t ubase = G.off[w.u];
        const uint32_t du = (uint32_t)(G.off[w.u + 1] - ubase);
        const uint64_t pb = G.ub[w.u] - G.up[w.u];
        for (uint32_t j = w.j0 + lane; j < w.j1; j += 32) bulk_pair(G, n, du, j, G.adj[ubase + j], pb + j, acc);
    }
    // the one-warp vertices, 32 consecutive ones per grab
    for (;;) {
        uint32_t blk = 0;
        if (lane == 0) blk = atomicAdd(&P.ctr[3], 1u);
        blk = __shfl_sync(0xffffffffu, blk, 0);
        uint64_t base, end;
        if (MODE == kTriWave) {
            if (blk >= P.n_wblocks) break;
            const uint32_t r = find_req(P.n_reqs, blk, [&](uint32_t q) { return P.reqs[q].block_pre; });
            if (r != cur_graph) use_graph(r);
            const WaveReq& q = P.reqs[r];
            base = q.warp_begin + ((uint64_t)(blk - q.block_pre) << q.pad);
            end = base + (1u << q.pad) < q.warp_end ? base + (1u << q.pad) : q.warp_end;
        } else if (MODE == kTriBatch) {
            if (blk >= P.n_wblocks) break;
            const uint4 wbk = P.wblocks[blk];
            if (wbk.z != cur_graph) use_graph(wbk.z);
            base = wbk.x;
            end = wbk.y;
        } else {
            base = (uint64_t)P.wb + 32ull * blk;
            if (base >= P.we) break;
            end = base + 32u < P.we ? base + 32u : P.we;
        }
        const unsigned long long n = G.n;
        const uint64_t u = base + lane;
        const bool ok = u < end;
        uint64_t ubase = ok ? G.off[u] : 0ull;
        uint32_t du = ok ? (uint32_t)(G.off[u + 1] - ubase) : 0u;
        uint32_t upu = ok ? G.up[u] : 0u;
        uint32_t cnt = du - upu;                  // upper pairs of u (0 past the block)
        const uint64_t pstart = G.ub[base];       // table index of the block's first pair
        // compact the vertices with upper pairs into lanes 0 .. nv-1, keeping their order
        const uint32_t nz = __ballot_sync(0xffffffffu, cnt != 0u);
        if (!nz) continue;
        const uint32_t nv = __popc(nz);
        const uint32_t src = __fns(nz, 0, lane + 1) & 31u;
        ubase = __shfl_sync(0xffffffffu, ubase, src);
        du = __shfl_sync(0xffffffffu, du, src);
        upu = __shfl_sync(0xffffffffu, upu, src);
        cnt = __shfl_sync(0xffffffffu, cnt, src);
        if ((uint32_t)lane >= nv) cnt = 0u;
        uint32_t incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const uint32_t excl = incl - cnt;
        const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
        int seg_prev = -1;
        for (uint32_t r0 = 0; r0 < total; r0 += 32) {
            const bool st = (uint32_t)lane < nv && excl >= r0 && excl < r0 + 32u;
            const uint32_t M = __reduce_or_sync(0xffffffffu, st ? (1u << (excl - r0)) : 0u);
            const int seg = seg_prev + __popc(M & le_mask);
            seg_prev = __shfl_sync(0xffffffffu, seg, 31);
            const uint32_t sg = (uint32_t)seg & 31u;
            const uint32_t sP = __shfl_sync(0xffffffffu, excl, sg);
            const uint64_t sB = __shfl_sync(0xffffffffu, ubase, sg);
            const uint32_t sD = __shfl_sync(0xffffffffu, du, sg), sU = __shfl_sync(0xffffffffu, upu, sg);
            const uint32_t i = r0 + lane;
            if (i >= total) continue;
            const uint32_t j = sU + (i - sP);         // the pair's position in N[u]
            bulk_pair(G, n, sD, j, G.adj[sB + j], pstart + i, acc);
        }
    }
    if (MODE == kTriSingle || cur_graph != 0xffffffffu) flush_bulk(acc, raw, lane);
}

struct Table64 {
    uint8_t t[64];
};

// 16 classes from the bulk sums and the triangle tricodes (see the file comment); adds
// classes 1..15 into out16 (index 0 untouched).  One block of 64 threads.
// Batched: block g folds raw + kBatchStride g and hist + kBatchStride g into out16 + 16 g.
__global__ void k_tri_fold(const unsigned long long* __restrict__ raw, const unsigned long long* __restrict__ hist,
                           Table64 T, unsigned long long* out16) {
    __shared__ unsigned long long s[16];
    const uint32_t t = threadIdx.x;
    raw += (uint64_t)kBatchStride * blockIdx.x;
    hist += (uint64_t)kBatchStride * blockIdx.x;
    out16 += 16ull * blockIdx.x;
    if (t < 16) s[t] = 0ull;
    __syncthreads();
    if (t < 21) {
        const uint32_t c = t / 7 + 1, k = t % 7;
        const unsigned long long v = raw[t];
        uint32_t cls;
        if (k < 3) cls = T.t[c | ((k + 1) << 2)];          // v-only: dir(v,w) = k + 1
        else if (k < 6) cls = T.t[c | ((k - 2) << 4)];     // u-only: dir(u,w) = k - 2
        else cls = c == 3u ? 2u : 1u;                       // dyadic base: 102 if mutual, else 012
        if (v) atomicAdd(&s[cls], v);
    }
    const unsigned long long h = hist[t];
    if (h) {
        const uint32_t cab = t & 3u;                                   // tricode bits of the pair (a, b)
        const uint32_t dac = (t >> 4) & 3u;                            // dir(a,c) seen from a
        const uint32_t dbc = (t >> 2) & 3u;                            // dir(b,c) seen from b
        const uint32_t dcb = ((dbc & 1u) << 1) | (dbc >> 1);           // dir(c,b) seen from c
        const uint32_t cac = ((dac & 1u) << 1) | (dac >> 1);           // tricode bits of the pair (a, c)
        const unsigned long long m = 0ull - h;
        atomicAdd(&s[T.t[t]], h);                                      // the triad, at (a, b) with w = c
        atomicAdd(&s[T.t[cab | (dac << 4)]], m);                       // c is no u-only vertex of (a, b)
        atomicAdd(&s[T.t[cab | (dbc << 2)]], m);                       // nor a v-only one
        atomicAdd(&s[T.t[cac | (dcb << 2)]], m);                       // b is no v-only vertex of (a, c)
        atomicAdd(&s[cab == 3u ? 2u : 1u], h);                         // a common neighbour of each pair
        atomicAdd(&s[dac == 3u ? 2u : 1u], h);
        atomicAdd(&s[dbc == 3u ? 2u : 1u], h);
    }
    __syncthreads();
    if (t >= 1 && t < 16 && s[t]) atomicAdd(&out16[t], s[t]);
}

// Serving: fold each finished request's scratch (block r) into its 16 counts in mapped host
// memory (dst + 16 r, index 0 = 0) and zero the scratch for the slot's next request.
struct TriCollect {
    unsigned long long* src[kMaxWave];
    unsigned long long* dst;
    uint32_t n;
};

__global__ void k_tri_collect(TriCollect a, Table64 T) {
    __shared__ unsigned long long out[16];
    const uint32_t r = blockIdx.x, t = threadIdx.x;
    if (r >= a.n) return;
    if (t < 16) out[t] = 0ull;
    __syncthreads();
    unsigned long long* sc = a.src[r];
    // the same fold as k_tri_fold, into shared memory
    if (t < 21) {
        const uint32_t c = t / 7 + 1, k = t % 7;
        const unsigned long long v = sc[t];
        const uint32_t cls = k < 3 ? T.t[c | ((k + 1) << 2)] : (k < 6 ? T.t[c | ((k - 2) << 4)] : (c == 3u ? 2u : 1u));
        if (v) atomicAdd(&out[cls], v);
    }
    const unsigned long long h = sc[32 + t];
    if (h) {
        const uint32_t cab = t & 3u, dac = (t >> 4) & 3u, dbc = (t >> 2) & 3u;
        const uint32_t dcb = ((dbc & 1u) << 1) | (dbc >> 1), cac = ((dac & 1u) << 1) | (dac >> 1);
        const unsigned long long m = 0ull - h;
        atomicAdd(&out[T.t[t]], h);
        atomicAdd(&out[T.t[cab | (dac << 4)]], m);
        atomicAdd(&out[T.t[cab | (dbc << 2)]], m);
        atomicAdd(&out[T.t[cac | (dcb << 2)]], m);
        atomicAdd(&out[cab == 3u ? 2u : 1u], h);
        atomicAdd(&out[dac == 3u ? 2u : 1u], h);
        atomicAdd(&out[dbc == 3u ? 2u : 1u], h);
    }
    __syncthreads();
    if (t < 16) a.dst[16 * r + t] = t ? out[t] : 0ull;
    for (uint32_t k = t; k < kBatchStride; k += blockDim.x) sc[k] = 0ull;
}

std::atomic<uint64_t> g_tri_attr[4] = {};

size_t tri_smem(uint32_t chunk, bool old) {
    const size_t slots = 2ull * chunk;
    return sizeof(uint32_t) * (slots * (old ? 2 : 1) + (size_t)kWarps * kWarpSlots * (old ? 2 : 1) + kWarps * 64) +
           (old ? 9 * 64 : 0);
}

// form: 0 single graph, 1 caller-id states (64-state census), 2 batched, 3 serving wave
tc_status tri_prepare(int form, size_t smem) {
    int dev = 0;
    TC_CUDA(cudaGetDevice(&dev));
    const uint64_t bit = 1ull << (dev & 63);
    const void* fns[4] = {(const void*)k_triangles<false, kTriSingle>, (const void*)k_triangles<true, kTriSingle>,
                          (const void*)k_triangles<false, kTriBatch>, (const void*)k_triangles<false, kTriWave>};
    const void* fn = fns[form];
    int optin = 0;
    TC_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    cudaFuncAttributes fa;
    TC_CUDA(cudaFuncGetAttributes(&fa, fn));
    const int lim = optin - (int)fa.sharedSizeBytes;
    if ((int)smem > lim) return fail(TC_ERR_ARG, "chunk_entries too large for this GPU's shared memory");
    if (!(g_tri_attr[form].load() & bit)) {
        TC_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
        g_tri_attr[form].fetch_or(bit);
    }
    return TC_OK;
}

tc_status fold_table(Table64* T) {
    const uint8_t* ht = host_tricode_table();
    if (!ht) return fail(TC_ERR_ARG, "tricode table derivation failed");
    std::memcpy(T->t, ht, 64);
    return TC_OK;
}

}  // namespace

tc_status triangles_launch(const GraphDev& gd, const Opts& o, const Item* items, uint32_t n_items, uint32_t warp_begin,
                           uint32_t warp_end, uint32_t* ctr, const uint32_t* old, const uint8_t* d_perm_state,
                           unsigned long long* d_hist64, unsigned long long* d_vcost, cudaStream_t st,
                           unsigned long long* d_phase) {
    const bool is_old = old != nullptr;
    const size_t smem = tri_smem(o.chunk, is_old);
    TC_TRY(tri_prepare(is_old ? 1 : 0, smem));
    TriParams P;
    std::memset(&P, 0, sizeof(P));
    P.g = gd;
    P.items = items;
    P.n_items = n_items;
    P.warp_begin = warp_begin;
    P.warp_end = warp_end;
    P.wshift = warp_block_shift(warp_end - warp_begin, (unsigned)census_grid(o));
    P.chunk = o.chunk;
    P.ctr = ctr;
    P.old = old;
    P.perm_state = d_perm_state;
    P.hist = d_hist64;
    P.vcost = d_vcost;
    P.phase = d_phase;
    const unsigned grid = (unsigned)census_grid(o);
    if (is_old) k_triangles<true, kTriSingle><<<grid, kThreads, smem, st>>>(P);
    else k_triangles<false, kTriSingle><<<grid, kThreads, smem, st>>>(P);
    TC_LAUNCH("k_triangles");
    return TC_OK;
}

tc_status triangle_census_enqueue(GraphStore& g, const Opts& o, const Item* items, uint32_t n_items,
                                  uint32_t warp_begin, uint32_t warp_end, cudaStream_t st, unsigned long long* d_out16,
                                  unsigned long long* d_vcost, unsigned long long* d_phase) {
    if (g.e_sym == 0) return TC_OK;
    if (!g.vs.p) return fail(TC_ERR_ARG, "the triangle form needs the per upper pair tables");
    if (!g.tri.p) TC_TRY(g.tri.alloc_persistent(sizeof(unsigned long long) * kBatchStride));
    unsigned long long* raw = g.tri.as<unsigned long long>();   // [0, 21) bulk sums, [32, 96) triangle tricodes
    unsigned long long* hist = raw + 32;
    TC_CUDA(cudaMemsetAsync(raw, 0, sizeof(unsigned long long) * kBatchStride, st));
    TC_CUDA(cudaMemsetAsync(g.ctr.p, 0, sizeof(uint32_t) * 4, st));
    const GraphDev gd = g.dev();
    const uint64_t units = (uint64_t)n_items + (warp_end - warp_begin + 31u) / 32u;
    if (units) {
        BulkParams B;
        std::memset(&B, 0, sizeof(B));
        B.g = gd;
        B.items = items;
        B.n_items = n_items;
        B.wb = warp_begin;
        B.we = warp_end;
        B.ctr = g.ctr.as<uint32_t>();
        B.raw = raw;
        k_pair_bulk<kTriSingle><<<grid_for(units * 32, 256, 4u * (unsigned)sm_count()), 256, 0, st>>>(B);
        TC_LAUNCH("k_pair_bulk");
    }
    TC_TRY(triangles_launch(gd, o, items, n_items, warp_begin, warp_end, g.ctr.as<uint32_t>(), nullptr, nullptr, hist,
                            d_vcost, st, d_phase));
    Table64 T;
    TC_TRY(fold_table(&T));
    k_tri_fold<<<1, 64, 0, st>>>(raw, hist, T, d_out16);
    TC_LAUNCH("k_tri_fold");
    return TC_OK;
}

tc_status triangle_census_batch(const GraphDev* d_graphs, uint32_t k, const Item* items, uint32_t n_items,
                                const uint4* wblocks, uint32_t n_wblocks, const Opts& o, uint32_t* ctr,
                                unsigned long long* d_scratch, unsigned long long* d_out, cudaStream_t st) {
    if (k == 0) return TC_OK;
    const size_t smem = tri_smem(o.chunk, false);
    TC_TRY(tri_prepare(2, smem));
    TC_CUDA(cudaMemsetAsync(d_scratch, 0, sizeof(unsigned long long) * kBatchStride * k, st));
    const uint64_t units = (uint64_t)n_items + n_wblocks;
    if (units) {
        BulkParams B;
        std::memset(&B, 0, sizeof(B));
        B.items = items;
        B.n_items = n_items;
        B.graphs = d_graphs;
        B.wblocks = wblocks;
        B.n_wblocks = n_wblocks;
        B.ctr = ctr;
        B.raw = d_scratch;
        k_pair_bulk<kTriBatch><<<grid_for(units * 32, 256, 4u * (unsigned)sm_count()), 256, 0, st>>>(B);
        TC_LAUNCH("k_pair_bulk (batched)");
        TriParams P;
        std::memset(&P, 0, sizeof(P));
        P.items = items;
        P.n_items = n_items;
        P.chunk = o.chunk;
        P.ctr = ctr;
        P.hist = d_scratch + 32;
        P.graphs = d_graphs;
        P.wblocks = wblocks;
        P.n_wblocks = n_wblocks;
        k_triangles<false, kTriBatch><<<(unsigned)census_grid(o), kThreads, smem, st>>>(P);
        TC_LAUNCH("k_triangles (batched)");
    }
    Table64 T;
    TC_TRY(fold_table(&T));
    k_tri_fold<<<k, 64, 0, st>>>(d_scratch, d_scratch + 32, T, d_out);
    TC_LAUNCH("k_tri_fold (batched)");
    return TC_OK;
}

tc_status triangle_census_wave(const WaveReq* d_reqs, uint32_t n_reqs, uint32_t total_items, uint32_t total_blocks,
                               const Opts& o, unsigned grid, uint32_t* ctr, cudaStream_t st) {
    if (n_reqs > kMaxWave) return fail(TC_ERR_RANGE, "wave larger than kMaxWave requests");
    const size_t smem = tri_smem(o.chunk, false);
    TC_TRY(tri_prepare(3, smem));
    BulkParams B;
    std::memset(&B, 0, sizeof(B));
    B.n_items = total_items;
    B.n_wblocks = total_blocks;
    B.reqs = d_reqs;
    B.n_reqs = n_reqs;
    B.ctr = ctr;
    const uint64_t units = (uint64_t)total_items + total_blocks;
    k_pair_bulk<kTriWave><<<grid_for(units * 32, 256, 4u * (unsigned)sm_count()), 256, 0, st>>>(B);
    TC_LAUNCH("k_pair_bulk (wave)");
    TriParams P;
    std::memset(&P, 0, sizeof(P));
    P.n_items = total_items;
    P.n_wblocks = total_blocks;
    P.reqs = d_reqs;
    P.n_reqs = n_reqs;
    P.chunk = o.chunk;
    P.ctr = ctr;
    k_triangles<false, kTriWave><<<grid, kThreads, smem, st>>>(P);
    TC_LAUNCH("k_triangles (wave)");
    return TC_OK;
}

tc_status triangle_collect(unsigned long long* const* scratch, uint32_t n, unsigned long long* d_dst, cudaStream_t st) {
    if (n == 0) return TC_OK;
    if (n > kMaxWave) return fail(TC_ERR_RANGE, "more finished requests than a wave holds");
    TriCollect a;
    std::memset(&a, 0, sizeof(a));
    for (uint32_t k = 0; k < n; ++k) a.src[k] = scratch[k];
    a.dst = d_dst;
    a.n = n;
    Table64 T;
    TC_TRY(fold_table(&T));
    k_tri_collect<<<n, 64, 0, st>>>(a, T);
    TC_LAUNCH("k_tri_collect");
    return TC_OK;
}

}  // namespace tc
