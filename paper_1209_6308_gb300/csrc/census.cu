// census.cu - the triad census hot path (Fig. 5, steps 2 - 2.1.4.2) on the GPU.
//
// Vertices are in descending-degree ids, so for every connected pair (u, v) with u < v
// (step 2.1) u is the endpoint of larger degree.  For each pair the kernel accounts for every
// third vertex w of S = N[u] u N[v] \ {u, v} (step 2.1.1, the union of Sec. 6 / Fig. 8) once:
//   - the v side: entries w of N[v] are looked up in N[u], staged in shared memory (a direct
//     map of two direction bits per id for the lowest ids, an open-addressing hash for the
//     rest).  A common w > v is a triad with both u-w and v-w links (classified through the
//     64-entry tricode table, step 2.1.4.1); a w in N[v] only, with w > u, is a triad through
//     v alone (the canonical rule of step 2.1.4).  With the per upper pair tables of the graph
//     the walk starts past u, and the triads through v alone are the table's direction-class
//     counts of N[v] past u minus the common neighbours found; the common neighbours below u
//     reach the pair's dyadic count as credits from the pairs (w, u) that found its triangle.
//   - the u side: the w in N[u] past v (the rest of S that the canonical rule keeps) are
//     triads through u alone, whose class depends only on dir(u,v) and dir(u,w).
//     TC_ALGO_SUFFIX takes their counts per direction class (from the per-pair table, or from
//     prefix counts of the staged chunk), less the common ones the v side already counted;
//     TC_ALGO_UNION walks them one by one.
// The dyadic triads of the pair (steps 2.1.2-2.1.3) add n - |S| - 2 = n - d_u - d_v + |common|
// to 012 or 102.  Counts go to per-lane packed 8-bit class counters, flushed by warp
// reductions into per-lane 64-bit class totals, and at the end to 16 64-bit atomics per CTA
// (the private census vectors of Sec. 6).
//
// Work decomposition ("manhattan collapse" of Sec. 7): vertices with deg > warp_max_deg
// become CTA items (u, range of pairs), cut by exact pair work (plan.cuh).  N[u] is staged
// one chunk at a time; when a hub's list takes several chunks, each pair keeps a cursor into
// its sorted N[v] and every chunk consumes the N[v] entries below the next chunk's first id,
// so each N[v] entry is read once per pair with no search.  Vertices with smaller degree are
// handled one warp per vertex after the items run out, in the same persistent launch.
#include <atomic>
#include <cstring>
#include <vector>

#include "graph.cuh"
#include "plan.cuh"

namespace tc {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr uint32_t kEmpty = 0u;              // stored entries always have dir != 0
#ifndef TC_UNROLL
#define TC_UNROLL 3
#endif
#ifndef TC_MIN_BLOCKS
#define TC_MIN_BLOCKS 3
#endif
constexpr int kUnroll = TC_UNROLL;           // v-side entries in flight per lane (per trip)
constexpr uint32_t kTrip = 32u * TC_UNROLL;  // entries of N[v] per warp trip

// Membership of the staged chunk of N[u]: ids below kMapIds (the highest-degree vertices, which
// make up most of the N[v] entries walked) sit in a direct map of two direction bits per id;
// the rest in the open-addressing hash.
// MAP selects the map; without it (graphs whose walks meet mostly ids past the map's range)
// every entry of the chunk goes to the hash.
template <int ALGO, bool MAP> constexpr uint32_t map_ids() {
    return MAP ? (ALGO == TC_ALGO_UNION ? kMapIdsUnion : kMapIdsSuffix) : 0u;
}
// Hash slots per staged entry.  The suffix form probes the hash for every walked id beyond the
// map, and a warp waits for its longest probe chain: at most a quarter full, the chains stay
// short (scale-20 census 19.13 -> 17.94 ms against half full at twice the chunk).
template <int ALGO, bool MAP> constexpr uint32_t hash_factor() { return ALGO == TC_ALGO_UNION ? 2u : 4u; }

__device__ uint8_t d_tricode_class[64];

struct Params {
    GraphDev g;
    const Item* items;
    uint32_t n_items;
    uint32_t warp_begin, warp_end;
    uint32_t wshift;               // warp tier: a warp takes 2^wshift consecutive vertices per grab
    uint32_t chunk;
    uint32_t warp_max;
    uint32_t* ctr;                 // [0] next item, [1] next warp-tier vertex block
    unsigned long long* out;       // 16 accumulators
    unsigned long long* vcost;     // optional [n]: SM cycles spent per vertex u (items summed)
    unsigned long long* phase;     // optional [3 * gridDim]: globaltimer at start, end of items, end
    // batched launch: item.pad is the graph index, warp-tier blocks are (u0, u1, graph), and
    // graph g's counts go to out[16 g ..]
    const GraphDev* graphs;
    const uint4* wblocks;
    uint32_t n_wblocks;
    // wave launch (serving): request r's items and warp-tier blocks, counts to out[16 r ..]
    const WaveReq* reqs;
    uint32_t n_reqs;
};

enum { kModeSingle = 0, kModeBatch = 1, kModeWave = 2 };

// index r of the last request whose prefix is <= i (prefixes ascend, pre[0] = 0)
template <typename F>
__device__ __forceinline__ uint32_t wave_find(uint32_t count, uint32_t i, F pre) {
    uint32_t lo = 0, hi = count;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (pre(mid) <= i) lo = mid; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// tricode bits of the u-v link from dir(u,v) (bit 0 u->v, bit 1 v->u): 2 = u->v, 1 = v->u
__device__ __forceinline__ uint32_t code_uv(uint32_t duv) { return ((duv & 1u) << 1) | (duv >> 1); }
__device__ __forceinline__ uint32_t hash_slot(uint32_t x, int hb) { return (x * 2654435761u) >> (32 - hb); }

__device__ __forceinline__ unsigned long long pack3(uint32_t c1, uint32_t c2, uint32_t c3) {
    return (unsigned long long)c1 | ((unsigned long long)c2 << 21) | ((unsigned long long)c3 << 42);
}

// counts of direction classes 1, 2, 3 among the 32 lanes' values (0 = none), packed
__device__ __forceinline__ unsigned long long ballot3(uint32_t e) {
    return pack3(__popc(__ballot_sync(0xffffffffu, e == 1u)), __popc(__ballot_sync(0xffffffffu, e == 2u)),
                 __popc(__ballot_sync(0xffffffffu, e == 3u)));
}

// Per-lane counting state.
//   racc   lane c < 16 holds the 64-bit total of class c.
//   lo/hi  packed 8-bit counters per class (lo: classes 0-7, hi: 8-15) for triads classified one
//          at a time (common neighbours past v, and the union walk's u-only triads), flushed
//          into racc by a warp reduction before any byte can overflow.
struct Counts {
    unsigned long long lo, hi, racc;
    uint32_t trips;   // warp-uniform: batches since the last flush, each adding <= kUnroll per byte
};

// Per-pair counts of one lane, 16-bit fields 1..3 keyed by a direction class d:
//   vo[d]  third vertices w reached through v only, w > u, with dir(v,w) = d
//   fo[d]  common neighbours w > v with dir(u,w) = d (their u-only count is taken back)
//   cm     common neighbours (toward |N[u] n N[v]|)
struct PairAcc {
    unsigned long long vo, fo;
    uint32_t cm, trips;
};

// A trip adds at most kUnroll to any packed byte or per-pair field of a lane.
constexpr uint32_t kFlushTrips = 255u / kUnroll;             // packed 8-bit class counters
constexpr uint32_t kPairSpillTrips = 65000u / kUnroll;       // per-pair 16-bit fields

__device__ __forceinline__ void pk_add(Counts& k, uint32_t cls) {
    const unsigned long long inc = 1ull << ((cls & 7u) << 3);
    if (cls & 8u) k.hi += inc; else k.lo += inc;
}

__device__ __forceinline__ void pk_flush(Counts& k, int lane) {
#pragma unroll
    for (int c = 0; c < 16; ++c) {
        const unsigned long long pp = c < 8 ? k.lo : k.hi;
        const uint32_t sum = __reduce_add_sync(0xffffffffu, (uint32_t)((pp >> ((c & 7) * 8)) & 255ull));
        if (lane == c) k.racc += sum;
    }
    k.lo = k.hi = 0;
    k.trips = 0;
}

__device__ __forceinline__ void pk_maybe_flush(Counts& k, int lane) {
    if (k.trips >= kFlushTrips) pk_flush(k, lane);
}

// Fold one pair's per-lane counts into the class lanes.  suf holds the pair's u-only triads
// per dir(u,w) class (packed 21-bit fields; 0 for the union walk, which counts them one by
// one), dy the dyadic base n - d_u - d_v (0 after the pair's first chunk); the common
// neighbours complete the dyadic count n - |S| - 2 (steps 2.1.2 - 2.1.3).
// VT (per-pair tables): the walk covers only the w > u of N[v], vo holds the common
// neighbours by dir(v,w), and vsv = (class-1 count, class-2 count, length) of N[v] past u (zero
// except in the pair's first fold), so the v-only triads are the suffix counts minus vo (mod
// 2^64 across folds); the common neighbours w < u of the pair were credited by the pairs
// (w, u) that met this pair's triangle, so the dyadic count takes only the walked ones.
// usv (VT): the u side the same way, (class-1, class-2 counts, length) of N[u] past v, or zero
// (later folds, and the union walk, which counts the u side one by one).
template <bool VT>
__device__ __forceinline__ void pair_fold(Counts& k, PairAcc& pa, int lane, uint32_t duv, uint32_t cuv,
                                          const uint8_t* sT, unsigned long long suf, unsigned long long dy,
                                          uint3 vsv = make_uint3(0u, 0u, 0u), uint3 usv = make_uint3(0u, 0u, 0u)) {
    uint32_t cm = VT ? 0u : __reduce_add_sync(0xffffffffu, pa.cm);
#pragma unroll
    for (uint32_t d = 1; d <= 3; ++d) {
        const uint32_t vs = __reduce_add_sync(0xffffffffu, (uint32_t)((pa.vo >> (16 * d)) & 0xffffull));
        const uint32_t fs = __reduce_add_sync(0xffffffffu, (uint32_t)((pa.fo >> (16 * d)) & 0xffffull));
        const int cv = sT[cuv | (d << 2)], cu = sT[cuv | (d << 4)];
        if (VT) {
            cm += vs;
            const uint32_t tot = d == 1 ? vsv.x : d == 2 ? vsv.y : vsv.z - vsv.x - vsv.y;
            if (lane == cv) k.racc += (unsigned long long)tot - (unsigned long long)vs;
        } else {
            if (lane == cv) k.racc += vs;
        }
        if (VT) {
            const uint32_t tot = d == 1 ? usv.x : d == 2 ? usv.y : usv.z - usv.x - usv.y;
            if (lane == cu) k.racc += (unsigned long long)tot - (unsigned long long)fs;
        } else {
            if (lane == cu) k.racc += ((suf >> (21 * (d - 1))) & 0x1fffffull) - (unsigned long long)fs;
        }
    }
    if (lane == (duv == 3u ? 2 : 1)) k.racc += dy + cm;
    pa.vo = pa.fo = 0;
    pa.cm = 0;
    pa.trips = 0;
}

// B entries [k0 + 32r + lane], cut at dv and, for a chunk with a successor, at hi_key
template <bool HAS_HI>
__device__ __forceinline__ void load_trip(uint32_t (&x)[kUnroll], const uint32_t* __restrict__ B, uint32_t k0,
                                          uint32_t dv, uint32_t hi_key, int lane) {
#pragma unroll
    for (int r = 0; r < kUnroll; ++r) {
        const uint32_t k = k0 + 32 * r + lane;
        uint32_t e = k < dv ? __ldg(B + k) : 0u;
        if (HAS_HI && e >= hi_key) e = 0u;
        x[r] = e;
    }
}

// Classify one trip of N[v] entries (0 = no entry) against the staged hash of N[u]:
//   found:  a common neighbour; counts toward |N[u] n N[v]| and, past v, is a triad with both
//           links (its u-only count from the u side is taken back);
//   else:   reached through v only; kept when w > u (the canonical rule of step 2.1.4).
// VT: every entry walked is past u; a common neighbour is counted by dir(v,w) (the v-only
// triads come from the pair's suffix counts), and one past v also credits the pair (v, w)
// with the common neighbour u, in the dyadic class of dir(v,w).
template <bool VT, uint32_t MAPIDS>
__device__ __forceinline__ void classify_trip(const uint32_t (&cur)[kUnroll], const uint32_t* sH,
                                              const uint32_t* sMap, int hb, uint32_t hmask, uint32_t u, uint32_t v,
                                              uint32_t cuv, const uint8_t* sT, Counts& k, PairAcc& pa) {
    uint32_t h[kUnroll], e[kUnroll];
#pragma unroll
    for (int r = 0; r < kUnroll; ++r) {
        const uint32_t x = cur[r] >> 2;
        h[r] = hash_slot(x, hb);
        if (!cur[r]) {
            e[r] = kEmpty;
        } else if (x < MAPIDS) {   // direct map: the entry's direction bits, 0 if absent
            const uint32_t dir = (sMap[x >> 4] >> ((x & 15u) << 1)) & 3u;
            e[r] = dir ? ((cur[r] & ~3u) | dir) : kEmpty;
        } else {
            e[r] = sH[h[r]];
        }
    }
#pragma unroll
    for (int r = 0; r < kUnroll; ++r) {
        while (e[r] != kEmpty && (e[r] >> 2) != (cur[r] >> 2)) {
            h[r] = (h[r] + 1) & hmask;
            e[r] = sH[h[r]];
        }
    }
#pragma unroll
    for (int r = 0; r < kUnroll; ++r) {
        const uint32_t x = cur[r] >> 2, dvw = cur[r] & 3u;
        if (VT) {
            if (e[r] != kEmpty) {
                pa.vo += 1ull << (dvw << 4);
                if (x > v) {
                    const uint32_t duw = e[r] & 3u;
                    pk_add(k, sT[cuv | (dvw << 2) | (duw << 4)]);
                    pa.fo += 1ull << (duw << 4);
                    pk_add(k, dvw == 3u ? 2u : 1u);
                }
            }
        } else if (e[r] != kEmpty) {
            ++pa.cm;
            if (x > v) {
                const uint32_t duw = e[r] & 3u;
                pk_add(k, sT[cuv | (dvw << 2) | (duw << 4)]);
                pa.fo += 1ull << (duw << 4);
            }
        } else if (cur[r] && x > u) {
            pa.vo += 1ull << (dvw << 4);
        }
    }
    ++k.trips;
    ++pa.trips;
}

// The v side of one pair (u, v) in a chunked hub: every w of N[v] from position k0 up to the
// chunk's id bound is looked up in the staged hash of N[u].  Returns the position after the
// last entry taken.
template <bool VT, uint32_t MAPIDS>
__device__ __forceinline__ uint32_t v_side_chunk(const uint32_t* __restrict__ B, uint32_t k0, uint32_t dv,
                                                 uint32_t hi_key, const uint32_t* sH, const uint32_t* sMap, int hb,
                                                 uint32_t hmask,
                                                 uint32_t u, uint32_t v, uint32_t duv, uint32_t cuv, const uint8_t* sT,
                                                 Counts& k, PairAcc& pa, int lane) {
    uint32_t cur[kUnroll], nxt[kUnroll];
    load_trip<true>(cur, B, k0, dv, hi_key, lane);
    for (;;) {
        pk_maybe_flush(k, lane);
        if (pa.trips >= kPairSpillTrips) pair_fold<VT>(k, pa, lane, duv, cuv, sT, 0ull, 0ull);
        load_trip<true>(nxt, B, k0 + kTrip, dv, hi_key, lane);
        classify_trip<VT, MAPIDS>(cur, sH, sMap, hb, hmask, u, v, cuv, sT, k, pa);
        uint32_t taken = 0;
#pragma unroll
        for (int r = 0; r < kUnroll; ++r) taken += __popc(__ballot_sync(0xffffffffu, cur[r] != 0u));
        k0 += taken;
        if (taken < kTrip) break;
#pragma unroll
        for (int r = 0; r < kUnroll; ++r) cur[r] = nxt[r];
    }
    return k0;
}

// Lanes 0-15 add their class totals to graph output `out` (batched launches switch graphs).
__device__ __forceinline__ void flush_graph(Counts& k, int lane, unsigned long long* out) {
    pk_flush(k, lane);
    if (lane < 16 && k.racc) atomicAdd(&out[lane], k.racc);
    k.racc = 0;
}

// VT: the graphs carry the per upper pair tables (GraphDev::ub, rp, vs): each N[v] walk starts
// past u, and the v-only triads come from the tables' suffix counts.
template <int ALGO, int MODE, bool VT, bool MAP>
__global__ void __launch_bounds__(kThreads, TC_MIN_BLOCKS) k_census(Params P) {
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t chunk = P.chunk;
    constexpr uint32_t kHashFactor = hash_factor<ALGO, MAP>();
    constexpr uint32_t kMap = map_ids<ALGO, MAP>();
    // map-first items (suffix form with tables): the map is staged once per item and only the
    // entries past it are chunked; the union walk keeps per-chunk staging for its sorted copy
    constexpr bool MF = VT && MAP && ALGO == TC_ALGO_SUFFIX;
    // TC_ALGO_UNION keeps the sorted chunk for its walk; the suffix form needs the hash, the
    // direction bit planes and their block prefix counts
    uint32_t* sA = reinterpret_cast<uint32_t*>(smem);                                  // [chunk] (union)
    uint32_t* sH = sA + (ALGO == TC_ALGO_UNION ? chunk : 0u);                          // [kHashFactor*chunk]
    uint32_t* sMap = sH + kHashFactor * chunk;                                         // [kMap/16]
    uint32_t* sLo = sMap + kMap / 16;                                                  // [chunk/32] dir bit 0
    uint32_t* sHi = sLo + chunk / 32;                                                  // [chunk/32] dir bit 1
    unsigned long long* sCk = reinterpret_cast<unsigned long long*>(sHi + chunk / 32); // [chunk/32+1]
    uint32_t* sCur = reinterpret_cast<uint32_t*>(sCk + chunk / 32 + 1);               // [kMaxItemPairs]
    unsigned long long* sC = reinterpret_cast<unsigned long long*>(sCur + kMaxItemPairs);  // [16]
    uint8_t* sT = reinterpret_cast<uint8_t*>(sC + 16);                                // [64]
    __shared__ uint32_t s_item, s_next, s_pl;
    __shared__ WaveReq sReq[MODE == kModeWave ? kMaxWave : 1];
    constexpr bool MULTI = MODE != kModeSingle;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid < 16) sC[tid] = 0;
    if (tid < 64) sT[tid] = d_tricode_class[tid];
    if (MODE == kModeWave)
        for (uint32_t i = tid; i < P.n_reqs; i += kThreads) sReq[i] = P.reqs[i];
    if (P.phase && tid == 0) P.phase[3 * blockIdx.x] = global_ns();
    __syncthreads();

    uint64_t n = P.g.n;
    const uint64_t* __restrict__ off = P.g.off;
    const uint32_t* __restrict__ adj = P.g.adj;
    const uint32_t* __restrict__ upv = P.g.up;
    const uint64_t* __restrict__ ubp = P.g.ub;
    const uint32_t* __restrict__ rpp = P.g.rp;
    const uint2* __restrict__ vsp = P.g.vs;
    const uint2* __restrict__ usp = P.g.us;
    uint32_t cur_graph = 0xffffffffu;          // batched: the graph whose totals the lanes hold
    unsigned long long* gout = P.out;
    Counts cnt;
    cnt.lo = cnt.hi = cnt.racc = 0;
    cnt.trips = 0;
    PairAcc pa;
    pa.vo = pa.fo = 0;
    pa.cm = pa.trips = 0;
    auto use_graph = [&](uint32_t gi) {
        if (cur_graph != 0xffffffffu) flush_graph(cnt, lane, gout);
        cur_graph = gi;
        const GraphDev G = MODE == kModeWave ? sReq[gi].g : P.graphs[gi];
        n = G.n;
        off = G.off;
        adj = G.adj;
        upv = G.up;
        ubp = G.ub;
        rpp = G.rp;
        vsp = G.vs;
        usp = G.us;
        gout = MODE == kModeWave ? sReq[gi].out : P.out + 16ull * gi;
    };

    // ---------------------------------------------------------------- CTA items
    for (;;) {
        if (tid == 0) s_item = atomicAdd(&P.ctr[0], 1u);
        __syncthreads();
        const uint32_t it = s_item;
        if (it >= P.n_items) break;
        Item w;
        if (MODE == kModeWave) {
            const uint32_t r = wave_find(P.n_reqs, it, [&](uint32_t q) { return sReq[q].item_pre; });
            w = sReq[r].items[it - sReq[r].item_pre];
            if (r != cur_graph) use_graph(r);
        } else {
            w = P.items[it];
            if (MODE == kModeBatch && w.pad != cur_graph) use_graph(w.pad);
        }
        const long long t_item = clock64();
        const uint32_t u = w.u;
        const uint64_t ubase = off[u];
        const uint32_t du = (uint32_t)(off[u + 1] - ubase);
        // MF: the map holds every entry of N[u] with an id below kMap - a prefix of the
        // ascending list, staged once per item - and only the entries past it are chunked
        // into the hash, so a hub mostly made of high-degree neighbours needs few chunks
        uint32_t pL = 0;
        if (MF) {
            for (uint32_t k = tid; k < kMap / 16; k += kThreads) sMap[k] = 0u;
            if (tid == 0) s_pl = 0;
            __syncthreads();
            for (uint32_t q = warp; q * 32u < du; q += kWarps) {
                const uint32_t idx = q * 32u + lane;
                const uint32_t e = idx < du ? adj[ubase + idx] : 0u, x = e >> 2;
                const bool in = idx < du && x < kMap;
                if (in) atomicOr(&sMap[x >> 4], (e & 3u) << ((x & 15u) << 1));
                const uint32_t bm = __ballot_sync(0xffffffffu, in);
                if (lane == 0 && bm) atomicAdd(&s_pl, (uint32_t)__popc(bm));
                if (bm != 0xffffffffu) break;   // later rows hold only ids >= kMap
            }
            __syncthreads();
            pL = s_pl;
        }
        const uint32_t nchunks = MF ? (du > pL ? (du - pL + chunk - 1) / chunk : 1u) : (du + chunk - 1) / chunk;
        const uint32_t npairs = w.j1 - w.j0;                      // <= kMaxItemPairs
        const uint32_t G = max(1u, min(32u, npairs / (4u * kWarps)));
        // table index of the item's first pair
        const uint64_t pb = VT ? ubp[u] + (w.j0 - upv[u]) : 0ull;
        if (nchunks > 1)
            for (uint32_t i = tid; i < npairs; i += kThreads) sCur[i] = VT ? rpp[pb + i] + 1u : 0u;

        for (uint32_t c = 0; c < nchunks; ++c) {
            const uint32_t a0 = MF ? pL + c * chunk : c * chunk, a1 = min(du, a0 + chunk), LA = a1 - a0;
            const uint32_t* __restrict__ Ach = adj + ubase + a0;
            int hb = 6;
            while ((1u << hb) < kHashFactor * LA) ++hb;
            const uint32_t H = 1u << hb, hmask = H - 1;
            for (uint32_t k = tid; k < H; k += kThreads) sH[k] = kEmpty;
            if (!MF)
                for (uint32_t k = tid; k < kMap / 16; k += kThreads) sMap[k] = 0u;
            if (tid == 0) s_next = 0;
            __syncthreads();
            // stage the chunk: hash (both forms), sorted copy (union), direction bit planes (suffix)
            const uint32_t nq = (LA + 31) / 32;
            for (uint32_t q = warp; q < nq; q += kWarps) {
                const uint32_t idx = q * 32 + lane;
                const uint32_t e = idx < LA ? Ach[idx] : 0u;
                if (idx < LA) {
                    if (ALGO == TC_ALGO_UNION) sA[idx] = e;
                    const uint32_t x = e >> 2;
                    if (x < kMap) {
                        atomicOr(&sMap[x >> 4], (e & 3u) << ((x & 15u) << 1));
                    } else {
                        uint32_t h = hash_slot(x, hb);
                        while (atomicCAS(&sH[h], kEmpty, e) != kEmpty) h = (h + 1) & hmask;
                    }
                }
                if (ALGO == TC_ALGO_SUFFIX && !MF) {
                    const uint32_t bl = __ballot_sync(0xffffffffu, e & 1u), bh = __ballot_sync(0xffffffffu, e & 2u);
                    if (lane == 0) {
                        sLo[q] = bl;
                        sHi[q] = bh;
                        sCk[q + 1] = pack3(__popc(bl & ~bh), __popc(bh & ~bl), __popc(bl & bh));
                    }
                }
            }
            __syncthreads();
            if (ALGO == TC_ALGO_SUFFIX && !MF) {
                if (warp == 0) {   // inclusive scan of the block counts -> counts before each block
                    unsigned long long carry = 0;
                    for (uint32_t b = 0; b < nq; b += 32) {
                        unsigned long long x = (b + lane < nq) ? sCk[b + lane + 1] : 0ull;
#pragma unroll
                        for (int o = 1; o < 32; o <<= 1) {
                            unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
                            if (lane >= o) x += y;
                        }
                        if (b + lane < nq) sCk[b + lane + 1] = x + carry;
                        carry += __shfl_sync(0xffffffffu, x, 31);
                    }
                    if (lane == 0) sCk[0] = 0;
                }
                __syncthreads();
            }

            // N[v] entries with id >= the next chunk's first id belong to later chunks
            const bool has_hi = a1 < du;
            const uint32_t hi_key = has_hi ? (adj[ubase + a1] & ~3u) : 0u;
            for (;;) {
                uint32_t base = 0;
                if (lane == 0) base = atomicAdd(&s_next, G);
                base = __shfl_sync(0xffffffffu, base, 0);
                if (base >= npairs) break;
                // prefetch the grabbed pairs: lane l holds pair base + l
                const uint32_t np = min(G, npairs - base);
                const bool okl = (uint32_t)lane < np;
                const uint32_t euv_l = okl ? adj[ubase + w.j0 + base + lane] : 0u;
                const uint64_t vb_l = okl ? off[euv_l >> 2] : 0ull;
                const uint32_t dv_l = okl ? (uint32_t)(off[(euv_l >> 2) + 1] - vb_l) : 0u;
                const uint32_t cur_l = (okl && nchunks > 1) ? sCur[base + lane] : 0u;
                // tables of the grabbed pairs, needed for their first chunk
                uint32_t rp_l = 0;
                uint2 vs_l = make_uint2(0u, 0u), us_l = make_uint2(0u, 0u);
                if (VT && c == 0 && okl) {
                    rp_l = rpp[pb + base + lane];
                    vs_l = vsp[pb + base + lane];
                    if (MF) us_l = usp[pb + base + lane];
                }
                // u side of pair t of this grab and the fold of its counts
                auto finish_pair = [&](uint32_t t, uint32_t duv, uint32_t cuv, uint32_t dv) {
                    const uint32_t j = w.j0 + base + t;
                    uint32_t s0 = (j + 1 > a0 ? j + 1 : a0) - a0;        // chunk entries past v
                    if (s0 > LA) s0 = LA;
                    unsigned long long suf = 0;
                    uint3 usv = make_uint3(0u, 0u, 0u);
                    if (MF) {
                        // the whole u side in the pair's first fold, from the table
                        if (c == 0)
                            usv = make_uint3(__shfl_sync(0xffffffffu, us_l.x, t), __shfl_sync(0xffffffffu, us_l.y, t),
                                             du - 1u - j);
                    } else if (ALGO == TC_ALGO_UNION) {
                        for (uint32_t kb = s0; kb < LA; kb += 32) {
                            pk_maybe_flush(cnt, lane);
                            const uint32_t k = kb + lane;
                            if (k < LA) pk_add(cnt, sT[cuv | ((sA[k] & 3u) << 4)]);
                            ++cnt.trips;
                        }
                    } else {
                        const uint32_t q = s0 >> 5, r = s0 & 31u;
                        const uint32_t m = (1u << r) - 1u;
                        const uint32_t bl = r ? (sLo[q] & m) : 0u, bh = r ? (sHi[q] & m) : 0u;
                        suf = sCk[nq] - sCk[q] - pack3(__popc(bl & ~bh), __popc(bh & ~bl), __popc(bl & bh));
                        if (VT) {   // the table form's fold takes the chunk's u side as counts
                            const uint32_t s1 = (uint32_t)(suf & 0x1fffffull), s2 = (uint32_t)((suf >> 21) & 0x1fffffull),
                                           s3 = (uint32_t)((suf >> 42) & 0x1fffffull);
                            usv = make_uint3(s1, s2, s1 + s2 + s3);
                        }
                    }
                    uint3 vsv = make_uint3(0u, 0u, 0u);
                    if (VT && c == 0) {
                        vsv.x = __shfl_sync(0xffffffffu, vs_l.x, t);
                        vsv.y = __shfl_sync(0xffffffffu, vs_l.y, t);
                        vsv.z = dv - 1u - __shfl_sync(0xffffffffu, rp_l, t);
                    }
                    pair_fold<VT>(cnt, pa, lane, duv, cuv, sT, suf, c == 0 ? n - du - dv : 0ull, vsv, usv);
                };
                if (has_hi) {
                    // chunked hub: each pair resumes at its cursor and stops at the chunk's id bound
                    for (uint32_t t = 0; t < np; ++t) {
                        const uint32_t euv = __shfl_sync(0xffffffffu, euv_l, t);
                        const uint64_t vb = __shfl_sync(0xffffffffu, vb_l, t);
                        const uint32_t dv = __shfl_sync(0xffffffffu, dv_l, t);
                        const uint32_t start = __shfl_sync(0xffffffffu, cur_l, t);
                        const uint32_t v = euv >> 2, duv = euv & 3u, cuv = code_uv(duv);
                        const uint32_t kend = v_side_chunk<VT, kMap>(adj + vb, start, dv, hi_key, sH, sMap, hb, hmask, u, v, duv, cuv,
                                                               sT, cnt, pa, lane);
                        if (lane == 0) sCur[base + t] = kend;
                        finish_pair(t, duv, cuv, dv);
                    }
                } else {
                    // the rest of each N[v]: one flattened (pair, trip) loop whose next trip's
                    // loads, possibly of the next pair, are in flight while this one is classified
                    // each pair's walk starts at its cursor (hub chunks), past u (tables) or at 0
                    auto start_of = [&](uint32_t q) -> uint32_t {
                        if (nchunks > 1) return __shfl_sync(0xffffffffu, cur_l, q);
                        if (VT) return __shfl_sync(0xffffffffu, rp_l, q) + 1u;
                        return 0u;
                    };
                    uint32_t t = 0, k0 = start_of(0);
                    uint32_t euv = __shfl_sync(0xffffffffu, euv_l, 0);
                    uint64_t vb = __shfl_sync(0xffffffffu, vb_l, 0);
                    uint32_t dv = __shfl_sync(0xffffffffu, dv_l, 0);
                    uint32_t cur[kUnroll], nxt[kUnroll];
                    load_trip<false>(cur, adj + vb, k0, dv, 0u, lane);
                    for (;;) {
                        pk_maybe_flush(cnt, lane);
                        const uint32_t v = euv >> 2, duv = euv & 3u, cuv = code_uv(duv);
                        if (pa.trips >= kPairSpillTrips) pair_fold<VT>(cnt, pa, lane, duv, cuv, sT, 0ull, 0ull);
                        uint32_t nt = t, nk0 = k0 + kTrip;
                        if (nk0 >= dv) {
                            nt = t + 1;
                            nk0 = nt < np ? start_of(nt) : 0u;
                        }
                        const bool more = nt < np;
                        uint32_t neuv = euv, ndv = dv;
                        uint64_t nvb = vb;
                        if (nt != t && more) {
                            neuv = __shfl_sync(0xffffffffu, euv_l, nt);
                            nvb = __shfl_sync(0xffffffffu, vb_l, nt);
                            ndv = __shfl_sync(0xffffffffu, dv_l, nt);
                        }
                        if (more) load_trip<false>(nxt, adj + nvb, nk0, ndv, 0u, lane);
                        classify_trip<VT, kMap>(cur, sH, sMap, hb, hmask, u, v, cuv, sT, cnt, pa);
                        if (nt != t) {
                            if (nchunks > 1 && lane == 0) sCur[base + t] = dv;
                            finish_pair(t, duv, cuv, dv);
                        }
                        if (!more) break;
                        t = nt;
                        k0 = nk0;
                        euv = neuv;
                        vb = nvb;
                        dv = ndv;
#pragma unroll
                        for (int r = 0; r < kUnroll; ++r) cur[r] = nxt[r];
                    }
                }
            }
            __syncthreads();   // all warps are done with this chunk before it is replaced
        }
        if (!MULTI && P.vcost && tid == 0) atomicAdd(&P.vcost[u], (unsigned long long)(clock64() - t_item));
    }
    if (P.phase && tid == 0) P.phase[3 * blockIdx.x + 1] = global_ns();

    // ---------------------------------------------------------------- one warp per vertex
    uint32_t* wA = reinterpret_cast<uint32_t*>(smem) + warp * P.warp_max;
    for (;;) {
        uint32_t u0, u1;
        if (MODE == kModeWave) {
            uint32_t b = 0;
            if (lane == 0) b = atomicAdd(&P.ctr[1], 1u);
            b = __shfl_sync(0xffffffffu, b, 0);
            if (b >= P.n_wblocks) break;
            const uint32_t r = wave_find(P.n_reqs, b, [&](uint32_t q) { return sReq[q].block_pre; });
            if (r != cur_graph) use_graph(r);
            u0 = sReq[r].warp_begin + ((b - sReq[r].block_pre) << sReq[r].pad);
            u1 = min(u0 + (1u << sReq[r].pad), sReq[r].warp_end);
        } else if (MODE == kModeBatch) {
            uint32_t b = 0;
            if (lane == 0) b = atomicAdd(&P.ctr[1], 1u);
            b = __shfl_sync(0xffffffffu, b, 0);
            if (b >= P.n_wblocks) break;
            const uint4 wb = P.wblocks[b];
            if (wb.z != cur_graph) use_graph(wb.z);
            u0 = wb.x;
            u1 = wb.y;
        } else {
            uint32_t ub = 0;
            if (lane == 0) ub = atomicAdd(&P.ctr[1], 1u << P.wshift);
            ub = __shfl_sync(0xffffffffu, ub, 0);
            if (ub >= P.warp_end - P.warp_begin) break;
            u0 = P.warp_begin + ub;
            u1 = min(u0 + (1u << P.wshift), P.warp_end);
        }
        for (uint32_t u = u0; u < u1; ++u) {
            const uint64_t ubase = off[u];
            const uint32_t du = (uint32_t)(off[u + 1] - ubase);
            const uint32_t p0 = upv[u];
            if (p0 >= du) continue;
            const long long t_vert = clock64();
            __syncwarp();
            for (uint32_t k = lane; k < du; k += 32) wA[k] = adj[ubase + k];
            __syncwarp();
            for (uint32_t jb = p0; jb < du; jb += 32) {
                const uint32_t jl = jb + lane;
                const bool okl = jl < du;
                const uint32_t euv_l = okl ? wA[jl] : 0u;
                const uint64_t vb_l = okl ? off[euv_l >> 2] : 0ull;
                const uint32_t dv_l = okl ? (uint32_t)(off[(euv_l >> 2) + 1] - vb_l) : 0u;
                uint32_t rp_l = 0;
                uint2 vs_l = make_uint2(0u, 0u);
                if (VT && okl) {
                    const uint64_t ti = ubp[u] + (jl - p0);
                    rp_l = rpp[ti];
                    vs_l = vsp[ti];
                }
                const uint32_t np = min(32u, du - jb);
                for (uint32_t t = 0; t < np; ++t) {
                    const uint32_t euv = __shfl_sync(0xffffffffu, euv_l, t);
                    const uint64_t vb = __shfl_sync(0xffffffffu, vb_l, t);
                    const uint32_t dv = __shfl_sync(0xffffffffu, dv_l, t);
                    const uint32_t v = euv >> 2, duv = euv & 3u, cuv = code_uv(duv);
                    const uint32_t* __restrict__ B = adj + vb;
                    const uint32_t j = jb + t;
                    uint3 vsv = make_uint3(0u, 0u, 0u);
                    uint32_t kstart = 0;
                    if (VT) {
                        kstart = __shfl_sync(0xffffffffu, rp_l, t) + 1u;
                        vsv = make_uint3(__shfl_sync(0xffffffffu, vs_l.x, t), __shfl_sync(0xffffffffu, vs_l.y, t),
                                         dv - kstart);
                    }
                    for (uint32_t kb = kstart; kb < dv; kb += 32) {
                        pk_maybe_flush(cnt, lane);
                        if (pa.trips >= kPairSpillTrips) pair_fold<VT>(cnt, pa, lane, duv, cuv, sT, 0ull, 0ull);
                        const uint32_t k = kb + lane;
                        if (k < dv) {
                            const uint32_t xe = __ldg(B + k), x = xe >> 2, dvw = xe & 3u;
                            uint32_t lo = 0, hi = du;
                            while (lo < hi) {
                                const uint32_t mid = (lo + hi) >> 1;
                                if ((wA[mid] >> 2) < x) lo = mid + 1; else hi = mid;
                            }
                            if (lo < du && (wA[lo] >> 2) == x) {
                                if (VT) pa.vo += 1ull << (dvw << 4);
                                else ++pa.cm;
                                if (x > v) {
                                    const uint32_t duw = wA[lo] & 3u;
                                    pk_add(cnt, sT[cuv | (dvw << 2) | (duw << 4)]);
                                    pa.fo += 1ull << (duw << 4);
                                    if (VT) pk_add(cnt, dvw == 3u ? 2u : 1u);
                                }
                            } else if (!VT && x > u) {
                                pa.vo += 1ull << (dvw << 4);
                            }
                        }
                        ++cnt.trips;
                        ++pa.trips;
                    }
                    unsigned long long suf = 0;
                    if (ALGO == TC_ALGO_UNION) {
                        for (uint32_t kb = j + 1; kb < du; kb += 32) {
                            pk_maybe_flush(cnt, lane);
                            const uint32_t k = kb + lane;
                            if (k < du) pk_add(cnt, sT[cuv | ((wA[k] & 3u) << 4)]);
                            ++cnt.trips;
                        }
                    } else {
                        for (uint32_t b = (j + 1) & ~31u; b < du; b += 32) {
                            const uint32_t k = b + lane;
                            suf += ballot3((k > j && k < du) ? (wA[k] & 3u) : 0u);
                        }
                    }
                    uint3 usv = make_uint3(0u, 0u, 0u);
                    if (VT && ALGO == TC_ALGO_SUFFIX) {   // deg(u) <= 64: the packed counts are exact
                        const uint32_t s1 = (uint32_t)(suf & 0x1fffffull), s2 = (uint32_t)((suf >> 21) & 0x1fffffull),
                                       s3 = (uint32_t)((suf >> 42) & 0x1fffffull);
                        usv = make_uint3(s1, s2, s1 + s2 + s3);
                    }
                    pair_fold<VT>(cnt, pa, lane, duv, cuv, sT, suf, n - du - dv, vsv, usv);
                }
            }
            if (!MULTI && P.vcost && lane == 0) P.vcost[u] += (unsigned long long)(clock64() - t_vert);
        }
    }

    // ---------------------------------------------------------------- totals
    if (MULTI) {
        if (cur_graph != 0xffffffffu) flush_graph(cnt, lane, gout);
    } else {
        pk_flush(cnt, lane);
        if (lane < 16 && cnt.racc) atomicAdd(&sC[lane], cnt.racc);
        __syncthreads();
        if (tid < 16 && sC[tid]) atomicAdd(&P.out[tid], sC[tid]);
    }
    if (P.phase && tid == 0) P.phase[3 * blockIdx.x + 2] = global_ns();
}

// ---------------------------------------------------------------- schedule (plan) kernels
__global__ void k_count_gt(const uint64_t* off, uint32_t n, uint32_t thr, uint32_t* cnt) {
    uint32_t c = 0;
    for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < n; x += (uint64_t)gridDim.x * blockDim.x)
        c += (off[x + 1] - off[x]) > thr;
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(cnt, c);
}

// Items of the CTA-tier vertices u < u_end (plan.cuh), one warp per task: a block of at most
// kMaxItemPairs upper pairs of one vertex.  The learned schedule fixes each vertex's item count
// from its predicted cost.
__device__ __forceinline__ double learned_items(const float* cost, uint64_t x, uint32_t item_work) {
    return cost ? fmax(1.0, ceil((double)cost[x] / (double)item_work)) : 0.0;
}

// tcnt[x] = the tasks of vertex x: its upper pairs in blocks of kMaxItemPairs
__global__ void k_task_count(const uint64_t* __restrict__ off, const uint32_t* __restrict__ up, uint32_t u_end,
                             uint32_t* tcnt) {
    for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < u_end; x += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t upper = (uint32_t)(off[x + 1] - off[x]) - up[x];
        tcnt[x] = (upper + kMaxItemPairs - 1) / kMaxItemPairs;
    }
}

// owner[t] = the vertex of task t (tasks numbered by vertex, then block)
__global__ void k_task_owner(const uint32_t* __restrict__ tbase, const uint32_t* __restrict__ tcnt, uint32_t u_end,
                             uint32_t* owner) {
    for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < u_end; x += (uint64_t)gridDim.x * blockDim.x)
        for (uint32_t b = 0, t = tbase[x]; b < tcnt[x]; ++b) owner[t + b] = (uint32_t)x;
}

// The pair range [j0, j1) of task t, owned by vertex x.
struct Task {
    uint32_t x, b, j0, j1;
};
__device__ __forceinline__ Task task_of(const GraphDev& g, const uint32_t* owner, const uint32_t* tbase, uint64_t t) {
    Task k;
    k.x = owner[t];
    k.b = (uint32_t)(t - tbase[k.x]);
    const uint32_t du = (uint32_t)(g.off[k.x + 1] - g.off[k.x]);
    k.j0 = g.up[k.x] + k.b * kMaxItemPairs;
    k.j1 = du - k.j0 > kMaxItemPairs ? k.j0 + kMaxItemPairs : du;
    return k;
}

// pu[pair] = each pair's work (by table index), tw[t] = task t's total; total[0] += the sum
// (sizes the items when the options leave item_work to the graph).
__global__ void k_plan_work(GraphDev g, const uint32_t* __restrict__ owner, const uint32_t* __restrict__ tbase,
                            const uint32_t* __restrict__ n_tasks, uint32_t chunk, int algo, unsigned long long* tw,
                            uint32_t* pu, unsigned long long* total) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint32_t T = *n_tasks;
    unsigned long long sum = 0;
    for (uint64_t t = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; t < T; t += warps) {
        const Task k = task_of(g, owner, tbase, t);
        const uint64_t ubase = g.off[k.x];
        const uint32_t du = (uint32_t)(g.off[k.x + 1] - ubase), upx = g.up[k.x];
        const uint32_t chunks = (du + chunk - 1) / chunk;
        const uint64_t tb = g.ub[k.x] - upx;
        unsigned long long w = 0;
        for (uint32_t j = k.j0 + lane; j < k.j1; j += 32) {
            const uint64_t c = pair_units(g, k.x, ubase, du, upx, j, chunks, algo);
            const uint32_t c32 = c < 0xffffffffull ? (uint32_t)c : 0xffffffffu;
            pu[tb + j] = c32;
            w += c32;
        }
        for (int o = 16; o; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
        sum += w;
        if (lane == 0) tw[t] = w;
    }
    if (lane == 0 && sum) atomicAdd(total, sum);
}

// One warp: the work of vertex x's tasks before task b (pre) and in all (W).
__device__ __forceinline__ void task_frame(const uint32_t* tbase, const uint32_t* tcnt, const unsigned long long* tw,
                                           const Task& k, unsigned long long& pre, unsigned long long& W) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t base = tbase[k.x], nt = tcnt[k.x];
    unsigned long long a = 0, p = 0;
    for (uint32_t i = lane; i < nt; i += 32) {
        const unsigned long long v = tw[base + i];
        a += v;
        if (i < k.b) p += v;
    }
    for (int o = 16; o; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        p += __shfl_xor_sync(0xffffffffu, p, o);
    }
    pre = p;
    W = a;
}

struct PlanArgs {
    const uint32_t *owner, *tbase, *tcnt, *n_tasks, *pu;
    const unsigned long long *tw, *total;
    const float* cost;
    uint32_t item_work;   // 0: adaptive_item_work(total, grid)
    uint32_t grid;
};

// cnt[t] = the items of task t (with emit: the items themselves, at items + pos[t])
template <bool EMIT>
__global__ void k_plan_items(GraphDev g, PlanArgs a, const uint32_t* __restrict__ pos, uint32_t* cnt, Item* items) {
    const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint32_t T = *a.n_tasks;
    const uint32_t iw = a.item_work ? a.item_work : adaptive_item_work(*a.total, a.grid);
    for (uint64_t t = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; t < T; t += warps) {
        const Task k = task_of(g, a.owner, a.tbase, t);
        unsigned long long pre, W;
        task_frame(a.tbase, a.tcnt, a.tw, k, pre, W);
        const float S = plan_items(W, iw, learned_items(a.cost, k.x, iw));
        const uint64_t tb = g.ub[k.x] - g.up[k.x];
        const uint32_t* pu = a.pu;
        auto units = [&](uint32_t j) { return (unsigned long long)pu[tb + j]; };
        if (EMIT) {
            Item* out = items + pos[t];
            const uint32_t c = plan_block(k.j0, k.j1, pre, W, S, units,
                                          [&](uint32_t j, uint32_t rank) { out[rank] = Item{k.x, j, 0u, 0u}; });
            plan_ends(out, c, k.j1);
        } else {
            const uint32_t c = plan_block(k.j0, k.j1, pre, W, S, units, [](uint32_t, uint32_t) {});
            if ((threadIdx.x & 31) == 0) cnt[t] = c;
        }
    }
}

// ---------------------------------------------------------------- shards (multi-GPU partition)
// The work of the census is a sequence: the plan's CTA items in order, then the one-warp-per-
// vertex tier's vertices in id order.  A shard is a contiguous range of that sequence of about
// 1/world of its work (Sec. 6-7: the pairs (u, v) are independent, so any partition of them
// sums to the census).  Work is counted in the plan's units (plan.cuh).

// units[i] = the work of item i, one warp per item (clamped to 2^32 - 1)
__global__ void k_item_units(GraphDev g, const Item* __restrict__ items, uint32_t n_items, uint32_t chunk, int algo,
                             uint32_t* units) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t i = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; i < n_items; i += warps) {
        const Item it = items[i];
        const uint64_t ubase = g.off[it.u];
        const uint32_t du = (uint32_t)(g.off[it.u + 1] - ubase), upu = g.up[it.u];
        const uint32_t chunks = (du + chunk - 1) / chunk;
        unsigned long long w = 0;
        for (uint32_t j = it.j0 + lane; j < it.j1; j += 32) w += pair_units(g, it.u, ubase, du, upu, j, chunks, algo);
        for (int o = 16; o; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
        if (lane == 0) units[i] = w < 0xffffffffull ? (uint32_t)w : 0xffffffffu;
    }
}

// units[x] = the work of warp-tier vertex wb + x (its at most warp_max_deg pairs)
__global__ void k_vertex_units(GraphDev g, uint32_t wb, uint32_t we, int algo, uint32_t* units) {
    for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < we - wb; x += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t u = wb + (uint32_t)x;
        const uint64_t ubase = g.off[u];
        const uint32_t du = (uint32_t)(g.off[u + 1] - ubase), upu = g.up[u];
        unsigned long long w = 0;
        for (uint32_t j = upu; j < du; ++j) w += pair_units(g, u, ubase, du, upu, j, 1u, algo);
        units[x] = w < 0xffffffffull ? (uint32_t)w : 0xffffffffu;
    }
}

// smallest i in [0, n] with pre[i] >= t (pre ascending, n + 1 entries)
__device__ __forceinline__ uint32_t lower_bound_u64(const uint64_t* pre, uint32_t n, unsigned long long t) {
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (pre[mid] < t) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Shard r's start in the sequence: out[2r] = first item, out[2r+1] = first warp-tier vertex
// (relative to the tier's start), for r = 0..world (r = world: the ends).  The cut for r sits
// at r/world of the total work; a cut inside the items starts the shard at the first item
// whose prefix reaches it, one inside the vertices likewise.
__global__ void k_shard_bounds(const uint64_t* __restrict__ ipre, uint32_t ni, const uint64_t* __restrict__ vpre,
                               uint32_t nv, uint32_t world, uint32_t* out) {
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r <= world; r += gridDim.x * blockDim.x) {
        const unsigned long long Ti = ipre[ni], T = Ti + vpre[nv];
        const unsigned long long t = (T / world) * r + (T % world) * r / world;
        uint32_t i = ni, v = 0;
        if (r == world) {
            v = nv;
        } else if (t <= Ti) {
            i = lower_bound_u64(ipre, ni, t);
        } else {
            v = lower_bound_u64(vpre, nv, t - Ti);
        }
        out[2 * r] = i;
        out[2 * r + 1] = v;
    }
}

std::atomic<uint64_t> g_table_uploaded{0};
constexpr int kForms = 5;   // single graph without tables; single graph with tables, with and without the
                            // map; batch and wave (tables and map)
std::atomic<uint64_t> g_attr_set[2 * kForms] = {};
std::atomic<int> g_dyn_limit[2 * kForms] = {};   // per kernel form: optin - static smem

size_t census_smem(uint32_t algo, uint32_t chunk, bool map) {
    const bool uni = algo == TC_ALGO_UNION;
    const unsigned long long hf = uni ? hash_factor<TC_ALGO_UNION, true>()
                                      : (map ? hash_factor<TC_ALGO_SUFFIX, true>() : hash_factor<TC_ALGO_SUFFIX, false>());
    const unsigned long long mw = uni ? (map ? map_ids<TC_ALGO_UNION, true>() : 0u)
                                      : (map ? map_ids<TC_ALGO_SUFFIX, true>() : 0u);
    const unsigned long long words = ((uni ? 1ull : 0ull) + hf) * chunk + mw / 16;
    return sizeof(uint32_t) * words + sizeof(uint32_t) * (chunk / 16) + sizeof(unsigned long long) * (chunk / 32 + 1) +
           sizeof(uint32_t) * kMaxItemPairs + sizeof(unsigned long long) * 16 + 64;
}

tc_status prepare_device(cudaStream_t st, int algo, size_t smem) {
    int dev = 0;
    TC_CUDA(cudaGetDevice(&dev));
    const uint64_t bit = 1ull << (dev & 63);
    if (!(g_table_uploaded.load() & bit)) {
        const uint8_t* t = host_tricode_table();
        if (!t) return fail(TC_ERR_ARG, "tricode table derivation failed");
        TC_CUDA(cudaMemcpyToSymbolAsync(d_tricode_class, t, 64, 0, cudaMemcpyHostToDevice, st));
        TC_CUDA(cudaStreamSynchronize(st));
        g_table_uploaded.fetch_or(bit);
    }
    int optin = 0;
    TC_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const int limit = optin - 256;   // leave room for the kernel's static shared variables
    if ((int)smem > limit) return fail(TC_ERR_ARG, "chunk_entries too large for this GPU's shared memory");
    const void* fns[2 * kForms] = {
        (const void*)k_census<TC_ALGO_UNION, kModeSingle, false, true>,
        (const void*)k_census<TC_ALGO_SUFFIX, kModeSingle, false, true>,
        (const void*)k_census<TC_ALGO_UNION, kModeSingle, true, true>,
        (const void*)k_census<TC_ALGO_SUFFIX, kModeSingle, true, true>,
        (const void*)k_census<TC_ALGO_UNION, kModeSingle, true, false>,
        (const void*)k_census<TC_ALGO_SUFFIX, kModeSingle, true, false>,
        (const void*)k_census<TC_ALGO_UNION, kModeBatch, true, true>,
        (const void*)k_census<TC_ALGO_SUFFIX, kModeBatch, true, true>,
        (const void*)k_census<TC_ALGO_UNION, kModeWave, true, true>,
        (const void*)k_census<TC_ALGO_SUFFIX, kModeWave, true, true>};
    for (int b = 0; b < kForms; ++b) {
        const int idx = 2 * b + algo;
        if (!(g_attr_set[idx].load() & bit)) {
            // dynamic + static shared memory may not exceed the opt-in limit; the wave form
            // keeps its request descriptors in static shared memory
            cudaFuncAttributes fa;
            TC_CUDA(cudaFuncGetAttributes(&fa, fns[idx]));
            const int lim_f = optin - (int)fa.sharedSizeBytes;
            TC_CUDA(cudaFuncSetAttribute(fns[idx], cudaFuncAttributeMaxDynamicSharedMemorySize, lim_f));
            g_dyn_limit[idx].store(lim_f);
            g_attr_set[idx].fetch_or(bit);
        }
        if ((int)smem > g_dyn_limit[idx].load())
            return fail(TC_ERR_ARG, "chunk_entries too large for this GPU's shared memory");
    }
    return TC_OK;
}

}  // namespace

tc_status get_plan(GraphStore& g, const Opts& o, cudaStream_t st, Plan** out) {
    for (auto& p : g.plans)
        if (p.valid && p.key == o) { *out = &p; return TC_OK; }
    if (o.schedule == TC_SCHED_LEARNED && !g.cost.p)
        return fail(TC_ERR_ARG, "learned schedule requested but no cost model is attached");
    if (o.algo == TC_ALGO_TRIANGLE && !g.vs.p) return fail(TC_ERR_ARG, "the triangle form needs the per upper pair tables");
    Plan& p = g.plans[g.next_plan];
    g.next_plan = (g.next_plan + 1) % GraphStore::kPlans;
    p.valid = false;
    p.shard_world = 0;
    p.shard_bounds.clear();
    p.items.release();
    p.key = o;
    const GraphDev gd = g.dev();
    DevBuf cnt1;
    TC_TRY(cnt1.alloc(sizeof(uint32_t), st));
    TC_CUDA(cudaMemsetAsync(cnt1.p, 0, sizeof(uint32_t), st));
    k_count_gt<<<grid_for(g.n, 256, 4096), 256, 0, st>>>(gd.off, g.n, o.warp_max_deg, cnt1.as<uint32_t>());
    TC_LAUNCH("k_count_gt");
    uint32_t u_end = 0;
    TC_CUDA(cudaMemcpyAsync(&u_end, cnt1.p, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    TC_CUDA(cudaStreamSynchronize(st));
    p.warp_begin = u_end;
    p.warp_end = g.n_active;
    p.n_items = 0;
    if (u_end) {
        // tasks: blocks of at most kMaxItemPairs upper pairs, at most u_end + e_sym / kMaxItemPairs
        const uint64_t tmax = (uint64_t)u_end + g.e_sym / kMaxItemPairs + 1;
        if (tmax >= (1ull << 32)) return fail(TC_ERR_RANGE, "too many plan tasks");
        DevBuf tcnt, tbase, ntask, owner, tw, wt, pu, cnt, pos, tot;
        TC_TRY(tcnt.alloc(sizeof(uint32_t) * u_end, st));
        TC_TRY(tbase.alloc(sizeof(uint32_t) * u_end, st));
        TC_TRY(ntask.alloc(sizeof(uint32_t), st));
        TC_TRY(owner.alloc(sizeof(uint32_t) * tmax, st));
        TC_TRY(tw.alloc(sizeof(unsigned long long) * tmax, st));
        TC_TRY(wt.alloc(sizeof(unsigned long long), st));
        TC_TRY(pu.alloc(sizeof(uint32_t) * (g.e_sym ? g.e_sym : 1), st));   // pair units by table index
        TC_TRY(cnt.alloc(sizeof(uint32_t) * tmax, st));
        TC_TRY(pos.alloc(sizeof(uint32_t) * tmax, st));
        TC_TRY(tot.alloc(sizeof(uint32_t), st));
        TC_CUDA(cudaMemsetAsync(wt.p, 0, sizeof(unsigned long long), st));
        TC_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(uint32_t) * tmax, st));
        const unsigned vgrid = grid_for(u_end, 256, 4096);
        k_task_count<<<vgrid, 256, 0, st>>>(gd.off, gd.up, u_end, tcnt.as<uint32_t>());
        TC_LAUNCH("k_task_count");
        TC_TRY(scan_u32(tcnt.as<uint32_t>(), tbase.as<uint32_t>(), u_end, ntask.as<uint32_t>(), st));
        k_task_owner<<<vgrid, 256, 0, st>>>(tbase.as<uint32_t>(), tcnt.as<uint32_t>(), u_end, owner.as<uint32_t>());
        TC_LAUNCH("k_task_owner");
        const unsigned tgrid = grid_for(tmax * 32, 256, 8192);
        k_plan_work<<<tgrid, 256, 0, st>>>(gd, owner.as<uint32_t>(), tbase.as<uint32_t>(), ntask.as<uint32_t>(), o.chunk,
                                           (int)o.algo, tw.as<unsigned long long>(), pu.as<uint32_t>(),
                                           wt.as<unsigned long long>());
        TC_LAUNCH("k_plan_work");
        PlanArgs pa;
        pa.owner = owner.as<uint32_t>();
        pa.tbase = tbase.as<uint32_t>();
        pa.tcnt = tcnt.as<uint32_t>();
        pa.n_tasks = ntask.as<uint32_t>();
        pa.pu = pu.as<uint32_t>();
        pa.tw = tw.as<unsigned long long>();
        pa.total = wt.as<unsigned long long>();
        pa.cost = (o.schedule == TC_SCHED_LEARNED) ? g.cost.as<float>() : nullptr;
        pa.item_work = o.item_work;
        pa.grid = (uint32_t)census_grid(o);
        k_plan_items<false><<<tgrid, 256, 0, st>>>(gd, pa, nullptr, cnt.as<uint32_t>(), nullptr);
        TC_LAUNCH("k_plan_items (count)");
        TC_TRY(scan_u32(cnt.as<uint32_t>(), pos.as<uint32_t>(), tmax, tot.as<uint32_t>(), st));
        TC_CUDA(cudaMemcpyAsync(&p.n_items, tot.p, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
        TC_CUDA(cudaStreamSynchronize(st));
        TC_TRY(p.items.alloc_persistent(sizeof(Item) * (p.n_items ? p.n_items : 1)));
        if (p.n_items) {
            k_plan_items<true><<<tgrid, 256, 0, st>>>(gd, pa, pos.as<uint32_t>(), nullptr, p.items.as<Item>());
            TC_LAUNCH("k_plan_items (emit)");
        }
        TC_CUDA(cudaStreamSynchronize(st));
    }
    p.valid = true;
    *out = &p;
    return TC_OK;
}

int census_grid(const Opts& o) { return sm_count() * (int)o.ctas_per_sm; }

uint32_t warp_block_shift(uint64_t vertices, unsigned grid) {
    // the largest grab of at most 32 vertices that still leaves every warp about four grabs:
    // with fewer, one warp walking 32 vertices' pairs in series sets the kernel's duration
    const uint64_t target = vertices / (4ull * grid * kWarps);
    uint32_t s = 5;
    while (s > 0 && (1ull << s) > target) --s;
    return s;
}

tc_status census_launch_batch(const GraphDev* d_graphs, const Item* items, uint32_t n_items, const uint4* wblocks,
                              uint32_t n_wblocks, const Opts& o, uint32_t* ctr, unsigned long long* d_out, cudaStream_t st) {
    const size_t smem = census_smem(o.algo, o.chunk, true);
    Params P;
    std::memset(&P, 0, sizeof(P));
    P.items = items;
    P.n_items = n_items;
    P.chunk = o.chunk;
    P.warp_max = o.warp_max_deg;
    P.ctr = ctr;
    P.out = d_out;
    P.graphs = d_graphs;
    P.wblocks = wblocks;
    P.n_wblocks = n_wblocks;
    const unsigned grid = (unsigned)census_grid(o);
    if (o.algo == TC_ALGO_UNION) k_census<TC_ALGO_UNION, kModeBatch, true, true><<<grid, kThreads, smem, st>>>(P);
    else k_census<TC_ALGO_SUFFIX, kModeBatch, true, true><<<grid, kThreads, smem, st>>>(P);
    TC_LAUNCH("k_census (batched)");
    return TC_OK;
}

tc_status census_launch_wave(const WaveReq* d_reqs, uint32_t n_reqs, uint32_t total_items, uint32_t total_blocks,
                             const Opts& o, unsigned grid, uint32_t* ctr, cudaStream_t st) {
    if (n_reqs > kMaxWave) return fail(TC_ERR_RANGE, "wave larger than kMaxWave requests");
    const size_t smem = census_smem(o.algo, o.chunk, true);
    Params P;
    std::memset(&P, 0, sizeof(P));
    P.n_items = total_items;
    P.chunk = o.chunk;
    P.warp_max = o.warp_max_deg;
    P.ctr = ctr;
    P.out = nullptr;
    P.n_wblocks = total_blocks;
    P.reqs = d_reqs;
    P.n_reqs = n_reqs;
    if (o.algo == TC_ALGO_UNION) k_census<TC_ALGO_UNION, kModeWave, true, true><<<grid, kThreads, smem, st>>>(P);
    else k_census<TC_ALGO_SUFFIX, kModeWave, true, true><<<grid, kThreads, smem, st>>>(P);
    TC_LAUNCH("k_census (wave)");
    return TC_OK;
}

tc_status census_prepare(cudaStream_t st, const Opts& o) {
    return prepare_device(st, (int)o.algo, census_smem(o.algo, o.chunk, true));
}

// The map pays when it answers most of the walk's lookups: at least half of the N[v] entries
// walked have ids below its range (counted when the tables are built).
bool census_use_map(const GraphStore& g) { return 2 * g.sum_walk_map >= g.sum_walk; }

// Whether a single-graph census of g takes the map form (always without the per-pair tables).
bool census_map(const GraphStore& g, const Opts& o) {
    const bool vt = g.vs.p != nullptr;
    return !vt || o.map_mode == 1 || (o.map_mode == 0 && census_use_map(g));
}

// An automatic chunk of the suffix form is 2048 entries with the map; without it, where every
// entry of the chunk goes to the hash, 4096 (scale 26: 6.25 s against 7.86 s at 2048).
void census_fit_chunk(const GraphStore& g, Opts& o) {
    if (o.chunk_auto && o.algo == TC_ALGO_SUFFIX && !census_map(g, o)) o.chunk = 4096;
}

tc_status census_launch_raw(const GraphDev& gd, const Opts& o, const Item* items, uint32_t n_items, uint32_t warp_begin,
                            uint32_t warp_end, uint32_t* ctr, unsigned long long* d_out16, cudaStream_t st) {
    const bool vt = gd.vs != nullptr, map = true;
    const size_t smem = census_smem(o.algo, o.chunk, map);
    TC_TRY(prepare_device(st, (int)o.algo, smem));
    Params P;
    P.g = gd;
    P.items = items;
    P.n_items = n_items;
    P.warp_begin = warp_begin;
    P.warp_end = warp_end;
    P.wshift = warp_block_shift(warp_end - warp_begin, (unsigned)census_grid(o));
    P.chunk = o.chunk;
    P.warp_max = o.warp_max_deg;
    P.ctr = ctr;
    P.out = d_out16;
    P.vcost = nullptr;
    P.phase = nullptr;
    P.graphs = nullptr;
    P.wblocks = nullptr;
    P.n_wblocks = 0;
    P.reqs = nullptr;
    P.n_reqs = 0;
    const unsigned grid = (unsigned)census_grid(o);
    if (o.algo == TC_ALGO_UNION) {
        if (!vt) k_census<TC_ALGO_UNION, kModeSingle, false, true><<<grid, kThreads, smem, st>>>(P);
        else if (map) k_census<TC_ALGO_UNION, kModeSingle, true, true><<<grid, kThreads, smem, st>>>(P);
        else k_census<TC_ALGO_UNION, kModeSingle, true, false><<<grid, kThreads, smem, st>>>(P);
    } else {
        if (!vt) k_census<TC_ALGO_SUFFIX, kModeSingle, false, true><<<grid, kThreads, smem, st>>>(P);
        else if (map) k_census<TC_ALGO_SUFFIX, kModeSingle, true, true><<<grid, kThreads, smem, st>>>(P);
        else k_census<TC_ALGO_SUFFIX, kModeSingle, true, false><<<grid, kThreads, smem, st>>>(P);
    }
    TC_LAUNCH("k_census");
    return TC_OK;
}

tc_status plan_shards(GraphStore& g, const Opts& o, Plan& p, uint32_t world, cudaStream_t st) {
    if (p.shard_world == world) return TC_OK;
    const GraphDev gd = g.dev();
    const uint32_t ni = p.n_items, nv = p.warp_end - p.warp_begin;
    DevBuf iu, vu, ipre, vpre, bounds;
    TC_TRY(iu.alloc(sizeof(uint32_t) * (ni ? ni : 1), st));
    TC_TRY(vu.alloc(sizeof(uint32_t) * (nv ? nv : 1), st));
    TC_TRY(ipre.alloc(sizeof(uint64_t) * (ni + 1ull), st));
    TC_TRY(vpre.alloc(sizeof(uint64_t) * (nv + 1ull), st));
    TC_TRY(bounds.alloc(sizeof(uint32_t) * 2ull * (world + 1ull), st));
    if (ni) {
        k_item_units<<<grid_for((uint64_t)ni * 32, 256, 8192), 256, 0, st>>>(gd, p.items.as<Item>(), ni, o.chunk,
                                                                             (int)o.algo, iu.as<uint32_t>());
        TC_LAUNCH("k_item_units");
    }
    if (nv) {
        k_vertex_units<<<grid_for(nv, 256, 8192), 256, 0, st>>>(gd, p.warp_begin, p.warp_end, (int)o.algo,
                                                                vu.as<uint32_t>());
        TC_LAUNCH("k_vertex_units");
    }
    TC_TRY(scan_u32_to_u64(iu.as<uint32_t>(), ipre.as<uint64_t>(), ni, st));
    TC_TRY(scan_u32_to_u64(vu.as<uint32_t>(), vpre.as<uint64_t>(), nv, st));
    k_shard_bounds<<<grid_for(world + 1ull, 256, 64), 256, 0, st>>>(ipre.as<uint64_t>(), ni, vpre.as<uint64_t>(), nv,
                                                                     world, bounds.as<uint32_t>());
    TC_LAUNCH("k_shard_bounds");
    std::vector<uint32_t> h(2ull * (world + 1ull));
    TC_CUDA(cudaMemcpyAsync(h.data(), bounds.p, sizeof(uint32_t) * h.size(), cudaMemcpyDeviceToHost, st));
    TC_CUDA(cudaStreamSynchronize(st));
    p.shard_bounds.swap(h);
    p.shard_world = world;
    return TC_OK;
}

tc_status census_enqueue(GraphStore& g, const Opts& o, const Plan& p, cudaStream_t st, unsigned long long* d_out16,
                         unsigned long long* d_vcost, unsigned long long* d_phase) {
    return census_enqueue_range(g, o, p.items.as<Item>(), p.n_items, p.warp_begin, p.warp_end, st, d_out16, d_vcost,
                                d_phase);
}

tc_status census_enqueue_range(GraphStore& g, const Opts& o, const Item* items, uint32_t n_items, uint32_t warp_begin,
                               uint32_t warp_end, cudaStream_t st, unsigned long long* d_out16,
                               unsigned long long* d_vcost, unsigned long long* d_phase) {
    if (g.e_sym == 0) return TC_OK;
    if (o.algo == TC_ALGO_TRIANGLE)
        return triangle_census_enqueue(g, o, items, n_items, warp_begin, warp_end, st, d_out16, d_vcost, d_phase);
    const bool vt = g.vs.p != nullptr;
    const bool map = census_map(g, o);
    const size_t smem = census_smem(o.algo, o.chunk, map);
    TC_TRY(prepare_device(st, (int)o.algo, smem));
    TC_CUDA(cudaMemsetAsync(g.ctr.p, 0, sizeof(uint32_t) * 4, st));
    Params P;
    P.g = g.dev();
    P.items = items;
    P.n_items = n_items;
    P.warp_begin = warp_begin;
    P.warp_end = warp_end;
    P.wshift = warp_block_shift(warp_end - warp_begin, (unsigned)census_grid(o));
    P.chunk = o.chunk;
    P.warp_max = o.warp_max_deg;
    P.ctr = g.ctr.as<uint32_t>();
    P.out = d_out16;
    P.vcost = d_vcost;
    P.phase = d_phase;
    P.graphs = nullptr;
    P.wblocks = nullptr;
    P.n_wblocks = 0;
    P.reqs = nullptr;
    P.n_reqs = 0;
    const unsigned grid = (unsigned)census_grid(o);
    if (o.algo == TC_ALGO_UNION) {
        if (!vt) k_census<TC_ALGO_UNION, kModeSingle, false, true><<<grid, kThreads, smem, st>>>(P);
        else if (map) k_census<TC_ALGO_UNION, kModeSingle, true, true><<<grid, kThreads, smem, st>>>(P);
        else k_census<TC_ALGO_UNION, kModeSingle, true, false><<<grid, kThreads, smem, st>>>(P);
    } else {
        if (!vt) k_census<TC_ALGO_SUFFIX, kModeSingle, false, true><<<grid, kThreads, smem, st>>>(P);
        else if (map) k_census<TC_ALGO_SUFFIX, kModeSingle, true, true><<<grid, kThreads, smem, st>>>(P);
        else k_census<TC_ALGO_SUFFIX, kModeSingle, true, false><<<grid, kThreads, smem, st>>>(P);
    }
    TC_LAUNCH("k_census");
    return TC_OK;
}

}  // namespace tc
