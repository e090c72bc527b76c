// build.cu - device construction of the compact graph structure of Sec. 6 (Fig. 7):
// one edge array holding every vertex's sorted neighbour list, a start offset per vertex,
// and the two low bits of each stored id giving the arc direction (01 owner->neighbour,
// 10 neighbour->owner, 11 both).
//
// From an arc list: validate ids, drop self-loops, key each arc by its unordered pair with
// one direction bit, radix sort, merge equal pairs by OR-ing their direction bits, count
// degrees, relabel vertices by descending degree (ties by original id), emit both
// directions of every pair in the new ids, radix sort by (owner, neighbour), and read off
// the offsets.  A CSR input is validated (sorted, flagged, loop-free, symmetric) and then
// goes through the same relabel.
#include <algorithm>

#include "graph.cuh"
#include "tc_internal.cuh"

namespace tc {
namespace {

constexpr int kB = 256;

__device__ __forceinline__ uint32_t swap_dir(uint32_t d) { return ((d & 1u) << 1) | ((d >> 1) & 1u); }

// stats[0] self-loops, stats[1] ids out of range
__global__ void k_make_keys(const uint32_t* src, const uint32_t* dst, uint64_t m, uint32_t n, int B,
                            uint64_t* keys, unsigned long long* stats) {
    uint32_t loops = 0, bad = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t a = src[i], b = dst[i];
        uint64_t key = ~0ull;
        if (a >= n || b >= n) ++bad;
        else if (a == b) ++loops;
        else {
            uint64_t lo = a < b ? a : b, hi = a < b ? b : a;
            uint64_t dir = a < b ? 1u : 2u;           // 01: lo->hi, 10: hi->lo
            key = (lo << (B + 2)) | (hi << 2) | dir;
        }
        keys[i] = key;
    }
    for (int o = 16; o; o >>= 1) {
        loops += __shfl_xor_sync(0xffffffffu, loops, o);
        bad += __shfl_xor_sync(0xffffffffu, bad, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (loops) atomicAdd(&stats[0], (unsigned long long)loops);
        if (bad) atomicAdd(&stats[1], (unsigned long long)bad);
    }
}

__global__ void k_head_flags(const uint64_t* keys, uint64_t cnt, uint32_t* flag) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < cnt; i += (uint64_t)gridDim.x * blockDim.x)
        flag[i] = (i == 0 || (keys[i] >> 2) != (keys[i - 1] >> 2)) ? 1u : 0u;
}

// Runs of equal pairs -> one pair key (lo<<B | hi) and the OR of their direction bits.
__global__ void k_unique(const uint64_t* keys, uint64_t cnt, const uint32_t* flag, const uint32_t* pos,
                         uint64_t* ukey, uint32_t* udir) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < cnt; i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t r = pos[i] + flag[i] - 1u;
        if (flag[i]) ukey[r] = keys[i] >> 2;
        atomicOr(&udir[r], (uint32_t)(keys[i] & 3u));
    }
}

// degrees; stats[2] mutual pairs.  The pairs are sorted by their smaller id, so the lanes of a
// warp mostly share it: one atomic per run of equal ids (a hub's run would otherwise serialise
// thousands of atomics on one address).
__global__ void k_degrees(const uint64_t* ukey, const uint32_t* udir, uint64_t E, int B, uint32_t* deg,
                          unsigned long long* stats) {
    const uint64_t mask = (1ull << B) - 1;
    const uint32_t lane = threadIdx.x & 31;
    uint32_t mut = 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t r0 = blockIdx.x * (uint64_t)blockDim.x + (threadIdx.x & ~31u); r0 < E; r0 += stride) {
        const uint64_t r = r0 + lane;   // uniform loop over the warp: every lane takes part in the match
        const bool ok = r < E;
        const uint64_t k = ok ? ukey[r] : ~0ull;
        const uint32_t lo = (uint32_t)(k >> B);
        const uint32_t peers = __match_any_sync(0xffffffffu, ok ? lo : 0xffffffffu);
        if (ok && (peers & ((1u << lane) - 1u)) == 0) atomicAdd(&deg[lo], (uint32_t)__popc(peers));
        if (ok) {
            atomicAdd(&deg[k & mask], 1u);
            mut += (udir[r] == 3u);
        }
    }
    for (int o = 16; o; o >>= 1) mut += __shfl_xor_sync(0xffffffffu, mut, o);
    if ((threadIdx.x & 31) == 0 && mut) atomicAdd(&stats[2], (unsigned long long)mut);
}

__global__ void k_relabel_keys(const uint32_t* deg, uint32_t n, int B, uint64_t* rk) {
    const uint64_t top = (1ull << B) - 1;
    for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < n; x += (uint64_t)gridDim.x * blockDim.x)
        rk[x] = ((top - deg[x]) << B) | x;
}

__global__ void k_perm(const uint64_t* rk, uint32_t n, int B, const uint32_t* deg, uint32_t* new_of_old,
                       uint32_t* new_deg) {
    const uint64_t mask = (1ull << B) - 1;
    for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < n; r += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t x = (uint32_t)(rk[r] & mask);
        new_of_old[x] = (uint32_t)r;
        new_deg[r] = deg[x];
    }
}

// Both directions of each pair in the new ids: (owner << (B+2)) | (nbr << 2) | dir(owner).
__global__ void k_entries(const uint64_t* ukey, const uint32_t* udir, uint64_t E, int B, const uint32_t* new_of_old,
                          uint64_t* ek) {
    const uint64_t mask = (1ull << B) - 1;
    for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < E; r += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t k = ukey[r];
        uint64_t a = new_of_old[k >> B], b = new_of_old[k & mask];
        uint32_t d = udir[r];
        ek[2 * r] = (a << (B + 2)) | (b << 2) | d;
        ek[2 * r + 1] = (b << (B + 2)) | (a << 2) | swap_dir(d);
    }
}

__global__ void k_adj_from_entries(const uint64_t* ek, uint64_t cnt, int B, uint32_t* adj) {
    const uint64_t mask = (1ull << (B + 2)) - 1;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < cnt; i += (uint64_t)gridDim.x * blockDim.x)
        adj[i] = (uint32_t)(ek[i] & mask);
}

// up[x] = number of neighbours with id < x (lists ascend, so a lower_bound).
__global__ void k_up(const uint64_t* off, const uint32_t* adj, uint32_t n, uint32_t* up) {
    for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < n; x += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t lo = off[x], hi = off[x + 1], b = lo;
        uint32_t key = (uint32_t)x << 2;
        while (lo < hi) {
            uint64_t mid = (lo + hi) >> 1;
            if (adj[mid] < key) lo = mid + 1; else hi = mid;
        }
        up[x] = (uint32_t)(lo - b);
    }
}

// stats[3] sum deg^2, stats[4] sum over upper pairs of deg(v), stats[5] max degree,
// stats[7] vertices with deg > 0, stats[10] sum of up (up - 1) / 2 (the entries the triangle form
// walks: for every upper pair (b, c), the neighbours of c below b)
__global__ void k_graph_sums(const uint64_t* off, const uint32_t* adj, const uint32_t* up, uint32_t n,
                             unsigned long long* stats) {
    unsigned long long d2 = 0, dv = 0, tw = 0;
    uint32_t mx = 0, act = 0;
    for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < n; x += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t d = off[x + 1] - off[x];
        d2 += d * d;
        mx = max(mx, (uint32_t)d);
        act += (d > 0);
        // x is the v of every pair (u, x) with u < x: the first up[x] neighbours
        dv += (unsigned long long)up[x] * d;
        tw += (unsigned long long)up[x] * (up[x] ? up[x] - 1ull : 0ull) / 2ull;
    }
    for (int o = 16; o; o >>= 1) {
        d2 += __shfl_xor_sync(0xffffffffu, d2, o);
        dv += __shfl_xor_sync(0xffffffffu, dv, o);
        tw += __shfl_xor_sync(0xffffffffu, tw, o);
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        act += __shfl_xor_sync(0xffffffffu, act, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (act) atomicAdd(&stats[7], (unsigned long long)act);
        atomicAdd(&stats[3], d2);
        atomicAdd(&stats[4], dv);
        atomicAdd(&stats[10], tw);
        atomicMax(&stats[5], (unsigned long long)mx);
    }
}

constexpr uint32_t kLongList = 4096;   // longer lists: k_pair_tables_long, a CTA per vertex
constexpr int kLongThreads = 1024;

// Per upper pair tables.  One warp per vertex v (lists of at most kLongList entries; longer ones
// are k_pair_tables_long's) takes N[v] in 32-entry blocks from the end,
// keeping running counts of the direction classes of the entries behind the block and adding,
// per lane, the block's entries after its own by ballot: so the lane at position k knows the
// counts of the entries after k.  At a lower neighbour u = N[v][k] (k < up[v]) those are the
// third vertices w > u reached from v: the lane writes them to sfx[lb[v] + k] (lb[v] = the
// lower entries of the vertices before v), where k_pair_rp picks them up for the upper pair
// (u, v).  At an upper neighbour
// (k >= up[v]) they are the third vertices w > N[v][k] reached from v, the u side of the pair
// (v, N[v][k]): us = (class-1, class-2 counts).  wk[0] += the suffix lengths at lower
// neighbours (the N[v] entries a census walks), wk[1] += those of them with ids below
// kMapIdsSuffix: with c the entries of N[v] below it (a prefix), the walk past position k
// meets max(0, c - k - 1) of them.
__global__ void k_pair_tables(const uint64_t* __restrict__ off, const uint32_t* __restrict__ adj,
                              const uint32_t* __restrict__ up, const uint64_t* __restrict__ ub,
                              const uint64_t* __restrict__ lb, uint32_t n, uint2* sfx, uint2* us,
                              unsigned long long* wk) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint32_t after = lane == 31 ? 0u : ~((2u << lane) - 1u);   // lanes above this one
    unsigned long long walk = 0, walk_map = 0;
    for (uint64_t v = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; v < n; v += warps) {
        const uint64_t ob = off[v];
        const uint32_t dv = (uint32_t)(off[v + 1] - ob), lv = up[v];
        if (dv > kLongList) continue;                                 // k_pair_tables_long's
        uint32_t c1 = 0, c2 = 0, cmap = 0;
        for (uint32_t cs = dv & ~31u; dv && cs <= dv; cs -= 32) {   // blocks from the last one down
            const uint32_t k = cs + lane;
            const uint32_t e = k < dv ? adj[ob + k] : 0u;
            const uint32_t b1 = __ballot_sync(0xffffffffu, (e & 3u) == 1u);
            const uint32_t b2 = __ballot_sync(0xffffffffu, (e & 3u) == 2u);
            if (k < lv) {
                sfx[lb[v] + k] = make_uint2(c1 + __popc(b1 & after), c2 + __popc(b2 & after));
                walk += dv - k - 1;
            } else if (k < dv) {
                us[ub[v] + (k - lv)] = make_uint2(c1 + __popc(b1 & after), c2 + __popc(b2 & after));
            }
            c1 += __popc(b1);
            c2 += __popc(b2);
            cmap += __popc(__ballot_sync(0xffffffffu, k < dv && (e >> 2) < kMapIdsSuffix));
            if (cs == 0) break;
        }
        const unsigned long long m = min(lv, cmap);
        if (lane == 0) walk_map += m * cmap - m * (m + 1) / 2;
    }
    for (int o = 16; o; o >>= 1) walk += __shfl_xor_sync(0xffffffffu, walk, o);
    if (lane == 0 && walk) atomicAdd(wk, walk);
    if (lane == 0 && walk_map) atomicAdd(wk + 1, walk_map);
}

// The same tables for the vertices with more than kLongList entries, a prefix of the ids
// (degrees descend), one CTA per vertex: a warp per list walks at most kLongList / 32 blocks in
// series.  Each warp takes a contiguous segment of N[v] (a multiple of 32 entries), counts its
// class-1 and class-2 entries, and then walks it backward from the counts of the segments after
// it, as k_pair_tables walks a whole list.
__global__ void __launch_bounds__(kLongThreads) k_pair_tables_long(
        const uint64_t* __restrict__ off, const uint32_t* __restrict__ adj, const uint32_t* __restrict__ up,
        const uint64_t* __restrict__ ub, const uint64_t* __restrict__ lb, uint32_t n, uint2* sfx, uint2* us,
        unsigned long long* wk) {
    __shared__ uint32_t s_c1[kLongThreads / 32], s_c2[kLongThreads / 32], s_map[kLongThreads / 32];
    const uint64_t v = blockIdx.x;
    if (v >= n) return;
    const uint64_t ob = off[v];
    const uint32_t dv = (uint32_t)(off[v + 1] - ob), lv = up[v];
    if (dv <= kLongList) return;                                      // the same for the whole CTA
    const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint32_t after = lane == 31 ? 0u : ~((2u << lane) - 1u);
    const uint32_t seg = ((dv + nw - 1) / nw + 31u) & ~31u;
    const uint32_t s0 = min(dv, wid * seg), s1 = min(dv, s0 + seg);
    uint32_t a1 = 0, a2 = 0, am = 0;
#pragma unroll 4
    for (uint32_t k = s0 + lane; k < s1; k += 32) {
        const uint32_t e = adj[ob + k];
        a1 += (e & 3u) == 1u;
        a2 += (e & 3u) == 2u;
        am += (e >> 2) < kMapIdsSuffix;
    }
    a1 = __reduce_add_sync(0xffffffffu, a1);
    a2 = __reduce_add_sync(0xffffffffu, a2);
    am = __reduce_add_sync(0xffffffffu, am);
    if (lane == 0) {
        s_c1[wid] = a1;
        s_c2[wid] = a2;
        s_map[wid] = am;
    }
    __syncthreads();
    uint32_t c1 = 0, c2 = 0, cmap = 0;
    for (uint32_t w = 0; w < nw; ++w) {
        if (w > wid) {
            c1 += s_c1[w];
            c2 += s_c2[w];
        }
        cmap += s_map[w];
    }
    unsigned long long walk = 0;
    if (s1 > s0) {
        for (uint32_t cs = (s1 - 1) & ~31u;; cs -= 32) {            // s0 is a multiple of 32
            const uint32_t k = cs + lane;
            const uint32_t e = k < s1 ? adj[ob + k] : 0u;
            const uint32_t b1 = __ballot_sync(0xffffffffu, (e & 3u) == 1u);
            const uint32_t b2 = __ballot_sync(0xffffffffu, (e & 3u) == 2u);
            if (k < lv) {
                sfx[lb[v] + k] = make_uint2(c1 + __popc(b1 & after), c2 + __popc(b2 & after));
                walk += dv - k - 1;
            } else if (k < s1) {
                us[ub[v] + (k - lv)] = make_uint2(c1 + __popc(b1 & after), c2 + __popc(b2 & after));
            }
            c1 += __popc(b1);
            c2 += __popc(b2);
            if (cs == s0) break;
        }
    }
    for (int o = 16; o; o >>= 1) walk += __shfl_xor_sync(0xffffffffu, walk, o);
    if (lane == 0 && walk) atomicAdd(wk, walk);
    if (threadIdx.x == 0) {
        const unsigned long long m = min(lv, cmap);
        const unsigned long long wm = m * cmap - m * (m + 1) / 2;
        if (wm) atomicAdd(wk + 1, wm);
    }
}

// Position of u in the lower part L = N[v][0, len) of a list (u is there: u < v and u ~ v).
// The degree order puts u, of degree at least v's, near the front of L, so the search gallops
// from the front (probes 1, 3, 7, ...) and then bisects the last gap: a hub's position costs a
// probe or two in the first sector of L.
__device__ __forceinline__ uint32_t lower_position(const uint32_t* __restrict__ L, uint32_t len, uint32_t u) {
    uint32_t lo = 0, hi = 1;
    while (hi < len && (L[hi] >> 2) < u) {
        lo = hi + 1;
        hi = 2 * hi + 1;
    }
    hi = min(hi, len);
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if ((L[mid] >> 2) < u) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// rp and vs of the upper pairs of u: for pair (u, v = N[u][j]), rp = the position k of u in
// N[v] and vs = sfx[lb[v] + k] (the class counts of N[v] past u, from k_pair_tables).  Entries
// j of each upper list in order, so the table writes are coalesced.  The upper pairs of one
// vertex u go to one warp (lists of at most kLongList entries) or, for longer lists, to one
// CTA (rp_long; those vertices are a prefix of the ids).
template <bool LONG>
__global__ void k_pair_rp(const uint64_t* __restrict__ off, const uint32_t* __restrict__ adj,
                          const uint32_t* __restrict__ up, const uint64_t* __restrict__ ub,
                          const uint64_t* __restrict__ lb, const uint2* __restrict__ sfx, uint32_t n, uint32_t* rp,
                          uint2* vs) {
    const uint32_t lanes = LONG ? blockDim.x : 32u;
    const uint32_t lane = LONG ? threadIdx.x : (threadIdx.x & 31u);
    // LONG: one CTA per vertex of the prefix the grid covers (the long lists are among them)
    const uint64_t stride = LONG ? n : ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t u = LONG ? blockIdx.x : (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; u < n; u += stride) {
        const uint64_t ob = off[u];
        const uint32_t du = (uint32_t)(off[u + 1] - ob), upu = up[u];
        if ((du > kLongList) != LONG) continue;      // uniform over the warp / CTA
        const uint64_t tb = ub[u];
        for (uint32_t j = upu + lane; j < du; j += lanes) {
            const uint32_t v = adj[ob + j] >> 2;
            const uint32_t k = lower_position(adj + off[v], up[v], (uint32_t)u);
            rp[tb + (j - upu)] = k;
            vs[tb + (j - upu)] = sfx[lb[v] + k];
        }
    }
}

// upper pairs per vertex: deg - up
__global__ void k_upper_of(const uint64_t* off, const uint32_t* up, uint32_t n, uint32_t* cnt) {
    for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < n; x += (uint64_t)gridDim.x * blockDim.x)
        cnt[x] = (uint32_t)(off[x + 1] - off[x]) - up[x];
}

// ---- CSR input validation: stats[6] = number of violations
__global__ void k_check_csr(const uint64_t* off, const uint32_t* adj, uint32_t n, uint64_t total,
                            unsigned long long* stats) {
    uint32_t badc = 0;
    for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < n; x += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t b = off[x], e = off[x + 1];
        if (e < b || e > total) { ++badc; continue; }
        for (uint64_t i = b; i < e; ++i) {
            uint32_t w = adj[i], id = w >> 2, d = w & 3u;
            if (id >= n || id == x || d == 0 || (i > b && (adj[i - 1] >> 2) >= id)) { ++badc; break; }
            // symmetry: x must appear in N[id] with mirrored direction bits
            uint64_t lo = off[id], hi = off[id + 1];
            if (hi < lo || hi > total) { ++badc; break; }
            uint32_t key = (uint32_t)x << 2;
            while (lo < hi) {
                uint64_t mid = (lo + hi) >> 1;
                if ((adj[mid] & ~3u) < key) lo = mid + 1; else hi = mid;
            }
            if (lo >= off[id + 1] || adj[lo] != (key | swap_dir(d))) { ++badc; break; }
        }
    }
    for (int o = 16; o; o >>= 1) badc += __shfl_xor_sync(0xffffffffu, badc, o);
    if ((threadIdx.x & 31) == 0 && badc) atomicAdd(&stats[6], (unsigned long long)badc);
}

// Upper entries (x < id) of a valid CSR -> pair keys and direction bits relative to lo = x.
__global__ void k_csr_pairs(const uint64_t* off, const uint32_t* adj, uint32_t n, int B, const uint32_t* upos,
                            uint64_t* ukey, uint32_t* udir, uint32_t* deg, unsigned long long* stats) {
    uint32_t mut = 0;
    for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < n; x += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t b = off[x], e = off[x + 1];
        deg[x] = (uint32_t)(e - b);
        uint32_t r = upos[x];
        for (uint64_t i = b; i < e; ++i) {
            uint32_t w = adj[i], id = w >> 2;
            if (id > x) {
                ukey[r] = ((uint64_t)x << B) | id;
                udir[r] = w & 3u;
                mut += ((w & 3u) == 3u);
                ++r;
            }
        }
    }
    for (int o = 16; o; o >>= 1) mut += __shfl_xor_sync(0xffffffffu, mut, o);
    if ((threadIdx.x & 31) == 0 && mut) atomicAdd(&stats[2], (unsigned long long)mut);
}

__global__ void k_upper_counts(const uint64_t* off, const uint32_t* adj, uint32_t n, uint32_t* cnt) {
    for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < n; x += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t c = 0;
        for (uint64_t i = off[x]; i < off[x + 1]; ++i) c += ((adj[i] >> 2) > x);
        cnt[x] = c;
    }
}


// Steps shared by both inputs: E unique pairs (ukey = lo<<B | hi, udir relative to lo) and
// degrees -> relabel, CSR, up[], stats.
tc_status finish_graph(GraphStore& g, uint64_t E, int B, uint64_t* ukey, uint32_t* udir, uint32_t* deg,
                       DevBuf& stats, cudaStream_t st) {
    const uint32_t n = g.n;
    const unsigned gridE = grid_for(E, kB, 1u << 16), gridN = grid_for(n, kB, 1u << 16);
    // relabel by descending degree
    DevBuf rk, rtmp, ndeg;
    TC_TRY(rk.alloc(sizeof(uint64_t) * n, st));
    TC_TRY(rtmp.alloc(sizeof(uint64_t) * n, st));
    TC_TRY(ndeg.alloc(sizeof(uint32_t) * n, st));
    TC_TRY(g.new_of_old.alloc_persistent(sizeof(uint32_t) * n));
    k_relabel_keys<<<gridN, kB, 0, st>>>(deg, n, B, rk.as<uint64_t>());
    TC_LAUNCH("k_relabel_keys");
    uint64_t* kp = rk.as<uint64_t>();
    uint64_t* tp = rtmp.as<uint64_t>();
    TC_TRY(radix_sort_u64(&kp, &tp, n, 0, 2 * B, st));
    k_perm<<<gridN, kB, 0, st>>>(kp, n, B, deg, g.new_of_old.as<uint32_t>(), ndeg.as<uint32_t>());
    TC_LAUNCH("k_perm");
    rk.release();
    rtmp.release();
    // offsets
    TC_TRY(g.off.alloc_persistent(sizeof(uint64_t) * (n + 1ull)));
    TC_TRY(scan_u32_to_u64(ndeg.as<uint32_t>(), g.off.as<uint64_t>(), n, st));
    // entries in new ids, sorted by (owner, neighbour)
    uint64_t total = 2 * E;
    DevBuf ek, etmp;
    TC_TRY(ek.alloc(sizeof(uint64_t) * (total ? total : 1), st));
    TC_TRY(etmp.alloc(sizeof(uint64_t) * (total ? total : 1), st));
    if (E) {
        k_entries<<<gridE, kB, 0, st>>>(ukey, udir, E, B, g.new_of_old.as<uint32_t>(), ek.as<uint64_t>());
        TC_LAUNCH("k_entries");
    }
    kp = ek.as<uint64_t>();
    tp = etmp.as<uint64_t>();
    TC_TRY(radix_sort_u64(&kp, &tp, total, 2, 2 * B + 2, st));
    TC_TRY(g.adj.alloc_persistent(sizeof(uint32_t) * (total ? total : 1)));
    if (total) {
        k_adj_from_entries<<<grid_for(total, kB, 1u << 16), kB, 0, st>>>(kp, total, B, g.adj.as<uint32_t>());
        TC_LAUNCH("k_adj_from_entries");
    }
    ek.release();
    etmp.release();
    TC_TRY(g.up.alloc_persistent(sizeof(uint32_t) * n));
    k_up<<<gridN, kB, 0, st>>>(g.off.as<uint64_t>(), g.adj.as<uint32_t>(), n, g.up.as<uint32_t>());
    TC_LAUNCH("k_up");
    k_graph_sums<<<gridN, kB, 0, st>>>(g.off.as<uint64_t>(), g.adj.as<uint32_t>(), g.up.as<uint32_t>(), n,
                                       stats.as<unsigned long long>());
    TC_LAUNCH("k_graph_sums");
    // per upper pair tables: ub = exclusive scan of the upper pairs per vertex
    {
        DevBuf ucnt;
        TC_TRY(ucnt.alloc(sizeof(uint32_t) * (n ? n : 1), st));
        TC_TRY(g.ub.alloc_persistent(sizeof(uint64_t) * (n + 1ull)));
        TC_TRY(g.rp.alloc_persistent(sizeof(uint32_t) * (E ? E : 1)));
        TC_TRY(g.vs.alloc_persistent(sizeof(uint2) * (E ? E : 1)));
        TC_TRY(g.us.alloc_persistent(sizeof(uint2) * (E ? E : 1)));
        if (n) {
            k_upper_of<<<gridN, kB, 0, st>>>(g.off.as<uint64_t>(), g.up.as<uint32_t>(), n, ucnt.as<uint32_t>());
            TC_LAUNCH("k_upper_of");
        }
        TC_TRY(scan_u32_to_u64(ucnt.as<uint32_t>(), g.ub.as<uint64_t>(), n, st));
        if (E) {
            // lower entries before each vertex (lb[n] = E), and their suffix counts
            DevBuf lb, sfx;
            TC_TRY(lb.alloc(sizeof(uint64_t) * (n + 1ull), st));
            TC_TRY(sfx.alloc(sizeof(uint2) * E, st));
            TC_TRY(scan_u32_to_u64(g.up.as<uint32_t>(), lb.as<uint64_t>(), n, st));
            // the walk lengths go to stats[8..9]
            k_pair_tables<<<grid_for((uint64_t)n * 32, kB, 1u << 16), kB, 0, st>>>(
                g.off.as<uint64_t>(), g.adj.as<uint32_t>(), g.up.as<uint32_t>(), g.ub.as<uint64_t>(),
                lb.as<uint64_t>(), n, sfx.as<uint2>(), g.us.as<uint2>(), stats.as<unsigned long long>() + 8);
            TC_LAUNCH("k_pair_tables");
            // lists longer than kLongList: at most 2E / kLongList of them, the first ids
            const uint64_t n_long = std::min<uint64_t>(n, 2ull * E / kLongList + 1);
            k_pair_tables_long<<<(unsigned)n_long, kLongThreads, 0, st>>>(
                g.off.as<uint64_t>(), g.adj.as<uint32_t>(), g.up.as<uint32_t>(), g.ub.as<uint64_t>(),
                lb.as<uint64_t>(), n, sfx.as<uint2>(), g.us.as<uint2>(), stats.as<unsigned long long>() + 8);
            TC_LAUNCH("k_pair_tables_long");
            k_pair_rp<false><<<grid_for((uint64_t)n * 32, kB, 1u << 16), kB, 0, st>>>(
                g.off.as<uint64_t>(), g.adj.as<uint32_t>(), g.up.as<uint32_t>(), g.ub.as<uint64_t>(),
                lb.as<uint64_t>(), sfx.as<uint2>(), n, g.rp.as<uint32_t>(), g.vs.as<uint2>());
            TC_LAUNCH("k_pair_rp");
            k_pair_rp<true><<<(unsigned)n_long, kLongThreads, 0, st>>>(
                g.off.as<uint64_t>(), g.adj.as<uint32_t>(), g.up.as<uint32_t>(), g.ub.as<uint64_t>(),
                lb.as<uint64_t>(), sfx.as<uint2>(), n, g.rp.as<uint32_t>(), g.vs.as<uint2>());
            TC_LAUNCH("k_pair_rp_long");
        }
    }
    unsigned long long hs[11];
    TC_CUDA(cudaMemcpyAsync(hs, stats.p, sizeof(hs), cudaMemcpyDeviceToHost, st));
    TC_CUDA(cudaStreamSynchronize(st));
    g.sum_tri_walk = hs[10];
    g.sum_walk = hs[8];
    g.sum_walk_map = hs[9];
    g.e_sym = E;
    g.mutual = hs[2];
    g.arcs = E + hs[2];
    g.sum_d2 = hs[3];
    g.sum_dv_upper = hs[4];
    g.max_deg = (uint32_t)hs[5];
    g.loops = hs[0];
    // degrees descend with the new id, so the vertices with deg > 0 are [0, n_active)
    g.n_active = (uint32_t)hs[7];
    return TC_OK;
}

}  // namespace

int bits_for(uint32_t n) {
    int B = 1;
    while ((1ull << B) < n) ++B;
    return B;
}

namespace {

// Runs of one pair among mv keys sorted by pair (direction bits in bits 0..1, runs adjacent)
// -> E unique pairs (ukey = lo<<B | hi) with the OR of their direction bits.
tc_status pairs_from_sorted(const uint64_t* kp, uint64_t mv, DevBuf& ukey, DevBuf& udir, uint32_t& E, cudaStream_t st) {
    DevBuf flag, pos, total;
    TC_TRY(flag.alloc(sizeof(uint32_t) * (mv ? mv : 1), st));
    TC_TRY(pos.alloc(sizeof(uint32_t) * (mv ? mv : 1), st));
    TC_TRY(total.alloc(sizeof(uint32_t), st));
    E = 0;
    if (mv) {
        k_head_flags<<<grid_for(mv, kB, 1u << 16), kB, 0, st>>>(kp, mv, flag.as<uint32_t>());
        TC_LAUNCH("k_head_flags");
        TC_TRY(scan_u32(flag.as<uint32_t>(), pos.as<uint32_t>(), mv, total.as<uint32_t>(), st));
        TC_CUDA(cudaMemcpyAsync(&E, total.p, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
        TC_CUDA(cudaStreamSynchronize(st));
    }
    TC_TRY(ukey.alloc(sizeof(uint64_t) * (E ? E : 1), st));
    TC_TRY(udir.alloc(sizeof(uint32_t) * (E ? E : 1), st));
    TC_CUDA(cudaMemsetAsync(udir.p, 0, sizeof(uint32_t) * (E ? E : 1), st));
    if (mv) {
        k_unique<<<grid_for(mv, kB, 1u << 16), kB, 0, st>>>(kp, mv, flag.as<uint32_t>(), pos.as<uint32_t>(),
                                                             ukey.as<uint64_t>(), udir.as<uint32_t>());
        TC_LAUNCH("k_unique");
    }
    return TC_OK;
}

// Degrees of the E unique pairs, then the relabelled CSR and its tables.
tc_status graph_from_pairs(GraphStore& g, int B, uint32_t E, DevBuf& ukey, DevBuf& udir, DevBuf& stats,
                           cudaStream_t st) {
    DevBuf deg;
    TC_TRY(deg.alloc(sizeof(uint32_t) * (g.n ? g.n : 1), st));
    TC_CUDA(cudaMemsetAsync(deg.p, 0, sizeof(uint32_t) * (g.n ? g.n : 1), st));
    if (E) {
        k_degrees<<<grid_for(E, kB, 1u << 16), kB, 0, st>>>(ukey.as<uint64_t>(), udir.as<uint32_t>(), E, B,
                                                             deg.as<uint32_t>(), stats.as<unsigned long long>());
        TC_LAUNCH("k_degrees");
    }
    return finish_graph(g, E, B, ukey.as<uint64_t>(), udir.as<uint32_t>(), deg.as<uint32_t>(), stats, st);
}

}  // namespace

tc_status build_from_arcs(GraphStore& g, uint64_t m, const uint32_t* d_src, const uint32_t* d_dst, cudaStream_t st) {
    const uint32_t n = g.n;
    const int B = bits_for(n);
    if (m >= (1ull << 32)) return fail(TC_ERR_RANGE, "more than 2^32-1 arcs");
    DevBuf stats, keys, tmp;
    TC_TRY(stats.alloc(sizeof(unsigned long long) * 11, st));
    TC_CUDA(cudaMemsetAsync(stats.p, 0, sizeof(unsigned long long) * 11, st));
    TC_TRY(keys.alloc(sizeof(uint64_t) * (m ? m : 1), st));
    TC_TRY(tmp.alloc(sizeof(uint64_t) * (m ? m : 1), st));
    if (m) {
        k_make_keys<<<grid_for(m, kB, 1u << 16), kB, 0, st>>>(d_src, d_dst, m, n, B, keys.as<uint64_t>(),
                                                               stats.as<unsigned long long>());
        TC_LAUNCH("k_make_keys");
    }
    unsigned long long hs[2];
    TC_CUDA(cudaMemcpyAsync(hs, stats.p, sizeof(hs), cudaMemcpyDeviceToHost, st));
    TC_CUDA(cudaStreamSynchronize(st));
    if (hs[1]) return fail(TC_ERR_RANGE, "arc list holds a vertex id >= n");
    uint64_t mv = m - hs[0];
    uint64_t* kp = keys.as<uint64_t>();
    uint64_t* tp = tmp.as<uint64_t>();
    TC_TRY(radix_sort_u64(&kp, &tp, m, 2, 2 * B + 2, st));
    // unique pairs (the self-loops' all-ones keys sort past the mv valid ones)
    DevBuf ukey, udir;
    uint32_t E = 0;
    TC_TRY(pairs_from_sorted(kp, mv, ukey, udir, E, st));
    keys.release();
    tmp.release();
    TC_TRY(graph_from_pairs(g, B, E, ukey, udir, stats, st));
    g.dups = m - g.loops - g.arcs;
    return TC_OK;
}

tc_status build_from_sorted_arcs(GraphStore& g, const uint64_t* d_keys, uint64_t m, cudaStream_t st) {
    const int B = bits_for(g.n);
    if (m >= (1ull << 32)) return fail(TC_ERR_RANGE, "more than 2^32-1 arcs");
    DevBuf stats, ukey, udir;
    TC_TRY(stats.alloc(sizeof(unsigned long long) * 11, st));
    TC_CUDA(cudaMemsetAsync(stats.p, 0, sizeof(unsigned long long) * 11, st));
    uint32_t E = 0;
    TC_TRY(pairs_from_sorted(d_keys, m, ukey, udir, E, st));
    TC_TRY(graph_from_pairs(g, B, E, ukey, udir, stats, st));
    g.dups = m - g.arcs;
    return TC_OK;
}

tc_status build_from_csr(GraphStore& g, const uint64_t* d_off, const uint32_t* d_adj, cudaStream_t st) {
    const uint32_t n = g.n;
    const int B = bits_for(n);
    uint64_t total_h = 0, first = 0;
    TC_CUDA(cudaMemcpyAsync(&total_h, d_off + n, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    TC_CUDA(cudaMemcpyAsync(&first, d_off, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    TC_CUDA(cudaStreamSynchronize(st));
    if (first != 0) return fail(TC_ERR_ARG, "CSR offsets must start at 0");
    if (total_h & 1) return fail(TC_ERR_ARG, "CSR is not symmetric (odd number of entries)");
    if (total_h >= (1ull << 32)) return fail(TC_ERR_RANGE, "more than 2^32-1 CSR entries");
    DevBuf stats;
    TC_TRY(stats.alloc(sizeof(unsigned long long) * 11, st));
    TC_CUDA(cudaMemsetAsync(stats.p, 0, sizeof(unsigned long long) * 11, st));
    const unsigned gridN = grid_for(n, kB, 1u << 16);
    k_check_csr<<<gridN, kB, 0, st>>>(d_off, d_adj, n, total_h, stats.as<unsigned long long>());
    TC_LAUNCH("k_check_csr");
    unsigned long long hs[8];
    TC_CUDA(cudaMemcpyAsync(hs, stats.p, sizeof(hs), cudaMemcpyDeviceToHost, st));
    TC_CUDA(cudaStreamSynchronize(st));
    if (hs[6]) return fail(TC_ERR_ARG, "CSR is not canonical (unsorted, loop, zero direction, id >= n or asymmetric)");
    uint64_t E = total_h / 2;
    DevBuf cnt, upos, ukey, udir, deg, etot;
    TC_TRY(cnt.alloc(sizeof(uint32_t) * n, st));
    TC_TRY(upos.alloc(sizeof(uint32_t) * n, st));
    TC_TRY(etot.alloc(sizeof(uint32_t), st));
    k_upper_counts<<<gridN, kB, 0, st>>>(d_off, d_adj, n, cnt.as<uint32_t>());
    TC_LAUNCH("k_upper_counts");
    TC_TRY(scan_u32(cnt.as<uint32_t>(), upos.as<uint32_t>(), n, etot.as<uint32_t>(), st));
    TC_TRY(ukey.alloc(sizeof(uint64_t) * (E ? E : 1), st));
    TC_TRY(udir.alloc(sizeof(uint32_t) * (E ? E : 1), st));
    TC_TRY(deg.alloc(sizeof(uint32_t) * n, st));
    k_csr_pairs<<<gridN, kB, 0, st>>>(d_off, d_adj, n, B, upos.as<uint32_t>(), ukey.as<uint64_t>(),
                                      udir.as<uint32_t>(), deg.as<uint32_t>(), stats.as<unsigned long long>());
    TC_LAUNCH("k_csr_pairs");
    TC_TRY(finish_graph(g, E, B, ukey.as<uint64_t>(), udir.as<uint32_t>(), deg.as<uint32_t>(), stats, st));
    g.dups = 0;
    g.loops = 0;
    return TC_OK;
}

}  // namespace tc
