// census64.cu - the 64-state triad census (Sec. 3, Fig. 2): how many triads are in each of the
// 64 labelled states, before isomorphic states are merged into the 16 classes.  A triad's
// actors take the roles (x, y, z) in increasing vertex id of the caller's labels, and the state
// has the tricode's bits: 1 y->x, 2 x->y, 4 y->z, 8 z->y, 16 x->z, 32 z->x.
//
// Every triad is counted by its links, in bulk where its state allows it:
//   - two links (a wedge with centre c): the state depends only on the two links' direction
//     classes seen from c and on where the ends' ids fall against c's.  With c's neighbours
//     sorted by the caller's ids, ordered class-pair counts among the neighbours below c
//     (c is z), among those above c (c is x), and the products of the class counts below and
//     above (c is y) count every pair of neighbours of c once;
//   - three links (a triangle): found once each by the triangle walk of triangles.cu, its
//     state read in the caller's id order.  Each triangle was also counted as a wedge at each
//     of its three vertices: those three are taken back;
//   - one link (a pair (a, b), a < b, and a third vertex linked to neither): the third vertex
//     below a, between or above b puts the link in the roles (y,z), (x,z) or (x,y).  Per pair
//     the three ranges hold a, b - a - 1 and n - 1 - b vertices; summed per direction class,
//     less the triads with more links that hold the same link in the same roles;
//   - no link: C(n,3) less the rest (128-bit).
// The sorted neighbour lists in caller ids come from one radix sort of (caller id of the row,
// caller id of the neighbour) keys of the stored lists.
#include <cstring>
#include <vector>

#include "graph.cuh"

namespace tc {
namespace {

// old[new_of_old[x]] = x: the original id of each stored vertex
__global__ void k_old_of(const uint32_t* __restrict__ new_of_old, uint32_t n, uint32_t* old) {
    for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < n; x += (uint64_t)gridDim.x * blockDim.x)
        old[new_of_old[x]] = (uint32_t)x;
}

// deg_old[x] = the degree of the vertex with caller id x
__global__ void k_deg_old(const uint64_t* __restrict__ off, const uint32_t* __restrict__ new_of_old, uint32_t n,
                          uint32_t* deg_old) {
    for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < n; x += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t r = new_of_old[x];
        deg_old[x] = (uint32_t)(off[r + 1] - off[r]);
    }
}

// One key per stored entry (row r, neighbour s): (old[r] << (B + 2)) | (old[s] << 2) | dir, with
// dir seen from r (1 r->s, 2 s->r).  One warp per row.
__global__ void k_keys64(GraphDev g, const uint32_t* __restrict__ old, int B, uint64_t* keys) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t r = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; r < g.n; r += warps) {
        const uint64_t b = g.off[r], e = g.off[r + 1];
        const uint64_t hi = (uint64_t)old[r] << (B + 2);
        for (uint64_t k = b + lane; k < e; k += 32) {
            const uint32_t x = g.adj[k];
            keys[k] = hi | ((uint64_t)old[x >> 2] << 2) | (x & 3u);
        }
    }
}

// The raw sums, per class pair (d1, d2), d = 1..3 (index 3 (d1-1) + d2-1):
//   raw[0..9)   PB: pairs p < q < c of neighbours of c, class(p) = d1, class(q) = d2 (c is z)
//   raw[9..18)  PA: pairs c < p < q                                         (c is x)
//   raw[18..27) X:  (neighbours below c of class d1) x (above c of class d2)  (c is y)
//   raw[27..36) R:  per pair (a, b), a < b, of direction class k = d1 (1 a->b, 2 b->a, 3 both):
//               position d2 = 1 above b (n - 1 - b), 2 between (b - a - 1), 3 below a (a)
// Classes are seen from c (1 c->nbr, 2 nbr->c).  One warp per vertex (caller ids).
__global__ void k_wedges64(const uint64_t* __restrict__ keys, const uint64_t* __restrict__ off_old, uint32_t n, int B,
                           unsigned long long* raw) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint64_t idmask = (1ull << B) - 1ull;
    const uint32_t lt = (1u << lane) - 1u;
    unsigned long long pb[3][3], pa[3][3], xx[3][3], rr[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) pb[i][j] = pa[i][j] = xx[i][j] = rr[i][j] = 0ull;
    for (uint64_t cx = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; cx < n; cx += warps) {
        const uint32_t c = (uint32_t)cx;
        const uint64_t kb = off_old[c], ke = off_old[c + 1];
        uint32_t rb[3] = {0u, 0u, 0u}, ra[3] = {0u, 0u, 0u};
        for (uint64_t k0 = kb; k0 < ke; k0 += 32) {
            const uint64_t k = k0 + lane;
            const bool valid = k < ke;
            const uint64_t key = valid ? keys[k] : 0ull;
            const uint32_t nb = (uint32_t)((key >> 2) & idmask), d = (uint32_t)(key & 3ull);
            const bool below = valid && nb < c, above = valid && nb > c;
            uint32_t bb[3], ba[3];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                bb[q] = __ballot_sync(0xffffffffu, below && d == (uint32_t)(q + 1));
                ba[q] = __ballot_sync(0xffffffffu, above && d == (uint32_t)(q + 1));
            }
#pragma unroll
            for (int q1 = 0; q1 < 3; ++q1) {
                const uint32_t before_b = rb[q1] + __popc(bb[q1] & lt), before_a = ra[q1] + __popc(ba[q1] & lt);
#pragma unroll
                for (int q2 = 0; q2 < 3; ++q2) {
                    if (below && d == (uint32_t)(q2 + 1)) pb[q1][q2] += before_b;
                    if (above && d == (uint32_t)(q2 + 1)) pa[q1][q2] += before_a;
                }
            }
            if (above) {
                const unsigned long long vals[3] = {(unsigned long long)n - 1ull - nb, (unsigned long long)(nb - c - 1u),
                                                    (unsigned long long)c};
#pragma unroll
                for (int q1 = 0; q1 < 3; ++q1)
                    if (d == (uint32_t)(q1 + 1))
#pragma unroll
                        for (int q2 = 0; q2 < 3; ++q2) rr[q1][q2] += vals[q2];
            }
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                rb[q] += __popc(bb[q]);
                ra[q] += __popc(ba[q]);
            }
        }
        if (lane == 0)
#pragma unroll
            for (int q1 = 0; q1 < 3; ++q1)
#pragma unroll
                for (int q2 = 0; q2 < 3; ++q2) xx[q1][q2] += (unsigned long long)rb[q1] * ra[q2];
    }
#pragma unroll
    for (int q1 = 0; q1 < 3; ++q1)
#pragma unroll
        for (int q2 = 0; q2 < 3; ++q2) {
            unsigned long long v[4] = {pb[q1][q2], pa[q1][q2], xx[q1][q2], rr[q1][q2]};
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                unsigned long long s = v[t];
                for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                if (lane == 0 && s) atomicAdd(&raw[9 * t + 3 * q1 + q2], s);
            }
        }
}

// states of wedges and one-link triads (see the file comment); d = direction class seen
// from the centre (1 centre->end, 2 end->centre)
inline uint32_t st_center_z(uint32_t d1, uint32_t d2) {   // ends p < q < c: p = x, q = y
    return (d1 & 2u ? 16u : 0u) | (d1 & 1u ? 32u : 0u) | (d2 & 2u ? 4u : 0u) | (d2 & 1u ? 8u : 0u);
}
inline uint32_t st_center_x(uint32_t d1, uint32_t d2) {   // c < p < q: p = y, q = z
    return (d1 & 1u ? 2u : 0u) | (d1 & 2u ? 1u : 0u) | (d2 & 1u ? 16u : 0u) | (d2 & 2u ? 32u : 0u);
}
inline uint32_t st_center_y(uint32_t dp, uint32_t dq) {   // p < c < q: p = x, q = z
    return (dp & 2u ? 2u : 0u) | (dp & 1u ? 1u : 0u) | (dq & 1u ? 4u : 0u) | (dq & 2u ? 8u : 0u);
}

// The state of a triangle tricode (roles (a, b, c) of the walk) once its actors are ordered by
// caller id: rank pattern 3 ra + rb (ra, rb = the ranks of a and b, c's is the rest).
std::vector<uint8_t> perm_states() {
    // bit b of a tricode is the arc kArc[b] between the roles a = 0, b = 1, c = 2; in sorted
    // roles x = 0, y = 1, z = 2 the arc (i -> j) has the state bit kBit[i][j]
    const int kArc[6][2] = {{1, 0}, {0, 1}, {1, 2}, {2, 1}, {0, 2}, {2, 0}};
    const int kBit[3][3] = {{0, 2, 16}, {1, 0, 4}, {32, 8, 0}};
    std::vector<uint8_t> t(9 * 64, 0);
    for (int ra = 0; ra < 3; ++ra)
        for (int rb = 0; rb < 3; ++rb) {
            if (ra == rb) continue;
            const int rank[3] = {ra, rb, 3 - ra - rb};
            for (int code = 0; code < 64; ++code) {
                int s = 0;
                for (int b = 0; b < 6; ++b)
                    if (code >> b & 1) s |= kBit[rank[kArc[b][0]]][rank[kArc[b][1]]];
                t[(3 * ra + rb) * 64 + code] = (uint8_t)s;
            }
        }
    return t;
}

}  // namespace
}  // namespace tc

using namespace tc;

extern "C" {

tc_status tc_census64(tc_graph* g, void* stream, tc_u128 out[64]) {
    if (!g || !out) return fail(TC_ERR_ARG, "null argument");
    cudaStream_t st = (cudaStream_t)stream;
    std::unique_lock<std::mutex> lk(g->s.busy, std::try_to_lock);
    if (!lk.owns_lock()) return fail(TC_ERR_BUSY, "graph is in use by another call");
    GraphStore& G = g->s;
    unsigned long long raw[36] = {}, tri[64] = {};
    if (G.e_sym) {
        int B = 1;
        while (B < 32 && (1ull << B) < G.n) ++B;
        const uint64_t E2 = 2ull * G.e_sym;
        DevBuf old, deg, offo, keys, tmp, acc, perm;
        TC_TRY(old.alloc(sizeof(uint32_t) * G.n, st));
        TC_TRY(deg.alloc(sizeof(uint32_t) * G.n, st));
        TC_TRY(offo.alloc(sizeof(uint64_t) * (G.n + 1ull), st));
        TC_TRY(keys.alloc(sizeof(uint64_t) * E2, st));
        TC_TRY(tmp.alloc(sizeof(uint64_t) * E2, st));
        TC_TRY(acc.alloc(sizeof(unsigned long long) * (36 + 64), st));
        TC_TRY(perm.alloc(9 * 64, st));
        const std::vector<uint8_t> ps = perm_states();
        TC_CUDA(cudaMemcpyAsync(perm.p, ps.data(), ps.size(), cudaMemcpyHostToDevice, st));
        TC_CUDA(cudaMemsetAsync(acc.p, 0, sizeof(unsigned long long) * (36 + 64), st));
        const GraphDev gd = G.dev();
        k_old_of<<<grid_for(G.n, 256, 4096), 256, 0, st>>>(G.new_of_old.as<uint32_t>(), G.n, old.as<uint32_t>());
        TC_LAUNCH("k_old_of");
        k_deg_old<<<grid_for(G.n, 256, 4096), 256, 0, st>>>(gd.off, G.new_of_old.as<uint32_t>(), G.n,
                                                            deg.as<uint32_t>());
        TC_LAUNCH("k_deg_old");
        TC_TRY(scan_u32_to_u64(deg.as<uint32_t>(), offo.as<uint64_t>(), G.n, st));
        k_keys64<<<grid_for((uint64_t)G.n * 32, 256, 8192), 256, 0, st>>>(gd, old.as<uint32_t>(), B,
                                                                          keys.as<uint64_t>());
        TC_LAUNCH("k_keys64");
        uint64_t* kp = keys.as<uint64_t>();
        uint64_t* tp = tmp.as<uint64_t>();
        TC_TRY(radix_sort_u64(&kp, &tp, E2, 2, 2 * B + 2, st));
        unsigned long long* d_raw = acc.as<unsigned long long>();
        k_wedges64<<<grid_for((uint64_t)G.n * 32, 256, 8u * (unsigned)sm_count()), 256, 0, st>>>(
            kp, offo.as<uint64_t>(), G.n, B, d_raw);
        TC_LAUNCH("k_wedges64");
        // triangles, in caller-id states, through the triangle form's plan
        tc_options to;
        std::memset(&to, 0, sizeof(to));
        to.algo = TC_ALGO_TRIANGLE;
        to.chunk_entries = 2048;
        to.ctas_per_sm = 4;   // the caller-id hash doubles the shared memory of a CTA
        Opts o;
        TC_TRY(resolve_opts(&to, nullptr, &o));
        Plan* p = nullptr;
        TC_TRY(get_plan(G, o, st, &p));
        TC_CUDA(cudaMemsetAsync(G.ctr.p, 0, sizeof(uint32_t) * 4, st));
        TC_TRY(triangles_launch(gd, o, p->items.as<Item>(), p->n_items, p->warp_begin, p->warp_end,
                                G.ctr.as<uint32_t>(), old.as<uint32_t>(), perm.as<uint8_t>(), d_raw + 36, nullptr, st));
        unsigned long long h[100];
        TC_CUDA(cudaMemcpyAsync(h, acc.p, sizeof(h), cudaMemcpyDeviceToHost, st));
        TC_CUDA(cudaStreamSynchronize(st));
        std::memcpy(raw, h, sizeof(raw));
        std::memcpy(tri, h + 36, sizeof(tri));
    }
    // assemble the states in 128-bit signed arithmetic
    __int128 C[64] = {};
    for (uint32_t d1 = 1; d1 <= 3; ++d1)
        for (uint32_t d2 = 1; d2 <= 3; ++d2) {
            const uint32_t i = 3 * (d1 - 1) + (d2 - 1);
            C[st_center_z(d1, d2)] += raw[i];
            C[st_center_x(d1, d2)] += raw[9 + i];
            C[st_center_y(d1, d2)] += raw[18 + i];
        }
    for (uint32_t t = 0; t < 64; ++t) {
        if (!tri[t]) continue;
        C[t] += tri[t];
        C[t & ~3u] -= tri[t];    // the wedge at z (x-y unlinked)
        C[t & ~12u] -= tri[t];   // at x (y-z unlinked)
        C[t & ~48u] -= tri[t];   // at y (x-z unlinked)
    }
    // one link: per direction class k of the pair (a, b), the range counts less the connected
    // triads holding that link in those roles
    __int128 S[64] = {};
    for (uint32_t s = 0; s < 64; ++s) S[s] = C[s];
    for (uint32_t k = 1; k <= 3; ++k) {
        const uint32_t ab = k & 1u, ba = k >> 1;
        const uint32_t s_above = (ab ? 2u : 0u) | (ba ? 1u : 0u);      // roles (x, y)
        const uint32_t s_between = (ab ? 16u : 0u) | (ba ? 32u : 0u);  // roles (x, z)
        const uint32_t s_below = (ab ? 4u : 0u) | (ba ? 8u : 0u);      // roles (y, z)
        __int128 a = raw[27 + 3 * (k - 1) + 0], b = raw[27 + 3 * (k - 1) + 1], c = raw[27 + 3 * (k - 1) + 2];
        for (uint32_t s = 0; s < 64; ++s) {
            if (!C[s]) continue;
            if ((s & 3u) == s_above) a -= C[s];
            if ((s & 48u) == s_between) b -= C[s];
            if ((s & 12u) == s_below) c -= C[s];
        }
        S[s_above] += a;
        S[s_between] += b;
        S[s_below] += c;
    }
    __int128 rest = 0;
    for (int s = 1; s < 64; ++s) rest += S[s];
    out[0] = to_u128(choose3(G.n) - (unsigned __int128)rest);
    for (int s = 1; s < 64; ++s) out[s] = to_u128((unsigned __int128)S[s]);
    return TC_OK;
}

}  // extern "C"
