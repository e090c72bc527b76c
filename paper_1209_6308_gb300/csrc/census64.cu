// census64.cu - the 64-state triad census (Sec. 3, Fig. 2): how many triads are in each of the
// 64 labelled states, before isomorphic states are merged into the 16 classes.  A triad's
// actors take the roles (u, v, w) in increasing vertex id of the caller's labels, and the state
// has the tricode's bits: 1 v->u, 2 u->v, 4 v->w, 8 w->v, 16 u->w, 32 w->u.
//
// The graph is stored in degree-relabelled ids, so roles come from the original ids
// (new_of_old inverted).  Every triad with at least two links is counted at its first linked
// pair in the order (x,y) < (x,z) < (y,z) of its sorted vertices x<y<z: a thread takes one
// linked pair (one upper CSR entry), merges the two neighbour lists, and counts each third
// vertex linked to either end whose triad starts at this pair.  Third vertices linked to
// neither end form one-link triads, whose state depends only on where the third vertex's id
// falls (below, between or above the pair's ids): their count per range is the range's size
// less the merged vertices in it.  The null state is C(n,3) less the rest, on the host.
#include "graph.cuh"

namespace tc {
namespace {

// old[new_of_old[x]] = x: the original id of each stored vertex
__global__ void k_old_of(const uint32_t* __restrict__ new_of_old, uint32_t n, uint32_t* old) {
    for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < n; x += (uint64_t)gridDim.x * blockDim.x)
        old[new_of_old[x]] = (uint32_t)x;
}

__device__ __forceinline__ uint32_t state_bits(bool yx, bool xy, bool yz, bool zy, bool xz, bool zx) {
    return (yx ? 1u : 0u) | (xy ? 2u : 0u) | (yz ? 4u : 0u) | (zy ? 8u : 0u) | (xz ? 16u : 0u) | (zx ? 32u : 0u);
}

// One thread per CSR entry; entries with id above the row's are the linked pairs.
__global__ void k_census64(GraphDev g, const uint32_t* __restrict__ old, unsigned long long* out64) {
    __shared__ unsigned long long h[64];
    for (int t = threadIdx.x; t < 64; t += blockDim.x) h[t] = 0;
    __syncthreads();
    const uint64_t total = g.off[g.n];
    const uint64_t n = g.n;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < total; i += (uint64_t)gridDim.x * blockDim.x) {
        // the row of entry i: the largest r with off[r] <= i (off[0] = 0 <= i < off[n])
        uint32_t lo = 0, hi = g.n;
        while (hi - lo > 1) {
            const uint32_t mid = lo + (hi - lo) / 2;
            if (g.off[mid] <= i) lo = mid; else hi = mid;
        }
        const uint32_t r = lo;
        const uint32_t e = g.adj[i], s = e >> 2;
        if (s <= r) continue;
        // the pair in original ids: a < b, ab = arc a->b, ba = arc b->a (entry bits: 1 r->s, 2 s->r)
        const uint32_t orr = old[r], os = old[s];
        const bool r_first = orr < os;
        const uint32_t a = r_first ? orr : os, b = r_first ? os : orr;
        const bool rs = (e & 1u) != 0, sr = (e & 2u) != 0;
        const bool ab = r_first ? rs : sr, ba = r_first ? sr : rs;
        const uint32_t* Nr = g.adj + g.off[r];
        const uint32_t* Ns = g.adj + g.off[s];
        const uint32_t dr = (uint32_t)(g.off[r + 1] - g.off[r]), ds = (uint32_t)(g.off[s + 1] - g.off[s]);
        unsigned long long below = 0, between = 0, above = 0;
        uint32_t p = 0, q = 0;
        while (p < dr || q < ds) {
            const uint32_t xr = p < dr ? (Nr[p] >> 2) : 0xffffffffu, xs = q < ds ? (Ns[q] >> 2) : 0xffffffffu;
            uint32_t c, lr = 0, ls = 0;   // link bits of (r, c) and (s, c): 1 end->c, 2 c->end
            if (xr < xs) {
                c = xr;
                lr = Nr[p] & 3u;
                ++p;
            } else if (xs < xr) {
                c = xs;
                ls = Ns[q] & 3u;
                ++q;
            } else {
                c = xr;
                lr = Nr[p] & 3u;
                ls = Ns[q] & 3u;
                ++p;
                ++q;
            }
            if (c == r || c == s) continue;
            const uint32_t oc = old[c];
            const uint32_t la = r_first ? lr : ls, lb = r_first ? ls : lr;   // links (a, c), (b, c)
            const bool ac = la & 1u, ca = la & 2u, bc = lb & 1u, cb = lb & 2u;
            if (oc < a) {
                // sorted (c, a, b): its first linked pair involves c, so it is counted there
                ++below;
            } else if (oc < b) {
                // sorted (a, c, b): first linked pair (a, b) unless a-c is linked
                ++between;
                if (!la) atomicAdd(&h[state_bits(ca, ac, cb, bc, ab, ba)], 1ull);
            } else {
                // sorted (a, b, c): (a, b) comes first
                ++above;
                atomicAdd(&h[state_bits(ba, ab, bc, cb, ac, ca)], 1ull);
            }
        }
        // third vertices linked to neither end: the pair's link alone, in the roles its
        // position gives (v-w below, u-w between, u-v above)
        const unsigned long long n_below = a, n_between = b - a - 1, n_above = n - b - 1;
        if (n_below > below) atomicAdd(&h[state_bits(false, false, ab, ba, false, false)], n_below - below);
        if (n_between > between) atomicAdd(&h[state_bits(false, false, false, false, ab, ba)], n_between - between);
        if (n_above > above) atomicAdd(&h[state_bits(ba, ab, false, false, false, false)], n_above - above);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 64; t += blockDim.x)
        if (h[t]) atomicAdd(&out64[t], h[t]);
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
    const GraphStore& G = g->s;
    unsigned long long h[64] = {};
    if (G.e_sym) {
        DevBuf old, acc;
        TC_TRY(old.alloc(sizeof(uint32_t) * G.n, st));
        TC_TRY(acc.alloc(sizeof(unsigned long long) * 64, st));
        TC_CUDA(cudaMemsetAsync(acc.p, 0, sizeof(unsigned long long) * 64, st));
        k_old_of<<<grid_for(G.n, 256, 4096), 256, 0, st>>>(G.new_of_old.as<uint32_t>(), G.n, old.as<uint32_t>());
        TC_LAUNCH("k_old_of");
        k_census64<<<grid_for(2ull * G.e_sym, 256, 8u * (unsigned)sm_count()), 256, 0, st>>>(
            G.dev(), old.as<uint32_t>(), acc.as<unsigned long long>());
        TC_LAUNCH("k_census64");
        TC_CUDA(cudaMemcpyAsync(h, acc.p, sizeof(h), cudaMemcpyDeviceToHost, st));
        TC_CUDA(cudaStreamSynchronize(st));
    }
    unsigned __int128 rest = 0;
    for (int t = 1; t < 64; ++t) rest += h[t];
    out[0] = to_u128(choose3(G.n) - rest);
    for (int t = 1; t < 64; ++t) out[t] = to_u128(h[t]);
    return TC_OK;
}

}  // extern "C"
