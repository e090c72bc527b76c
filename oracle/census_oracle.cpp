// census_oracle.cpp - TEST INFRASTRUCTURE ONLY: the CPU oracle for the directed triad
// census.  Only the tests, the smoke check and the benchmark's CPU-baseline leg may load
// or run it; the GPU library never does and shares no code, table or header with it.
//
// What it computes: the exact 16-type triad census of a digraph G=(V,E), i.e. for each of
// the 16 isomorphism classes of 3-vertex digraphs, the number of 3-subsets of V whose
// induced subdigraph is in that class (paper Sec. 3: n(n-1)(n-2)/6 triads in total, 64
// labelled states folded to 16 classes).  Three independent routes:
//
//   1. or_census_bm     - Batagelj and Mrvar's census as listed in Fig. 5 (Sec. 4), written
//                         plainly: explicit union S built by the two-pointer walk of Sec. 6
//                         (Fig. 8), dyadic count n-|S|-2, canonical third-vertex rule,
//                         IsoTricode via a 64-entry table, null count by subtraction in
//                         128-bit.  Single-threaded.
//   2. or_census_brute  - the O(n^3) definition (Sec. 4, first paragraph): every a<b<c,
//                         classified by canonical form.  For small n only.
//   3. or_invariants    - O(m) graph statistics that fix weighted sums of the census
//                         (dyad totals, 2-stars, 2-paths, triangles); the tests combine
//                         them with per-class constants.
//
// The 64-state census (Sec. 3, Fig. 2: the labelled triad states before the fold to 16
// classes), two more independent routes:
//   4. or_census64_brute - every a<b<c, its state read over the roles (a, b, c).  Small n.
//   5. or_census64       - per linked pair (a, b), a<b: the merge of N(a) and N(b) gives
//                          every third vertex linked to a or b; such a triad is counted at
//                          its first linked pair in the order (x,y) < (x,z) < (y,z) of its
//                          sorted vertices x<y<z.  Third vertices linked to neither are
//                          counted per position (below a, between, above b) as the range's
//                          size less the merged vertices in it; the null state by
//                          subtraction.  Neither Fig. 5's third-vertex rule nor anything of
//                          the GPU method is used.
//   Reading: the paper names 64 states of a triad's three actors without fixing which actor
//   takes which role; the state here orders them by vertex id, the caller's labels (roles
//   u = smallest, v = middle, w = largest id, bits as the tricode).  Folded through the
//   16-class table, the 64-state census gives the 16-class census.
//
// The tricode -> class table is derived twice, by different methods, and the tests check
// that the two agree: or_table_rules (mutual/asymmetric/null dyad counts plus direction
// tests) and or_table_canonical (minimum code over the 6 vertex permutations matched
// against 16 hand-built class representatives).
//
// Readings of the paper used here (where it is silent or garbled):
//   - S in step 2.1.1 excludes u and v (Sec. 6 defines the third node over the union of
//     both neighbourhoods minus {u, v}); otherwise n-|S|-2 would be wrong.
//   - The relation is a set: self-loops and repeated arcs are ignored.
//   - Census order (0-based): 003 012 102 021D 021U 021C 111D 111U 030T 030C 201 120D
//     120U 120C 210 300 (step 5 fixes index 1 = null, step 2.1.2 fixes 2 = asymmetric
//     dyad and 3 = mutual dyad; the rest follows the usual M-A-N order).
//   - Tricode bits: 1 = v->u, 2 = u->v, 4 = v->w, 8 = w->v, 16 = u->w, 32 = w->u.
//   - n is given explicitly and counts isolated vertices.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <ctime>
#include <utility>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef unsigned __int128 u128;

namespace {

enum Cls { T003, T012, T102, T021D, T021U, T021C, T111D, T111U, T030T, T030C, T201, T120D, T120U, T120C, T210, T300 };

// ------------------------------------------------------------------ table by rules
// Decode a tricode into a 3x3 arc matrix over the roles (u=0, v=1, w=2).
void code_to_adj(int code, bool a[3][3]) {
    std::memset(a, 0, 9 * sizeof(bool));
    a[1][0] = code & 1;   // v->u
    a[0][1] = code & 2;   // u->v
    a[1][2] = code & 4;   // v->w
    a[2][1] = code & 8;   // w->v
    a[0][2] = code & 16;  // u->w
    a[2][0] = code & 32;  // w->u
}

int classify_by_rules(int code) {
    bool a[3][3];
    code_to_adj(code, a);
    const int pairs[3][2] = {{0, 1}, {0, 2}, {1, 2}};
    int M = 0, A = 0;
    for (auto& p : pairs) {
        bool f = a[p[0]][p[1]], b = a[p[1]][p[0]];
        if (f && b) ++M; else if (f || b) ++A;
    }
    int outd[3] = {0, 0, 0}, ind[3] = {0, 0, 0};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            if (a[i][j]) { ++outd[i]; ++ind[j]; }
    if (M == 0 && A == 0) return T003;
    if (M == 0 && A == 1) return T012;
    if (M == 1 && A == 0) return T102;
    if (M == 0 && A == 2) {
        // the two arcs share one vertex (the centre): out-star, in-star or path
        for (int x = 0; x < 3; ++x) {
            if (outd[x] == 2) return T021D;
            if (ind[x] == 2) return T021U;
        }
        return T021C;
    }
    if (M == 1 && A == 1) {
        // the outsider is the vertex outside the mutual pair; D if it sends into the pair
        for (auto& p : pairs) {
            if (a[p[0]][p[1]] && a[p[1]][p[0]]) {
                int z = 3 - p[0] - p[1];
                return (outd[z] == 1) ? T111D : T111U;
            }
        }
    }
    if (M == 0 && A == 3) {
        for (int x = 0; x < 3; ++x)
            if (outd[x] == 2) return T030T;
        return T030C;
    }
    if (M == 2 && A == 0) return T201;
    if (M == 1 && A == 2) {
        for (auto& p : pairs) {
            if (a[p[0]][p[1]] && a[p[1]][p[0]]) {
                int x = 3 - p[0] - p[1];   // outsider, joined to both by asymmetric arcs
                if (outd[x] == 2) return T120D;
                if (ind[x] == 2) return T120U;
                return T120C;
            }
        }
    }
    if (M == 2 && A == 1) return T210;
    if (M == 3) return T300;
    return -1;
}

// ------------------------------------------------------------------ table by canonical form
int adj_to_code(const bool a[3][3]) {
    return (a[1][0] ? 1 : 0) | (a[0][1] ? 2 : 0) | (a[1][2] ? 4 : 0) | (a[2][1] ? 8 : 0) |
           (a[0][2] ? 16 : 0) | (a[2][0] ? 32 : 0);
}

int canonical_code(int code) {
    bool a[3][3];
    code_to_adj(code, a);
    int p[3] = {0, 1, 2}, best = 64;
    do {
        bool b[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) b[i][j] = a[p[i]][p[j]];
        best = std::min(best, adj_to_code(b));
    } while (std::next_permutation(p, p + 3));
    return best;
}

// One representative digraph per class, written straight from the class definitions
// (x=0, y=1, z=2; each pair is an arc x->y).
struct Rep { int cls; int narcs; int arcs[6][2]; };
const Rep kReps[16] = {
    {T003, 0, {}},
    {T012, 1, {{0, 1}}},
    {T102, 2, {{0, 1}, {1, 0}}},
    {T021D, 2, {{0, 1}, {0, 2}}},                          // out-star from x
    {T021U, 2, {{1, 0}, {2, 0}}},                          // in-star into x
    {T021C, 2, {{0, 1}, {1, 2}}},                          // path x->y->z
    {T111D, 3, {{0, 1}, {1, 0}, {2, 1}}},                  // x<->y, z->y
    {T111U, 3, {{0, 1}, {1, 0}, {1, 2}}},                  // x<->y, y->z
    {T030T, 3, {{0, 1}, {1, 2}, {0, 2}}},                  // transitive
    {T030C, 3, {{0, 1}, {1, 2}, {2, 0}}},                  // cycle
    {T201, 4, {{0, 1}, {1, 0}, {0, 2}, {2, 0}}},           // two mutual, one null
    {T120D, 4, {{1, 2}, {2, 1}, {0, 1}, {0, 2}}},          // y<->z, x->y, x->z
    {T120U, 4, {{1, 2}, {2, 1}, {1, 0}, {2, 0}}},          // y<->z, y->x, z->x
    {T120C, 4, {{1, 2}, {2, 1}, {0, 1}, {2, 0}}},          // y<->z, x->y, z->x
    {T210, 5, {{0, 1}, {1, 0}, {1, 2}, {2, 1}, {0, 2}}},   // two mutual, x->z
    {T300, 6, {{0, 1}, {1, 0}, {0, 2}, {2, 0}, {1, 2}, {2, 1}}},
};

// ------------------------------------------------------------------ the digraph
struct Tagged { uint32_t id; bool out; bool in; };   // out: owner->id, in: id->owner

struct Digraph {
    uint32_t n = 0;
    std::vector<std::vector<uint32_t>> out;   // sorted out-neighbours
    std::vector<std::vector<Tagged>> N;       // sorted neighbour lists (either direction)
    uint64_t arcs = 0, loops = 0, dups = 0;
    mutable uint64_t pair_work_cache = ~0ull;   // merge length of the whole census (timing samples)

    bool arc(uint32_t x, uint32_t y) const {
        return std::binary_search(out[x].begin(), out[x].end(), y);
    }
};

// Returns false if an id is out of range.
bool build_digraph(uint32_t n, uint64_t m, const uint32_t* src, const uint32_t* dst, Digraph& g) {
    g.n = n;
    std::vector<std::pair<uint32_t, uint32_t>> e;
    e.reserve(m);
    for (uint64_t i = 0; i < m; ++i) {
        if (src[i] >= n || dst[i] >= n) return false;
        if (src[i] == dst[i]) { ++g.loops; continue; }
        e.emplace_back(src[i], dst[i]);
    }
    // (generated inputs arrive sorted by (src, dst): skip the sort then, the result is the same)
    if (!std::is_sorted(e.begin(), e.end())) std::sort(e.begin(), e.end());
    e.erase(std::unique(e.begin(), e.end()), e.end());
    g.arcs = e.size();
    g.dups = m - g.loops - g.arcs;
    // out[x]: the arcs are sorted by source, so x's out-neighbours are one run of e; in[x]: a
    // counting placement by target.  Both filled (and the lists merged) vertex by vertex, the
    // vertices shared among OpenMP threads when there are many: the lists are the same.
    const int64_t N64 = (int64_t)n;
    std::vector<uint64_t> ostart(n + 1ull, 0), istart(n + 1ull, 0);
    for (auto& p : e) { ++ostart[p.first + 1ull]; ++istart[p.second + 1ull]; }
    for (uint64_t x = 0; x < n; ++x) { ostart[x + 1] += ostart[x]; istart[x + 1] += istart[x]; }
    std::vector<uint32_t> inflat(e.size());
    {
        std::vector<uint64_t> pos(istart.begin(), istart.end() - 1);
        for (auto& p : e) inflat[pos[p.second]++] = p.first;   // e is sorted: each run ascends
    }
    g.out.assign(n, {});
    std::vector<std::vector<uint32_t>> in(n);
    g.N.assign(n, {});
#pragma omp parallel for schedule(dynamic, 4096) if (n > 100000)
    for (int64_t xi = 0; xi < N64; ++xi) {
        const uint32_t x = (uint32_t)xi;
        g.out[x].reserve(ostart[x + 1] - ostart[x]);
        for (uint64_t k = ostart[x]; k < ostart[x + 1]; ++k) g.out[x].push_back(e[k].second);
        in[x].assign(inflat.begin() + istart[x], inflat.begin() + istart[x + 1]);
        std::sort(in[x].begin(), in[x].end());
        // merge out[x] and in[x] into one tagged sorted list
        size_t i = 0, j = 0;
        const auto& o = g.out[x];
        const auto& q = in[x];
        g.N[x].reserve(o.size() + q.size());
        while (i < o.size() || j < q.size()) {
            if (j == q.size() || (i < o.size() && o[i] < q[j])) { g.N[x].push_back({o[i], true, false}); ++i; }
            else if (i == o.size() || q[j] < o[i]) { g.N[x].push_back({q[j], false, true}); ++j; }
            else { g.N[x].push_back({o[i], true, true}); ++i; ++j; }
        }
        std::vector<uint32_t>().swap(in[x]);
    }
    return true;
}

double now_seconds() {
    timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

u128 choose3(uint64_t n) {
    if (n < 3) return 0;
    u128 a = n, b = n - 1, c = n - 2;
    return a * b * c / 6;
}

void store(const u128 c[16], uint64_t* out) {
    for (int t = 0; t < 16; ++t) { out[2 * t] = (uint64_t)c[t]; out[2 * t + 1] = (uint64_t)(c[t] >> 64); }
}

int g_table[64];
bool g_table_ready = false;
void ensure_table() {
    if (g_table_ready) return;
    for (int c = 0; c < 64; ++c) g_table[c] = classify_by_rules(c);
    g_table_ready = true;
}

int iso_tricode(const Digraph& g, uint32_t u, uint32_t v, uint32_t w) {
    int code = (g.arc(v, u) ? 1 : 0) | (g.arc(u, v) ? 2 : 0) | (g.arc(v, w) ? 4 : 0) |
               (g.arc(w, v) ? 8 : 0) | (g.arc(u, w) ? 16 : 0) | (g.arc(w, u) ? 32 : 0);
    return g_table[code];
}

struct SElem { uint32_t w; bool in_u; };

// Steps 2.1 .. 2.1.4.2 of Fig. 5 for one vertex u; adds into census and returns the merge
// length (|N[u]| + |N[v]| summed over the pairs handled).
uint64_t bm_vertex(const Digraph& g, uint32_t u, u128 census[16], std::vector<SElem>& S) {
    const uint64_t n = g.n;
    uint64_t work = 0;
    const auto& Nu = g.N[u];
    for (const Tagged& tv : Nu) {
        uint32_t v = tv.id;
        if (!(u < v)) continue;                                   // step 2.1
        const auto& Nv = g.N[v];
        work += Nu.size() + Nv.size();
        // step 2.1.1: S := N[u] union N[v] minus {u, v}, by the two-pointer walk of Fig. 8
        S.clear();
        size_t i = 0, j = 0;
        while (i < Nu.size() || j < Nv.size()) {
            uint32_t w;
            bool in_u;
            if (j == Nv.size() || (i < Nu.size() && Nu[i].id < Nv[j].id)) { w = Nu[i].id; in_u = true; ++i; }
            else if (i == Nu.size() || Nv[j].id < Nu[i].id) { w = Nv[j].id; in_u = false; ++j; }
            else { w = Nu[i].id; in_u = true; ++i; ++j; }        // common neighbour
            if (w == u || w == v) continue;
            S.push_back({w, in_u});
        }
        // steps 2.1.2 - 2.1.3: dyadic triads of the connected pair
        int tri = (g.arc(u, v) && g.arc(v, u)) ? T102 : T012;
        census[tri] += (u128)(n - S.size() - 2);
        // step 2.1.4: each third vertex, counted once through the canonical choice
        for (const SElem& s : S) {
            uint32_t w = s.w;
            if (v < w || (u < w && w < v && !s.in_u)) census[iso_tricode(g, u, v, w)] += 1;
        }
    }
    return work;
}

// |N[u]| + |N[v]| summed over the pairs u < v (the merge length of the whole census), once per graph
uint64_t pair_work(const Digraph& g) {
    if (g.pair_work_cache == ~0ull) {
        uint64_t tot = 0;
        for (uint32_t u = 0; u < g.n; ++u)
            for (const Tagged& tv : g.N[u])
                if (u < tv.id) tot += g.N[u].size() + g.N[tv.id].size();
        g.pair_work_cache = tot;
    }
    return g.pair_work_cache;
}

void bm_finish(uint64_t n, u128 census[16]) {
    u128 sum = 0;                                                // steps 3 - 4
    for (int t = 1; t < 16; ++t) sum += census[t];
    census[T003] = choose3(n) - sum;                             // step 5
}

// ------------------------------------------------------------------ 64-state census
// The state of {a<b<c} over the roles (u, v, w) = (a, b, c), bits as the tricode.
int state_of(bool ab, bool ba, bool bc, bool cb, bool ac, bool ca) {
    return (ba ? 1 : 0) | (ab ? 2 : 0) | (bc ? 4 : 0) | (cb ? 8 : 0) | (ac ? 16 : 0) | (ca ? 32 : 0);
}

void store64(const u128 c[64], uint64_t* out) {
    for (int t = 0; t < 64; ++t) { out[2 * t] = (uint64_t)c[t]; out[2 * t + 1] = (uint64_t)(c[t] >> 64); }
}

// Direction of a link seen from one end x: out = x->other, in = other->x.
struct Link { bool out, in; };

}  // namespace

extern "C" {

// Route 4: the O(n^3) definition of the 64-state census.
int or_census64_brute(uint32_t n, uint64_t m, const uint32_t* src, const uint32_t* dst, uint64_t* out) {
    if (n > 4096) return -2;
    std::vector<uint8_t> adj((size_t)n * n, 0);
    for (uint64_t i = 0; i < m; ++i) {
        if (src[i] >= n || dst[i] >= n) return -1;
        if (src[i] != dst[i]) adj[(size_t)src[i] * n + dst[i]] = 1;
    }
    auto A = [&](uint32_t x, uint32_t y) { return adj[(size_t)x * n + y] != 0; };
    std::vector<u128> census(64, 0);
    for (uint32_t a = 0; a < n; ++a)
        for (uint32_t b = a + 1; b < n; ++b)
            for (uint32_t c = b + 1; c < n; ++c)
                census[state_of(A(a, b), A(b, a), A(b, c), A(c, b), A(a, c), A(c, a))] += 1;
    store64(census.data(), out);
    return 0;
}

// Route 5: per linked pair, first-linked-pair rule for connected triads, range counts for
// the triads whose only link is the pair, null state by subtraction.
int or_census64(uint32_t n, uint64_t m, const uint32_t* src, const uint32_t* dst, uint64_t* out) {
    Digraph g;
    if (!build_digraph(n, m, src, dst, g)) return -1;
    std::vector<u128> census(64, 0);
    for (uint32_t a = 0; a < n; ++a) {
        for (const Tagged& tb : g.N[a]) {
            const uint32_t b = tb.id;
            if (b <= a) continue;
            const bool ab = tb.out, ba = tb.in;   // a->b, b->a
            // merge N(a) and N(b) without a and b: every third vertex linked to a or b
            const auto& Na = g.N[a];
            const auto& Nb = g.N[b];
            size_t i = 0, j = 0;
            uint64_t below = 0, between = 0, above = 0;   // merged vertices per range
            while (i < Na.size() || j < Nb.size()) {
                uint32_t c;
                Link la{false, false}, lb{false, false};   // a-c and b-c: out = a->c / b->c
                if (j == Nb.size() || (i < Na.size() && Na[i].id < Nb[j].id)) {
                    c = Na[i].id; la = {Na[i].out, Na[i].in}; ++i;
                } else if (i == Na.size() || Nb[j].id < Na[i].id) {
                    c = Nb[j].id; lb = {Nb[j].out, Nb[j].in}; ++j;
                } else {
                    c = Na[i].id; la = {Na[i].out, Na[i].in}; lb = {Nb[j].out, Nb[j].in}; ++i; ++j;
                }
                if (c == a || c == b) continue;
                const bool lac = la.out || la.in, lbc = lb.out || lb.in;
                if (c < a) ++below; else if (c < b) ++between; else ++above;
                // sorted vertices x<y<z and the first linked pair among (x,y), (x,z), (y,z)
                uint32_t x, y, z;
                if (c < a) { x = c; y = a; z = b; } else if (c < b) { x = a; y = c; z = b; } else { x = a; y = b; z = c; }
                auto linked = [&](uint32_t p, uint32_t q) {
                    if ((p == a && q == b) || (p == b && q == a)) return true;
                    if (p == a || q == a) return lac;
                    return lbc;
                };
                uint32_t p0, q0;
                if (linked(x, y)) { p0 = x; q0 = y; } else if (linked(x, z)) { p0 = x; q0 = z; } else { p0 = y; q0 = z; }
                if (!(p0 == a && q0 == b)) continue;   // counted at its first linked pair
                // arcs among a, b, c
                auto arc = [&](uint32_t p, uint32_t q) {
                    if (p == a && q == b) return ab;
                    if (p == b && q == a) return ba;
                    if (p == a && q == c) return la.out;
                    if (p == c && q == a) return la.in;
                    if (p == b && q == c) return lb.out;
                    return lb.in;   // c -> b
                };
                census[state_of(arc(x, y), arc(y, x), arc(y, z), arc(z, y), arc(x, z), arc(z, x))] += 1;
            }
            // third vertices linked to neither a nor b: the pair's link alone
            const uint64_t n_below = a, n_between = b - a - 1, n_above = (uint64_t)n - b - 1;
            census[state_of(false, false, ab, ba, false, false)] += n_below - below;        // roles (c, a, b)
            census[state_of(false, false, false, false, ab, ba)] += n_between - between;    // roles (a, c, b)
            census[state_of(ab, ba, false, false, false, false)] += n_above - above;        // roles (a, b, c)
        }
    }
    u128 rest = 0;
    for (int t = 1; t < 64; ++t) rest += census[t];
    census[0] = choose3(n) - rest;
    store64(census.data(), out);
    return 0;
}


// Tricode -> class tables.  Return 0 on success, -1 if a code is left unclassified.
int or_table_rules(uint8_t T[64]) {
    for (int c = 0; c < 64; ++c) {
        int k = classify_by_rules(c);
        if (k < 0) return -1;
        T[c] = (uint8_t)k;
    }
    return 0;
}

int or_table_canonical(uint8_t T[64]) {
    int rep_canon[16];
    for (int r = 0; r < 16; ++r) {
        bool a[3][3] = {};
        for (int k = 0; k < kReps[r].narcs; ++k) a[kReps[r].arcs[k][0]][kReps[r].arcs[k][1]] = true;
        rep_canon[kReps[r].cls] = canonical_code(adj_to_code(a));
    }
    for (int c = 0; c < 64; ++c) {
        int cc = canonical_code(c), found = -1;
        for (int k = 0; k < 16; ++k)
            if (rep_canon[k] == cc) { if (found >= 0) return -1; found = k; }
        if (found < 0) return -1;
        T[c] = (uint8_t)found;
    }
    return 0;
}

// Fig. 5 census.  out: 16 counts as (lo, hi) 64-bit halves.  Returns 0, or -1 when an id
// is >= n.  stats (may be null): distinct arcs, self-loops dropped, duplicates dropped.
int or_census_bm(uint32_t n, uint64_t m, const uint32_t* src, const uint32_t* dst, uint64_t* out,
                 uint64_t* stats) {
    ensure_table();
    Digraph g;
    if (!build_digraph(n, m, src, dst, g)) return -1;
    u128 census[16] = {};                                        // step 1
    std::vector<SElem> S;
    for (uint32_t u = 0; u < n; ++u) bm_vertex(g, u, census, S); // step 2
    bm_finish(n, census);
    store(census, out);
    if (stats) { stats[0] = g.arcs; stats[1] = g.loops; stats[2] = g.dups; }
    return 0;
}

// The paper's CPU parallel form (Secs. 6-7): the u and v loops collapsed into one flat loop
// over connected pairs, dynamic scheduling, and private census vectors summed at the end.
// Identical arithmetic to or_census_bm per pair.
int or_census_bm_parallel(uint32_t n, uint64_t m, const uint32_t* src, const uint32_t* dst,
                          uint64_t* out, int threads) {
    ensure_table();
    Digraph g;
    if (!build_digraph(n, m, src, dst, g)) return -1;
    u128 census[16] = {};
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel
    {
        u128 priv[16] = {};
        std::vector<SElem> S;
#pragma omp for schedule(dynamic, 64)
        for (int64_t u = 0; u < (int64_t)n; ++u) bm_vertex(g, (uint32_t)u, priv, S);
#pragma omp critical
        for (int t = 0; t < 16; ++t) census[t] += priv[t];
    }
#else
    (void)threads;
    std::vector<SElem> S;
    for (uint32_t u = 0; u < n; ++u) bm_vertex(g, u, census, S);
#endif
    bm_finish(n, census);
    store(census, out);
    return 0;
}

// Timing samples of the Fig. 5 census on a graph built once (or_graph_new): runs steps
// 2.1 - 2.1.4 for the vertices u with u % stride == offset only (no 003 step) and returns
// the seconds spent in that loop; work_sample / work_total receive the merge length
// (|N[u]| + |N[v]| over the pairs) of the sample and of the whole graph.
void* or_graph_new(uint32_t n, uint64_t m, const uint32_t* src, const uint32_t* dst) {
    ensure_table();
    Digraph* g = new Digraph();
    if (!build_digraph(n, m, src, dst, *g)) { delete g; return nullptr; }
    return g;
}

void or_graph_free(void* h) { delete static_cast<Digraph*>(h); }

double or_census_bm_sample(void* h, uint32_t stride, uint32_t offset, uint64_t* out, uint64_t* work_sample,
                           uint64_t* work_total) {
    const Digraph& g = *static_cast<Digraph*>(h);
    const uint64_t tot = pair_work(g);
    u128 census[16] = {};
    std::vector<SElem> S;
    double t0 = now_seconds();
    uint64_t w = 0;
    for (uint32_t u = offset; u < g.n; u += stride) w += bm_vertex(g, u, census, S);
    double t1 = now_seconds();
    store(census, out);
    *work_sample = w;
    *work_total = tot;
    return t1 - t0;
}

// The same timing sample with the loop over the sampled vertices shared by OpenMP threads
// (dynamic schedule, private census vectors summed at the end: the paper's CPU form, Sec. 6-7).
// *threads_used receives the number of threads that ran.  Wall seconds of the loop.
double or_census_bm_sample_parallel(void* h, uint32_t stride, uint32_t offset, int threads, uint64_t* out,
                                    uint64_t* work_sample, uint64_t* work_total, int* threads_used) {
    const Digraph& g = *static_cast<Digraph*>(h);
    const uint64_t tot = pair_work(g);
    u128 census[16] = {};
    uint64_t w = 0;
    int used = 1;
    if (stride == 0) stride = 1;
    const int64_t count = offset < g.n ? (int64_t)((g.n - 1 - offset) / stride) + 1 : 0;
    double t0 = now_seconds();
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel reduction(+ : w)
    {
#pragma omp single
        used = omp_get_num_threads();
        u128 priv[16] = {};
        std::vector<SElem> S;
#pragma omp for schedule(dynamic, 1)
        for (int64_t k = 0; k < count; ++k) w += bm_vertex(g, offset + (uint32_t)k * stride, priv, S);
#pragma omp critical
        for (int t = 0; t < 16; ++t) census[t] += priv[t];
    }
#else
    (void)threads;
    std::vector<SElem> S;
    for (int64_t k = 0; k < count; ++k) w += bm_vertex(g, offset + (uint32_t)k * stride, census, S);
#endif
    double t1 = now_seconds();
    store(census, out);
    *work_sample = w;
    *work_total = tot;
    if (threads_used) *threads_used = used;
    return t1 - t0;
}

// The O(n^3) definition: every 3-subset a<b<c, classified by canonical form.
int or_census_brute(uint32_t n, uint64_t m, const uint32_t* src, const uint32_t* dst, uint64_t* out) {
    if (n > 4096) return -2;
    uint8_t T[64];
    if (or_table_canonical(T) != 0) return -3;
    std::vector<uint8_t> adj((size_t)n * n, 0);
    for (uint64_t i = 0; i < m; ++i) {
        if (src[i] >= n || dst[i] >= n) return -1;
        if (src[i] != dst[i]) adj[(size_t)src[i] * n + dst[i]] = 1;
    }
    auto A = [&](uint32_t x, uint32_t y) { return adj[(size_t)x * n + y] != 0; };
    u128 census[16] = {};
    for (uint32_t a = 0; a < n; ++a)
        for (uint32_t b = a + 1; b < n; ++b)
            for (uint32_t c = b + 1; c < n; ++c) {
                int code = (A(b, a) ? 1 : 0) | (A(a, b) ? 2 : 0) | (A(b, c) ? 4 : 0) | (A(c, b) ? 8 : 0) |
                           (A(a, c) ? 16 : 0) | (A(c, a) ? 32 : 0);
                census[T[code]] += 1;
            }
    store(census, out);
    return 0;
}

// O(m) statistics, each as (lo, hi):
//   0 mutual dyads M, 1 asymmetric dyads A, 2 null dyads C(n,2)-M-A,
//   3 sum_v C(dout,2), 4 sum_v C(din,2), 5 sum_v (din*dout - mutual partners of v),
//   6 undirected triangles, 7 distinct arcs.
// The O(m) statistics; with_triangles = 0 leaves the triangle count (the one superlinear part)
// at 0, for graphs too large to count them on the CPU.
int or_invariants_opt(uint32_t n, uint64_t m, const uint32_t* src, const uint32_t* dst, uint64_t* out,
                      int with_triangles) {
    Digraph g;
    if (!build_digraph(n, m, src, dst, g)) return -1;
    u128 M = 0, A = 0, out2 = 0, in2 = 0, paths = 0, tri = 0;
    std::vector<uint64_t> din(n, 0);
    for (uint32_t x = 0; x < n; ++x)
        for (uint32_t y : g.out[x]) din[y]++;
    for (uint32_t x = 0; x < n; ++x) {
        uint64_t dout = g.out[x].size(), mut = 0;
        for (const Tagged& t : g.N[x]) {
            if (t.out && t.in) ++mut;
            if (x < t.id) { if (t.out && t.in) ++M; else ++A; }
        }
        out2 += (u128)dout * (dout - (dout ? 1 : 0)) / 2;
        in2 += (u128)din[x] * (din[x] - (din[x] ? 1 : 0)) / 2;
        paths += (u128)din[x] * dout - mut;
    }
    // triangles, each once: orient every pair from lower to higher (degree, id) rank and
    // count, for each oriented pair a->b, the common out-neighbours of a and b
    std::vector<uint64_t> deg(with_triangles ? n : 0);
    for (uint32_t x = 0; x < deg.size(); ++x) deg[x] = g.N[x].size();
    auto before = [&](uint32_t x, uint32_t y) { return deg[x] < deg[y] || (deg[x] == deg[y] && x < y); };
    std::vector<std::vector<uint32_t>> fwd(with_triangles ? n : 0);
    for (uint32_t x = 0; x < fwd.size(); ++x) {
        for (const Tagged& t : g.N[x])
            if (before(x, t.id)) fwd[x].push_back(t.id);
        std::sort(fwd[x].begin(), fwd[x].end());
    }
    for (uint32_t a = 0; a < fwd.size(); ++a)
        for (uint32_t b : fwd[a]) {
            auto ia = fwd[a].begin(), ib = fwd[b].begin();
            while (ia != fwd[a].end() && ib != fwd[b].end()) {
                if (*ia < *ib) ++ia; else if (*ib < *ia) ++ib; else { ++tri; ++ia; ++ib; }
            }
        }
    u128 pairs = (u128)n * (n ? n - 1 : 0) / 2;
    u128 vals[8] = {M, A, pairs - M - A, out2, in2, paths, tri, (u128)g.arcs};
    for (int k = 0; k < 8; ++k) { out[2 * k] = (uint64_t)vals[k]; out[2 * k + 1] = (uint64_t)(vals[k] >> 64); }
    return 0;
}

int or_invariants(uint32_t n, uint64_t m, const uint32_t* src, const uint32_t* dst, uint64_t* out) {
    return or_invariants_opt(n, m, src, dst, out, 1);
}

}  // extern "C"
