// graph.cuh - the tc_graph object: device CSR (Sec. 6, Fig. 7), statistics, cached census
// plans and the per-graph census workspace.
#pragma once

#include <mutex>
#include <vector>

#include "tc_internal.cuh"

namespace tc {

// Census options.  chunk and ctas_per_sm may be 0 (= automatic) until finalised for the
// chosen kernel family: the suffix form keeps a hash of 4 slots per staged entry (2048
// entries by default), the union walk one of 2 slots plus the sorted chunk (4096).
struct Opts {
    uint32_t algo = TC_ALGO_UNION;
    uint32_t schedule = TC_SCHED_PLAIN;
    uint32_t warp_max_deg = 64;
    uint32_t chunk = 0;
    uint32_t item_work = 0;   // 0: sized to the graph (adaptive_item_work)
    uint32_t ctas_per_sm = 0;
    uint32_t map_mode = 0;    // 0 auto, 1 always, 2 never (single-graph census with tables)
    bool chunk_auto = false;  // chunk was left to the library (census_fit_chunk may widen it)
    bool operator==(const Opts& o) const {
        return algo == o.algo && schedule == o.schedule && warp_max_deg == o.warp_max_deg && chunk == o.chunk &&
               item_work == o.item_work && ctas_per_sm == o.ctas_per_sm && map_mode == o.map_mode;
    }
};

// Overlay the non-zero fields of `in` on `base`, fill the automatic values and validate.
tc_status resolve_opts(const tc_options* in, const Opts* base, Opts* out);
// Work units per CTA item when none is set: about four items per CTA of the launch, so a large
// census re-stages hub lists rarely and a small one still spreads over every SM.
__host__ __device__ inline uint32_t adaptive_item_work(unsigned long long total_units, unsigned grid) {
    unsigned long long w = total_units / (4ull * (grid ? grid : 1u));
    if (w < (1ull << 14)) w = 1ull << 14;
    if (w > (1ull << 22)) w = 1ull << 22;
    return (uint32_t)w;
}
// Overlay only (automatic values kept), for a graph's stored defaults.
Opts merge_opts(const tc_options* in, const Opts* base);

// A census plan: the CTA work items for the vertices with deg > warp_max_deg, and the
// id range of the vertices handled one warp per vertex.
struct Plan {
    bool valid = false;
    Opts key;
    DevBuf items;
    uint32_t n_items = 0;
    uint32_t warp_begin = 0, warp_end = 0;
    // shards of the plan's work for shard_world ranks (plan_shards): rank r runs items
    // [shard_bounds[2r], shard_bounds[2r+2]) and warp-tier vertices warp_begin +
    // [shard_bounds[2r+1], shard_bounds[2r+3]); 0 = not computed
    uint32_t shard_world = 0;
    std::vector<uint32_t> shard_bounds;
};

struct GraphStore {
    uint32_t n = 0, n_active = 0, max_deg = 0;
    uint64_t arcs = 0, e_sym = 0, mutual = 0, loops = 0, dups = 0, sum_d2 = 0, sum_dv_upper = 0, sum_walk = 0;
    uint64_t sum_walk_map = 0;   // walked entries with ids below kMapIdsSuffix
    uint64_t sum_tri_walk = 0;   // sum of up (up - 1) / 2: the entries the triangle form walks
    DevBuf off, adj, up, new_of_old;
    DevBuf ub, rp, vs, us;   // per upper pair tables (see GraphDev)
    DevBuf ctr;        // census work counters (uint32 x 4)
    DevBuf acc;        // census accumulators (uint64 x 16)
    DevBuf cost;       // optional per-vertex predicted cost (float x n) for the learned schedule
    DevBuf tri;        // triangle form: bulk sums and triangle tricode histogram (uint64 x 96)
    Opts opts;
    static constexpr int kPlans = 4;
    Plan plans[kPlans];
    int next_plan = 0;
    unsigned long long* h_counts = nullptr;   // pinned staging for 16 counts
    std::mutex busy;

    GraphDev dev() const {
        GraphDev d;
        d.n = n;
        d.n_active = n_active;
        d.off = off.as<uint64_t>();
        d.adj = adj.as<uint32_t>();
        d.up = up.as<uint32_t>();
        d.ub = ub.as<uint64_t>();
        d.rp = rp.as<uint32_t>();
        d.vs = vs.as<uint2>();
        d.us = us.as<uint2>();
        return d;
    }
};

}  // namespace tc

struct tc_graph {
    tc::GraphStore s;
};

namespace tc {

// One request's slice in a serving wave: its graph, a range of its plan's CTA items, a range
// of its one-warp-per-vertex tier (taken 2^pad vertices per warp-tier block), the prefixes of
// items / warp-tier blocks of the slices before it in the wave, and its output (16 uint64 the
// kernel adds to).
struct WaveReq {
    GraphDev g;
    const Item* items;
    unsigned long long* out;
    uint32_t n_items, item_pre, warp_begin, warp_end, block_pre, pad;
};
// slices per wave launch; 32 descriptors (2.3 KB of static shared memory) keep three CTAs
// per SM at the default chunk
constexpr uint32_t kMaxWave = 32;

tc_status build_from_arcs(GraphStore& g, uint64_t m, const uint32_t* d_src, const uint32_t* d_dst, cudaStream_t st);
tc_status build_from_csr(GraphStore& g, const uint64_t* d_off, const uint32_t* d_adj, cudaStream_t st);
// From m distinct arc keys sorted ascending, each (lo << (B+2)) | (hi << 2) | dir with lo < hi the
// pair's ids, B = bits_for(n) and dir 1 for lo -> hi, 2 for hi -> lo (a mutual pair has both).
tc_status build_from_sorted_arcs(GraphStore& g, const uint64_t* d_keys, uint64_t m, cudaStream_t st);
// Bits of a vertex id in the build's keys: the least B >= 1 with 2^B >= n.
int bits_for(uint32_t n);
// A graph (as tc_graph_create_arcs makes it, options `opt`) from m sorted distinct arc keys on
// the device, as build_from_sorted_arcs takes them; synchronises `st`.
tc_status graph_create_sorted(uint32_t n, const uint64_t* d_keys, uint64_t m, cudaStream_t st, const tc_options* opt,
                              tc_graph** out);

// Enqueue one census on `st`; counts of classes 1..15 are added to d_out16 (which the
// caller zeroes; index 0 is never touched).  No host synchronisation, no allocation once
// the plan for `o` exists (get_plan allocates it on first use).
tc_status get_plan(GraphStore& g, const Opts& o, cudaStream_t st, Plan** out);
// The single-graph census's form (map or not) and, for an automatic chunk, its size: call
// before get_plan, whose items depend on the chunk.
bool census_map(const GraphStore& g, const Opts& o);
void census_fit_chunk(const GraphStore& g, Opts& o);
// d_vcost (optional, [n] uint64, caller-zeroed) receives the SM cycles spent per vertex u;
// d_phase (optional, [3 * CTAs] uint64) the globaltimer at start, end of items, end per CTA.
tc_status census_enqueue(GraphStore& g, const Opts& o, const Plan& p, cudaStream_t st, unsigned long long* d_out16,
                         unsigned long long* d_vcost = nullptr, unsigned long long* d_phase = nullptr);
// The same census over a part of a plan: items[0, n_items) and warp-tier vertices
// [warp_begin, warp_end) (a shard; census_enqueue runs the whole plan).
tc_status census_enqueue_range(GraphStore& g, const Opts& o, const Item* items, uint32_t n_items, uint32_t warp_begin,
                               uint32_t warp_end, cudaStream_t st, unsigned long long* d_out16,
                               unsigned long long* d_vcost = nullptr, unsigned long long* d_phase = nullptr);
// TC_ALGO_TRIANGLE (triangles.cu): the bulk pair sums and the triangle tricode histogram over
// the given items and warp-tier range, and the fold into d_out16[1..15].
tc_status triangle_census_enqueue(GraphStore& g, const Opts& o, const Item* items, uint32_t n_items,
                                  uint32_t warp_begin, uint32_t warp_end, cudaStream_t st, unsigned long long* d_out16,
                                  unsigned long long* d_vcost, unsigned long long* d_phase = nullptr);
// Batched triangle form: k graphs (d_graphs), items tagged with the graph (pad), warp-tier
// blocks (u0, u1, graph); d_scratch holds 96 uint64 per graph (zeroed here), graph g's counts of
// classes 1..15 are added to d_out[16 g ..] (caller-zeroed); ctr: 4 zeroed uint32.
tc_status triangle_census_batch(const GraphDev* d_graphs, uint32_t k, const Item* items, uint32_t n_items,
                                const uint4* wblocks, uint32_t n_wblocks, const Opts& o, uint32_t* ctr,
                                unsigned long long* d_scratch, unsigned long long* d_out, cudaStream_t st);
// Serving wave of the triangle form: the request slices' bulk sums and triangle tricodes into each
// request's 96-uint64 scratch (WaveReq.out); ctr: 4 zeroed uint32.
tc_status triangle_census_wave(const WaveReq* d_reqs, uint32_t n_reqs, uint32_t total_items, uint32_t total_blocks,
                               const Opts& o, unsigned grid, uint32_t* ctr, cudaStream_t st);
// Fold n finished requests' scratch into 16 counts each at d_dst + 16 k (index 0 = 0) and zero the
// scratch.
tc_status triangle_collect(unsigned long long* const* scratch, uint32_t n, unsigned long long* d_dst, cudaStream_t st);
// The triangle walk alone: histogram of the 64 tricodes (old == nullptr) or of the 64 states in
// the caller's id order (old = original id per vertex, d_perm_state = [9][64] state of a
// tricode per rank pattern) of every triangle, added into d_hist64; ctr: 4 zeroed uint32.
tc_status triangles_launch(const GraphDev& gd, const Opts& o, const Item* items, uint32_t n_items, uint32_t warp_begin,
                           uint32_t warp_end, uint32_t* ctr, const uint32_t* old, const uint8_t* d_perm_state,
                           unsigned long long* d_hist64, unsigned long long* d_vcost, cudaStream_t st,
                           unsigned long long* d_phase = nullptr);
// Cut p's work into `world` contiguous shards of about equal work (cached in p for that world);
// synchronises st when it computes them.
tc_status plan_shards(GraphStore& g, const Opts& o, Plan& p, uint32_t world, cudaStream_t st);
int census_grid(const Opts& o);
// log2 of the vertices a warp takes per grab in the one-warp-per-vertex tier, for `vertices`
// such vertices and a grid of `grid` CTAs (0..5).
uint32_t warp_block_shift(uint64_t vertices, unsigned grid);
// Batched census: one launch over several graphs (d_graphs on the device); item.pad is the
// graph index, wblocks are (u0, u1, graph, 0) warp-tier blocks; graph g's counts are added to
// d_out[16 g ..] (caller-zeroed); ctr: 4 zeroed uint32.  census_prepare must have run.
tc_status census_launch_batch(const GraphDev* d_graphs, const Item* items, uint32_t n_items, const uint4* wblocks,
                              uint32_t n_wblocks, const Opts& o, uint32_t* ctr, unsigned long long* d_out, cudaStream_t st);
// Wave census (serving): n_reqs request slices (device descriptors) with total_items CTA
// items and total_blocks warp-tier blocks; slice r's counts are added to d_reqs[r].out;
// ctr: 4 zeroed uint32.  census_prepare must have run.
tc_status census_launch_wave(const WaveReq* d_reqs, uint32_t n_reqs, uint32_t total_items, uint32_t total_blocks,
                             const Opts& o, unsigned grid, uint32_t* ctr, cudaStream_t st);
// Per-device set-up of the census kernels (table upload, shared-memory limit); synchronises st.
tc_status census_prepare(cudaStream_t st, const Opts& o);
// Launch the census kernel on explicit buffers (no allocation): the work items, the id range
// of the one-warp-per-vertex tier and 4 zeroed uint32 work counters are the caller's.
tc_status census_launch_raw(const GraphDev& gd, const Opts& o, const Item* items, uint32_t n_items, uint32_t warp_begin,
                            uint32_t warp_end, uint32_t* ctr, unsigned long long* d_out16, cudaStream_t st);

// The library's tricode -> class table (derived in tables.cu); census.cu copies it into
// its device memory before the first census.
const uint8_t* host_tricode_table();

}  // namespace tc
