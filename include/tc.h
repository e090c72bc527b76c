/*
 * tc.h - C ABI of the GB300 triad-census library (libtc.so).
 *
 * Computes the exact 16-type directed triad census of Batagelj and Mrvar (paper Sec. 4,
 * Fig. 5) on one GPU.  The graph is held as the compact structure of Sec. 6 (Fig. 7): one
 * edge array, a start offset per vertex, and the neighbour id stored with two low direction
 * bits.  All signatures use plain C types and pointers; nothing here depends on PyTorch.
 *
 * Census index order (0-based), used by every output array:
 *   0 003   1 012   2 102   3 021D  4 021U  5 021C  6 111D  7 111U
 *   8 030T  9 030C 10 201  11 120D 12 120U 13 120C 14 210  15 300
 * (Fig. 5 step 5 fixes index 0 = null triads, step 2.1.2 fixes 1 = one asymmetric dyad and
 * 2 = one mutual dyad; the others follow the usual mutual-asymmetric-null order.)
 *
 * Conventions for every entry point:
 *   - Return a tc_status; TC_OK is 0.  On failure nothing is written to the outputs, and
 *     tc_last_error() returns a message for the calling thread.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *   - Device memory comes from the library's own stream-ordered pool on each device; freed
 *     blocks stay in the pool (up to a quarter of the device's memory) for later calls.
 *     A graph's buffers are owned by the tc_graph until tc_graph_destroy, which first waits
 *     for the device (as cudaFree does); temporaries are released in stream order.
 *   - The caller keeps ownership of every buffer it passes; inputs are copied.
 *   - Vertex ids are uint32 and must be < n; n must be <= 2^30 because each stored id
 *     carries two direction bits (Sec. 6).
 */
#ifndef TC_H
#define TC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tc_graph tc_graph;                 /* opaque; owns its device CSR */
typedef struct { uint64_t lo, hi; } tc_u128;      /* unsigned 128-bit count, little-endian halves */

typedef enum {
    TC_OK = 0,
    TC_ERR_ARG = 1,       /* null pointer, malformed CSR, bad option */
    TC_ERR_RANGE = 2,     /* a vertex id >= n, n > 2^30, or a count beyond a documented limit */
    TC_ERR_OOM = 3,       /* device (or pinned host) allocation failed */
    TC_ERR_CUDA = 4,      /* a CUDA runtime call or kernel launch failed */
    TC_ERR_TIMEOUT = 5,   /* a bounded device-side wait gave up */
    TC_ERR_BUSY = 6       /* the object is in use by another call */
} tc_status;

/* Which census kernel family runs the hot loop (step 2.1.4 of Fig. 5). */
typedef enum {
    /* Visit every third vertex w of S = N[u] u N[v] \ {u,v} and classify it through the
     * 64-entry tricode table (Fig. 5 with the two-list walk of Sec. 6, Fig. 8). */
    TC_ALGO_UNION = 0,
    /* Same census; the w that only u reaches and that lie past v are classified in bulk
     * from per-list direction-class counts instead of one by one (only dir(u,v) and
     * dir(u,w) decide their class), so each pair costs O(|N[v]|). */
    TC_ALGO_SUFFIX = 1,
    /* Same census; the one-sided third vertices of each pair are counted in bulk as in
     * TC_ALGO_SUFFIX, and the common neighbours of all pairs are found once per triangle
     * (a < b < c met once, walking the lower-id neighbours of c against those of b), whose
     * tricode fixes the triad and its corrections to the three pairs' bulk and dyadic
     * counts (steps 2.1.2 - 2.1.4).  Needs the per upper pair tables every built graph has;
     * warp_max_deg <= 128. */
    TC_ALGO_TRIANGLE = 2
} tc_algo;

/* How the connected pairs (u,v) are grouped into GPU work items. */
typedef enum {
    TC_SCHED_PLAIN = 0,    /* degree-threshold tiers; a vertex's pairs split into items by their exact work
                              (the N[v] entries walked plus per-pair overheads) */
    TC_SCHED_LEARNED = 1   /* the same, with each vertex's item count from the learned cost model */
} tc_schedule;

/* Options; zero-initialise and set what you need (0 selects the default). */
typedef struct {
    uint32_t algo;            /* tc_algo, default TC_ALGO_UNION */
    uint32_t schedule;        /* tc_schedule, default TC_SCHED_PLAIN */
    uint32_t warp_max_deg;    /* vertices u with deg <= this run one warp per u (default 64) */
    uint32_t chunk_entries;   /* neighbour entries of u staged per CTA: power of 2 in [512, 16384],
                                 at most 8192 for TC_ALGO_SUFFIX (default 2048 for TC_ALGO_SUFFIX,
                                 4096 for TC_ALGO_UNION) */
    uint32_t item_work;       /* work per CTA item, in list entries walked plus pair overheads
                                 (0 = sized to the graph: about four items per CTA, 2^14 to 2^22) */
    uint32_t ctas_per_sm;     /* persistent CTAs per SM (default 3) */
    uint32_t map_mode;        /* direct id map of the staged lists in a single-graph census: 0 = when at
                                 least half the walked lookups fall in its range, 1 = always, 2 = never */
    uint32_t reserved[9];
} tc_options;

/* Statistics of a built graph (all counts after cleaning). */
typedef struct {
    uint32_t n;               /* vertices, isolated ones included */
    uint32_t max_deg;         /* largest symmetric degree */
    uint64_t arcs;            /* distinct directed arcs; a mutual pair counts 2 */
    uint64_t e_sym;           /* connected (unordered) pairs = upper pairs u<v */
    uint64_t mutual;          /* mutual pairs */
    uint64_t loops_dropped;   /* self-loops in the input */
    uint64_t dups_dropped;    /* repeated arcs in the input */
    uint64_t sum_d2;          /* sum over vertices of deg^2 = merge steps of the full union walk */
    uint64_t sum_dv_upper;    /* sum over upper pairs u<v of deg(v) */
    uint64_t bytes_alg;       /* algorithmic bytes of one census (below) */
    uint64_t sum_walk;        /* sum over upper pairs u<v of |{w in N(v): w > u}|: the N[v] entries
                                 a census walks */
    uint64_t sum_walk_map;    /* those of them with ids below 2^17 (answered by the direct id map) */
    uint64_t sum_tri_walk;    /* sum over upper pairs (b, c) of the neighbours of c with (relabelled) ids
                                 below b: the entries TC_ALGO_TRIANGLE walks */
    uint64_t bytes_alg_tri;   /* algorithmic bytes of one TC_ALGO_TRIANGLE census (below) */
} tc_graph_info;
/* bytes_alg = 16(n+1) + 44 e_sym + 4 sum_walk + 128: the CSR read once (offsets 8(n+1), lists
 * 8 e_sym), the per-pair tables (8(n+1) + 20 e_sym), 16 B of bookkeeping per pair, 4 B per
 * N[v] entry walked, and the 16 counters.
 * bytes_alg_tri = 32(n+1) + 60 e_sym + 4 sum_tri_walk + 1280: per vertex 32 B (offsets, lower-
 * neighbour counts and table starts, read by the bulk pass and by the walk); per upper pair
 * 60 B (the bulk pass: the pair's entry, its 20 B of tables and the other end's two offsets;
 * the walk: the entry again, the other end's offset, the pair's position table entry, and the
 * pair's share of the staged lower lists); 4 B per entry walked; the 96 counters and the fold. */

/* Build a graph from an arc list (Sec. 6, Fig. 7).  src[i] -> dst[i] for i < m; self-loops
 * and repeated arcs are dropped and counted.  Ids >= n give TC_ERR_RANGE.  src/dst are
 * device pointers if ptr_is_device, else host pointers: page-locked host arrays (cudaHostAlloc,
 * cudaHostRegister) are read once by the build's first kernel directly over the host link,
 * pageable ones are copied to the device on `stream` first.
 * Vertices are relabelled by descending symmetric degree (ties by original id); the census
 * does not depend on labels.  opt may be NULL.  The call synchronises `stream`. */
tc_status tc_graph_create_arcs(uint32_t n, uint64_t m, const uint32_t* src, const uint32_t* dst,
                               int ptr_is_device, void* stream, const tc_options* opt, tc_graph** out);

/* Build a graph from a CSR already in the Fig. 7 form: off[n+1] (uint64) and
 * adj_flagged[off[n]] where each entry is (id << 2) | dir, dir 1 = owner->id, 2 = id->owner,
 * 3 = both.  Every list must be strictly ascending by id, loop-free, with dir != 0, and the
 * lists must be symmetric (x in N[y] iff y in N[x], with mirrored dir bits); otherwise
 * TC_ERR_ARG.  Pointers are device or host as for tc_graph_create_arcs. */
tc_status tc_graph_create_csr(uint32_t n, const uint64_t* off, const uint32_t* adj_flagged,
                              int ptr_is_device, void* stream, const tc_options* opt, tc_graph** out);

/* Full census (Fig. 5): 16 counts, the null count (index 0) computed as C(n,3) minus the
 * rest in 128-bit (steps 3-5).  Enqueues the kernels on `stream` and synchronises it. */
tc_status tc_census(tc_graph* g, void* stream, tc_u128 out[16]);

/* Same census with options overriding the graph's creation options (algo, schedule,
 * tiers) for this call only.  opt may be NULL. */
tc_status tc_census_opts(tc_graph* g, void* stream, const tc_options* opt, tc_u128 out[16]);

/* Asynchronous census: enqueues the kernels on `stream` and writes, when they finish,
 * counts of classes 1..15 to d_out16[1..15] (device memory, uint64) and 0 to d_out16[0].
 * The null count needs 128-bit arithmetic: obtain it with tc_null_count.  Does not
 * synchronise; d_out16 must stay valid until the stream reaches the end of the census. */
tc_status tc_census_async(tc_graph* g, void* stream, const tc_options* opt, uint64_t* d_out16);

/* Instrumented census, for scheduling and for training the learned cost model: the same
 * counts as tc_census_async into d_out16, plus the SM cycles spent on each vertex u (as the
 * smaller endpoint of its pairs, Fig. 5 step 2) added into d_vcost[n] (device uint64, indexed
 * by the relabelled id of tc_graph_device_csr; the caller zeroes it).  d_phase (device uint64,
 * may be NULL) receives, for each of the tc_census_grid() CTAs, the global timer in ns at
 * its start, at the end of its CTA work items and at its end (in the TC_ALGO_TRIANGLE form,
 * those of the triangle walk's launch).  Does not synchronise. */
tc_status tc_census_profile(tc_graph* g, void* stream, const tc_options* opt, uint64_t* d_out16,
                            uint64_t* d_vcost, uint64_t* d_phase);

/* One rank's share of a census sharded over `world` GPUs (paper Sec. 6-7: the connected pairs
 * (u, v) of Fig. 5 step 2.1 are independent units of work, so any partition of them sums to the
 * census).  The census's work - the plan's CTA work items in order, then the vertices handled
 * one warp each, in id order - is cut into `world` contiguous shards of about equal work
 * (the plan's exact per-pair work units), and this call runs shard `rank` (0 <= rank < world,
 * else TC_ERR_ARG).  Every rank holds the same graph.  d_out16 (device, 16 uint64) receives
 * this shard's counts of classes 1..15 (index 0 = 0), as tc_census_async does; summing the
 * world shards' outputs (an all-reduce of 16 uint64) gives the census's classes 1..15, and
 * tc_null_count of that sum gives the null count.  The first call for a plan and a world
 * computes the shards and synchronises `stream`; later calls only enqueue.  TC_ERR_BUSY if the
 * graph is in use by another call; TC_ERR_RANGE if world > 2^20. */
tc_status tc_census_shard(tc_graph* g, void* stream, const tc_options* opt, uint32_t rank, uint32_t world,
                          uint64_t* d_out16);

/* Where the shards of tc_census_shard start: bounds[2r] = the first CTA work item and
 * bounds[2r+1] = the first one-warp-per-vertex id of shard r, for r = 0..world (r = world: the
 * item count and the end of that tier's id range).  Host array of 2 (world + 1) uint32.
 * Synchronises `stream` when the shards are not yet computed. */
tc_status tc_census_shard_bounds(tc_graph* g, void* stream, const tc_options* opt, uint32_t world, uint32_t* bounds);

/* Number of CTAs the census launches on the current device for these options (opt may be
 * NULL): the length / 3 of d_phase above. */
uint32_t tc_census_grid(const tc_options* opt);

/* Null count C(n,3) - sum(counts[1..15]) in 128-bit (Fig. 5 steps 3-5), on the host. */
tc_u128 tc_null_count(uint32_t n, const uint64_t counts16[16]);

/* The 64-state census (Sec. 3, Fig. 2): out[s] = the number of triads in labelled state s, the
 * arc pattern among the three actors before isomorphic states are merged into the 16 classes.
 * The paper does not fix which actor takes which role; here they take the roles (u, v, w) in
 * increasing vertex id of the caller's labels, and s has the tricode's bits: 1 v->u, 2 u->v,
 * 4 v->w, 8 w->v, 16 u->w, 32 w->u (so out[0] is the null triads, C(n,3) less the rest).
 * Merging the states through tc_tricode_table gives tc_census's 16 counts.  out: 64 host
 * tc_u128 values.  Synchronises the stream.  Errors: TC_ERR_ARG (null argument), TC_ERR_BUSY
 * (the graph is in use by another call), TC_ERR_OOM, TC_ERR_CUDA. */
tc_status tc_census64(tc_graph* g, void* stream, tc_u128 out[64]);

/* The census by its matrix form (Sec. 4 names Moody's matrix census as the dense alternative to
 * Fig. 5): with S the one-way arcs, M the mutual and N the null dyads as 0/1 matrices, each class
 * count is a sum of an elementwise product of one of them with one of the products NN, S'S, SS',
 * SS, NM, MM, divided by the class's symmetries (003 = sum(N o NN)/6, 012 = sum(S o NN), ...,
 * 300 = sum(M o MM)/6).  All 16 counts come from their own sums (the null count too).  The
 * matrices are bit-packed and each product's masked sums are fused into its tiles: O(n^3 / 64)
 * work, a dense cross-check of the Fig. 5 kernels for graphs of n <= 2^14 vertices (larger n:
 * TC_ERR_RANGE).  out: 16 host tc_u128.  Synchronises the stream.  TC_ERR_BUSY if the graph is
 * in use by another call, TC_ERR_OOM, TC_ERR_CUDA. */
tc_status tc_census_matrix(tc_graph* g, void* stream, tc_u128 out[16]);

/* Census of k graphs in one persistent launch (builds a tc_batch, runs it once, frees it).
 * out16xk receives 16 uint64 per graph in the callers' order (index 0 set to the low 64 bits
 * of the null count); out003_k (may be NULL) receives each full 128-bit null count.  Host
 * pointers.  Synchronises `stream`. */
tc_status tc_census_batch(tc_graph* const* gs, uint32_t k, void* stream, uint64_t* out16xk,
                          tc_u128* out003_k);

/* A reusable batch: one combined work plan for the k graphs (largest graph first; CTA items of
 * every graph, then one-warp-per-vertex blocks of every graph, drawn by one persistent launch
 * from two device work counters) and that launch captured in a CUDA graph.  The graphs must
 * outlive the batch.  opt may be NULL (the defaults of tc_options).  Synchronises `stream`. */
typedef struct tc_batch tc_batch;
tc_status tc_batch_create(tc_graph* const* gs, uint32_t k, const tc_options* opt, void* stream, tc_batch** out);

/* Replay the captured launch on `stream`; if d_out16xk (device, 16 uint64 per graph) is not
 * NULL the counts of classes 1..15 (index 0 = 0) are copied there in the callers' order. */
tc_status tc_batch_census_async(tc_batch* b, void* stream, uint64_t* d_out16xk);

/* Replay and return host counts as for tc_census_batch.  Synchronises `stream`. */
tc_status tc_batch_census(tc_batch* b, void* stream, uint64_t* out16xk, tc_u128* out003_k);

/* Autotuner: time the batch under candidate kernel forms and tile and tier thresholds by
 * coordinate descent from the batch's current options - algo {union, suffix, triangle},
 * warp_max_deg {16..256}, chunk_entries {1024..8192}, ctas_per_sm {2..8}, item_work {sized to the
 * graphs, 2^14..2^22} - one at a time, keeping the best value of each, for up to three passes
 * or until a pass gains under 1% (at most max_trials timed plans, 0 = no limit; each timed as
 * the median of three replays after one untimed one).  Keeps the fastest plan in the batch and
 * reports its options and median time per launch in ms.  Synchronises `stream`. */
tc_status tc_batch_autotune(tc_batch* b, void* stream, uint32_t max_trials, tc_options* best, float* best_ms);

/* The trials of the batch's last autotune, in the order they ran (options and median ms). */
typedef struct {
    tc_options opts;
    float ms;
} tc_autotune_trial;
tc_status tc_batch_autotune_history(const tc_batch* b, tc_autotune_trial* out, uint32_t max, uint32_t* count);

/* Work counts of the batch's current plan (either pointer may be NULL). */
tc_status tc_batch_stats(const tc_batch* b, uint32_t* n_items, uint32_t* n_warp_blocks);

void tc_batch_destroy(tc_batch* b);

tc_status tc_graph_stats(const tc_graph* g, tc_graph_info* info);

/* Device pointers of the built CSR in the relabelled ids, and the relabelling:
 * new_of_old[old id] = new id.  Valid until tc_graph_destroy.  Any out pointer may be NULL. */
tc_status tc_graph_device_csr(const tc_graph* g, const uint64_t** off, const uint32_t** adj,
                              const uint32_t** new_of_old);

/* Copy the built CSR (relabelled ids, Fig. 7 layout) and the relabelling to host memory:
 * off_host[n+1], adj_host[2*e_sym], new_of_old_host[n].  Any pointer may be NULL to skip
 * that array.  Synchronous (uses the legacy default stream). */
tc_status tc_graph_export_csr(const tc_graph* g, uint64_t* off_host, uint32_t* adj_host, uint32_t* new_of_old_host);

void tc_graph_destroy(tc_graph* g);
const char* tc_status_str(tc_status s);
const char* tc_last_error(void);

/* Census that allocates nothing, for callers that cannot call cudaMalloc (allocation is
 * forbidden or must not block where they run, or all device memory is already reserved by
 * their own pool).  The paper has no counterpart to this entry point.
 *
 * Input: a device CSR in this library's form, as tc_graph_device_csr returns it: d_off[n+1]
 * (uint64, starting at 0 and never decreasing) and d_adj[d_off[n]] (uint32 (id << 2) | dir,
 * ids < n, no self-loops, dir != 0, strictly ascending per list, symmetric with mirrored dir
 * bits), with vertex degrees not increasing with the id.  Every one of these rules is checked
 * on the device before the census runs (the checks read only inside the lists that the offsets
 * define), and a CSR that breaks one gives TC_ERR_ARG with nothing launched after the check.
 * Output: d_out16 (device, 16 uint64) as for tc_census_async (index 0 = 0; get the null count
 * with tc_null_count).
 * Scratch: one fixed 8 MiB device array inside the library, so n <= 2^20 (larger n gives
 * TC_ERR_RANGE, as does a graph needing more than 2^18 work items).  Every GPU that loads the
 * library holds the array until the process exits.  The first call on a device looks up the
 * array's device address; make that first call before any stream capture.  All calls share
 * the array and it keeps the last call's contents, so calls that overlap on the GPU race:
 * serialise them.  The call synchronises `stream` while it checks the CSR and sizes the work,
 * then enqueues the census and returns. */
tc_status tc_census_csr_noalloc(uint32_t n, const uint64_t* d_off, const uint32_t* d_adj, void* stream,
                                uint64_t* d_out16);

/* ------------------------------------------------------------------ learned schedule
 * A small network predicts, per vertex u, the SM cycles its pairs (u, v > u) cost the census
 * (Fig. 5 step 2 unit); the plan then takes u's number of work items from that prediction
 * (schedule TC_SCHED_LEARNED) instead of from the exact work total (the cuts still follow the
 * pairs' exact work).  It only reorders work: counts
 * are the same either way.  Network: features log1p(out-degree, in-degree, degree, sum of
 * neighbour degrees) -> 32 -> 32 -> 1 (tanh), FP16 weights, FP32 accumulation, output
 * log(cycles); trained on the GPU with Adam on cycles measured by tc_census_profile. */
typedef struct tc_costmodel tc_costmodel;
uint32_t tc_costmodel_num_params(void);   /* 1249: W1[32][4] b1[32] W2[32][32] b2[32] W3[32] b3 */
tc_status tc_costmodel_create(uint64_t seed, tc_costmodel** out);
void tc_costmodel_destroy(tc_costmodel* c);
/* FP32 master weights in the layout above (host arrays); set also refreshes the FP16 copy. */
tc_status tc_costmodel_set_params(tc_costmodel* c, const float* host);
tc_status tc_costmodel_get_params(const tc_costmodel* c, float* host);
/* Input standardisation (x - mean) / std, target centring, and kappa = plan units per cycle. */
tc_status tc_costmodel_set_norm(tc_costmodel* c, const float mean[4], const float std_[4], float target_mean,
                                float kappa);
tc_status tc_costmodel_get_norm(const tc_costmodel* c, float mean[4], float std_[4], float* target_mean, float* kappa);
/* Fit the standardisation to training samples (device arrays) and set kappa. */
tc_status tc_costmodel_fit_norm(tc_costmodel* c, const float* d_x4, const float* d_y, uint32_t count, float kappa,
                                void* stream);
/* Per-vertex features of a graph into d_feat4[4 n] (device, relabelled ids).  Asynchronous. */
tc_status tc_graph_features(const tc_graph* g, void* stream, float* d_feat4);
/* Training samples from a profiled census: every vertex split into CTA work items (degree
 * above the graph's warp-tier threshold) with d_vcost > 0 contributes its
 * features to d_x4 and log(cycles) to d_y (device, at most `capacity`, any order); *count
 * receives the number written; est_sum / cycle_sum (may be NULL) the plain schedule's work
 * units and the measured cycles summed over those vertices (their ratio calibrates kappa). */
tc_status tc_costmodel_samples(const tc_graph* g, const uint64_t* d_vcost, const float* d_feat4, uint32_t capacity,
                               void* stream, float* d_x4, float* d_y, uint32_t* count, double* est_sum,
                               double* cycle_sum);
/* Mean squared error on log(cycles) and its gradient w.r.t. the parameters (host outputs,
 * either may be NULL), computed with the FP16 weights and FP32 accumulation. */
tc_status tc_costmodel_grad(tc_costmodel* c, const float* d_x4, const float* d_y, uint32_t count, void* stream,
                            float* host_grad, float* host_loss);
/* `steps` full-batch Adam steps (learning rate lr); *final_loss (may be NULL) after training. */
tc_status tc_costmodel_train(tc_costmodel* c, const float* d_x4, const float* d_y, uint32_t count, uint32_t steps,
                             float lr, void* stream, float* final_loss);
/* Predicted cycles for count feature rows into d_out (device). */
tc_status tc_costmodel_predict(const tc_costmodel* c, const float* d_x4, uint32_t count, void* stream, float* d_out);
/* Compute the graph's features, predict each vertex's cost (cycles x kappa) and keep it for
 * plans made with schedule TC_SCHED_LEARNED.  Synchronises `stream`. */
tc_status tc_graph_attach_costmodel(tc_graph* g, const tc_costmodel* c, void* stream);

/* ------------------------------------------------------------------ serving
 * A census server keeps graphs resident on the GPU and answers census requests on them (the
 * paper's monitoring use runs the census repeatedly at fixed intervals, Sec. 3) with
 * continuous batching: an engine thread runs each request as slices of its work items
 * (Fig. 5 step 2 pairs), up to 32 slices of different requests per launch ("wave") of the
 * census kernel, each wave sized to a target device time (at least the time of its heaviest
 * item).  In the TC_ALGO_TRIANGLE form a wave is the bulk pair sums and the triangle walk over
 * the wave's slices, which add to each request's raw sums and tricode histogram, and, for
 * the requests the wave finishes, one block each that folds those into the 16 counts.  New requests join the next wave; shortest remaining work goes first, and the oldest
 * request, once older than starve_ms, gets up to half of each wave.  With two or more lanes,
 * lane 0 runs the requests larger than half a quantum's work in waves that leave one CTA slot
 * per SM free, and the other lanes (high-priority streams) run the small ones in that slot.
 * Counts are exactly those of tc_census.
 *
 * Thread safety: submit, poll, drain and stats may be called from any thread; add/remove
 * from any thread.  A registered graph must not be destroyed before tc_server_remove_graph,
 * and the census options of the server apply to every graph (a TC_SCHED_LEARNED server needs
 * a cost model attached to each graph before it is added). */
typedef struct tc_server tc_server;

typedef struct {
    tc_options census;        /* kernel options shared by every resident graph */
    uint64_t budget_bytes;    /* cap on resident graph bytes (0 = 90% of device memory) */
    uint32_t max_active;      /* requests in execution at once, one output slot each (0 = 1024) */
    uint32_t max_pending;     /* queued requests beyond which submit returns TC_ERR_BUSY (0 = 65536) */
    uint32_t quantum_us;      /* target device time of one wave (0 = 1000) */
    uint32_t lanes;           /* CUDA streams waves are issued on, 1..4 (0 = 3): one bulk lane, the rest express */
    uint32_t starve_ms;       /* age after which a request is served before all younger ones (0 = 50) */
    uint32_t max_item_units;  /* work items above max(this, 4 deg(u)) cost units are split for serving (0 = 2^20) */
    uint32_t reserved[8];
} tc_server_options;

typedef struct {
    uint64_t id;              /* the id tc_server_submit returned */
    uint32_t graph;           /* the graph id of the request */
    int32_t status;           /* tc_status of the request (TC_OK, or TC_ERR_CUDA if its wave failed) */
    uint64_t counts[16];      /* census in the order above; counts[0] = 003 mod 2^64 */
    tc_u128 c003;             /* the null count in full */
    uint64_t submit_ns;       /* tc_server_now_ns() clock: submitted, */
    uint64_t start_ns;        /*   first slice launched, */
    uint64_t done_ns;         /*   result seen complete by the engine */
    uint32_t waves;           /* waves the request took part in */
    uint32_t lane;            /* stream index it ran on */
} tc_serve_result;

typedef struct {
    uint64_t submitted, completed, refused;   /* refused: graphs turned away by admission */
    uint64_t waves, slices;
    uint64_t resident_bytes, budget_bytes;
    uint32_t graphs, active, pending, inflight_waves;
    double gpu_ms;            /* summed device time of the waves (CUDA events) */
    double ns_per_unit;       /* calibrated device ns per element unit of the slice cost model */
    int32_t error;            /* first engine error (tc_status), 0 if none */
    uint32_t reserved[7];
} tc_server_info;

/* Monotonic clock (ns) of the result timestamps. */
uint64_t tc_server_now_ns(void);
/* Start a server on the current device (opt may be NULL).  Starts the engine thread. */
tc_status tc_server_create(const tc_server_options* opt, tc_server** out);
/* Register a built graph: makes its work plan under the server's options, copies the plan and
 * computes each work item's cost on `stream` (synchronised).  Admission: TC_ERR_OOM, with
 * nothing registered, if the server's resident bytes (CSR, relabelling and plan copy of every
 * registered graph) would exceed budget_bytes.  *graph_id receives the id requests name. */
tc_status tc_server_add_graph(tc_server* s, tc_graph* g, void* stream, uint32_t* graph_id);
/* Unregister a graph (TC_ERR_BUSY while requests for it are queued or running). */
tc_status tc_server_remove_graph(tc_server* s, uint32_t graph_id);
/* Queue a census of graph graph_id; *request_id (may be NULL) receives its id.  TC_ERR_ARG for
 * an unknown graph, TC_ERR_BUSY when max_pending requests are queued.  Never blocks on the GPU. */
tc_status tc_server_submit(tc_server* s, uint32_t graph_id, uint64_t* request_id);
/* Up to `max` finished results, waiting at most timeout_ms for the first; *count = number
 * written (0 on timeout).  Each result is returned once. */
tc_status tc_server_poll(tc_server* s, tc_serve_result* out, uint32_t max, uint32_t timeout_ms, uint32_t* count);
/* Wait, at most timeout_ms, until every submitted request has finished (TC_ERR_TIMEOUT if
 * not); returns the first engine error if one occurred.  Results stay queued for poll. */
tc_status tc_server_drain(tc_server* s, uint32_t timeout_ms);
tc_status tc_server_stats(tc_server* s, tc_server_info* info);
/* One wave of the engine, for tracing: launch and completion time (tc_server_now_ns clock),
 * device time (CUDA events), the slice cost model's units in it and the budget it was sized
 * to, and its counts of slices, finished requests, CTA items and 32-vertex warp-tier blocks. */
typedef struct {
    uint64_t launch_ns, done_ns;
    uint64_t units, budget;
    float gpu_ms;
    uint32_t lane, slices, finished, items, blocks;
} tc_wave_record;
/* The last min(max, 8192) waves, oldest first; *count = number written. */
tc_status tc_server_trace(tc_server* s, tc_wave_record* out, uint32_t max, uint32_t* count);
/* Total cost units (element units) of a registered graph's census and its work counts. */
tc_status tc_server_graph_units(tc_server* s, uint32_t graph_id, uint64_t* units, uint32_t* n_items,
                                uint32_t* n_blocks);
/* Stop the engine: queued requests that have not started are dropped, started ones finish;
 * then free the server (registered graphs are not destroyed). */
void tc_server_destroy(tc_server* s);

/* ------------------------------------------------------------------ interval census
 * The census of a network observed as a stream of timestamped arcs, taken at chosen times over
 * a sliding window (the paper's monitoring application, Sec. 3: the census at fixed intervals).
 * The census at time t covers the arcs with t - window < time <= t, as a set (self-loops and
 * repeated arcs dropped) on the n vertices; it is exactly tc_census of those arcs.  The arcs of
 * the window stay on the device, and so does the window's arc set between censuses (its
 * distinct arcs, sorted, with their multiplicities): a census updates the set with the arcs
 * that entered and left the window since the last one (a sort of those only and a merge), then
 * builds the window's graph from the set and counts it.  Not thread-safe: one caller at a time
 * per stream. */
typedef struct tc_stream tc_stream;
/* window > 0 in the caller's time unit; opt (may be NULL) as for tc_graph_create_arcs and
 * tc_census; `stream` is the CUDA stream every copy, build and census of this object uses. */
tc_status tc_stream_create(uint32_t n, uint64_t window, const tc_options* opt, void* stream, tc_stream** out);
/* Append m arcs src[i] -> dst[i] at times t[i] (host arrays, copied before return).  Times must
 * not decrease, within the call and across calls (TC_ERR_ARG); ids >= n give TC_ERR_RANGE;
 * on error nothing is appended. */
tc_status tc_stream_push(tc_stream* s, uint64_t m, const uint32_t* src, const uint32_t* dst, const uint64_t* t);
/* Census of the window ending at t_now (Fig. 5, out as for tc_census); *arcs_in_window (may be
 * NULL) receives the number of arcs pushed into the window, before loops and repeats are
 * dropped.  t_now must not decrease across calls (TC_ERR_ARG): arcs older than the window are
 * freed once the window's arc set is updated, even if the build or the count then fails.
 * Synchronises the stream. */
tc_status tc_stream_census(tc_stream* s, uint64_t t_now, tc_u128 out[16], uint64_t* arcs_in_window);
typedef struct {
    uint64_t live_arcs;      /* arcs held: pushed and not older than the last census's window */
    uint64_t capacity;       /* device capacity in arcs */
    uint64_t censuses;       /* censuses taken */
    uint64_t distinct_arcs;  /* distinct arcs (loops excluded) in the last census's window */
    uint64_t rebuilds;       /* censuses that made the arc set from the whole window (the first,
                                and any whose change was as large as the window) */
    uint64_t repairs;        /* updates that found the set disagreeing with the window and made
                                it afresh (0 unless something is wrong) */
    uint64_t last_added;     /* arcs keyed as entering by the last census */
    uint64_t last_evicted;   /* arcs keyed as leaving by the last census */
} tc_stream_info;
tc_status tc_stream_stats(const tc_stream* s, tc_stream_info* info);
void tc_stream_destroy(tc_stream* s);

/* The 64-entry tricode -> class table the kernels use (for inspection and tests). */
void tc_tricode_table(uint8_t out[64]);

#ifdef __cplusplus
}
#endif
#endif /* TC_H */
