// server.cu - census serving: resident graphs, a request queue and continuous batching of
// the Fig. 5 census into short "wave" launches of the persistent kernel.
//
// The census of one graph is a sum over its work items (CTA items of the hub tier and
// 32-vertex blocks of the one-warp-per-vertex tier), so it can be cut anywhere between items.
// The engine thread therefore runs every request as a sequence of slices: each wave is one
// launch of the census kernel over up to kMaxWave slices of different requests, sized to a
// target device time (the "quantum") with a cost model in element units that is calibrated
// online from the waves' own CUDA-event durations.  Requests join at the next wave after they
// arrive and leave when their last slice retires, so a small census never waits for a large
// one to finish, and the device always has a full wave queued.  Slices are chosen shortest
// remaining work first, with requests older than starve_ms served first.
//
// Lanes: each request is pinned to one CUDA stream ("lane") at its first slice, and every
// slice of it runs there, so its 16 counters (one slot of a device array, added to by each
// slice) are complete, in stream order, when the wave holding its last slice has run.  That
// wave ends with a small kernel that copies the finished slots to mapped host memory and
// zeroes them for reuse.  With two or more lanes, lane 0 is the bulk lane: requests larger
// than half of the quantum's work run there, in waves of one CTA fewer per SM than the census
// grid; the other lanes are express lanes on high-priority streams for the small requests,
// which thus start in the CTA slot the bulk waves leave free instead of waiting for a long
// bulk wave (whose duration is bounded below by its longest hub item) to end.
//
// Memory admission: tc_server_add_graph admits a graph only while the resident bytes (CSR,
// relabelling, the server's copy of the work plan) stay within the budget; refused graphs get
// TC_ERR_OOM and the server keeps serving the others.  The paper runs the census at fixed
// intervals for monitoring (Sec. 3); this layer serves such repeated requests.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "graph.cuh"

namespace tc {
namespace {

uint64_t steady_ns() {
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch()).count();
}

constexpr uint64_t kPairUnits = 16;   // per-pair overhead in element units (offsets, the pair fold)

// N[v] entries the census walks for the upper pair (u, v = N[u][j]): those past u when the
// graph has per-pair tables, else all of N[v]; the triangle form walks those below u.
__device__ __forceinline__ uint64_t walked(const GraphDev& g, uint32_t u, uint32_t j, uint32_t v, int algo) {
    if (algo == TC_ALGO_TRIANGLE) return g.rp[g.ub[u] + (j - g.up[u])];
    const uint64_t dv = g.off[v + 1] - g.off[v];
    return g.rp ? dv - 1 - g.rp[g.ub[u] + (j - g.up[u])] : dv;
}

// Cost of CTA item i in element units: staging N[u] once, then N[v] plus a fixed overhead per
// pair and per pair and chunk of N[u] (the pair's cursor), and the union walk's u side, which
// visits about half of N[u] per pair.  One warp per item.
__global__ void k_item_cost(GraphDev g, const Item* __restrict__ items, uint32_t n_items, int algo, uint32_t chunk,
                            unsigned long long* cost) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t i = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; i < n_items; i += warps) {
        const Item it = items[i];
        const uint64_t ub = g.off[it.u];
        const uint64_t du = g.off[it.u + 1] - ub;
        unsigned long long c = 0;
        for (uint32_t j = it.j0 + lane; j < it.j1; j += 32) {
            const uint32_t v = g.adj[ub + j] >> 2;
            c += walked(g, it.u, j, v, algo) + kPairUnits + (algo == TC_ALGO_UNION ? du / 2 : 0);
        }
        c = __reduce_add_sync(0xffffffffu, (unsigned)(c & 0xffffffffu)) +
            ((unsigned long long)__reduce_add_sync(0xffffffffu, (unsigned)(c >> 32)) << 32);
        const uint64_t chunks = (du + chunk - 1) / chunk;
        if (lane == 0) cost[i] = c + du + (uint64_t)(it.j1 - it.j0) * chunks * kPairUnits;
    }
}

// Cost of each 32-vertex block [w0 + 32 b, w0 + 32 b + 32) of the warp tier: per vertex, its
// list plus N[v] and the pair overhead for each upper neighbour v.
__global__ void k_block_cost(GraphDev g, uint32_t w0, uint32_t w1, uint32_t n_blocks, int algo,
                             unsigned long long* cost) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t b = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; b < n_blocks; b += warps) {
        const uint64_t u = w0 + 32 * b + lane;
        unsigned long long c = 0;
        if (u < w1) {
            const uint64_t ub = g.off[u], du = g.off[u + 1] - ub;
            c = du;
            for (uint64_t j = ub + g.up[u]; j < ub + du; ++j) {
                const uint32_t v = g.adj[j] >> 2;
                c += walked(g, (uint32_t)u, (uint32_t)(j - ub), v, algo) + kPairUnits +
                     (algo == TC_ALGO_UNION ? du / 2 : 0);
            }
        }
        c = __reduce_add_sync(0xffffffffu, (unsigned)(c & 0xffffffffu)) +
            ((unsigned long long)__reduce_add_sync(0xffffffffu, (unsigned)(c >> 32)) << 32);
        if (lane == 0) cost[b] = c;
    }
}

// Cost of every pair of the listed items (pair p of the concatenation: item it[q] with
// pre[q] <= p < pre[q+1]), in the units of k_item_cost without the item's staging term.
__global__ void k_pair_cost(GraphDev g, const Item* __restrict__ items, const uint32_t* __restrict__ it,
                            const uint64_t* __restrict__ pre, uint32_t nq, uint64_t total, int algo, uint32_t chunk,
                            unsigned long long* cost) {
    for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < total; p += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t lo = 0, hi = nq;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (pre[mid] <= p) lo = mid; else hi = mid;
        }
        const Item w = items[it[lo]];
        const uint32_t j = w.j0 + (uint32_t)(p - pre[lo]);
        const uint64_t ub = g.off[w.u], du = g.off[w.u + 1] - ub;
        const uint32_t v = g.adj[ub + j] >> 2;
        cost[p] = walked(g, w.u, j, v, algo) + kPairUnits + ((du + chunk - 1) / chunk) * kPairUnits +
                  (algo == TC_ALGO_UNION ? du / 2 : 0);
    }
}

// Copy the finished requests' counters to host memory and zero their slots for reuse.
struct CollectArgs {
    unsigned long long* src[kMaxWave];
    unsigned long long* dst;   // mapped host memory, 16 per finished request
    uint32_t n;
};

__global__ void k_collect(CollectArgs a) {
    const uint32_t r = threadIdx.x >> 4, c = threadIdx.x & 15;
    if (r < a.n) {
        a.dst[16 * r + c] = a.src[r][c];
        a.src[r][c] = 0;
    }
}

unsigned __int128 choose3(uint64_t n) {
    if (n < 3) return 0;
    unsigned __int128 a = n, b = n - 1, c = n - 2;
    return a * b * c / 6;
}

struct SGraph {
    uint32_t id = 0;
    uint32_t n = 0;
    uint64_t arcs = 0;
    GraphDev gd{};
    DevBuf items;                        // the server's copy of the plan's CTA items
    uint32_t n_items = 0, warp_begin = 0, warp_end = 0, n_blocks = 0;
    std::vector<uint64_t> item_pre, block_pre;   // cost prefix sums, n_items + 1 / n_blocks + 1
    uint64_t bytes = 0;
    uint32_t refs = 0;                   // requests of this graph in the server (under mu)
    uint64_t units() const { return item_pre.back() + block_pre.back(); }
};

struct Req {
    uint64_t id = 0;
    SGraph* G = nullptr;
    uint64_t t_submit = 0, t_start = 0;
    uint32_t ic = 0, bc = 0;             // next item / warp-tier block to launch
    uint32_t slot = 0;
    int lane = -1;
    uint32_t waves = 0, inflight = 0;
    uint64_t left = 0;                   // units not yet launched
    tc_status status = TC_OK;
};

struct Wave {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    WaveReq* h_desc = nullptr;           // pinned: kMaxWave descriptors + 4 zero counters
    unsigned char* d_desc = nullptr;     // device copy
    unsigned long long* h_res = nullptr; // mapped pinned [kMaxWave][16]
    unsigned long long* d_res = nullptr; // its device address
    std::vector<Req*> slices, finishing;
    uint64_t units = 0, budget = 0, launch_ns = 0;
    uint32_t items = 0, blocks = 0, work = 0;
    bool used = false;
};

constexpr uint32_t kTrace = 8192;        // wave records kept for tc_server_trace

constexpr size_t kDescBytes = sizeof(WaveReq) * kMaxWave + 16;
constexpr int kDepth = 2;                // waves in flight per lane
constexpr int kMaxLanes = 4;

struct Lane {
    cudaStream_t st = nullptr;
    Wave waves[kDepth];
    std::deque<Wave*> inflight;          // in launch order
};

}  // namespace
}  // namespace tc

struct tc_server {
    tc::Opts opts;
    uint64_t budget = 0, resident = 0;
    uint32_t max_active = 1024, max_pending = 65536, lanes_n = 2;
    uint64_t quantum_ns = 1000000, starve_ns = 50000000;
    uint64_t max_item_units = 1u << 20;
    int device = 0;
    unsigned grid = 0;          // census grid (every CTA slot)
    unsigned grid_bulk = 0;     // bulk-lane waves when express lanes exist

    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::unordered_map<uint32_t, std::unique_ptr<tc::SGraph>> graphs;
    uint32_t next_graph = 0;
    std::deque<std::unique_ptr<tc::Req>> pending;
    std::deque<tc_serve_result> done;
    uint64_t next_req = 1;
    bool stop = false;
    uint64_t n_submitted = 0, n_completed = 0, n_refused = 0, n_waves = 0, n_slices = 0;
    uint32_t n_active_shared = 0, n_inflight_shared = 0;   // engine state mirrored under mu
    double gpu_ms = 0.0;
    double ns_per_unit = 0.004;
    tc_status err = TC_OK;
    std::string err_msg;
    std::vector<tc_wave_record> trace;   // ring of the last kTrace waves (under mu)
    uint64_t trace_next = 0;

    // engine-owned
    std::vector<std::unique_ptr<tc::Req>> active;
    std::vector<uint32_t> free_slots;
    tc::DevBuf slots;                    // [max_active][slot_stride] uint64
    uint32_t slot_stride = 16;           // 16 counters, or the triangle form's 96-uint64 scratch
    tc::Lane lanes[tc::kMaxLanes];
    std::thread engine;
};

namespace tc {
namespace {

void record_error(tc_server* s, tc_status st, const std::string& msg) {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->err == TC_OK) {
        s->err = st;
        s->err_msg = msg;
    }
}

// The last slice boundary e in [b, n] with pre[e] - pre[b] <= budget; when even one unit
// does not fit, b + 1 if `must` (the first slice of a wave always makes progress), else b.
uint32_t slice_end(const std::vector<uint64_t>& pre, uint32_t b, uint32_t n, uint64_t budget, bool must) {
    if (b >= n) return n;
    const uint64_t lim = pre[b] + budget;
    auto it = std::upper_bound(pre.begin() + b + 1, pre.begin() + n + 1, lim);
    const uint32_t e = (uint32_t)(it - pre.begin()) - 1;
    return e > b ? e : (must ? b + 1 : b);
}

void finish(tc_server* s, Req* r, const unsigned long long* c16, uint64_t t_done, int lane) {
    tc_serve_result res;
    std::memset(&res, 0, sizeof(res));
    res.id = r->id;
    res.graph = r->G->id;
    res.status = (int32_t)r->status;
    unsigned __int128 sum = 0;
    if (c16) {
        for (int t = 1; t < 16; ++t) {
            res.counts[t] = c16[t];
            sum += c16[t];
        }
        const unsigned __int128 z = choose3(r->G->n) - sum;
        res.c003.lo = (uint64_t)z;
        res.c003.hi = (uint64_t)(z >> 64);
        res.counts[0] = (uint64_t)z;
    }
    res.submit_ns = r->t_submit;
    res.start_ns = r->t_start;
    res.done_ns = t_done;
    res.waves = r->waves;
    res.lane = (uint32_t)(lane < 0 ? 0 : lane);
    std::lock_guard<std::mutex> lk(s->mu);
    s->done.push_back(res);
    s->n_completed++;
    r->G->refs--;
}

// Retire the completed waves at the head of each lane; returns whether any retired.
bool retire(tc_server* s) {
    bool any = false;
    for (uint32_t L = 0; L < s->lanes_n; ++L) {
        Lane& ln = s->lanes[L];
        while (!ln.inflight.empty()) {
            Wave* w = ln.inflight.front();
            const cudaError_t q = cudaEventQuery(w->e1);
            if (q == cudaErrorNotReady) break;
            const uint64_t t_done = steady_ns();
            if (q != cudaSuccess) {
                record_error(s, TC_ERR_CUDA, std::string("wave completion: ") + cudaGetErrorString(q));
                for (Req* r : w->slices) r->status = TC_ERR_CUDA;
            } else {
                float ms = 0.f;
                if (cudaEventElapsedTime(&ms, w->e0, w->e1) == cudaSuccess) {
                    std::lock_guard<std::mutex> lk(s->mu);
                    s->gpu_ms += ms;
                    // calibrate element units -> device time only on waves that fill the GPU
                    // (a wave's time is bounded below by its longest item, so sparse waves
                    // would overstate the cost per unit), with each step limited to 2x
                    const double budget = (double)s->quantum_ns / s->ns_per_unit;
                    const bool calib = s->lanes_n < 2 || L == 0;
                    if (calib && w->work >= (s->lanes_n < 2 ? s->grid : s->grid_bulk) &&
                        (double)w->units > 0.25 * budget) {
                        const double r = std::min(2.0 * s->ns_per_unit,
                                                  std::max(0.5 * s->ns_per_unit, (double)ms * 1e6 / (double)w->units));
                        s->ns_per_unit = 0.75 * s->ns_per_unit + 0.25 * r;
                    }
                    tc_wave_record rec;
                    std::memset(&rec, 0, sizeof(rec));
                    rec.launch_ns = w->launch_ns;
                    rec.done_ns = t_done;
                    rec.units = w->units;
                    rec.budget = w->budget;
                    rec.gpu_ms = ms;
                    rec.lane = L;
                    rec.slices = (uint32_t)w->slices.size();
                    rec.finished = (uint32_t)w->finishing.size();
                    rec.items = w->items;
                    rec.blocks = w->blocks;
                    if (s->trace.size() < kTrace) s->trace.push_back(rec);
                    else s->trace[s->trace_next % kTrace] = rec;
                    s->trace_next++;
                }
            }
            for (Req* r : w->slices) r->inflight--;
            bool fin = false;
            for (size_t k = 0; k < w->finishing.size(); ++k) {
                Req* r = w->finishing[k];
                finish(s, r, r->status == TC_OK ? w->h_res + 16 * k : nullptr, t_done, r->lane);
                s->free_slots.push_back(r->slot);
                fin = true;
            }
            // requests of a failed wave with slices still unlaunched end here, with their
            // partial counters cleared before the slot is reused
            for (Req* r : w->slices) {
                if (r->status != TC_OK && r->left > 0 && r->inflight == 0) {
                    r->left = 0;
                    cudaMemsetAsync(s->slots.as<unsigned long long>() + (uint64_t)s->slot_stride * r->slot, 0, 8ull * s->slot_stride, ln.st);
                    finish(s, r, nullptr, t_done, r->lane);
                    s->free_slots.push_back(r->slot);
                    fin = true;
                }
            }
            if (fin) {
                auto& A = s->active;
                A.erase(std::remove_if(A.begin(), A.end(),
                                       [](const std::unique_ptr<Req>& r) {
                                           return r->inflight == 0 && r->left == 0;
                                       }),
                        A.end());
                s->cv_done.notify_all();
            }
            w->slices.clear();
            w->finishing.clear();
            w->used = false;
            ln.inflight.pop_front();
            any = true;
        }
    }
    return any;
}

// Move queued requests into execution while output slots are free.  A request with no work
// (no connected pairs: every triad is null) finishes here.
void admit(tc_server* s) {
    std::vector<std::unique_ptr<Req>> empty;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        while (!s->pending.empty() && !s->free_slots.empty()) {
            std::unique_ptr<Req> r = std::move(s->pending.front());
            s->pending.pop_front();
            r->left = r->G->units();
            if (r->left == 0) {
                empty.push_back(std::move(r));
                continue;
            }
            r->slot = s->free_slots.back();
            s->free_slots.pop_back();
            s->active.push_back(std::move(r));
        }
    }
    if (empty.empty()) return;
    const unsigned long long zero[16] = {0};
    const uint64_t t = steady_ns();
    for (auto& r : empty) {
        r->t_start = t;
        finish(s, r.get(), zero, t, -1);
    }
    s->cv_done.notify_all();
}

// Whether lane L may take request r: its own lane, or, for a request not yet started, the
// bulk lane (0) for large requests and an express lane for small ones (one lane takes all).
bool eligible(const tc_server* s, const Req* r, int L, uint64_t express_units) {
    if (r->left == 0 || r->status != TC_OK) return false;
    if (r->lane >= 0) return r->lane == L;
    if (s->lanes_n < 2) return true;
    return (L == 0) == (r->left > express_units);
}

uint64_t express_units(tc_server* s) {
    std::lock_guard<std::mutex> lk(s->mu);
    return (uint64_t)((double)s->quantum_ns / s->ns_per_unit / 2.0);
}

bool has_work(const tc_server* s, int L, uint64_t xu) {
    for (const auto& r : s->active)
        if (eligible(s, r.get(), L, xu)) return true;
    return false;
}

// Build and launch one wave on lane L from the requests it may take.
void launch_wave(tc_server* s, int L) {
    Lane& ln = s->lanes[L];
    Wave* w = nullptr;
    for (auto& x : ln.waves)
        if (!x.used) { w = &x; break; }
    if (!w) return;
    const uint64_t now = steady_ns();
    const uint64_t xu = express_units(s);
    const bool split = s->lanes_n >= 2, bulk = !split || L == 0;
    const unsigned lane_grid = split && L == 0 ? s->grid_bulk : s->grid;
    std::vector<Req*> cand;
    for (auto& r : s->active)
        if (eligible(s, r.get(), L, xu)) cand.push_back(r.get());
    // shortest remaining work first; the oldest request, once older than starve_ns, goes
    // first with at most half of the wave's budget, so it progresses without holding the lane
    std::sort(cand.begin(), cand.end(), [](const Req* a, const Req* b) {
        if (a->left != b->left) return a->left < b->left;
        return a->id < b->id;
    });
    Req* starved = nullptr;
    for (Req* r : cand)
        if (now - r->t_submit > s->starve_ns && (!starved || r->t_submit < starved->t_submit)) starved = r;
    if (starved) {
        cand.erase(std::find(cand.begin(), cand.end(), starved));
        cand.insert(cand.begin(), starved);
    }
    double nspu;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        nspu = s->ns_per_unit;
    }
    const uint64_t budget0 = (uint64_t)std::max(1.0, (double)s->quantum_ns / nspu);
    // A wave lasts at least as long as its heaviest item (one CTA runs it), so once a wave
    // holds an item of h units it may hold h x grid units at no cost in time: the effective
    // budget is max(quantum budget, h x grid), and heavy-item requests fill the GPU by
    // themselves while the rest of that time goes to other requests.  Items are in plan order
    // (heaviest vertices first), so a slice's first item is its heaviest.
    uint64_t heavy = 0, units = 0;
    auto eff_budget = [&]() { return std::max<uint64_t>(budget0, heavy * lane_grid); };
    uint32_t n = 0, tot_items = 0, tot_blocks = 0, work = 0;
    const size_t zero_ctr_off = sizeof(WaveReq) * kMaxWave;
    for (Req* r : cand) {
        if (n == kMaxWave) break;
        if (n > 0 && units >= eff_budget()) break;
        SGraph& G = *r->G;
        const uint32_t i0 = r->ic, b0 = r->bc;
        uint32_t i1 = i0, b1 = b0;
        uint64_t took = 0;
        if (i0 < G.n_items && bulk) heavy = std::max<uint64_t>(heavy, G.item_pre[i0 + 1] - G.item_pre[i0]);
        const uint64_t left_b = eff_budget() > units ? eff_budget() - units : 0;
        const uint64_t cap = (r == starved && cand.size() > 1) ? std::max<uint64_t>(left_b / 2, 1) : left_b;
        if (i0 < G.n_items) {
            i1 = slice_end(G.item_pre, i0, G.n_items, cap, n == 0);
            took = G.item_pre[i1] - G.item_pre[i0];
        }
        if (i1 == G.n_items && b0 < G.n_blocks) {
            b1 = slice_end(G.block_pre, b0, G.n_blocks, took < cap ? cap - took : 0, n == 0 && i1 == i0);
            took += G.block_pre[b1] - G.block_pre[b0];
        }
        if (i1 == i0 && b1 == b0) continue;   // its next unit does not fit; try the others
        WaveReq& d = w->h_desc[n];
        d.g = G.gd;
        d.items = G.items.as<Item>() + i0;
        d.out = s->slots.as<unsigned long long>() + (uint64_t)s->slot_stride * r->slot;
        d.n_items = i1 - i0;
        d.item_pre = tot_items;
        d.warp_begin = G.warp_begin + 32u * b0;
        d.warp_end = std::min(G.warp_begin + 32u * b1, G.warp_end);
        if (b1 == b0) d.warp_end = d.warp_begin;
        d.block_pre = 0;
        d.pad = 0;
        tot_items += i1 - i0;
        tot_blocks += b1 - b0;
        work += (i1 - i0) + 4 * (b1 - b0);
        units += took;
        r->ic = i1;
        r->bc = b1;
        r->left = (r->left > took) ? r->left - took : 0;
        if (r->ic == G.n_items && r->bc == G.n_blocks) r->left = 0;
        if (r->lane < 0) {
            r->lane = L;
            r->t_start = now;
        }
        r->waves++;
        r->inflight++;
        w->slices.push_back(r);
        if (r->left == 0) w->finishing.push_back(r);
        ++n;
    }
    if (n == 0) return;
    // warp-tier blocks: the cost model slices in 32-vertex blocks; the kernel takes smaller
    // ones when the wave has few warp-tier vertices, so no warp walks 32 vertices alone
    uint64_t wverts = 0;
    for (uint32_t k = 0; k < n; ++k) wverts += w->h_desc[k].warp_end - w->h_desc[k].warp_begin;
    const uint32_t ws = warp_block_shift(wverts, lane_grid);
    tot_blocks = 0;
    for (uint32_t k = 0; k < n; ++k) {
        WaveReq& d = w->h_desc[k];
        d.pad = ws;
        d.block_pre = tot_blocks;
        tot_blocks += (d.warp_end - d.warp_begin + (1u << ws) - 1) >> ws;
    }
    std::memset(reinterpret_cast<unsigned char*>(w->h_desc) + zero_ctr_off, 0, 16);
    w->units = units;
    w->budget = eff_budget();
    w->items = tot_items;
    w->blocks = tot_blocks;
    w->work = work;
    w->launch_ns = now;
    w->used = true;
    cudaStream_t st = ln.st;
    unsigned grid = std::min<unsigned>(lane_grid, std::max<unsigned>(1u, tot_items + (tot_blocks + 7) / 8));
    cudaError_t e = cudaMemcpyAsync(w->d_desc, w->h_desc, kDescBytes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaEventRecord(w->e0, st);
    tc_status ks = TC_OK;
    const bool tri = s->opts.algo == TC_ALGO_TRIANGLE;
    if (e == cudaSuccess)
        ks = tri ? triangle_census_wave(reinterpret_cast<const WaveReq*>(w->d_desc), n, tot_items, tot_blocks, s->opts,
                                        grid, reinterpret_cast<uint32_t*>(w->d_desc + zero_ctr_off), st)
                 : census_launch_wave(reinterpret_cast<const WaveReq*>(w->d_desc), n, tot_items, tot_blocks, s->opts,
                                      grid, reinterpret_cast<uint32_t*>(w->d_desc + zero_ctr_off), st);
    if (e == cudaSuccess && ks == TC_OK && !w->finishing.empty()) {
        unsigned long long* src[kMaxWave];
        for (size_t k = 0; k < w->finishing.size(); ++k)
            src[k] = s->slots.as<unsigned long long>() + (uint64_t)s->slot_stride * w->finishing[k]->slot;
        if (tri) {
            ks = triangle_collect(src, (uint32_t)w->finishing.size(), w->d_res, st);
        } else {
            CollectArgs a;
            std::memset(&a, 0, sizeof(a));
            for (size_t k = 0; k < w->finishing.size(); ++k) a.src[k] = src[k];
            a.dst = w->d_res;
            a.n = (uint32_t)w->finishing.size();
            k_collect<<<1, 16 * kMaxWave, 0, st>>>(a);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess && ks == TC_OK) e = cudaEventRecord(w->e1, st);
    if (e != cudaSuccess || ks != TC_OK) {
        record_error(s, ks != TC_OK ? ks : TC_ERR_CUDA,
                     e != cudaSuccess ? std::string("wave launch: ") + cudaGetErrorString(e) : std::string("wave launch failed"));
        // nothing of this wave is known to run: fail its requests now, or, for those with
        // earlier slices still in flight, when those retire (left > 0 marks them for retire())
        for (Req* r : w->slices) {
            r->status = TC_ERR_CUDA;
            r->inflight--;
            r->left = r->inflight ? std::max<uint64_t>(r->left, 1) : 0;
        }
        const uint64_t t = steady_ns();
        for (Req* r : w->slices) {
            if (r->inflight == 0) {
                cudaMemsetAsync(s->slots.as<unsigned long long>() + (uint64_t)s->slot_stride * r->slot, 0, 8ull * s->slot_stride, st);
                finish(s, r, nullptr, t, r->lane);
                s->free_slots.push_back(r->slot);
            }
        }
        auto& A = s->active;
        A.erase(std::remove_if(A.begin(), A.end(),
                               [](const std::unique_ptr<Req>& r) { return r->status != TC_OK && r->inflight == 0; }),
                A.end());
        w->slices.clear();
        w->finishing.clear();
        w->used = false;
        s->cv_done.notify_all();
        return;
    }
    ln.inflight.push_back(w);
    std::lock_guard<std::mutex> lk(s->mu);
    s->n_waves++;
    s->n_slices += n;
}

void engine_main(tc_server* s) {
    cudaSetDevice(s->device);
    for (;;) {
        bool did = retire(s);
        admit(s);
        // lanes with the fewest waves in flight first, so new requests go to the idlest stream
        int order[kMaxLanes];
        for (uint32_t L = 0; L < s->lanes_n; ++L) order[L] = (int)L;
        std::sort(order, order + s->lanes_n,
                  [&](int a, int b) { return s->lanes[a].inflight.size() < s->lanes[b].inflight.size(); });
        const uint64_t xu = express_units(s);
        for (uint32_t k = 0; k < s->lanes_n; ++k) {
            const int L = order[k];
            if (s->lanes[L].inflight.size() < (size_t)kDepth && has_work(s, L, xu)) {
                const uint64_t before = s->n_waves;
                launch_wave(s, L);
                did |= s->n_waves != before;
            }
        }
        size_t inflight = 0;
        for (uint32_t L = 0; L < s->lanes_n; ++L) inflight += s->lanes[L].inflight.size();
        std::unique_lock<std::mutex> lk(s->mu);
        s->n_active_shared = (uint32_t)s->active.size();
        s->n_inflight_shared = (uint32_t)inflight;
        if (s->pending.empty() && s->active.empty() && inflight == 0) {
            s->cv_done.notify_all();
            if (s->stop) break;
            s->cv_work.wait(lk, [&] { return s->stop || !s->pending.empty(); });
            continue;
        }
        if (!did) {
            if (inflight > 0) {
                lk.unlock();
                std::this_thread::yield();   // waves in flight: poll their events
            } else {
                // active requests wait only for slots of lanes that are all busy: not reachable
                // with waves retired, but never spin without a bound
                s->cv_work.wait_for(lk, std::chrono::microseconds(50));
            }
        }
    }
}

}  // namespace
}  // namespace tc

using namespace tc;

extern "C" {

uint64_t tc_server_now_ns(void) { return steady_ns(); }

tc_status tc_server_create(const tc_server_options* opt, tc_server** out) {
    if (!out) return fail(TC_ERR_ARG, "null argument");
    *out = nullptr;
    tc_server_options o;
    std::memset(&o, 0, sizeof(o));
    if (opt) o = *opt;
    if (o.lanes > (uint32_t)kMaxLanes) return fail(TC_ERR_ARG, "lanes must be <= 4");
    std::unique_ptr<tc_server> s(new tc_server());
    TC_TRY(resolve_opts(&o.census, nullptr, &s->opts));
    if (s->opts.schedule != TC_SCHED_PLAIN && s->opts.schedule != TC_SCHED_LEARNED)
        return fail(TC_ERR_ARG, "unknown schedule");
    s->max_active = o.max_active ? o.max_active : 1024;
    s->max_pending = o.max_pending ? o.max_pending : 65536;
    s->lanes_n = o.lanes ? o.lanes : 3;
    s->quantum_ns = (uint64_t)(o.quantum_us ? o.quantum_us : 1000) * 1000ull;
    s->starve_ns = (uint64_t)(o.starve_ms ? o.starve_ms : 50) * 1000000ull;
    s->max_item_units = o.max_item_units ? o.max_item_units : (1u << 20);
    TC_CUDA(cudaGetDevice(&s->device));
    size_t fr = 0, total = 0;
    TC_CUDA(cudaMemGetInfo(&fr, &total));
    s->budget = o.budget_bytes ? o.budget_bytes : (uint64_t)(0.9 * (double)total);
    s->grid = (unsigned)census_grid(s->opts);
    const unsigned sms = (unsigned)sm_count();
    s->grid_bulk = s->opts.ctas_per_sm > 1 ? sms * (s->opts.ctas_per_sm - 1) : sms;
    int prio_lo = 0, prio_hi = 0;
    TC_CUDA(cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi));
    s->slot_stride = s->opts.algo == TC_ALGO_TRIANGLE ? 96u : 16u;
    TC_TRY(s->slots.alloc_persistent(sizeof(unsigned long long) * (uint64_t)s->slot_stride * s->max_active));
    TC_CUDA(cudaMemset(s->slots.p, 0, s->slots.bytes));
    for (uint32_t i = 0; i < s->max_active; ++i) s->free_slots.push_back(s->max_active - 1 - i);
    bool ok = true;
    for (uint32_t L = 0; L < s->lanes_n && ok; ++L) {
        Lane& ln = s->lanes[L];
        ok = cudaStreamCreateWithPriority(&ln.st, cudaStreamNonBlocking, L == 0 ? prio_lo : prio_hi) == cudaSuccess;
        for (auto& w : ln.waves) {
            if (!ok) break;
            ok = cudaEventCreate(&w.e0) == cudaSuccess && cudaEventCreate(&w.e1) == cudaSuccess &&
                 cudaMallocHost((void**)&w.h_desc, kDescBytes) == cudaSuccess &&
                 cudaMalloc((void**)&w.d_desc, kDescBytes) == cudaSuccess &&
                 cudaHostAlloc((void**)&w.h_res, sizeof(unsigned long long) * 16 * kMaxWave, cudaHostAllocMapped) ==
                     cudaSuccess &&
                 cudaHostGetDevicePointer((void**)&w.d_res, w.h_res, 0) == cudaSuccess;
        }
    }
    if (!ok) {
        const cudaError_t e = cudaGetLastError();
        tc_server_destroy(s.release());
        return cuda_fail(e == cudaSuccess ? cudaErrorMemoryAllocation : e, "server streams and wave buffers");
    }
    const tc_status ps = s->opts.algo == TC_ALGO_TRIANGLE ? TC_OK : census_prepare(s->lanes[0].st, s->opts);
    if (ps != TC_OK) {
        const std::string why = tc_last_error();
        tc_server_destroy(s.release());
        return fail(ps, why);
    }
    try {
        s->engine = std::thread(engine_main, s.get());
    } catch (...) {
        tc_server_destroy(s.release());
        return fail(TC_ERR_OOM, "cannot start the server's engine thread");
    }
    *out = s.release();
    return TC_OK;
}

tc_status tc_server_add_graph(tc_server* s, tc_graph* g, void* stream, uint32_t* graph_id) {
    if (!s || !g || !graph_id) return fail(TC_ERR_ARG, "null argument");
    cudaStream_t st = (cudaStream_t)stream;
    std::unique_lock<std::mutex> glk(g->s.busy, std::try_to_lock);
    if (!glk.owns_lock()) return fail(TC_ERR_BUSY, "graph is in use by another call");
    Plan* p = nullptr;
    TC_TRY(get_plan(g->s, s->opts, st, &p));
    std::unique_ptr<SGraph> G(new SGraph());
    G->n = g->s.n;
    G->arcs = g->s.arcs;
    G->gd = g->s.dev();
    G->n_items = p->n_items;
    G->warp_begin = p->warp_begin;
    G->warp_end = p->warp_end;
    G->n_blocks = (p->warp_end - p->warp_begin + 31) / 32;
    const uint64_t item_bytes = sizeof(Item) * (uint64_t)std::max(p->n_items, 1u);
    G->bytes = g->s.off.bytes + g->s.adj.bytes + g->s.up.bytes + g->s.new_of_old.bytes + g->s.ub.bytes +
               g->s.rp.bytes + g->s.vs.bytes + g->s.us.bytes + item_bytes;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->resident + G->bytes > s->budget) {
            s->n_refused++;
            return fail(TC_ERR_OOM, "admission refused: " + std::to_string(G->bytes) + " bytes would exceed the budget (" +
                                        std::to_string(s->resident) + " of " + std::to_string(s->budget) + " resident)");
        }
        s->resident += G->bytes;   // reserved while the graph is prepared
    }
    auto unreserve = [&](tc_status r) {
        std::lock_guard<std::mutex> lk(s->mu);
        s->resident -= G->bytes;
        return r;
    };
    if (G->items.alloc_persistent(item_bytes) != TC_OK) return unreserve(TC_ERR_OOM);
    if (p->n_items && cudaMemcpyAsync(G->items.p, p->items.p, sizeof(Item) * p->n_items, cudaMemcpyDeviceToDevice, st) !=
                          cudaSuccess)
        return unreserve(cuda_fail(cudaGetLastError(), "copy of the work plan"));
    DevBuf ci, cb;
    if (ci.alloc(sizeof(unsigned long long) * std::max(G->n_items, 1u), st) != TC_OK ||
        cb.alloc(sizeof(unsigned long long) * std::max(G->n_blocks, 1u), st) != TC_OK)
        return unreserve(TC_ERR_OOM);
    if (G->n_items)
        k_item_cost<<<grid_for((uint64_t)G->n_items * 32, 256, 8192), 256, 0, st>>>(
            G->gd, G->items.as<Item>(), G->n_items, (int)s->opts.algo, s->opts.chunk, ci.as<unsigned long long>());
    if (G->n_blocks)
        k_block_cost<<<grid_for((uint64_t)G->n_blocks * 32, 256, 8192), 256, 0, st>>>(
            G->gd, G->warp_begin, G->warp_end, G->n_blocks, (int)s->opts.algo, cb.as<unsigned long long>());
    if (cudaGetLastError() != cudaSuccess) return unreserve(fail(TC_ERR_CUDA, "cost kernels failed to launch"));
    std::vector<uint64_t> hi(G->n_items), hb(G->n_blocks);
    if ((G->n_items && cudaMemcpyAsync(hi.data(), ci.p, sizeof(uint64_t) * G->n_items, cudaMemcpyDeviceToHost, st) !=
                           cudaSuccess) ||
        (G->n_blocks && cudaMemcpyAsync(hb.data(), cb.p, sizeof(uint64_t) * G->n_blocks, cudaMemcpyDeviceToHost, st) !=
                            cudaSuccess) ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return unreserve(cuda_fail(cudaGetLastError(), "cost of the work plan"));
    // A wave lasts as long as its heaviest item, and the plan splits a hub's pairs evenly by
    // count, so its first items (the pairs with other hubs) can be far heavier than the rest.
    // Items above max(max_item_units, 4 deg(u)) units are cut into consecutive pair ranges by
    // their pairs' exact costs; every piece stages N[u] again, which the floor of 4 deg(u)
    // keeps to a quarter of a piece at most.
    std::vector<uint32_t> heavy;
    std::vector<Item> hitems;
    if (G->n_items) {
        hitems.resize(G->n_items);
        if (cudaMemcpyAsync(hitems.data(), G->items.p, sizeof(Item) * G->n_items, cudaMemcpyDeviceToHost, st) !=
                cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return unreserve(cuda_fail(cudaGetLastError(), "copy of the work plan"));
    }
    for (uint32_t i = 0; i < G->n_items; ++i)
        if (hitems[i].j1 - hitems[i].j0 > 1 && hi[i] > s->max_item_units) heavy.push_back(i);
    if (!heavy.empty()) {
        std::vector<uint64_t> qpre(heavy.size() + 1, 0);
        for (size_t q = 0; q < heavy.size(); ++q) qpre[q + 1] = qpre[q] + (hitems[heavy[q]].j1 - hitems[heavy[q]].j0);
        const uint64_t total = qpre.back();
        DevBuf d_it, d_pre, d_pc;
        if (d_it.alloc(sizeof(uint32_t) * heavy.size(), st) != TC_OK || d_pre.alloc(sizeof(uint64_t) * qpre.size(), st) != TC_OK ||
            d_pc.alloc(sizeof(unsigned long long) * total, st) != TC_OK)
            return unreserve(TC_ERR_OOM);
        std::vector<uint64_t> pc(total);
        if (cudaMemcpyAsync(d_it.p, heavy.data(), sizeof(uint32_t) * heavy.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(d_pre.p, qpre.data(), sizeof(uint64_t) * qpre.size(), cudaMemcpyHostToDevice, st) != cudaSuccess)
            return unreserve(cuda_fail(cudaGetLastError(), "heavy item list"));
        k_pair_cost<<<grid_for(total, 256, 8192), 256, 0, st>>>(G->gd, G->items.as<Item>(), d_it.as<uint32_t>(),
                                                               d_pre.as<uint64_t>(), (uint32_t)heavy.size(), total,
                                                               (int)s->opts.algo, s->opts.chunk,
                                                               d_pc.as<unsigned long long>());
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(pc.data(), d_pc.p, sizeof(uint64_t) * total, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return unreserve(cuda_fail(cudaGetLastError(), "pair costs of heavy items"));
        std::vector<Item> nitems;
        std::vector<uint64_t> ncost;
        nitems.reserve(G->n_items + total / 4);
        size_t q = 0;
        for (uint32_t i = 0; i < G->n_items; ++i) {
            if (q < heavy.size() && heavy[q] == i) {
                const Item w = hitems[i];
                uint64_t pair_sum = 0;
                for (uint64_t p = qpre[q]; p < qpre[q + 1]; ++p) pair_sum += pc[p];
                const uint64_t stage = hi[i] > pair_sum ? hi[i] - pair_sum : 0;   // deg(u)
                const uint64_t cap = std::max<uint64_t>(s->max_item_units, 4 * stage);
                uint32_t start = w.j0;
                uint64_t acc = stage;
                for (uint32_t j = w.j0; j < w.j1; ++j) {
                    const uint64_t c = pc[qpre[q] + (j - w.j0)];
                    if (j > start && acc + c > cap) {
                        nitems.push_back(Item{w.u, start, j, 0});
                        ncost.push_back(acc);
                        start = j;
                        acc = stage;
                    }
                    acc += c;
                }
                nitems.push_back(Item{w.u, start, w.j1, 0});
                ncost.push_back(acc);
                ++q;
            } else {
                nitems.push_back(hitems[i]);
                ncost.push_back(hi[i]);
            }
        }
        if (nitems.size() != G->n_items) {
            const uint64_t add = sizeof(Item) * (nitems.size() - G->n_items);
            {
                std::lock_guard<std::mutex> lk(s->mu);
                if (s->resident + add > s->budget) {
                    s->n_refused++;
                    s->resident -= G->bytes;
                    return fail(TC_ERR_OOM, "admission refused: the split work plan exceeds the budget");
                }
                s->resident += add;
                G->bytes += add;
            }
            if (G->items.alloc_persistent(sizeof(Item) * nitems.size()) != TC_OK ||
                cudaMemcpyAsync(G->items.p, nitems.data(), sizeof(Item) * nitems.size(), cudaMemcpyHostToDevice, st) !=
                    cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess)
                return unreserve(cuda_fail(cudaGetLastError(), "split work plan"));
            G->n_items = (uint32_t)nitems.size();
            hi.swap(ncost);
        }
    }
    G->item_pre.assign(G->n_items + 1, 0);
    G->block_pre.assign(G->n_blocks + 1, 0);
    for (uint32_t i = 0; i < G->n_items; ++i) G->item_pre[i + 1] = G->item_pre[i] + std::max<uint64_t>(hi[i], 1);
    for (uint32_t b = 0; b < G->n_blocks; ++b) G->block_pre[b + 1] = G->block_pre[b] + std::max<uint64_t>(hb[b], 1);
    std::lock_guard<std::mutex> lk(s->mu);
    G->id = s->next_graph++;
    *graph_id = G->id;
    s->graphs[G->id] = std::move(G);
    return TC_OK;
}

tc_status tc_server_remove_graph(tc_server* s, uint32_t graph_id) {
    if (!s) return fail(TC_ERR_ARG, "null argument");
    std::unique_ptr<SGraph> G;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->graphs.find(graph_id);
        if (it == s->graphs.end()) return fail(TC_ERR_ARG, "unknown graph id");
        if (it->second->refs) return fail(TC_ERR_BUSY, "graph has requests in the server");
        s->resident -= it->second->bytes;
        G = std::move(it->second);
        s->graphs.erase(it);
    }
    return TC_OK;
}

tc_status tc_server_submit(tc_server* s, uint32_t graph_id, uint64_t* request_id) {
    if (!s) return fail(TC_ERR_ARG, "null argument");
    const uint64_t t = steady_ns();
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return fail(TC_ERR_BUSY, "server is stopping");
    auto it = s->graphs.find(graph_id);
    if (it == s->graphs.end()) return fail(TC_ERR_ARG, "unknown graph id");
    if (s->pending.size() >= s->max_pending) return fail(TC_ERR_BUSY, "request queue is full");
    std::unique_ptr<Req> r(new Req());
    r->id = s->next_req++;
    r->G = it->second.get();
    r->t_submit = t;
    r->G->refs++;
    if (request_id) *request_id = r->id;
    s->pending.push_back(std::move(r));
    s->n_submitted++;
    s->cv_work.notify_one();
    return TC_OK;
}

tc_status tc_server_poll(tc_server* s, tc_serve_result* out, uint32_t max, uint32_t timeout_ms, uint32_t* count) {
    if (!s || !count || (max && !out)) return fail(TC_ERR_ARG, "null argument");
    *count = 0;
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->done.empty() && timeout_ms)
        s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return !s->done.empty(); });
    uint32_t k = 0;
    while (k < max && !s->done.empty()) {
        out[k++] = s->done.front();
        s->done.pop_front();
    }
    *count = k;
    return TC_OK;
}

tc_status tc_server_drain(tc_server* s, uint32_t timeout_ms) {
    if (!s) return fail(TC_ERR_ARG, "null argument");
    std::unique_lock<std::mutex> lk(s->mu);
    const bool idle = s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] {
        return s->pending.empty() && s->n_submitted == s->n_completed;
    });
    if (!idle) return fail(TC_ERR_TIMEOUT, "requests still in execution after the drain limit");
    if (s->err != TC_OK) return fail(s->err, s->err_msg);
    return TC_OK;
}

tc_status tc_server_stats(tc_server* s, tc_server_info* info) {
    if (!s || !info) return fail(TC_ERR_ARG, "null argument");
    std::memset(info, 0, sizeof(*info));
    std::lock_guard<std::mutex> lk(s->mu);
    info->submitted = s->n_submitted;
    info->completed = s->n_completed;
    info->refused = s->n_refused;
    info->waves = s->n_waves;
    info->slices = s->n_slices;
    info->resident_bytes = s->resident;
    info->budget_bytes = s->budget;
    info->graphs = (uint32_t)s->graphs.size();
    info->active = s->n_active_shared;
    info->pending = (uint32_t)s->pending.size();
    info->inflight_waves = s->n_inflight_shared;
    info->gpu_ms = s->gpu_ms;
    info->ns_per_unit = s->ns_per_unit;
    info->error = (int32_t)s->err;
    return TC_OK;
}

tc_status tc_server_graph_units(tc_server* s, uint32_t graph_id, uint64_t* units, uint32_t* n_items,
                                uint32_t* n_blocks) {
    if (!s) return fail(TC_ERR_ARG, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->graphs.find(graph_id);
    if (it == s->graphs.end()) return fail(TC_ERR_ARG, "unknown graph id");
    if (units) *units = it->second->units();
    if (n_items) *n_items = it->second->n_items;
    if (n_blocks) *n_blocks = it->second->n_blocks;
    return TC_OK;
}

tc_status tc_server_trace(tc_server* s, tc_wave_record* out, uint32_t max, uint32_t* count) {
    if (!s || !count || (max && !out)) return fail(TC_ERR_ARG, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    const uint64_t have = std::min<uint64_t>(s->trace.size(), max);
    // oldest first among the last `have` records
    for (uint64_t k = 0; k < have; ++k) {
        const uint64_t idx = s->trace_next - have + k;
        out[k] = s->trace[idx % kTrace];
    }
    *count = (uint32_t)have;
    return TC_OK;
}

void tc_server_destroy(tc_server* s) {
    if (!s) return;
    if (s->engine.joinable()) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->stop = true;
            s->pending.clear();   // queued requests that never started are dropped
            s->cv_work.notify_all();
        }
        s->engine.join();         // waves already launched run to completion first
    }
    for (uint32_t L = 0; L < (uint32_t)kMaxLanes; ++L) {
        Lane& ln = s->lanes[L];
        if (ln.st) cudaStreamSynchronize(ln.st);
        for (auto& w : ln.waves) {
            if (w.e0) cudaEventDestroy(w.e0);
            if (w.e1) cudaEventDestroy(w.e1);
            if (w.h_desc) cudaFreeHost(w.h_desc);
            if (w.d_desc) cudaFree(w.d_desc);
            if (w.h_res) cudaFreeHost(w.h_res);
        }
        if (ln.st) cudaStreamDestroy(ln.st);
    }
    delete s;
}

}  // extern "C"
