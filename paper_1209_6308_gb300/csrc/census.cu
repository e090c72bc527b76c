// census.cu - the triad census hot path (Fig. 5, steps 2 - 2.1.4.2) on the GPU.
//
// Vertices are in descending-degree ids, so for every connected pair (u, v) with u < v
// (step 2.1) u is the endpoint of larger degree.  For each pair the kernel accounts for every
// third vertex w of S = N[u] u N[v] \ {u, v} (step 2.1.1, the union of Sec. 6 / Fig. 8) in
// two sweeps that together visit S exactly once:
//   - the v side: each w in N[v] is looked up in N[u] (staged in shared memory as a sorted
//     array plus an open-addressing hash).  A common w counts toward |N[u] n N[v]|; a common
//     w > v is a connected triad with both u-w and v-w links; a w in N[v] only, with w > u,
//     is a connected triad through v alone (the canonical rule of step 2.1.4).
//   - the u side: the w in N[u] past v (the rest of S that the canonical rule keeps: w > v)
//     are classified as triads through u alone; the common ones among them were already
//     counted with both links by the v side, which therefore also removes their u-only count.
//   TC_ALGO_UNION walks the u side one w at a time and looks each class up in the 64-entry
//     tricode table (step 2.1.4.1).
//   TC_ALGO_SUFFIX gets the same u-side counts per direction class from prefix counts of the
//     staged list: for a w reached from u alone the class depends only on dir(u,v) and
//     dir(u,w), so the three counts, each sent through the same table, give the same census.
// The dyadic triads of the pair (steps 2.1.2-2.1.3) add n - |S| - 2 = n - d_u - d_v + |common|
// to 012 or 102.  Counts go to per-thread shared-memory histograms (class-major, one column
// per thread: no bank conflicts), per-warp 64-bit accumulators, and at the end 16 64-bit
// atomics per CTA (the private census vectors of Sec. 6).
//
// Work decomposition ("manhattan collapse" of Sec. 7): vertices with deg > warp_max_deg
// become CTA items (u, chunk of N[u] that fits in shared memory, range of v), sized by the
// schedule; a hub's list is split into chunks and every chunk takes the part of each N[v]
// that falls in its id range.  Vertices with smaller degree are handled one warp per vertex
// after the items run out, in the same persistent launch.
#include <atomic>

#include "graph.cuh"

namespace tc {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr uint32_t kEmpty = 0xffffffffu;
constexpr uint32_t kFlushAfter = 1u << 26;   // list entries per CTA between histogram flushes

__device__ uint8_t d_tricode_class[64];

struct Params {
    GraphDev g;
    const Item* items;
    uint32_t n_items;
    uint32_t warp_begin, warp_end;
    uint32_t chunk;
    uint32_t warp_max;
    uint32_t* ctr;                 // [0] next item, [1] next warp-tier vertex block
    unsigned long long* out;       // 16 accumulators
};

// tricode bits of the u-v link from dir(u,v) (bit 0 u->v, bit 1 v->u): 2 = u->v, 1 = v->u
__device__ __forceinline__ uint32_t code_uv(uint32_t duv) { return ((duv & 1u) << 1) | (duv >> 1); }
__device__ __forceinline__ uint32_t hash_slot(uint32_t x, int hb) { return (x * 2654435761u) >> (32 - hb); }

// first index of a flagged ascending list whose id is >= val
__device__ __forceinline__ uint32_t lower_bound_id(const uint32_t* a, uint32_t len, uint32_t val) {
    const uint32_t key = val << 2;
    uint32_t lo = 0, hi = len;
    while (lo < hi) {
        uint32_t mid = (lo + hi) >> 1;
        if (__ldg(a + mid) < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ unsigned long long pack3(uint32_t c1, uint32_t c2, uint32_t c3) {
    return (unsigned long long)c1 | ((unsigned long long)c2 << 21) | ((unsigned long long)c3 << 42);
}

// counts of direction classes 1, 2, 3 among the 32 lanes' values (0 = none), packed
__device__ __forceinline__ unsigned long long ballot3(uint32_t e) {
    return pack3(__popc(__ballot_sync(0xffffffffu, e == 1u)), __popc(__ballot_sync(0xffffffffu, e == 2u)),
                 __popc(__ballot_sync(0xffffffffu, e == 3u)));
}

__device__ __forceinline__ void hist_add(int* hist, uint32_t cls, int tid, int d) { hist[cls * kThreads + tid] += d; }

// Sum the per-thread histogram columns into the CTA's 64-bit accumulators and clear them.
__device__ __forceinline__ void flush_hist(int* hist, unsigned long long* cacc, int warp, int lane) {
    for (int cls = warp; cls < 16; cls += kWarps) {
        long long s = 0;
#pragma unroll
        for (int q = 0; q < kThreads / 32; ++q) {
            int i = cls * kThreads + lane + 32 * q;
            s += hist[i];
            hist[i] = 0;
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) cacc[cls] += (unsigned long long)s;
    }
}

template <int ALGO>
__global__ void __launch_bounds__(kThreads, 3) k_census(Params P) {
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t chunk = P.chunk;
    uint32_t* sA = reinterpret_cast<uint32_t*>(smem);                       // [chunk]   staged N[u] chunk
    uint32_t* sH = sA + chunk;                                               // [2*chunk] hash of the chunk
    unsigned long long* sCk = reinterpret_cast<unsigned long long*>(sH + 2 * chunk);  // [chunk/32+1]
    int* sHist = reinterpret_cast<int*>(sCk + chunk / 32 + 1);               // [16][kThreads]
    unsigned long long* sW = reinterpret_cast<unsigned long long*>(sHist + 16 * kThreads);  // [kWarps][16]
    unsigned long long* sC = sW + kWarps * 16;                               // [16]
    uint8_t* sT = reinterpret_cast<uint8_t*>(sC + 16);                       // [64]
    __shared__ uint32_t s_item, s_pending;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int i = tid; i < 16 * kThreads; i += kThreads) sHist[i] = 0;
    if (tid < kWarps * 16) sW[tid] = 0;
    if (tid < 16) sC[tid] = 0;
    if (tid < 64) sT[tid] = d_tricode_class[tid];
    if (tid == 0) s_pending = 0;
    __syncthreads();

    const uint64_t n = P.g.n;
    const uint64_t* __restrict__ off = P.g.off;
    const uint32_t* __restrict__ adj = P.g.adj;
    unsigned long long* wacc = sW + warp * 16;

    // ---------------------------------------------------------------- CTA items
    for (;;) {
        if (tid == 0) s_item = atomicAdd(&P.ctr[0], 1u);
        __syncthreads();
        const uint32_t it = s_item;
        if (it >= P.n_items) break;
        const Item w = P.items[it];
        const uint32_t u = w.u;
        const uint64_t ubase = off[u];
        const uint32_t du = (uint32_t)(off[u + 1] - ubase);
        const uint32_t LA = w.a1 - w.a0;
        int hb = 6;
        while ((1u << hb) < 2 * LA) ++hb;
        const uint32_t H = 1u << hb;
        for (uint32_t k = tid; k < LA; k += kThreads) sA[k] = adj[ubase + w.a0 + k];
        for (uint32_t k = tid; k < H; k += kThreads) sH[k] = kEmpty;
        __syncthreads();
        for (uint32_t k = tid; k < LA; k += kThreads) {
            const uint32_t e = sA[k];
            uint32_t h = hash_slot(e >> 2, hb);
            while (atomicCAS(&sH[h], kEmpty, e) != kEmpty) h = (h + 1) & (H - 1);
        }
        const uint32_t nq = (LA + 31) / 32;
        if (ALGO == TC_ALGO_SUFFIX) {
            for (uint32_t q = warp; q < nq; q += kWarps) {
                const uint32_t idx = q * 32 + lane;
                const unsigned long long c = ballot3(idx < LA ? (sA[idx] & 3u) : 0u);
                if (lane == 0) sCk[q + 1] = c;
            }
            __syncthreads();
            if (warp == 0) {   // inclusive scan of the block counts -> prefix before each block
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
        }
        __syncthreads();

        const uint32_t lo_val = w.a0 ? (sA[0] >> 2) : 0u;
        const bool has_hi = w.a1 < du;
        const uint32_t hi_val = has_hi ? (adj[ubase + w.a1] >> 2) : 0u;
        uint32_t pend = 0;
        for (uint32_t j = w.j0 + warp; j < w.j1; j += kWarps) {
            const uint32_t euv = adj[ubase + j];
            const uint32_t v = euv >> 2, duv = euv & 3u, cuv = code_uv(duv);
            const uint64_t vb = off[v];
            const uint32_t dv = (uint32_t)(off[v + 1] - vb);
            const uint32_t* __restrict__ B = adj + vb;
            const uint32_t b0 = w.a0 ? lower_bound_id(B, dv, lo_val) : 0u;
            const uint32_t b1 = has_hi ? lower_bound_id(B, dv, hi_val) : dv;
            uint32_t c = 0;
            for (uint32_t k = b0 + lane; k < b1; k += 32) {       // v side
                const uint32_t xe = B[k], x = xe >> 2, dvw = xe & 3u;
                uint32_t h = hash_slot(x, hb), e;
                bool found = false;
                while ((e = sH[h]) != kEmpty) {
                    if ((e >> 2) == x) { found = true; break; }
                    h = (h + 1) & (H - 1);
                }
                if (found) {
                    ++c;
                    if (x > v) {
                        const uint32_t duw = e & 3u;
                        hist_add(sHist, sT[cuv | (dvw << 2) | (duw << 4)], tid, 1);
                        hist_add(sHist, sT[cuv | (duw << 4)], tid, -1);
                    }
                } else if (x > u) {
                    hist_add(sHist, sT[cuv | (dvw << 2)], tid, 1);
                }
            }
            c = __reduce_add_sync(0xffffffffu, c);
            uint32_t s0 = (j + 1 > w.a0 ? j + 1 : w.a0) - w.a0;   // u side: chunk entries past v
            if (s0 > LA) s0 = LA;
            if (ALGO == TC_ALGO_UNION) {
                for (uint32_t k = s0 + lane; k < LA; k += 32) hist_add(sHist, sT[cuv | ((sA[k] & 3u) << 4)], tid, 1);
            } else {
                const uint32_t q = s0 >> 5, r = s0 & 31u, idx = q * 32 + lane;
                const unsigned long long part = ballot3((lane < r && idx < LA) ? (sA[idx] & 3u) : 0u);
                const unsigned long long suf = sCk[nq] - sCk[q] - part;
                if (lane == 0) {
#pragma unroll
                    for (uint32_t d = 1; d <= 3; ++d) {
                        const unsigned long long cnt = (suf >> (21 * (d - 1))) & 0x1fffffull;
                        if (cnt) wacc[sT[cuv | (d << 4)]] += cnt;
                    }
                }
            }
            if (lane == 0) {
                const unsigned long long dy = (w.a0 == 0 ? n - du - dv : 0ull) + c;
                wacc[duv == 3u ? 2 : 1] += dy;
                pend += (b1 - b0) + (ALGO == TC_ALGO_UNION ? LA - s0 : 0u);
            }
        }
        if (lane == 0) atomicAdd(&s_pending, pend);
        __syncthreads();
        if (s_pending > kFlushAfter) {
            flush_hist(sHist, sC, warp, lane);
            __syncthreads();
            if (tid == 0) s_pending = 0;
        }
    }

    // ---------------------------------------------------------------- one warp per vertex
    uint32_t* wA = sA + warp * P.warp_max;
    for (;;) {
        uint32_t ub = 0;
        if (lane == 0) ub = atomicAdd(&P.ctr[1], 32u);
        ub = __shfl_sync(0xffffffffu, ub, 0);
        const uint32_t u0 = P.warp_begin + ub;
        if (u0 >= P.warp_end || ub >= P.warp_end) break;
        const uint32_t u1 = min(u0 + 32u, P.warp_end);
        for (uint32_t u = u0; u < u1; ++u) {
            const uint64_t ubase = off[u];
            const uint32_t du = (uint32_t)(off[u + 1] - ubase);
            const uint32_t p0 = P.g.up[u];
            if (p0 >= du) continue;
            __syncwarp();
            for (uint32_t k = lane; k < du; k += 32) wA[k] = adj[ubase + k];
            __syncwarp();
            for (uint32_t j = p0; j < du; ++j) {
                const uint32_t euv = wA[j];
                const uint32_t v = euv >> 2, duv = euv & 3u, cuv = code_uv(duv);
                const uint64_t vb = off[v];
                const uint32_t dv = (uint32_t)(off[v + 1] - vb);
                const uint32_t* __restrict__ B = adj + vb;
                uint32_t c = 0;
                for (uint32_t k = lane; k < dv; k += 32) {
                    const uint32_t xe = B[k], x = xe >> 2, dvw = xe & 3u;
                    uint32_t lo = 0, hi = du;
                    while (lo < hi) {
                        uint32_t mid = (lo + hi) >> 1;
                        if ((wA[mid] >> 2) < x) lo = mid + 1; else hi = mid;
                    }
                    if (lo < du && (wA[lo] >> 2) == x) {
                        ++c;
                        if (x > v) {
                            const uint32_t duw = wA[lo] & 3u;
                            hist_add(sHist, sT[cuv | (dvw << 2) | (duw << 4)], tid, 1);
                            hist_add(sHist, sT[cuv | (duw << 4)], tid, -1);
                        }
                    } else if (x > u) {
                        hist_add(sHist, sT[cuv | (dvw << 2)], tid, 1);
                    }
                }
                c = __reduce_add_sync(0xffffffffu, c);
                if (ALGO == TC_ALGO_UNION) {
                    for (uint32_t k = j + 1 + lane; k < du; k += 32) hist_add(sHist, sT[cuv | ((wA[k] & 3u) << 4)], tid, 1);
                } else {
                    unsigned long long suf = 0;
                    for (uint32_t b = (j + 1) & ~31u; b < du; b += 32) {
                        const uint32_t k = b + lane;
                        suf += ballot3((k > j && k < du) ? (wA[k] & 3u) : 0u);
                    }
                    if (lane == 0) {
#pragma unroll
                        for (uint32_t d = 1; d <= 3; ++d) {
                            const unsigned long long cnt = (suf >> (21 * (d - 1))) & 0x1fffffull;
                            if (cnt) wacc[sT[cuv | (d << 4)]] += cnt;
                        }
                    }
                }
                if (lane == 0) wacc[duv == 3u ? 2 : 1] += (n - du - dv) + c;
            }
        }
    }

    __syncthreads();
    flush_hist(sHist, sC, warp, lane);
    __syncthreads();
    if (tid < 16) {
        unsigned long long t = sC[tid];
#pragma unroll
        for (int w = 0; w < kWarps; ++w) t += sW[w * 16 + tid];
        if (t) atomicAdd(&P.out[tid], t);
    }
}

// ---------------------------------------------------------------- schedule (plan) kernels
__global__ void k_count_gt(const uint64_t* off, uint32_t n, uint32_t thr, uint32_t* cnt) {
    uint32_t c = 0;
    for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < n; x += (uint64_t)gridDim.x * blockDim.x)
        c += (off[x + 1] - off[x]) > thr;
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(cnt, c);
}

// Items per vertex u < u_end: C chunks of N[u] times S ranges of v, with S from the
// estimated work of u's pairs (degrees for the plain schedule, the cost model if given).
__global__ void k_plan_count(GraphDev g, uint32_t u_end, uint32_t chunk, uint32_t item_work, int algo, float dbar,
                             const float* cost, uint32_t* cnt, uint32_t* split) {
    for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < u_end; x += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t du = (uint32_t)(g.off[x + 1] - g.off[x]);
        const uint32_t P = du - g.up[x];
        if (P == 0) { cnt[x] = 0; split[x] = 0; continue; }
        const uint32_t C = (du + chunk - 1) / chunk;
        double est;
        if (cost) est = (double)cost[x];
        else est = (double)P * ((double)dbar + 16.0) + (algo == TC_ALGO_UNION ? 0.5 * (double)P * (double)du : 0.0);
        double s = ceil(est / (double)C / (double)item_work);
        if (s < 1.0) s = 1.0;
        if (s > (double)P) s = (double)P;
        const uint32_t S = (uint32_t)s;
        cnt[x] = C * S;
        split[x] = S;
    }
}

__global__ void k_plan_emit(GraphDev g, uint32_t u_end, uint32_t chunk, const uint32_t* pos, const uint32_t* split,
                            Item* items) {
    for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < u_end; x += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t S = split[x];
        if (!S) continue;
        const uint32_t du = (uint32_t)(g.off[x + 1] - g.off[x]);
        const uint32_t up = g.up[x], P = du - up;
        const uint32_t C = (du + chunk - 1) / chunk;
        uint32_t o = pos[x];
        for (uint32_t c = 0; c < C; ++c) {
            const uint32_t a0 = c * chunk, a1 = min(du, a0 + chunk);
            for (uint32_t s = 0; s < S; ++s) {
                Item it;
                it.u = (uint32_t)x;
                it.a0 = a0;
                it.a1 = a1;
                it.j0 = up + (uint32_t)((uint64_t)P * s / S);
                it.j1 = up + (uint32_t)((uint64_t)P * (s + 1) / S);
                items[o++] = it;
            }
        }
    }
}

std::atomic<uint64_t> g_table_uploaded{0};
std::atomic<uint64_t> g_attr_set[2] = {{0}, {0}};

size_t census_smem(uint32_t chunk) {
    return sizeof(uint32_t) * 3ull * chunk + sizeof(unsigned long long) * (chunk / 32 + 1) +
           sizeof(int) * 16ull * kThreads + sizeof(unsigned long long) * (kWarps * 16 + 16) + 64;
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
    if (!(g_attr_set[algo].load() & bit)) {
        const void* fn = algo == TC_ALGO_UNION ? (const void*)k_census<TC_ALGO_UNION> : (const void*)k_census<TC_ALGO_SUFFIX>;
        TC_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, limit));
        g_attr_set[algo].fetch_or(bit);
    }
    return TC_OK;
}

}  // namespace

tc_status get_plan(GraphStore& g, const Opts& o, cudaStream_t st, Plan** out) {
    for (auto& p : g.plans)
        if (p.valid && p.key == o) { *out = &p; return TC_OK; }
    Plan& p = g.plans[g.next_plan];
    g.next_plan = (g.next_plan + 1) % GraphStore::kPlans;
    p.valid = false;
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
        DevBuf cnt, split, pos, tot;
        TC_TRY(cnt.alloc(sizeof(uint32_t) * u_end, st));
        TC_TRY(split.alloc(sizeof(uint32_t) * u_end, st));
        TC_TRY(pos.alloc(sizeof(uint32_t) * u_end, st));
        TC_TRY(tot.alloc(sizeof(uint32_t), st));
        const float dbar = g.n_active ? (float)(2.0 * (double)g.e_sym / (double)g.n_active) : 0.f;
        const float* cost = (o.schedule == TC_SCHED_LEARNED) ? g.cost.as<float>() : nullptr;
        if (o.schedule == TC_SCHED_LEARNED && !cost) return fail(TC_ERR_ARG, "learned schedule requested but no cost model is attached");
        k_plan_count<<<grid_for(u_end, 256, 4096), 256, 0, st>>>(gd, u_end, o.chunk, o.item_work, (int)o.algo, dbar, cost,
                                                                  cnt.as<uint32_t>(), split.as<uint32_t>());
        TC_LAUNCH("k_plan_count");
        TC_TRY(scan_u32(cnt.as<uint32_t>(), pos.as<uint32_t>(), u_end, tot.as<uint32_t>(), st));
        TC_CUDA(cudaMemcpyAsync(&p.n_items, tot.p, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
        TC_CUDA(cudaStreamSynchronize(st));
        TC_TRY(p.items.alloc_persistent(sizeof(Item) * (p.n_items ? p.n_items : 1)));
        if (p.n_items) {
            k_plan_emit<<<grid_for(u_end, 256, 4096), 256, 0, st>>>(gd, u_end, o.chunk, pos.as<uint32_t>(),
                                                                     split.as<uint32_t>(), p.items.as<Item>());
            TC_LAUNCH("k_plan_emit");
        }
        TC_CUDA(cudaStreamSynchronize(st));
    }
    p.valid = true;
    *out = &p;
    return TC_OK;
}

tc_status census_enqueue(GraphStore& g, const Opts& o, const Plan& p, cudaStream_t st, unsigned long long* d_out16) {
    if (g.e_sym == 0) return TC_OK;
    const size_t smem = census_smem(o.chunk);
    TC_TRY(prepare_device(st, (int)o.algo, smem));
    TC_CUDA(cudaMemsetAsync(g.ctr.p, 0, sizeof(uint32_t) * 4, st));
    Params P;
    P.g = g.dev();
    P.items = p.items.as<Item>();
    P.n_items = p.n_items;
    P.warp_begin = p.warp_begin;
    P.warp_end = p.warp_end;
    P.chunk = o.chunk;
    P.warp_max = o.warp_max_deg;
    P.ctr = g.ctr.as<uint32_t>();
    P.out = d_out16;
    const unsigned grid = (unsigned)(sm_count() * (int)o.ctas_per_sm);
    if (o.algo == TC_ALGO_UNION) k_census<TC_ALGO_UNION><<<grid, kThreads, smem, st>>>(P);
    else k_census<TC_ALGO_SUFFIX><<<grid, kThreads, smem, st>>>(P);
    TC_LAUNCH("k_census");
    return TC_OK;
}

}  // namespace tc
