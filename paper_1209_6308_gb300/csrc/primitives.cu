// primitives.cu - device scans and a stable LSD radix sort, used by the graph builder
// (symmetrise, dedupe, relabel and sort steps of the Sec. 6 compact structure).
//
// Scan: reduce-then-scan over tiles of 4096 values (256 threads x 16 per thread), the tile
// sums scanned by one CTA, then a downsweep.
// Radix sort: 8-bit digits.  Per pass: a tile histogram (digit-major counts), an exclusive
// scan of the counts, and a scatter that ranks each key stably inside its tile with a
// warp multi-split (eight ballots give the lanes sharing a digit), stages the tile in
// shared memory in digit order, then writes contiguous runs per digit.
#include <algorithm>

#include "tc_internal.cuh"

namespace tc {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanPer = 16;
constexpr int kScanTile = kScanThreads * kScanPer;
constexpr int kSortThreads = 256;
constexpr int kSortRounds = 16;
constexpr int kSortTile = kSortThreads * kSortRounds;

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

// Exclusive block scan of one value per thread (blockDim.x == 256 or 1024); returns the
// exclusive prefix and writes the block total to *total.
template <typename T>
__device__ __forceinline__ T block_excl_scan(T v, T* total) {
    __shared__ T warp_sums[32];
    __shared__ T s_total;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T inc = warp_incl_scan(v);
    if (lane == 31) warp_sums[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        T w = lane < nw ? warp_sums[lane] : T(0);
        T wi = warp_incl_scan(w);
        warp_sums[lane] = wi - w;
        if (lane == nw - 1) s_total = wi;
    }
    __syncthreads();
    T res = inc - v + warp_sums[warp];
    *total = s_total;
    __syncthreads();
    return res;
}

template <typename Tout>
__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t* in, uint64_t n, Tout* tile_sums) {
    uint64_t base = (uint64_t)blockIdx.x * kScanTile;
    Tout s = 0;
#pragma unroll
    for (int r = 0; r < kScanPer; ++r) {
        uint64_t i = base + (uint64_t)r * kScanThreads + threadIdx.x;
        if (i < n) s += in[i];
    }
    Tout tot;
    block_excl_scan<Tout>(s, &tot);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

// One CTA scans `cnt` tile sums in place (exclusive); writes the grand total to *total.
template <typename Tout>
__global__ void __launch_bounds__(1024) k_scan_tiles(Tout* sums, uint64_t cnt, Tout* total) {
    Tout carry = 0;
    for (uint64_t base = 0; base < cnt; base += 1024) {
        uint64_t i = base + threadIdx.x;
        Tout v = i < cnt ? sums[i] : Tout(0);
        Tout tot;
        Tout ex = block_excl_scan<Tout>(v, &tot);
        if (i < cnt) sums[i] = ex + carry;
        carry += tot;
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

template <typename Tout>
__global__ void __launch_bounds__(kScanThreads) k_scan_down(const uint32_t* in, uint64_t n, const Tout* tile_off, Tout* out) {
    __shared__ uint32_t tile[kScanTile];
    uint64_t base = (uint64_t)blockIdx.x * kScanTile;
#pragma unroll
    for (int r = 0; r < kScanPer; ++r) {
        uint64_t i = base + (uint64_t)r * kScanThreads + threadIdx.x;
        tile[r * kScanThreads + threadIdx.x] = i < n ? in[i] : 0u;
    }
    __syncthreads();
    // thread t owns the 16 consecutive values [16t, 16t+16) of the tile
    Tout loc[kScanPer];
    Tout s = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) { loc[k] = s; s += tile[threadIdx.x * kScanPer + k]; }
    Tout tot;
    Tout ex = block_excl_scan<Tout>(s, &tot) + tile_off[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        uint64_t i = base + (uint64_t)threadIdx.x * kScanPer + k;
        if (i < n) out[i] = ex + loc[k];
    }
}

template <typename Tout>
tc_status scan_impl(const uint32_t* in, Tout* out, uint64_t n, Tout* total, cudaStream_t st) {
    if (n == 0) {
        if (total) TC_CUDA(cudaMemsetAsync(total, 0, sizeof(Tout), st));
        return TC_OK;
    }
    uint64_t tiles = (n + kScanTile - 1) / kScanTile;
    if (tiles > 0x7fffffffull) return fail(TC_ERR_RANGE, "scan: too many elements");
    DevBuf sums;
    TC_TRY(sums.alloc(sizeof(Tout) * tiles, st));
    k_scan_reduce<Tout><<<(unsigned)tiles, kScanThreads, 0, st>>>(in, n, sums.as<Tout>());
    TC_LAUNCH("k_scan_reduce");
    k_scan_tiles<Tout><<<1, 1024, 0, st>>>(sums.as<Tout>(), tiles, total);
    TC_LAUNCH("k_scan_tiles");
    k_scan_down<Tout><<<(unsigned)tiles, kScanThreads, 0, st>>>(in, n, sums.as<Tout>(), out);
    TC_LAUNCH("k_scan_down");
    return TC_OK;
}

// ------------------------------------------------------------------ radix sort
__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const uint64_t* keys, uint64_t n, int shift,
                                                             uint32_t* counts, uint32_t tiles) {
    __shared__ uint32_t wh[kSortThreads / 32][256];
    const int warp = threadIdx.x >> 5;
    for (int d = threadIdx.x; d < (kSortThreads / 32) * 256; d += kSortThreads) (&wh[0][0])[d] = 0;
    __syncthreads();
    uint64_t base = (uint64_t)blockIdx.x * kSortTile;
    // all of the thread's keys are loaded before any is counted, so the tile's loads are in
    // flight together
    uint32_t dg[kSortRounds];
#pragma unroll
    for (int r = 0; r < kSortRounds; ++r) {
        uint64_t i = base + (uint64_t)r * kSortThreads + threadIdx.x;
        dg[r] = i < n ? (uint32_t)(keys[i] >> shift) & 255u : 256u;
    }
#pragma unroll
    for (int r = 0; r < kSortRounds; ++r)
        if (dg[r] < 256u) atomicAdd(&wh[warp][dg[r]], 1u);
    __syncthreads();
    uint32_t s = 0;
#pragma unroll
    for (int w = 0; w < kSortThreads / 32; ++w) s += wh[w][threadIdx.x];
    counts[(uint64_t)threadIdx.x * tiles + blockIdx.x] = s;
}

__global__ void __launch_bounds__(kSortThreads, 3) k_radix_scatter(const uint64_t* in, uint64_t* out, uint64_t n, int shift,
                                                                const uint32_t* counts, const uint32_t* offs,
                                                                uint32_t tiles) {
    __shared__ uint64_t s_keys[kSortTile];
    __shared__ uint32_t s_start[256];
    __shared__ uint32_t s_run[256];
    __shared__ uint32_t s_wc[kSortThreads / 32][256];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t lt_mask = (1u << lane) - 1u;
    uint64_t base = (uint64_t)blockIdx.x * kSortTile;

    uint32_t c = counts[(uint64_t)tid * tiles + blockIdx.x];
    uint32_t tot;
    s_start[tid] = block_excl_scan<uint32_t>(c, &tot);
    s_run[tid] = 0;
    __syncthreads();

    // the thread's keys of all rounds, loaded together (coalesced, one tile in flight)
    uint64_t kr[kSortRounds];
#pragma unroll
    for (int r = 0; r < kSortRounds; ++r) {
        uint64_t i = base + (uint64_t)r * kSortThreads + tid;
        kr[r] = i < n ? in[i] : 0ull;
    }
#pragma unroll
    for (int r = 0; r < kSortRounds; ++r) {
        uint64_t i = base + (uint64_t)r * kSortThreads + tid;
        bool valid = i < n;
        uint64_t k = kr[r];
        uint32_t d = (uint32_t)(k >> shift) & 255u;
#pragma unroll
        for (int q = 0; q < 8; ++q) s_wc[warp][lane + 32 * q] = 0;
        __syncwarp();
        uint32_t peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            uint32_t bal = __ballot_sync(0xffffffffu, (d >> b) & 1u);
            peers &= ((d >> b) & 1u) ? bal : ~bal;
        }
        uint32_t rank = __popc(peers & lt_mask);
        if (valid && rank == 0) s_wc[warp][d] = __popc(peers);
        __syncthreads();
        {
            uint32_t run = s_run[tid];
#pragma unroll
            for (int w = 0; w < kSortThreads / 32; ++w) {
                uint32_t cw = s_wc[w][tid];
                s_wc[w][tid] = run;
                run += cw;
            }
            s_run[tid] = run;
        }
        __syncthreads();
        if (valid) s_keys[s_start[d] + s_wc[warp][d] + rank] = k;
        __syncthreads();
    }
    uint64_t rem = n - base;
    uint32_t tile_n = rem < (uint64_t)kSortTile ? (uint32_t)rem : (uint32_t)kSortTile;
    for (uint32_t i = tid; i < tile_n; i += kSortThreads) {
        uint64_t k = s_keys[i];
        uint32_t d = (uint32_t)(k >> shift) & 255u;
        out[(uint64_t)offs[(uint64_t)d * tiles + blockIdx.x] + (i - s_start[d])] = k;
    }
}

}  // namespace

tc_status scan_u32(const uint32_t* in, uint32_t* out, uint64_t n, uint32_t* total, cudaStream_t st) {
    return scan_impl<uint32_t>(in, out, n, total, st);
}

tc_status scan_u32_to_u64(const uint32_t* in, uint64_t* out, uint64_t n, cudaStream_t st) {
    return scan_impl<uint64_t>(in, out, n, out + n, st);
}

tc_status radix_sort_u64(uint64_t** keys, uint64_t** tmp, uint64_t n, int lo_bit, int hi_bit, cudaStream_t st) {
    if (n <= 1 || hi_bit <= lo_bit) return TC_OK;
    if (n >= (1ull << 32)) return fail(TC_ERR_RANGE, "radix sort: more than 2^32-1 keys");
    uint64_t tiles64 = (n + kSortTile - 1) / kSortTile;
    uint32_t tiles = (uint32_t)tiles64;
    DevBuf counts, offs;
    TC_TRY(counts.alloc(sizeof(uint32_t) * 256ull * tiles, st));
    TC_TRY(offs.alloc(sizeof(uint32_t) * 256ull * tiles, st));
    for (int sh = lo_bit; sh < hi_bit; sh += 8) {
        k_radix_hist<<<tiles, kSortThreads, 0, st>>>(*keys, n, sh, counts.as<uint32_t>(), tiles);
        TC_LAUNCH("k_radix_hist");
        TC_TRY(scan_u32(counts.as<uint32_t>(), offs.as<uint32_t>(), 256ull * tiles, nullptr, st));
        k_radix_scatter<<<tiles, kSortThreads, 0, st>>>(*keys, *tmp, n, sh, counts.as<uint32_t>(),
                                                        offs.as<uint32_t>(), tiles);
        TC_LAUNCH("k_radix_scatter");
        std::swap(*keys, *tmp);
    }
    return TC_OK;
}

}  // namespace tc
