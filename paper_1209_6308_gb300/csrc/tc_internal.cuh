// tc_internal.cuh - shared declarations of the GPU triad-census library (device structs,
// error plumbing, primitive launchers).  Only the library's own .cu files include this.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/tc.h"

namespace tc {

// ------------------------------------------------------------------ errors
void set_error(const std::string& msg);
tc_status fail(tc_status s, const std::string& msg);
tc_status cuda_fail(cudaError_t e, const char* what);

#define TC_CUDA(call)                                                     \
    do {                                                                  \
        cudaError_t _e = (call);                                          \
        if (_e != cudaSuccess) return ::tc::cuda_fail(_e, #call);         \
    } while (0)
#define TC_LAUNCH(what)                                                   \
    do {                                                                  \
        cudaError_t _e = cudaGetLastError();                              \
        if (_e != cudaSuccess) return ::tc::cuda_fail(_e, what);          \
    } while (0)
#define TC_TRY(expr)                                                      \
    do {                                                                  \
        tc_status _s = (expr);                                            \
        if (_s != TC_OK) return _s;                                       \
    } while (0)

// Device buffer: alloc() is stream-ordered (freed on the same stream when released),
// alloc_persistent() is a plain cudaMalloc for buffers that outlive the creating stream.
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    cudaStream_t st = nullptr;
    bool async = false;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() { release(); }
    tc_status alloc(size_t b, cudaStream_t s);
    tc_status alloc_persistent(size_t b);
    void release();
    template <typename T> T* as() const { return static_cast<T*>(p); }
};

// ------------------------------------------------------------------ graph on the device
// Compact CSR of Sec. 6 (Fig. 7) in degree-descending ids: adj entries are (id << 2) | dir
// with dir bit 0 = owner->id and bit 1 = id->owner; lists ascend by id.
struct GraphDev {
    uint32_t n;
    uint32_t n_active;      // vertices with deg > 0 are exactly ids [0, n_active)
    const uint64_t* off;    // [n+1]
    const uint32_t* adj;    // [off[n]]
    const uint32_t* up;     // [n] number of neighbours with a smaller id (index of first v > u)
    // Per upper pair tables (null when absent): the upper pair (u, v = N[u][j]) with j >= up[u]
    // has index ub[u] + j - up[u]; rp[.] is the position of u in N[v], vs[.] the counts of
    // direction classes 1 and 2 among the entries of N[v] after u, us[.] those among the
    // entries of N[u] after v (class 3: the rest of each suffix).
    const uint64_t* ub;     // [n+1] upper pairs before each vertex
    const uint32_t* rp;     // [E]
    const uint2* vs;        // [E]
    const uint2* us;        // [E]
};

// One CTA work item of the census: vertex u and its pairs (u, N[u][j]) for j in [j0, j1)
// (all with N[u][j] > u).  N[u] is staged in shared memory one chunk at a time.
struct Item {
    uint32_t u, j0, j1, pad;
};
constexpr uint32_t kMaxItemPairs = 1024;   // pairs per item (one N[v] cursor each in shared memory)
// The census answers membership in N[u] for ids below these from a direct two-bit-per-id map
// of the staged list (the highest-degree vertices, since ids descend with the degree).
constexpr uint32_t kMapIdsSuffix = 1u << 17, kMapIdsUnion = 1u << 16;

// ------------------------------------------------------------------ primitives
// Exclusive scan of n uint32 values into uint32 (out may alias nothing); *total (device
// pointer, may be null) receives the sum.
tc_status scan_u32(const uint32_t* in, uint32_t* out, uint64_t n, uint32_t* total, cudaStream_t st);
// Exclusive scan of n uint32 values into uint64 offsets; out has n+1 entries (out[n] = sum).
tc_status scan_u32_to_u64(const uint32_t* in, uint64_t* out, uint64_t n, cudaStream_t st);
// Stable LSD radix sort of n 64-bit keys on bits [lo_bit, hi_bit); keys and tmp both hold n
// keys; the result ends in *keys (the pointers may be swapped).  n must be < 2^32.
tc_status radix_sort_u64(uint64_t** keys, uint64_t** tmp, uint64_t n, int lo_bit, int hi_bit, cudaStream_t st);

inline unsigned grid_for(uint64_t n, unsigned block, unsigned cap = 1u << 20) {
    uint64_t g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (unsigned)g;
}

int sm_count();

inline tc_u128 to_u128(unsigned __int128 x) {
    tc_u128 r;
    r.lo = (uint64_t)x;
    r.hi = (uint64_t)(x >> 64);
    return r;
}

// C(n, 3), the number of triads (Fig. 5 step 5's total), in 128 bits
inline unsigned __int128 choose3(uint64_t n) {
    if (n < 3) return 0;
    unsigned __int128 a = n, b = n - 1, c = n - 2;
    return a * b * c / 6;
}

}  // namespace tc
