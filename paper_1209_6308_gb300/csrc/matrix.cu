// matrix.cu - the matrix form of the census (paper Sec. 4 names Moody's matrix census as the
// dense way to compute it): every class count as sums of elementwise products of 0/1 dyad
// matrices with matrix products of them.  With S the one-way arcs (S[i][j] = 1 for i -> j
// only), M the mutual dyads and N the null dyads (i != j, no arc):
//   003 = sum(N o NN)/6    012 = sum(S o NN)        102 = sum(M o NN)/2
//   021D = sum(N o S'S)/2  021U = sum(N o SS')/2    021C = sum(N o SS)
//   111D = sum(S o NM)     111U = sum(S' o NM)      030T = sum(S o SS)      030C = sum(S' o SS)/3
//   201 = sum(N o MM)/2    120D = sum(M o S'S)/2    120U = sum(M o SS')/2   120C = sum(M o SS)
//   210 = sum(S o MM)      300 = sum(M o MM)/6
// (each a labelled count of the class's arc pattern over its symmetries; S' = S transposed).
// Six products, each reduced against up to four masks.  The matrices are 0/1, so they are held
// bit-packed, 64 columns per word, and a product entry (XY)[i][j] is the popcount of row i of X
// AND row j of Y' over the words: a dense contraction done in the integer pipes, 64 entries per
// instruction, with the masked sums fused into the tile so no product is ever stored.  All 16
// counts come from their own sums (the null count too), independently of the Fig. 5 method.
#include <cstring>

#include "graph.cuh"

namespace tc {
namespace {

constexpr uint32_t kMatrixMaxN = 1u << 14;
constexpr int kTile = 64;        // rows i and j of a block's tile
constexpr int kWords = 16;       // words of a row staged per step
constexpr int kThreadsM = 256;   // 16 x 16 threads, 4 x 4 entries each

// Bit rows of S, S', M for the relabelled graph (one warp per row), then N from them.
__global__ void k_dyad_bits(const uint64_t* __restrict__ off, const uint32_t* __restrict__ adj, uint32_t n, uint32_t W,
                            unsigned long long* S, unsigned long long* St, unsigned long long* M) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t i = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
        const uint64_t row = i * W;
        for (uint64_t k = off[i] + lane; k < off[i + 1]; k += 32) {
            const uint32_t e = adj[k], j = e >> 2, dir = e & 3u;   // dir seen from i: 1 i->j, 2 j->i
            unsigned long long* dst = dir == 3u ? M : (dir == 1u ? S : St);
            atomicOr(&dst[row + (j >> 6)], 1ull << (j & 63u));
        }
    }
}

__global__ void k_null_bits(uint32_t n, uint32_t W, const unsigned long long* __restrict__ S,
                            const unsigned long long* __restrict__ St, const unsigned long long* __restrict__ M,
                            unsigned long long* N) {
    const uint64_t total = (uint64_t)n * W;
    for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < total; x += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t i = (uint32_t)(x / W), w = (uint32_t)(x % W);
        unsigned long long v = ~(S[x] | St[x] | M[x]);
        const uint32_t lo = w * 64u;
        if (lo + 64u > n) v &= (n > lo) ? ((1ull << (n - lo)) - 1ull) : 0ull;   // columns past n
        if ((i >> 6) == w) v &= ~(1ull << (i & 63u));                           // no self-dyad
        N[x] = v;
    }
}

// sums[m] += sum over i, j < n of Z_m[i][j] * popcount(X row i AND Yt row j), m < n_masks.
struct MaskedProduct {
    const unsigned long long* X;
    const unsigned long long* Yt;
    const unsigned long long* Z[4];
    uint32_t n_masks;
};

__global__ void __launch_bounds__(kThreadsM) k_masked_product(MaskedProduct P, uint32_t n, uint32_t W,
                                                               unsigned long long* sums) {
    __shared__ unsigned long long sX[kTile][kWords + 1];
    __shared__ unsigned long long sY[kTile][kWords + 1];
    __shared__ unsigned long long sRed[4][kThreadsM / 32];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const uint32_t i0 = blockIdx.y * kTile, j0 = blockIdx.x * kTile;
    uint32_t acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0u;
    for (uint32_t w0 = 0; w0 < W; w0 += kWords) {
        // stage 64 rows x 16 words of X (rows i) and of Yt (rows j); zeros past n and W
        for (int k = tid; k < kTile * kWords; k += kThreadsM) {
            const int r = k / kWords, c = k % kWords;
            const uint32_t w = w0 + c;
            const uint32_t ri = i0 + r, rj = j0 + r;
            sX[r][c] = (ri < n && w < W) ? P.X[(uint64_t)ri * W + w] : 0ull;
            sY[r][c] = (rj < n && w < W) ? P.Yt[(uint64_t)rj * W + w] : 0ull;
        }
        __syncthreads();
#pragma unroll 4
        for (int c = 0; c < kWords; ++c) {
            unsigned long long xv[4], yv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) xv[a] = sX[ty * 4 + a][c];
#pragma unroll
            for (int b = 0; b < 4; ++b) yv[b] = sY[tx * 4 + b][c];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] += (uint32_t)__popcll(xv[a] & yv[b]);
        }
        __syncthreads();
    }
    // the masks of the tile's entries
    unsigned long long part[4] = {0ull, 0ull, 0ull, 0ull};
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const uint32_t i = i0 + ty * 4 + a;
        if (i >= n) continue;
        const uint32_t jb = j0 + tx * 4;   // four consecutive columns in one word
        if (jb >= n) continue;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            if ((uint32_t)m >= P.n_masks) break;
            const unsigned long long z = P.Z[m][(uint64_t)i * W + (jb >> 6)] >> (jb & 63u);
#pragma unroll
            for (int b = 0; b < 4; ++b)
                if ((z >> b) & 1ull) part[m] += acc[a][b];
        }
    }
    const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        unsigned long long v = part[m];
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) sRed[m][warp] = v;
    }
    __syncthreads();
    if (tid < 4 && (uint32_t)tid < P.n_masks) {
        unsigned long long v = 0;
        for (int q = 0; q < kThreadsM / 32; ++q) v += sRed[tid][q];
        if (v) atomicAdd(&sums[tid], v);
    }
}

}  // namespace
}  // namespace tc

using namespace tc;

extern "C" tc_status tc_census_matrix(tc_graph* g, void* stream, tc_u128 out[16]) {
    if (!g || !out) return fail(TC_ERR_ARG, "null argument");
    GraphStore& G = g->s;
    if (G.n > kMatrixMaxN)
        return fail(TC_ERR_RANGE, "tc_census_matrix: n = " + std::to_string(G.n) + " exceeds its limit of " +
                                      std::to_string(kMatrixMaxN) + " vertices");
    cudaStream_t st = (cudaStream_t)stream;
    std::unique_lock<std::mutex> lk(G.busy, std::try_to_lock);
    if (!lk.owns_lock()) return fail(TC_ERR_BUSY, "graph is in use by another call");
    const uint32_t n = G.n;
    unsigned long long h[24] = {};
    if (n >= 3) {
        const uint32_t W = (n + 63) / 64;
        const uint64_t words = (uint64_t)n * W;
        DevBuf bS, bSt, bM, bN, sums;
        TC_TRY(bS.alloc(sizeof(unsigned long long) * words, st));
        TC_TRY(bSt.alloc(sizeof(unsigned long long) * words, st));
        TC_TRY(bM.alloc(sizeof(unsigned long long) * words, st));
        TC_TRY(bN.alloc(sizeof(unsigned long long) * words, st));
        TC_TRY(sums.alloc(sizeof(unsigned long long) * 24, st));
        unsigned long long *S = bS.as<unsigned long long>(), *St = bSt.as<unsigned long long>(),
                           *M = bM.as<unsigned long long>(), *N = bN.as<unsigned long long>();
        TC_CUDA(cudaMemsetAsync(S, 0, sizeof(unsigned long long) * words, st));
        TC_CUDA(cudaMemsetAsync(St, 0, sizeof(unsigned long long) * words, st));
        TC_CUDA(cudaMemsetAsync(M, 0, sizeof(unsigned long long) * words, st));
        TC_CUDA(cudaMemsetAsync(sums.p, 0, sizeof(unsigned long long) * 24, st));
        if (G.e_sym) {
            k_dyad_bits<<<grid_for((uint64_t)n * 32, 256, 4096), 256, 0, st>>>(G.off.as<uint64_t>(), G.adj.as<uint32_t>(),
                                                                            n, W, S, St, M);
            TC_LAUNCH("k_dyad_bits");
        }
        k_null_bits<<<grid_for(words, 256, 8192), 256, 0, st>>>(n, W, S, St, M, N);
        TC_LAUNCH("k_null_bits");
        // the six products and their masks (S' as the rows of a product's right factor means
        // the factor is S, and so on; M and N are symmetric)
        const MaskedProduct prods[6] = {
            {N, N, {S, M, N, nullptr}, 3},        // NN:   012, 2 x 102, 6 x 003
            {St, St, {N, M, nullptr, nullptr}, 2},  // S'S:  2 x 021D, 2 x 120D
            {S, S, {N, M, nullptr, nullptr}, 2},    // SS':  2 x 021U, 2 x 120U
            {S, St, {N, S, St, M}, 4},              // SS:   021C, 030T, 3 x 030C, 120C
            {N, M, {S, St, nullptr, nullptr}, 2},   // NM:   111D, 111U
            {M, M, {N, S, M, nullptr}, 3},          // MM:   2 x 201, 210, 6 x 300
        };
        const dim3 grid((n + kTile - 1) / kTile, (n + kTile - 1) / kTile);
        for (int p = 0; p < 6; ++p) {
            k_masked_product<<<grid, kThreadsM, 0, st>>>(prods[p], n, W, sums.as<unsigned long long>() + 4 * p);
            TC_LAUNCH("k_masked_product");
        }
        TC_CUDA(cudaMemcpyAsync(h, sums.p, sizeof(h), cudaMemcpyDeviceToHost, st));
        TC_CUDA(cudaStreamSynchronize(st));
    }
    const unsigned long long c[16] = {
        h[2] / 6,  h[0],      h[1] / 2,  h[4] / 2,  h[8] / 2,  h[12],     h[16],     h[17],
        h[13],     h[14] / 3, h[20] / 2, h[5] / 2,  h[9] / 2,  h[15],     h[21],     h[22] / 6};
    for (int t = 0; t < 16; ++t) out[t] = to_u128(c[t]);
    if (n < 3) out[0] = to_u128(0);
    return TC_OK;
}
