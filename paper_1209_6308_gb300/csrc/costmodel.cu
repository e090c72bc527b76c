// costmodel.cu - the learned per-vertex cost model that schedules the census (which vertices'
// pairs are split into how many CTA work items).  It only reorders work: counts never depend
// on it.
//
// Features of vertex x (relabelled id): log1p of its out-degree, in-degree, symmetric degree
// and the sum of its neighbours' degrees.  Network: 4 -> 32 -> 32 -> 1, tanh hidden units,
// linear output predicting log(SM cycles) of x's census work (standardised inputs, centred
// target).  Weights are held as FP16 for the forward pass with FP32 accumulation; the Adam
// optimiser keeps an FP32 master copy.  Training, gradients and inference are kernels here.
//
// Parameter layout (floats): W1[32][4], b1[32], W2[32][32], b2[32], W3[32], b3.
#include <cuda_fp16.h>

#include <cmath>
#include <cstring>
#include <random>
#include <vector>

#include "graph.cuh"
#include "plan.cuh"

namespace tc {
namespace {

constexpr int kIn = 4, kH = 32;
constexpr int kW1 = 0, kB1 = kW1 + kH * kIn, kW2 = kB1 + kH, kB2 = kW2 + kH * kH, kW3 = kB2 + kH, kB3 = kW3 + kH;
constexpr int kNP = kB3 + 1;   // 1249 parameters
constexpr int kTile = 128;     // samples per block iteration in the gradient kernel
constexpr int kMT = 256;       // threads of the MLP kernels

struct Norm {
    float mean[kIn], inv_std[kIn];
    float tmean;
};

// ---------------------------------------------------------------- features
__global__ void k_features(const uint64_t* __restrict__ off, const uint32_t* __restrict__ adj, uint32_t n,
                           float4* __restrict__ feat) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x / 32);
    for (uint64_t x = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) / 32; x < n; x += warps) {
        const uint64_t b = off[x], e = off[x + 1];
        uint32_t o = 0, in = 0;
        double nb = 0.0;
        for (uint64_t i = b + lane; i < e; i += 32) {
            const uint32_t w = adj[i], y = w >> 2;
            o += w & 1u;
            in += (w >> 1) & 1u;
            nb += (double)(off[y + 1] - off[y]);
        }
        o = __reduce_add_sync(0xffffffffu, o);
        in = __reduce_add_sync(0xffffffffu, in);
        for (int s = 16; s; s >>= 1) nb += __shfl_xor_sync(0xffffffffu, nb, s);
        if (lane == 0) feat[x] = make_float4(log1pf((float)o), log1pf((float)in), log1pf((float)(e - b)), (float)log1p(nb));
    }
}

// Training samples: vertices with measured cycles; features, log(cycles), and the plain
// schedule's work units of the same vertex (for the cycles -> plan-units calibration).  One
// warp per vertex.
__global__ void k_samples(GraphDev g, const float4* __restrict__ feat, const unsigned long long* __restrict__ vcost,
                          uint32_t chunk, uint32_t warp_max, int algo, uint32_t cap, float4* __restrict__ sx,
                          float* __restrict__ sy, uint32_t* cnt, double* sums) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t x = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; x < g.n; x += warps) {
        const unsigned long long c = vcost[x];
        const uint64_t ubase = g.off[x];
        const uint32_t du = (uint32_t)(g.off[x + 1] - ubase), upx = g.up[x];
        if (!c || du <= warp_max) continue;   // CTA-item vertices only: what the plan splits
        const uint32_t chunks = (du + chunk - 1) / chunk;
        unsigned long long W = 0;
        for (uint32_t j = upx + lane; j < du; j += 32) W += pair_units(g, (uint32_t)x, ubase, du, upx, j, chunks, algo);
        for (int o = 16; o; o >>= 1) W += __shfl_xor_sync(0xffffffffu, W, o);
        if (lane == 0) {
            const uint32_t i = atomicAdd(cnt, 1u);
            if (i < cap) {
                sx[i] = feat[x];
                sy[i] = logf((float)c);
                atomicAdd(&sums[0], (double)W);
                atomicAdd(&sums[1], (double)c);
            }
        }
    }
}

// ---------------------------------------------------------------- MLP
__device__ __forceinline__ void load_params(const __half* __restrict__ wh, float* W) {
    for (int p = threadIdx.x; p < kNP; p += blockDim.x) W[p] = __half2float(wh[p]);
}

__device__ __forceinline__ float norm_in(const float4 f, int k, const Norm& nm) {
    const float v = k == 0 ? f.x : k == 1 ? f.y : k == 2 ? f.z : f.w;
    return (v - nm.mean[k]) * nm.inv_std[k];
}

// Loss = mean((y - t)^2) over the samples and its gradient, accumulated into G[0..kNP) and
// G[kNP] (loss); G must be zeroed.
__global__ void __launch_bounds__(kMT) k_mlp_grad(const float4* __restrict__ X, const float* __restrict__ T,
                                                  uint32_t count, const __half* __restrict__ wh, Norm nm, float* G) {
    extern __shared__ float sm[];
    float* W = sm;                                  // [kNP]
    float* gs = W + kNP;                            // [kNP + 1]
    float* x = gs + kNP + 1;                        // [kTile][kIn]
    float* h1 = x + kTile * kIn;                    // [kTile][kH + 1]
    float* h2 = h1 + kTile * (kH + 1);
    float* d2 = h2 + kTile * (kH + 1);
    float* d1 = d2 + kTile * (kH + 1);
    float* dy = d1 + kTile * (kH + 1);              // [kTile]
    const int tid = threadIdx.x;
    load_params(wh, W);
    for (int p = tid; p <= kNP; p += kMT) gs[p] = 0.f;
    const float inv_n = 1.f / (float)(count ? count : 1);
    __syncthreads();
    for (uint64_t base = (uint64_t)blockIdx.x * kTile; base < count; base += (uint64_t)gridDim.x * kTile) {
        for (int i = tid; i < kTile * kIn; i += kMT) {
            const int s = i / kIn, k = i % kIn;
            const uint64_t g = base + s;
            x[i] = g < count ? norm_in(X[g], k, nm) : 0.f;
        }
        __syncthreads();
        for (int i = tid; i < kTile * kH; i += kMT) {
            const int s = i / kH, j = i % kH;
            float z = W[kB1 + j];
#pragma unroll
            for (int k = 0; k < kIn; ++k) z += W[kW1 + j * kIn + k] * x[s * kIn + k];
            h1[s * (kH + 1) + j] = tanhf(z);
        }
        __syncthreads();
        for (int i = tid; i < kTile * kH; i += kMT) {
            const int s = i / kH, j = i % kH;
            float z = W[kB2 + j];
#pragma unroll 8
            for (int k = 0; k < kH; ++k) z += W[kW2 + j * kH + k] * h1[s * (kH + 1) + k];
            h2[s * (kH + 1) + j] = tanhf(z);
        }
        __syncthreads();
        float loss = 0.f;
        for (int s = tid; s < kTile; s += kMT) {
            const uint64_t g = base + s;
            float y = W[kB3];
#pragma unroll 8
            for (int k = 0; k < kH; ++k) y += W[kW3 + k] * h2[s * (kH + 1) + k];
            const float err = g < count ? y - (T[g] - nm.tmean) : 0.f;
            dy[s] = 2.f * err * inv_n;
            loss += err * err * inv_n;
        }
        if (loss != 0.f) atomicAdd(&gs[kNP], loss);
        __syncthreads();
        for (int i = tid; i < kTile * kH; i += kMT) {
            const int s = i / kH, j = i % kH;
            const float h = h2[s * (kH + 1) + j];
            d2[s * (kH + 1) + j] = dy[s] * W[kW3 + j] * (1.f - h * h);
        }
        __syncthreads();
        for (int i = tid; i < kTile * kH; i += kMT) {
            const int s = i / kH, j = i % kH;
            float a = 0.f;
#pragma unroll 8
            for (int k = 0; k < kH; ++k) a += d2[s * (kH + 1) + k] * W[kW2 + k * kH + j];
            const float h = h1[s * (kH + 1) + j];
            d1[s * (kH + 1) + j] = a * (1.f - h * h);
        }
        __syncthreads();
        // parameter gradients summed over the tile's samples
        for (int p = tid; p < kNP; p += kMT) {
            float a = 0.f;
            if (p < kB1) {
                const int j = (p - kW1) / kIn, k = (p - kW1) % kIn;
                for (int s = 0; s < kTile; ++s) a += d1[s * (kH + 1) + j] * x[s * kIn + k];
            } else if (p < kW2) {
                const int j = p - kB1;
                for (int s = 0; s < kTile; ++s) a += d1[s * (kH + 1) + j];
            } else if (p < kB2) {
                const int j = (p - kW2) / kH, k = (p - kW2) % kH;
                for (int s = 0; s < kTile; ++s) a += d2[s * (kH + 1) + j] * h1[s * (kH + 1) + k];
            } else if (p < kW3) {
                const int j = p - kB2;
                for (int s = 0; s < kTile; ++s) a += d2[s * (kH + 1) + j];
            } else if (p < kB3) {
                const int j = p - kW3;
                for (int s = 0; s < kTile; ++s) a += dy[s] * h2[s * (kH + 1) + j];
            } else {
                for (int s = 0; s < kTile; ++s) a += dy[s];
            }
            gs[p] += a;
        }
        __syncthreads();
    }
    for (int p = tid; p <= kNP; p += kMT)
        if (gs[p] != 0.f) atomicAdd(&G[p], gs[p]);
}

// Adam step on the FP32 master weights; refreshes the FP16 copy and clears the gradient.
__global__ void k_adam(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v, float* __restrict__ g,
                       __half* __restrict__ wh, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= kNP) return;
    const float gp = g[p];
    const float mp = b1 * m[p] + (1.f - b1) * gp, vp = b2 * v[p] + (1.f - b2) * gp * gp;
    m[p] = mp;
    v[p] = vp;
    const float wn = w[p] - lr * (mp / c1) / (sqrtf(vp / c2) + eps);
    w[p] = wn;
    wh[p] = __float2half(wn);
    g[p] = 0.f;
}

__global__ void k_zero(float* g, int count) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) g[i] = 0.f;
}

// Predicted cycles (exp of the network output) times `scale`.
__global__ void __launch_bounds__(kMT) k_mlp_infer(const float4* __restrict__ X, uint32_t count,
                                                   const __half* __restrict__ wh, Norm nm, float scale,
                                                   float* __restrict__ out) {
    __shared__ float W[kNP];
    load_params(wh, W);
    __syncthreads();
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < count; i += (uint64_t)gridDim.x * blockDim.x) {
        const float4 f = X[i];
        float xi[kIn], h1[kH];
#pragma unroll
        for (int k = 0; k < kIn; ++k) xi[k] = norm_in(f, k, nm);
#pragma unroll
        for (int j = 0; j < kH; ++j) {
            float z = W[kB1 + j];
#pragma unroll
            for (int k = 0; k < kIn; ++k) z += W[kW1 + j * kIn + k] * xi[k];
            h1[j] = tanhf(z);
        }
        float y = W[kB3];
        for (int j = 0; j < kH; ++j) {
            float z = W[kB2 + j];
#pragma unroll
            for (int k = 0; k < kH; ++k) z += W[kW2 + j * kH + k] * h1[k];
            y += W[kW3 + j] * tanhf(z);
        }
        out[i] = expf(y + nm.tmean) * scale;
    }
}

// sums of each feature, its square and of the target (double atomics per warp)
__global__ void k_norm_stats(const float4* __restrict__ X, const float* __restrict__ T, uint32_t count, double* acc) {
    double a[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < count; i += (uint64_t)gridDim.x * blockDim.x) {
        const float4 f = X[i];
        const float v[4] = {f.x, f.y, f.z, f.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) { a[k] += v[k]; a[4 + k] += (double)v[k] * v[k]; }
        a[8] += T[i];
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        for (int s = 16; s; s >>= 1) a[k] += __shfl_xor_sync(0xffffffffu, a[k], s);
        if ((threadIdx.x & 31) == 0) atomicAdd(&acc[k], a[k]);
    }
}

size_t grad_smem() { return sizeof(float) * (2 * kNP + 1 + kTile * kIn + 4 * kTile * (kH + 1) + kTile); }

}  // namespace
}  // namespace tc

struct tc_costmodel {
    tc::DevBuf w, m, v, g, wh;
    tc::Norm norm{};
    float kappa = 1.f;           // plan units per predicted cycle
    uint64_t step = 0;
};

using namespace tc;

namespace {
tc_status cm_prepare(cudaStream_t st) {
    (void)st;
    static bool done[64] = {};
    int dev = 0;
    TC_CUDA(cudaGetDevice(&dev));
    if (dev >= 0 && dev < 64 && !done[dev]) {
        TC_CUDA(cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)grad_smem()));
        done[dev] = true;
    }
    return TC_OK;
}
}  // namespace

extern "C" {

uint32_t tc_costmodel_num_params(void) { return (uint32_t)kNP; }

tc_status tc_costmodel_create(uint64_t seed, tc_costmodel** out) {
    if (!out) return fail(TC_ERR_ARG, "null argument");
    *out = nullptr;
    tc_costmodel* c = new tc_costmodel();
    std::vector<float> w(kNP, 0.f);
    std::mt19937_64 rng(seed);
    std::normal_distribution<float> nd(0.f, 1.f);
    for (int p = kW1; p < kB1; ++p) w[p] = nd(rng) * std::sqrt(1.f / kIn);
    for (int p = kW2; p < kB2; ++p) w[p] = nd(rng) * std::sqrt(1.f / kH);
    for (int p = kW3; p < kB3; ++p) w[p] = nd(rng) * std::sqrt(1.f / kH);
    for (int k = 0; k < kIn; ++k) { c->norm.mean[k] = 0.f; c->norm.inv_std[k] = 1.f; }
    tc_status s = c->w.alloc_persistent(sizeof(float) * kNP);
    if (s == TC_OK) s = c->m.alloc_persistent(sizeof(float) * kNP);
    if (s == TC_OK) s = c->v.alloc_persistent(sizeof(float) * kNP);
    if (s == TC_OK) s = c->g.alloc_persistent(sizeof(float) * (kNP + 1));
    if (s == TC_OK) s = c->wh.alloc_persistent(sizeof(__half) * kNP);
    if (s == TC_OK) s = tc_costmodel_set_params(c, w.data());
    if (s == TC_OK && (cudaMemset(c->m.p, 0, sizeof(float) * kNP) != cudaSuccess ||
                       cudaMemset(c->v.p, 0, sizeof(float) * kNP) != cudaSuccess ||
                       cudaMemset(c->g.p, 0, sizeof(float) * (kNP + 1)) != cudaSuccess))
        s = fail(TC_ERR_CUDA, "cost model: clearing optimiser state failed");
    if (s != TC_OK) {
        delete c;
        return s;
    }
    *out = c;
    return TC_OK;
}

void tc_costmodel_destroy(tc_costmodel* c) {
    if (!c) return;
    cudaDeviceSynchronize();
    delete c;
}

tc_status tc_costmodel_set_params(tc_costmodel* c, const float* host) {
    if (!c || !host) return fail(TC_ERR_ARG, "null argument");
    std::vector<__half> h(kNP);
    for (int p = 0; p < kNP; ++p) h[p] = __float2half(host[p]);
    TC_CUDA(cudaMemcpy(c->w.p, host, sizeof(float) * kNP, cudaMemcpyHostToDevice));
    TC_CUDA(cudaMemcpy(c->wh.p, h.data(), sizeof(__half) * kNP, cudaMemcpyHostToDevice));
    return TC_OK;
}

tc_status tc_costmodel_get_params(const tc_costmodel* c, float* host) {
    if (!c || !host) return fail(TC_ERR_ARG, "null argument");
    TC_CUDA(cudaMemcpy(host, c->w.p, sizeof(float) * kNP, cudaMemcpyDeviceToHost));
    return TC_OK;
}

tc_status tc_costmodel_set_norm(tc_costmodel* c, const float mean[4], const float std_[4], float target_mean,
                                float kappa) {
    if (!c || !mean || !std_) return fail(TC_ERR_ARG, "null argument");
    for (int k = 0; k < kIn; ++k) {
        if (!(std_[k] > 0.f)) return fail(TC_ERR_ARG, "feature standard deviation must be > 0");
        c->norm.mean[k] = mean[k];
        c->norm.inv_std[k] = 1.f / std_[k];
    }
    c->norm.tmean = target_mean;
    c->kappa = kappa;
    return TC_OK;
}

tc_status tc_costmodel_get_norm(const tc_costmodel* c, float mean[4], float std_[4], float* target_mean, float* kappa) {
    if (!c) return fail(TC_ERR_ARG, "null argument");
    for (int k = 0; k < kIn; ++k) {
        if (mean) mean[k] = c->norm.mean[k];
        if (std_) std_[k] = 1.f / c->norm.inv_std[k];
    }
    if (target_mean) *target_mean = c->norm.tmean;
    if (kappa) *kappa = c->kappa;
    return TC_OK;
}

tc_status tc_graph_features(const tc_graph* g, void* stream, float* d_feat4) {
    if (!g || !d_feat4) return fail(TC_ERR_ARG, "null argument");
    const GraphStore& s = g->s;
    if (!s.n) return TC_OK;
    k_features<<<grid_for((uint64_t)s.n * 32, 256, 1u << 16), 256, 0, (cudaStream_t)stream>>>(
        s.off.as<uint64_t>(), s.adj.as<uint32_t>(), s.n, reinterpret_cast<float4*>(d_feat4));
    TC_LAUNCH("k_features");
    return TC_OK;
}

tc_status tc_costmodel_samples(const tc_graph* g, const uint64_t* d_vcost, const float* d_feat4, uint32_t capacity,
                               void* stream, float* d_x4, float* d_y, uint32_t* count, double* est_sum,
                               double* cycle_sum) {
    if (!g || !d_vcost || !d_feat4 || !d_x4 || !d_y || !count) return fail(TC_ERR_ARG, "null argument");
    const GraphStore& s = g->s;
    cudaStream_t st = (cudaStream_t)stream;
    Opts o;
    TC_TRY(resolve_opts(nullptr, &s.opts, &o));
    DevBuf cnt, sums;
    TC_TRY(cnt.alloc(sizeof(uint32_t), st));
    TC_TRY(sums.alloc(sizeof(double) * 2, st));
    TC_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(uint32_t), st));
    TC_CUDA(cudaMemsetAsync(sums.p, 0, sizeof(double) * 2, st));
    if (s.n) {
        k_samples<<<grid_for((uint64_t)s.n * 32, 256, 1u << 16), 256, 0, st>>>(
            s.dev(), reinterpret_cast<const float4*>(d_feat4), reinterpret_cast<const unsigned long long*>(d_vcost),
            o.chunk, o.warp_max_deg, (int)o.algo, capacity, reinterpret_cast<float4*>(d_x4), d_y, cnt.as<uint32_t>(),
            sums.as<double>());
        TC_LAUNCH("k_samples");
    }
    uint32_t c = 0;
    double hs[2] = {0, 0};
    TC_CUDA(cudaMemcpyAsync(&c, cnt.p, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    TC_CUDA(cudaMemcpyAsync(hs, sums.p, sizeof(hs), cudaMemcpyDeviceToHost, st));
    TC_CUDA(cudaStreamSynchronize(st));
    *count = c < capacity ? c : capacity;
    if (est_sum) *est_sum = hs[0];
    if (cycle_sum) *cycle_sum = hs[1];
    return TC_OK;
}

tc_status tc_costmodel_fit_norm(tc_costmodel* c, const float* d_x4, const float* d_y, uint32_t count, float kappa,
                                void* stream) {
    if (!c || !d_x4 || !d_y || !count) return fail(TC_ERR_ARG, "null argument or no samples");
    cudaStream_t st = (cudaStream_t)stream;
    DevBuf acc;
    TC_TRY(acc.alloc(sizeof(double) * 9, st));
    TC_CUDA(cudaMemsetAsync(acc.p, 0, sizeof(double) * 9, st));
    k_norm_stats<<<grid_for(count, 256, 1024), 256, 0, st>>>(reinterpret_cast<const float4*>(d_x4), d_y, count,
                                                              acc.as<double>());
    TC_LAUNCH("k_norm_stats");
    double h[9];
    TC_CUDA(cudaMemcpyAsync(h, acc.p, sizeof(h), cudaMemcpyDeviceToHost, st));
    TC_CUDA(cudaStreamSynchronize(st));
    float mean[4], sd[4];
    for (int k = 0; k < 4; ++k) {
        const double m = h[k] / count, var = h[4 + k] / count - m * m;
        mean[k] = (float)m;
        sd[k] = (float)std::sqrt(var > 1e-12 ? var : 1e-12);
    }
    return tc_costmodel_set_norm(c, mean, sd, (float)(h[8] / count), kappa);
}

tc_status tc_costmodel_grad(tc_costmodel* c, const float* d_x4, const float* d_y, uint32_t count, void* stream,
                            float* host_grad, float* host_loss) {
    if (!c || (count && (!d_x4 || !d_y))) return fail(TC_ERR_ARG, "null argument");
    cudaStream_t st = (cudaStream_t)stream;
    TC_TRY(cm_prepare(st));
    k_zero<<<8, 256, 0, st>>>(c->g.as<float>(), kNP + 1);
    TC_LAUNCH("k_zero");
    if (count) {
        const unsigned grid = grid_for((count + kTile - 1) / kTile, 1, 2 * (unsigned)sm_count());
        k_mlp_grad<<<grid, kMT, grad_smem(), st>>>(reinterpret_cast<const float4*>(d_x4), d_y, count,
                                                   c->wh.as<__half>(), c->norm, c->g.as<float>());
        TC_LAUNCH("k_mlp_grad");
    }
    std::vector<float> h(kNP + 1);
    TC_CUDA(cudaMemcpyAsync(h.data(), c->g.p, sizeof(float) * (kNP + 1), cudaMemcpyDeviceToHost, st));
    TC_CUDA(cudaStreamSynchronize(st));
    if (host_grad) std::memcpy(host_grad, h.data(), sizeof(float) * kNP);
    if (host_loss) *host_loss = h[kNP];
    k_zero<<<8, 256, 0, st>>>(c->g.as<float>(), kNP + 1);
    TC_LAUNCH("k_zero");
    return TC_OK;
}

tc_status tc_costmodel_train(tc_costmodel* c, const float* d_x4, const float* d_y, uint32_t count, uint32_t steps,
                             float lr, void* stream, float* final_loss) {
    if (!c || !d_x4 || !d_y) return fail(TC_ERR_ARG, "null argument");
    if (!count) return fail(TC_ERR_ARG, "no training samples");
    cudaStream_t st = (cudaStream_t)stream;
    TC_TRY(cm_prepare(st));
    k_zero<<<8, 256, 0, st>>>(c->g.as<float>(), kNP + 1);
    TC_LAUNCH("k_zero");
    const unsigned grid = grid_for((count + kTile - 1) / kTile, 1, 2 * (unsigned)sm_count());
    const float b1 = 0.9f, b2 = 0.999f;
    for (uint32_t it = 0; it < steps; ++it) {
        k_mlp_grad<<<grid, kMT, grad_smem(), st>>>(reinterpret_cast<const float4*>(d_x4), d_y, count,
                                                   c->wh.as<__half>(), c->norm, c->g.as<float>());
        TC_LAUNCH("k_mlp_grad");
        ++c->step;
        const float c1 = 1.f - std::pow(b1, (float)c->step), c2 = 1.f - std::pow(b2, (float)c->step);
        k_adam<<<(kNP + 255) / 256, 256, 0, st>>>(c->w.as<float>(), c->m.as<float>(), c->v.as<float>(), c->g.as<float>(),
                                                   c->wh.as<__half>(), lr, b1, b2, 1e-8f, c1, c2);
        TC_LAUNCH("k_adam");
    }
    if (final_loss) {
        float loss = 0.f;
        TC_TRY(tc_costmodel_grad(c, d_x4, d_y, count, stream, nullptr, &loss));
        *final_loss = loss;
    }
    return TC_OK;
}

tc_status tc_costmodel_predict(const tc_costmodel* c, const float* d_x4, uint32_t count, void* stream, float* d_out) {
    if (!c || (count && (!d_x4 || !d_out))) return fail(TC_ERR_ARG, "null argument");
    if (!count) return TC_OK;
    k_mlp_infer<<<grid_for(count, kMT, 4096), kMT, 0, (cudaStream_t)stream>>>(
        reinterpret_cast<const float4*>(d_x4), count, c->wh.as<__half>(), c->norm, 1.f, d_out);
    TC_LAUNCH("k_mlp_infer");
    return TC_OK;
}

tc_status tc_graph_attach_costmodel(tc_graph* g, const tc_costmodel* c, void* stream) {
    if (!g || !c) return fail(TC_ERR_ARG, "null argument");
    GraphStore& s = g->s;
    cudaStream_t st = (cudaStream_t)stream;
    DevBuf feat;
    TC_TRY(feat.alloc(sizeof(float4) * (s.n ? s.n : 1), st));
    TC_TRY(tc_graph_features(g, stream, feat.as<float>()));
    TC_TRY(s.cost.alloc_persistent(sizeof(float) * (s.n ? s.n : 1)));
    if (s.n) {
        k_mlp_infer<<<grid_for(s.n, kMT, 4096), kMT, 0, st>>>(feat.as<float4>(), s.n, c->wh.as<__half>(), c->norm,
                                                             c->kappa, s.cost.as<float>());
        TC_LAUNCH("k_mlp_infer");
    }
    TC_CUDA(cudaStreamSynchronize(st));
    // plans made with the learned schedule depend on the model: drop them
    for (auto& p : s.plans)
        if (p.valid && p.key.schedule == TC_SCHED_LEARNED) p.valid = false;
    return TC_OK;
}

}  // extern "C"
