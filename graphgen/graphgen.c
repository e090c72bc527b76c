/*
 * graphgen.c - seeded synthetic directed-graph generators.
 *
 * These generators produce the arc lists that both the CPU oracle and the GPU census
 * library consume.  They hold none of the census arithmetic: their only job is to turn
 * a seed into a clean list of distinct, loop-free directed arcs with the shape of the
 * paper's scale-free workloads (Sec. 5: power-law out-degree distributions).
 *
 * Random numbers come from one counter-based generator: the splitmix64 finaliser
 * (Steele, Lea and Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014)
 * applied to key + (i+1)*0x9E3779B97F4A7C15.  Draw i of a stream depends only on
 * (seed, stream tag, i), so the parallel loops below give the same graph for any
 * thread count.
 *
 * Workload definitions implemented here:
 *   - R-MAT (Chakrabarti, Zhan, Faloutsos 2004): each arc descends `scale` levels of
 *     the adjacency matrix, choosing quadrant (src bit, dst bit) = (0,0) with prob. a,
 *     (0,1) with b, (1,0) with c and (1,1) with d = 1-a-b-c.  No noise.  Vertex ids are
 *     then relabelled by a seeded random permutation so locality is not free.
 *   - Chung-Lu: out-weight of vertex j is (j+1)^(-1/(gamma-1)), scaled to the requested
 *     mean degree and capped at n-1; in-weights are a seeded permutation of the
 *     out-weights; mean_deg*n arcs are drawn with source ~ w_out and target ~ w_in.
 *   - Cleaning: self-loops and duplicate arcs are dropped.
 *   - Reciprocation: afterwards every arc (x,y) whose reverse is absent gets (y,x)
 *     added with probability p, decided by draw i of a separate stream, where i is
 *     the arc's index in the sorted clean list.
 * Output arcs are sorted by (src, dst).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define GOLDEN 0x9E3779B97F4A7C15ull

static inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static inline uint64_t ctr_rand(uint64_t key, uint64_t i) { return mix64(key + (i + 1) * GOLDEN); }
static inline uint64_t stream_key(uint64_t seed, uint64_t tag) { return mix64(mix64(seed + GOLDEN) ^ tag); }
/* uniform double in [0,1) from the top 53 bits */
static inline double u01(uint64_t r) { return (double)(r >> 11) * (1.0 / 9007199254740992.0); }
/* uniform integer in [0, bound) by the multiply-high method (bias < bound / 2^64) */
static inline uint64_t below(uint64_t r, uint64_t bound) { return (uint64_t)(((unsigned __int128)r * bound) >> 64); }

enum { TAG_RMAT = 0x524d4154, TAG_PERM = 0x5045524d, TAG_RECIP = 0x52454350,
       TAG_CLW = 0x434c5750, TAG_CLA = 0x434c4152, TAG_SIZE = 0x53495a45 };

/* ---------------------------------------------------------------- sorting (keys) */
/* LSD radix sort of 64-bit keys with 16-bit digits; digits that are constant over the
 * whole array are skipped.  Each thread histograms and scatters its own contiguous block,
 * in thread order, so every pass is stable.  Returns a pointer to whichever buffer holds
 * the result. */
static uint64_t* radix_sort_u64(uint64_t* a, uint64_t* tmp, uint64_t cnt) {
    int T = 1;
#ifdef _OPENMP
    /* one thread when already inside a parallel region (nested regions get one thread) */
    T = (cnt >= (1u << 20) && !omp_in_parallel()) ? omp_get_max_threads() : 1;
#endif
    size_t* hist = (size_t*)malloc(sizeof(size_t) * 65536 * (size_t)T);
    for (int pass = 0; pass < 4; ++pass) {
        int sh = pass * 16;
        memset(hist, 0, sizeof(size_t) * 65536 * (size_t)T);
#pragma omp parallel num_threads(T)
        {
            int t = 0;
#ifdef _OPENMP
            t = omp_get_thread_num();
#endif
            uint64_t b0 = cnt * (uint64_t)t / (uint64_t)T, b1 = cnt * (uint64_t)(t + 1) / (uint64_t)T;
            size_t* h = hist + 65536 * (size_t)t;
            for (uint64_t i = b0; i < b1; ++i) h[(a[i] >> sh) & 0xffff]++;
        }
        int only = 0;
        for (int d = 0; d < 65536 && !only; ++d) {
            size_t tot = 0;
            for (int t = 0; t < T; ++t) tot += hist[65536 * (size_t)t + d];
            if (tot == cnt) only = 1;
        }
        if (only) continue;
        size_t s = 0;
        for (int d = 0; d < 65536; ++d)
            for (int t = 0; t < T; ++t) { size_t* h = &hist[65536 * (size_t)t + d]; size_t c = *h; *h = s; s += c; }
#pragma omp parallel num_threads(T)
        {
            int t = 0;
#ifdef _OPENMP
            t = omp_get_thread_num();
#endif
            uint64_t b0 = cnt * (uint64_t)t / (uint64_t)T, b1 = cnt * (uint64_t)(t + 1) / (uint64_t)T;
            size_t* h = hist + 65536 * (size_t)t;
            for (uint64_t i = b0; i < b1; ++i) tmp[h[(a[i] >> sh) & 0xffff]++] = a[i];
        }
        uint64_t* t = a; a = tmp; tmp = t;
    }
    free(hist);
    return a;
}

/* Keep the entries with flag set, in order (flag[i] in {0, 1}); returns the count. */
static uint64_t compact_flagged(uint64_t* k, const uint8_t* flag, uint64_t cnt) {
    uint64_t o = 0;
    for (uint64_t i = 0; i < cnt; ++i) if (flag[i]) k[o++] = k[i];
    return o;
}

/* Drop loops (already excluded by caller) and duplicates from sorted keys; returns count */
static uint64_t unique_sorted(uint64_t* k, uint64_t cnt) {
    uint64_t o = 0;
    for (uint64_t i = 0; i < cnt; ++i)
        if (o == 0 || k[i] != k[o - 1]) k[o++] = k[i];
    return o;
}

static int key_present(const uint64_t* k, uint64_t cnt, uint64_t x) {
    uint64_t lo = 0, hi = cnt;
    while (lo < hi) { uint64_t mid = (lo + hi) >> 1; if (k[mid] < x) lo = mid + 1; else hi = mid; }
    return lo < cnt && k[lo] == x;
}

/* keys (src<<32|dst), loop-free, possibly duplicated -> sorted clean reciprocated arcs */
static int64_t finish_arcs(uint64_t* keys, uint64_t cnt, double recip, uint64_t seed,
                           uint32_t** src_out, uint32_t** dst_out) {
    uint64_t* tmp = (uint64_t*)malloc(sizeof(uint64_t) * (cnt ? cnt : 1));
    if (!tmp) return -1;
    uint64_t* s = radix_sort_u64(keys, tmp, cnt);
    uint64_t* other = (s == keys) ? tmp : keys;
    uint64_t m = unique_sorted(s, cnt);
    /* reciprocation: decisions depend only on (seed, index in sorted clean list) */
    uint64_t rk = stream_key(seed, TAG_RECIP);
    uint8_t* addf = (uint8_t*)malloc(m ? m : 1);
    if (!addf) { free(tmp); return -1; }
#pragma omp parallel for schedule(static) if (m >= (1u << 16))
    for (int64_t i = 0; i < (int64_t)m; ++i) {
        uint64_t x = s[i] >> 32, y = s[i] & 0xffffffffull;
        uint64_t rev = (y << 32) | x;
        other[i] = rev;
        addf[i] = recip > 0.0 && u01(ctr_rand(rk, (uint64_t)i)) < recip && !key_present(s, m, rev);
    }
    uint64_t add = compact_flagged(other, addf, m);
    free(addf);
    uint64_t tot = m + add;
    uint64_t* all = (uint64_t*)malloc(sizeof(uint64_t) * (tot ? tot : 1));
    uint64_t* all_tmp = (uint64_t*)malloc(sizeof(uint64_t) * (tot ? tot : 1));
    if (!all || !all_tmp) { free(tmp); free(all); free(all_tmp); return -1; }
    memcpy(all, s, sizeof(uint64_t) * m);
    memcpy(all + m, other, sizeof(uint64_t) * add);
    free(tmp);
    uint64_t* fin = radix_sort_u64(all, all_tmp, tot);
    uint32_t* so = (uint32_t*)malloc(sizeof(uint32_t) * (tot ? tot : 1));
    uint32_t* d_o = (uint32_t*)malloc(sizeof(uint32_t) * (tot ? tot : 1));
    if (!so || !d_o) { free(all); free(all_tmp); free(so); free(d_o); return -1; }
    for (uint64_t i = 0; i < tot; ++i) { so[i] = (uint32_t)(fin[i] >> 32); d_o[i] = (uint32_t)fin[i]; }
    free(all); free(all_tmp);
    *src_out = so; *dst_out = d_o;
    return (int64_t)tot;
}

/* Seeded Fisher-Yates permutation of 0..n-1 */
static void seeded_perm(uint32_t* p, uint32_t n, uint64_t key) {
    for (uint32_t i = 0; i < n; ++i) p[i] = i;
    for (uint64_t i = n; i > 1; --i) {
        uint64_t j = below(ctr_rand(key, i), i);
        uint32_t t = p[i - 1]; p[i - 1] = p[j]; p[j] = t;
    }
}

void gg_free(void* p) { free(p); }

/* R-MAT digraph, cleaned and reciprocated.  Returns the arc count, or -1 on error. */
int64_t gg_rmat(uint32_t scale, uint32_t edge_factor, double a, double b, double c,
                double recip, uint64_t seed, int permute, uint32_t** src_out, uint32_t** dst_out) {
    if (scale < 1 || scale > 30) return -1;
    uint64_t n = 1ull << scale;
    uint64_t draws = n * edge_factor;
    uint64_t* keys = (uint64_t*)malloc(sizeof(uint64_t) * (draws ? draws : 1));
    uint32_t* perm = (uint32_t*)malloc(sizeof(uint32_t) * n);
    if (!keys || !perm) { free(keys); free(perm); return -1; }
    /* quadrant thresholds on a 32-bit uniform: two levels per 64-bit draw */
    const double two32 = 4294967296.0;
    uint64_t ta = (uint64_t)(a * two32), tab = (uint64_t)((a + b) * two32), tabc = (uint64_t)((a + b + c) * two32);
    uint64_t rk = stream_key(seed, TAG_RMAT);
    uint64_t words = (scale + 1) / 2;
    if (permute) seeded_perm(perm, (uint32_t)n, stream_key(seed, TAG_PERM));
    else for (uint64_t i = 0; i < n; ++i) perm[i] = (uint32_t)i;
    int64_t kept = 0;
    uint8_t* keep = (uint8_t*)malloc(draws ? draws : 1);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)draws; ++i) {
        uint64_t sidx = 0, didx = 0;
        for (uint64_t w = 0; w < words; ++w) {
            uint64_t r = ctr_rand(rk, (uint64_t)i * words + w);
            for (int h = 0; h < 2; ++h) {
                uint64_t lvl = w * 2 + h;
                if (lvl >= scale) break;
                uint64_t x = (r >> (32 * h)) & 0xffffffffull;
                uint64_t sb, db;
                if (x < ta) { sb = 0; db = 0; }
                else if (x < tab) { sb = 0; db = 1; }
                else if (x < tabc) { sb = 1; db = 0; }
                else { sb = 1; db = 1; }
                sidx |= sb << (scale - 1 - lvl);
                didx |= db << (scale - 1 - lvl);
            }
        }
        uint64_t s = perm[sidx], d = perm[didx];
        keys[i] = (s << 32) | d;
        keep[i] = (s != d);
    }
    kept = (int64_t)compact_flagged(keys, keep, draws);
    free(keep); free(perm);
    int64_t r = finish_arcs(keys, (uint64_t)kept, recip, seed, src_out, dst_out);
    free(keys);
    return r;
}

/* Chung-Lu digraph with power-law weights (exponent gamma), cleaned and reciprocated.
 * `graph_index` selects an independent sub-stream so that many graphs can share a seed. */
int64_t gg_chung_lu(uint32_t n, double mean_deg, double gamma, double recip, uint64_t seed,
                    uint64_t graph_index, uint32_t** src_out, uint32_t** dst_out) {
    if (n < 2) return -1;
    uint64_t gseed = mix64(seed ^ (graph_index * GOLDEN + 0x1234567ull));
    double* wout = (double*)malloc(sizeof(double) * n);
    double* cout_ = (double*)malloc(sizeof(double) * n);
    double* cin = (double*)malloc(sizeof(double) * n);
    uint32_t* perm = (uint32_t*)malloc(sizeof(uint32_t) * n);
    uint64_t draws = (uint64_t)llround(mean_deg * (double)n);
    uint64_t* keys = (uint64_t*)malloc(sizeof(uint64_t) * (draws ? draws : 1));
    if (!wout || !cout_ || !cin || !perm || !keys) { free(wout); free(cout_); free(cin); free(perm); free(keys); return -1; }
    double ex = 1.0 / (gamma - 1.0), sum = 0.0;
    for (uint32_t j = 0; j < n; ++j) { wout[j] = pow((double)j + 1.0, -ex); sum += wout[j]; }
    double sc = mean_deg * (double)n / sum;
    for (uint32_t j = 0; j < n; ++j) { wout[j] *= sc; if (wout[j] > (double)(n - 1)) wout[j] = (double)(n - 1); }
    seeded_perm(perm, n, stream_key(gseed, TAG_CLW));
    double so = 0.0, si = 0.0;
    for (uint32_t j = 0; j < n; ++j) { so += wout[j]; cout_[j] = so; si += wout[perm[j]]; cin[j] = si; }
    uint64_t ak = stream_key(gseed, TAG_CLA);
    uint8_t* keep = (uint8_t*)malloc(draws ? draws : 1);
    if (!keep) { free(wout); free(cout_); free(cin); free(perm); free(keys); return -1; }
#pragma omp parallel for schedule(static) if (draws >= (1u << 16))
    for (int64_t ii = 0; ii < (int64_t)draws; ++ii) {
        uint64_t i = (uint64_t)ii;
        double x = u01(ctr_rand(ak, 2 * i)) * so, y = u01(ctr_rand(ak, 2 * i + 1)) * si;
        uint32_t lo = 0, hi = n - 1;
        while (lo < hi) { uint32_t mid = (lo + hi) >> 1; if (cout_[mid] <= x) lo = mid + 1; else hi = mid; }
        uint32_t s = lo;
        lo = 0; hi = n - 1;
        while (lo < hi) { uint32_t mid = (lo + hi) >> 1; if (cin[mid] <= y) lo = mid + 1; else hi = mid; }
        uint32_t d = lo;
        keys[i] = ((uint64_t)s << 32) | d;
        keep[i] = (s != d);
    }
    uint64_t kept = compact_flagged(keys, keep, draws);
    free(keep);
    free(wout); free(cout_); free(cin); free(perm);
    int64_t r = finish_arcs(keys, kept, recip, gseed, src_out, dst_out);
    free(keys);
    return r;
}

/* k sizes floor(exp(U(ln lo, ln hi))), clamped to [lo, hi] */
void gg_loguniform_sizes(uint32_t k, double lo, double hi, uint64_t seed, uint32_t* out) {
    uint64_t key = stream_key(seed, TAG_SIZE);
    double a = log(lo), b = log(hi);
    for (uint32_t i = 0; i < k; ++i) {
        double v = floor(exp(a + (b - a) * u01(ctr_rand(key, i))));
        if (v < lo) v = lo;
        if (v > hi) v = hi;
        out[i] = (uint32_t)v;
    }
}

/* k Chung-Lu graphs of sizes n[i] (graph i uses sub-stream i), generated in parallel.
 * Arcs of graph i are written to src/dst [arc_off[i], arc_off[i+1]); returns the total arc
 * count or -1.  The caller frees *src_out, *dst_out, *arc_off_out with gg_free. */
int64_t gg_chung_lu_batch(uint32_t k, const uint32_t* n, double mean_deg, double gamma, double recip, uint64_t seed,
                          uint32_t** src_out, uint32_t** dst_out, uint64_t** arc_off_out) {
    uint32_t** ss = (uint32_t**)calloc(k ? k : 1, sizeof(uint32_t*));
    uint32_t** dd = (uint32_t**)calloc(k ? k : 1, sizeof(uint32_t*));
    int64_t* cnt = (int64_t*)calloc(k ? k : 1, sizeof(int64_t));
    uint64_t* off = (uint64_t*)malloc(sizeof(uint64_t) * (k + 1ull));
    if (!ss || !dd || !cnt || !off) { free(ss); free(dd); free(cnt); free(off); return -1; }
    int failed = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : failed)
    for (int64_t i = 0; i < (int64_t)k; ++i) {
        cnt[i] = gg_chung_lu(n[i], mean_deg, gamma, recip, seed, (uint64_t)i, &ss[i], &dd[i]);
        if (cnt[i] < 0) failed = 1;
    }
    int64_t tot = 0;
    off[0] = 0;
    for (uint32_t i = 0; i < k; ++i) { off[i + 1] = off[i] + (uint64_t)(cnt[i] > 0 ? cnt[i] : 0); }
    tot = (int64_t)off[k];
    uint32_t* so = (uint32_t*)malloc(sizeof(uint32_t) * (tot ? tot : 1));
    uint32_t* d_o = (uint32_t*)malloc(sizeof(uint32_t) * (tot ? tot : 1));
    if (!so || !d_o) failed = 1;
    for (uint32_t i = 0; i < k; ++i) {
        if (!failed && cnt[i] > 0) {
            memcpy(so + off[i], ss[i], sizeof(uint32_t) * cnt[i]);
            memcpy(d_o + off[i], dd[i], sizeof(uint32_t) * cnt[i]);
        }
        free(ss[i]);
        free(dd[i]);
    }
    free(ss); free(dd); free(cnt);
    if (failed) { free(so); free(d_o); free(off); return -1; }
    *src_out = so; *dst_out = d_o; *arc_off_out = off;
    return tot;
}
