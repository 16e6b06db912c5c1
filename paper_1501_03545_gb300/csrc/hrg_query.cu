// hrg_query.cu -- the neighbourhood queries of Algorithm 1 and the CSR rows.
//
// Algorithm 1 runs, for every vertex v in parallel, a range query for the
// hyperbolic circle of radius R around v and adds (v, w) for every w inside.
// Here a query visits every radial band, bounds its admissible angle by the
// closed-form window at the band's inner radius, reads the angular buckets
// that the window touches, and decides each candidate with
//   * an FP32 test of the scaled predicate with an undecided band of
//     relative half-width mu, and an FP64 recheck of the pairs inside it, or
//   * the FP64 predicate on every candidate (the plain double path).
// The same traversal runs twice: once to count degrees, once to write the
// neighbour ids into the caller's CSR, each row sorted by vertex id.
#include <cstdio>
#include "hrg_internal.h"

namespace hrg {

namespace {

enum { ST_CAND = 0, ST_RECHECK = 1, ST_EDGES = 2, ST_ERR = 7 };

// Candidate positions of query q in band j: up to two ranges [s0,e0) [s1,e1)
struct Ranges { int32_t s0, e0, s1, e1; uint64_t W; };

__device__ __forceinline__ Ranges band_ranges(const Plan &p, const int32_t *__restrict__ start, const PMS &q,
                                              uint64_t Aq, int j)
{
    Ranges rg;
    const int64_t b0 = p.base[j], b1 = p.base[j + 1];
    const int32_t s = __ldg(start + b0), e = __ldg(start + b1);
    rg.s1 = rg.e1 = 0;
    rg.W = kFullCircle;
    if (s == e) { rg.s0 = rg.e0 = 0; return rg; }
    const uint64_t W = window_halfwidth(p, q, j);
    rg.W = W;
    const int g = p.gbits[j];
    if (W == kFullCircle || g == 0) { rg.s0 = s; rg.e0 = e; return rg; }
    const uint64_t lo = Aq - W, hi = Aq + W;
    const int64_t blo = (int64_t)(lo >> (64 - g)), bhi = (int64_t)(hi >> (64 - g));
    if (lo <= hi) {
        rg.s0 = __ldg(start + b0 + blo);
        rg.e0 = __ldg(start + b0 + bhi + 1);
    } else {  // the window wraps through angle 0
        rg.s0 = __ldg(start + b0 + blo);
        rg.e0 = e;
        rg.s1 = s;
        rg.e1 = __ldg(start + b0 + bhi + 1);
    }
    return rg;
}

__device__ __forceinline__ bool within(uint64_t Aq, uint64_t Ac, uint64_t W)
{
    const uint64_t d = Ac - Aq;
    const uint64_t ad = (int64_t)d < 0 ? (0ull - d) : d;
    return ad <= W;
}

// Decide candidate position c for query qp.  Returns true for an edge.
template <bool F64>
__device__ __forceinline__ bool decide(const Plan &p, const QueryBufs &b, int32_t qp, const PMS &q,
                                       const PMS64 &q64, uint64_t Aq, int32_t c, uint64_t W,
                                       unsigned &n_cand, unsigned &n_re)
{
    if (c == qp) return false;
    const uint64_t Ac = __ldg(b.A + c);
    if (W != kFullCircle && !within(Aq, Ac, W)) return false;
    ++n_cand;
    if (F64) {
        const PMS64 c64 = b.pms64[c];
        return edge_pms64(p, q64, c64);
    } else {
        const PMS cc = b.pms[c];
        const float v = lhs32(q, cc, (int64_t)(Ac - Aq));
        if (v < p.rhs32 * (1.0f - p.mu)) return true;
        if (v > p.rhs32 * (1.0f + p.mu)) return false;
        ++n_re;
        return edge64(__ldg(b.r + q.id), __ldg(b.phi + q.id), __ldg(b.r + cc.id), __ldg(b.phi + cc.id),
                      p.coshR);
    }
}

__device__ __forceinline__ void add_stats(unsigned long long *stats, unsigned n_cand, unsigned n_re, unsigned n_edge)
{
    // warp-aggregated counters
    unsigned long long a = n_cand, r = n_re, e = n_edge;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        r += __shfl_down_sync(0xffffffffu, r, o);
        e += __shfl_down_sync(0xffffffffu, e, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (a) atomicAdd(&stats[ST_CAND], a);
        if (r) atomicAdd(&stats[ST_RECHECK], r);
        if (e) atomicAdd(&stats[ST_EDGES], e);
    }
}

__device__ __forceinline__ void classify_row(const QueryBufs &b, int32_t id, int32_t d)
{
    if (d > kSmemRow) {
        const int k = atomicAdd(&b.list_cnt[1], 1);
        b.big_rows[k] = id;
        atomicAdd((unsigned long long *)b.big_total, (unsigned long long)d);
    } else if (d > kRegRow) {
        const int k = atomicAdd(&b.list_cnt[0], 1);
        b.mid_rows[k] = id;
    }
}

// ---------------------------------------------------------------------------
// Thread per query (bands >= hub_bands).
// ---------------------------------------------------------------------------
template <bool F64, bool WRITE>
__global__ void __launch_bounds__(128) k_query_thread(Plan p, QueryBufs b, int32_t q_begin,
                                                      const int64_t *__restrict__ row_off,
                                                      int32_t *__restrict__ col_idx)
{
    const int32_t qp = q_begin + (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
    const bool active = qp < (int32_t)p.n;
    unsigned n_cand = 0, n_re = 0, n_edge = 0;
    if (active) {
        const PMS q = b.pms[qp];
        const uint64_t Aq = b.A[qp];
        PMS64 q64{};
        if (F64) q64 = b.pms64[qp];
        int64_t base = 0;
        int32_t deg = 0;
        if (WRITE) {
            base = row_off[q.id];
            deg = b.deg[q.id];
        }
        int32_t buf[kRegRow];
        int32_t cnt = 0;
        for (int j = 0; j < p.B; ++j) {
            const Ranges rg = band_ranges(p, b.start, q, Aq, j);
            for (int part = 0; part < 2; ++part) {
                const int32_t s = part ? rg.s1 : rg.s0, e = part ? rg.e1 : rg.e0;
                for (int32_t c = s; c < e; ++c) {
                    if (decide<F64>(p, b, qp, q, q64, Aq, c, rg.W, n_cand, n_re)) {
                        if (WRITE) {
                            const int32_t nb = b.pms[c].id;
                            if (deg <= kRegRow) {
                                // insertion into the sorted register list (cnt < deg <= kRegRow)
                                if (cnt < deg) {
                                    int32_t k = cnt;
                                    while (k > 0 && buf[k - 1] > nb) { buf[k] = buf[k - 1]; --k; }
                                    buf[k] = nb;
                                }
                            } else if (cnt < deg) {
                                col_idx[base + cnt] = nb;
                            }
                        }
                        ++cnt;
                    }
                }
            }
        }
        n_edge = cnt;
        if (WRITE) {
            if (cnt != deg) atomicOr((unsigned long long *)&b.stats[ST_ERR], 1ull);
            if (deg <= kRegRow)
                for (int32_t k = 0; k < cnt && k < deg; ++k) col_idx[base + k] = buf[k];
        } else {
            b.deg[q.id] = cnt;
            classify_row(b, q.id, cnt);
        }
    }
    if (!WRITE) add_stats(b.stats, n_cand, n_re, n_edge);
}

// ---------------------------------------------------------------------------
// CTA per query (hub bands): the candidates of each band are strided over
// the block's threads.
// ---------------------------------------------------------------------------
template <bool F64, bool WRITE>
__global__ void __launch_bounds__(256) k_query_cta(Plan p, QueryBufs b, const int64_t *__restrict__ row_off,
                                                   int32_t *__restrict__ col_idx)
{
    __shared__ int32_t s_cnt;
    __shared__ int32_t s_red[8];
    const int32_t qp = blockIdx.x;
    const PMS q = b.pms[qp];
    const uint64_t Aq = b.A[qp];
    PMS64 q64{};
    if (F64) q64 = b.pms64[qp];
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    int64_t base = 0;
    int32_t deg = 0;
    if (WRITE) {
        base = row_off[q.id];
        deg = b.deg[q.id];
    }
    unsigned n_cand = 0, n_re = 0;
    int32_t mine = 0;
    for (int j = 0; j < p.B; ++j) {
        const Ranges rg = band_ranges(p, b.start, q, Aq, j);
        for (int part = 0; part < 2; ++part) {
            const int32_t s = part ? rg.s1 : rg.s0, e = part ? rg.e1 : rg.e0;
            for (int32_t c = s + (int32_t)threadIdx.x; c < e; c += blockDim.x) {
                if (decide<F64>(p, b, qp, q, q64, Aq, c, rg.W, n_cand, n_re)) {
                    if (WRITE) {
                        const int32_t slot = atomicAdd(&s_cnt, 1);
                        if (slot < deg) col_idx[base + slot] = b.pms[c].id;
                    }
                    ++mine;
                }
            }
        }
    }
    // block sum of the degree
    int32_t v = mine;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t d = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) d += s_red[w];
        if (WRITE) {
            if (d != deg) atomicOr((unsigned long long *)&b.stats[ST_ERR], 1ull);
        } else {
            b.deg[q.id] = d;
            classify_row(b, q.id, d);
        }
    }
    if (!WRITE) add_stats(b.stats, n_cand, n_re, 0u);
    if (!WRITE && threadIdx.x == 0) {
        // edge count of this row (thread 0 adds it once)
        int32_t d = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) d += s_red[w];
        atomicAdd(&b.stats[ST_EDGES], (unsigned long long)d);
    }
}

// ---------------------------------------------------------------------------
// Row sorting.  Mid rows: one CTA, bitonic sort in shared memory.
// ---------------------------------------------------------------------------
__device__ void bitonic_smem(int32_t *s, int m)
{
    for (int k = 2; k <= m; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < m; i += blockDim.x) {
                const int l = i ^ j;
                if (l > i) {
                    const int32_t a = s[i], c = s[l];
                    const bool up = (i & k) == 0;
                    if ((a > c) == up) { s[i] = c; s[l] = a; }
                }
            }
            __syncthreads();
        }
    }
}

__global__ void __launch_bounds__(512) k_sort_mid(const QueryBufs b, const int64_t *__restrict__ row_off,
                                                  int32_t *__restrict__ col_idx)
{
    extern __shared__ int32_t sm[];
    const int32_t id = b.mid_rows[blockIdx.x];
    const int64_t base = row_off[id];
    const int len = (int)(row_off[id + 1] - base);
    int m = 1;
    while (m < len) m <<= 1;
    for (int i = threadIdx.x; i < m; i += blockDim.x) sm[i] = i < len ? col_idx[base + i] : 0x7fffffff;
    __syncthreads();
    bitonic_smem(sm, m);
    for (int i = threadIdx.x; i < len; i += blockDim.x) col_idx[base + i] = sm[i];
}

// Big rows: ids bucketed by value (bucket = id * nbk / n, order preserving),
// then every bucket (at most n / nbk <= kSmemRow ids) sorted in shared memory.
struct BigDesc { int64_t tmp_off; int32_t nbk; int32_t pad; };

__global__ void k_big_setup(const QueryBufs b, int n_big, const int64_t *__restrict__ row_off, int64_t n,
                            int32_t nbk, BigDesc *__restrict__ desc, int32_t *__restrict__ hist)
{
    // one thread per big row: tmp offsets are a prefix sum over big rows
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    int64_t acc = 0;
    for (int k = 0; k < n_big; ++k) {
        const int32_t id = b.big_rows[k];
        desc[k].tmp_off = acc;
        desc[k].nbk = nbk;
        acc += row_off[id + 1] - row_off[id];
    }
    (void)hist;
    (void)n;
}

__global__ void k_big_hist(const QueryBufs b, const int64_t *__restrict__ row_off, int64_t n, int32_t nbk,
                           const int32_t *__restrict__ col_idx, int32_t *__restrict__ hist)
{
    const int k = blockIdx.x;
    const int32_t id = b.big_rows[k];
    const int64_t base = row_off[id], len = row_off[id + 1] - base;
    int32_t *h = hist + (int64_t)k * nbk * 2;
    for (int64_t i = (int64_t)blockIdx.y * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.y * blockDim.x) {
        const int32_t v = col_idx[base + i];
        const int32_t bk = (int32_t)(((int64_t)v * nbk) / n);
        atomicAdd(&h[bk], 1);
    }
}

__global__ void k_big_scan(int32_t nbk, int32_t *__restrict__ hist)
{
    // one block per big row: exclusive scan of its nbk bucket counts into the
    // cursor half of the row's histogram area
    __shared__ int32_t carry;
    int32_t *h = hist + (int64_t)blockIdx.x * nbk * 2;
    int32_t *cur = h + nbk;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int32_t t0 = 0; t0 < nbk; t0 += blockDim.x) {
        const int32_t i = t0 + threadIdx.x;
        const int32_t v = i < nbk ? h[i] : 0;
        // block inclusive scan (simple shared-memory Hillis-Steele)
        __shared__ int32_t buf[1024];
        buf[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < (int)blockDim.x; o <<= 1) {
            const int32_t y = threadIdx.x >= (unsigned)o ? buf[threadIdx.x - o] : 0;
            __syncthreads();
            buf[threadIdx.x] += y;
            __syncthreads();
        }
        if (i < nbk) cur[i] = carry + buf[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry += buf[threadIdx.x];
        __syncthreads();
    }
}

__global__ void k_big_scatter(const QueryBufs b, const int64_t *__restrict__ row_off, int64_t n, int32_t nbk,
                              const BigDesc *__restrict__ desc, const int32_t *__restrict__ col_idx,
                              int32_t *__restrict__ hist, int32_t *__restrict__ tmp)
{
    const int k = blockIdx.x;
    const int32_t id = b.big_rows[k];
    const int64_t base = row_off[id], len = row_off[id + 1] - base;
    int32_t *cur = hist + (int64_t)k * nbk * 2 + nbk;
    int32_t *t = tmp + desc[k].tmp_off;
    for (int64_t i = (int64_t)blockIdx.y * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.y * blockDim.x) {
        const int32_t v = col_idx[base + i];
        const int32_t bk = (int32_t)(((int64_t)v * nbk) / n);
        const int32_t pos = atomicAdd(&cur[bk], 1);
        t[pos] = v;
    }
}

__global__ void __launch_bounds__(512) k_big_sort(const QueryBufs b, const int64_t *__restrict__ row_off,
                                                  int32_t nbk, const BigDesc *__restrict__ desc,
                                                  const int32_t *__restrict__ hist, const int32_t *__restrict__ tmp,
                                                  int32_t *__restrict__ col_idx)
{
    extern __shared__ int32_t sm[];
    const int k = blockIdx.x;
    const int32_t id = b.big_rows[k];
    const int64_t base = row_off[id];
    const int32_t *h = hist + (int64_t)k * nbk * 2;
    const int32_t *cur = h + nbk;  // after scatter: end of each bucket
    const int32_t *t = tmp + desc[k].tmp_off;
    for (int32_t bk = blockIdx.y; bk < nbk; bk += gridDim.y) {
        const int32_t cnt = h[bk];
        if (cnt == 0) continue;
        const int32_t beg = cur[bk] - cnt;
        int m = 1;
        while (m < cnt) m <<= 1;
        for (int i = threadIdx.x; i < m; i += blockDim.x) sm[i] = i < cnt ? t[beg + i] : 0x7fffffff;
        __syncthreads();
        bitonic_smem(sm, m);
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) col_idx[base + beg + i] = sm[i];
        __syncthreads();
    }
}

}  // namespace

static int32_t big_buckets(int64_t n)
{
    // bucket width n / nbk <= kSmemRow guarantees every bucket fits in shared memory
    int32_t nbk = 1;
    while ((int64_t)nbk * kSmemRow < n) nbk <<= 1;
    return nbk < 16 ? 16 : nbk;
}

}  // namespace hrg

namespace hrg {

cudaError_t launch_count_split(const Plan &p, const QueryBufs &b, bool fp64_only, int32_t p_hub, cudaStream_t s)
{
    const int32_t rest = (int32_t)p.n - p_hub;
    if (p_hub > 0) {
        if (fp64_only) k_query_cta<true, false><<<p_hub, 256, 0, s>>>(p, b, nullptr, nullptr);
        else k_query_cta<false, false><<<p_hub, 256, 0, s>>>(p, b, nullptr, nullptr);
    }
    if (rest > 0) {
        const int g = (rest + 127) / 128;
        if (fp64_only) k_query_thread<true, false><<<g, 128, 0, s>>>(p, b, p_hub, nullptr, nullptr);
        else k_query_thread<false, false><<<g, 128, 0, s>>>(p, b, p_hub, nullptr, nullptr);
    }
    return cudaGetLastError();
}

cudaError_t launch_write_split(const Plan &p, const QueryBufs &b, bool fp64_only, int32_t p_hub,
                               const int64_t *row_off, int32_t *col_idx, cudaStream_t s)
{
    const int32_t rest = (int32_t)p.n - p_hub;
    if (p_hub > 0) {
        if (fp64_only) k_query_cta<true, true><<<p_hub, 256, 0, s>>>(p, b, row_off, col_idx);
        else k_query_cta<false, true><<<p_hub, 256, 0, s>>>(p, b, row_off, col_idx);
    }
    if (rest > 0) {
        const int g = (rest + 127) / 128;
        if (fp64_only) k_query_thread<true, true><<<g, 128, 0, s>>>(p, b, p_hub, row_off, col_idx);
        else k_query_thread<false, true><<<g, 128, 0, s>>>(p, b, p_hub, row_off, col_idx);
    }
    return cudaGetLastError();
}

size_t big_sort_hist_words(int64_t n, int n_big) { return (size_t)n_big * big_buckets(n) * 2; }

cudaError_t launch_sort_rows(const Plan &p, const QueryBufs &b, int n_mid, int n_big, const int64_t *row_off,
                             int32_t *col_idx, int32_t *tmp, int64_t tmp_len, int32_t *bucket_ws,
                             int64_t bucket_ws_len, cudaStream_t s)
{
    static bool attr_set = false;
    const size_t smem = (size_t)16384 * sizeof(int32_t);
    if (!attr_set) {
        cudaFuncSetAttribute(k_sort_mid, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(k_big_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr_set = true;
    }
    if (n_mid > 0) k_sort_mid<<<n_mid, 512, smem, s>>>(b, row_off, col_idx);
    if (n_big > 0) {
        const int32_t nbk = big_buckets(p.n);
        BigDesc *desc = (BigDesc *)bucket_ws;
        int32_t *hist = bucket_ws + ((size_t)n_big * sizeof(BigDesc) + 3) / 4;
        const size_t hist_words = (size_t)n_big * nbk * 2;
        if ((int64_t)(((size_t)n_big * sizeof(BigDesc) + 3) / 4 + hist_words) > bucket_ws_len) return cudaErrorInvalidValue;
        cudaMemsetAsync(hist, 0, hist_words * sizeof(int32_t), s);
        k_big_setup<<<1, 1, 0, s>>>(b, n_big, row_off, p.n, nbk, desc, hist);
        dim3 g(n_big, 64);
        k_big_hist<<<g, 256, 0, s>>>(b, row_off, p.n, nbk, col_idx, hist);
        k_big_scan<<<n_big, 1024, 0, s>>>(nbk, hist);
        k_big_scatter<<<g, 256, 0, s>>>(b, row_off, p.n, nbk, desc, col_idx, hist, tmp);
        dim3 g2(n_big, 128);
        k_big_sort<<<g2, 512, smem, s>>>(b, row_off, nbk, desc, hist, tmp, col_idx);
        (void)tmp_len;
    }
    return cudaGetLastError();
}

}  // namespace hrg
