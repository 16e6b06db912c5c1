// hrg_sort.cu -- ascending vertex ids inside every CSR row.
//
// The query traversal emits a row's neighbours in (band, angle) order.  The
// canonical CSR lists each row ascending.  Rows of up to kCopySortRow entries
// kept by the rim count pass are sorted by the copy that stores them, rows of
// up to kRegRow entries by the traversal itself; the other rows (hub rows,
// longer rim rows, kept or traversed again) are sorted here:
//   * kRegRow < d <= kWarpRow:  one warp per row; up to 64 ids by a bitonic
//     network in the warp's registers, more by a bucket sort in the warp's
//     shared-memory slice (the ids of a row are spread evenly over [0, n), so
//     d/4 .. d/2 equal-width value buckets hold 2..4 ids each);
//   * kWarpRow < d <= kSmemRow: one CTA per row, the same bucket sort over
//     the whole CTA;
//   * d > kSmemRow: the row's ids are split by value into buckets of expected
//     size <= 4096 (bucket k holds ids in [k n / nbk, (k+1) n / nbk)), every
//     bucket is sorted by the CTA bucket sort; a bucket that still exceeds
//     kSmemRow (only for id-clustered injected point sets) is sorted by a
//     bitonic network in global memory.
// Value buckets are taken as umulhi(key, mul) with mul = floor(nb 2^32 /
// range): monotone in the key and below nb for every key < range.
#include <cstdio>
#include "hrg_internal.h"

namespace hrg {

namespace {

constexpr int kSortThreads = 256;
constexpr int kWarps = kSortThreads / 32;
constexpr int kSortRowsPerBlock = 16 * kWarps;
constexpr int kCtaThreads = 512;  // CTA bucket sort
constexpr int kCtaWarps = kCtaThreads / 32;
constexpr int kSetupThreads = 1024;  // k_big_setup needs whole warps (shuffle scans)

__device__ __forceinline__ uint32_t bucket_mul(uint32_t nb, uint32_t range)
{
    return (uint32_t)(((uint64_t)nb << 32) / (uint64_t)range);
}

// warp bitonic sort of a[0..L) in shared memory, any L (positions >= L act as
// +infinity: the first step of each merge pairs i with its mirror, so every
// block sorts ascending and those positions never move)
__device__ void warp_bitonic_any(uint32_t *a, int L, int lane)
{
    int M = 1;
    while (M < L) M <<= 1;
    for (int kk = 2; kk <= M; kk <<= 1)
        for (int j = kk >> 1; j > 0; j >>= 1) {
            for (int i = lane; i < M; i += 32) {
                const int l = (j == (kk >> 1)) ? (i ^ (kk - 1)) : (i ^ j);
                if (l > i && l < L) {
                    const uint32_t x = a[i], y = a[l];
                    if (x > y) { a[i] = y; a[l] = x; }
                }
            }
            __syncwarp();
        }
}

// insertion sort of a[s0..e0) by one thread
__device__ __forceinline__ void insertion(uint32_t *a, uint32_t s0, uint32_t e0)
{
    for (uint32_t i = s0 + 1; i < e0; ++i) {
        const uint32_t v = a[i];
        uint32_t k = i;
        while (k > s0 && a[k - 1] > v) { a[k] = a[k - 1]; --k; }
        a[k] = v;
    }
}

// Buckets [cnt[b-1], cnt[b]) of b in [b_begin, nb) stepping by 32*stride warps:
// up to 32 keys by the lane's own insertion sort, longer ones by the warp.
__device__ void sort_buckets(uint32_t *key, const uint32_t *cnt, uint32_t nb, uint32_t b_begin, uint32_t b_step,
                             int lane)
{
    for (uint32_t b0 = b_begin; b0 < nb; b0 += b_step) {
        const uint32_t b = b0 + lane;
        const uint32_t s0 = (b < nb && b) ? cnt[b - 1] : 0u, e0 = b < nb ? cnt[b] : 0u;
        if (b < nb && e0 - s0 > 1 && e0 - s0 <= 32) insertion(key, s0, e0);
        unsigned big = __ballot_sync(0xffffffffu, b < nb && e0 - s0 > 32);
        __syncwarp();
        while (big) {
            const int src_lane = __ffs(big) - 1;
            big &= big - 1;
            const uint32_t bs = __shfl_sync(0xffffffffu, s0, src_lane), be = __shfl_sync(0xffffffffu, e0, src_lane);
            warp_bitonic_any(key + bs, (int)(be - bs), lane);
        }
    }
}

// --------------------------------------------------------------------------
// Warp bucket sort of one row of kRegRow < d <= kWarpRow ids.
// --------------------------------------------------------------------------
constexpr int kWarpBuckets = kWarpRow / 4;

struct WarpSortSmem {
    uint32_t key[kWarpRow];
    uint32_t cnt[kWarpBuckets + 1];
};

// ids of row `id` lie in [0, n), n of the row's graph in a batch
__device__ __forceinline__ uint32_t row_range(int64_t n, const int32_t *graph_of, const int64_t *noff, int32_t id)
{
    if (!graph_of) return (uint32_t)n;
    const int g = __ldg(graph_of + id);
    return (uint32_t)(__ldg(noff + g + 1) - __ldg(noff + g));
}

// Rows of up to 64 ids: the bitonic network over the warp's registers.
__device__ __forceinline__ void warp_sort64(int32_t *row, int d, int lane)
{
    int32_t a = lane < d ? row[lane] : 0x7fffffff;
    int32_t b = lane + 32 < d ? row[lane + 32] : 0x7fffffff;
    warp_bitonic64(a, b, lane);
    if (lane < d) row[lane] = a;
    if (lane + 32 < d) row[lane + 32] = b;
}

template <int R>
__device__ __forceinline__ void warp_sort_regs(int32_t *row, int d, int lane)
{
    int32_t v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = lane + 32 * r < d ? row[lane + 32 * r] : 0x7fffffff;
    warp_bitonic_regs<R>(v, lane);
#pragma unroll
    for (int r = 0; r < R; ++r)
        if (lane + 32 * r < d) row[lane + 32 * r] = v[r];
}

// One row of the warp sort (33..kWarpRow ids).
__device__ __forceinline__ void warp_sort_row(WarpSortSmem &S, int32_t id, int64_t n,
                                              const int32_t *__restrict__ graph_of, const int64_t *__restrict__ noff,
                                              const int64_t *__restrict__ row_off, int32_t *col_idx, int lane)
{
    const int64_t base = row_off[id];
    const int d = (int)(row_off[id + 1] - base);
    int32_t *row = col_idx + base;
    if (d <= 64) {  // uniform per warp
        warp_sort64(row, d, lane);
        return;
    }
    if (d <= 256) {  // a bitonic network over the warp's registers: four or eight ids a lane
        if (d <= 128) warp_sort_regs<4>(row, d, lane);
        else warp_sort_regs<8>(row, d, lane);
        return;
    }
    uint32_t nb = 1;
    while (nb * 4 <= (uint32_t)d && nb < (uint32_t)kWarpBuckets) nb <<= 1;
    const uint32_t mul = bucket_mul(nb, row_range(n, graph_of, noff, id));
    for (uint32_t i = lane; i <= nb; i += 32) S.cnt[i] = 0;
    __syncwarp();
    for (int i = lane; i < d; i += 32) atomicAdd(&S.cnt[__umulhi((uint32_t)row[i], mul)], 1u);
    __syncwarp();
    {   // exclusive scan of cnt[0..nb): a run of nb/32 counters per lane
        const uint32_t per = (nb + 31) >> 5;
        const uint32_t b0 = min(nb, lane * per), b1 = min(nb, b0 + per);
        uint32_t s = 0;
        for (uint32_t i = b0; i < b1; ++i) s += S.cnt[i];
        uint32_t inc = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        uint32_t run = inc - s;
        for (uint32_t i = b0; i < b1; ++i) { const uint32_t v = S.cnt[i]; S.cnt[i] = run; run += v; }
    }
    __syncwarp();
    for (int i = lane; i < d; i += 32) {
        const uint32_t v = (uint32_t)row[i];
        S.key[atomicAdd(&S.cnt[__umulhi(v, mul)], 1u)] = v;
    }
    __syncwarp();
    sort_buckets(S.key, S.cnt, nb, 0, 32, lane);
    __syncwarp();
    for (int i = lane; i < d; i += 32) row[i] = (int32_t)S.key[i];
}

// kSortRowsPerBlock rows a block: warp w sorts row w first, then the next row
// not yet taken (a shared counter), so the block's warps end together
// although the rows' lengths differ.
__global__ void __launch_bounds__(kSortThreads) k_sort_warp(const int32_t *__restrict__ rows, const int32_t *__restrict__ cnt,
                                                            int64_t n, const int32_t *__restrict__ graph_of,
                                                            const int64_t *__restrict__ noff,
                                                            const int64_t *__restrict__ row_off, int32_t *col_idx)
{
    __shared__ WarpSortSmem sm[kWarps];
    __shared__ int32_t s_next;
    if (threadIdx.x == 0) s_next = kWarps;
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t r0 = (int64_t)blockIdx.x * kSortRowsPerBlock, nr = *cnt;
    for (int k = w; k < kSortRowsPerBlock && r0 + k < nr;) {
        warp_sort_row(sm[w], rows[r0 + k], n, graph_of, noff, row_off, col_idx, lane);
        __syncwarp();
        int32_t nx = 0;
        if (lane == 0) nx = atomicAdd(&s_next, 1);
        k = __shfl_sync(0xffffffffu, nx, 0);
    }
}

// --------------------------------------------------------------------------
// CTA bucket sort of m <= kSmemRow keys in [lo, lo + range): the ids of a
// row are spread evenly over their range, so ~m/2 equal-width buckets hold ~2
// keys each.  Count (shared atomics), scan, scatter, then every bucket is
// sorted on its own: by one thread (insertion) up to 32 keys, by one warp
// (bitonic) beyond, so skewed inputs stay correct.
// --------------------------------------------------------------------------
// Shared memory of the CTA sort of up to CAP keys: m keys use the smallest
// power of two above m/4 buckets, at most BK.  Rows take up to kSmemRow keys;
// the big rows' id buckets expect 2048..4096 keys each and take up to
// kItemCap (twice that: a larger bucket, which uniformly spread ids make
// vanishingly rare, goes to the global-memory network), so their CTAs need
// less shared memory and four fit on an SM.
template <int CAP, int BK>
struct SortSmemT {
    uint32_t tmp[CAP];
    uint32_t cnt[BK + 1];
    uint32_t wsum[kCtaWarps];
    static constexpr uint32_t kBuckets = BK;
};
using SortSmem = SortSmemT<kSmemRow, 4096>;  // rows of up to kSmemRow keys use at most 4096 buckets
constexpr int kItemCap = 8191;
using ItemSmem = SortSmemT<kItemCap, 2048>;

// in-place exclusive scan of c[0..nb) (nb at most the sort's bucket count) by the whole CTA
__device__ void cta_exclusive_scan(uint32_t *c, uint32_t nb, uint32_t *wsum)
{
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const uint32_t per = (nb + kCtaThreads - 1) / kCtaThreads;
    const uint32_t b0 = min(nb, t * per), b1 = min(nb, b0 + per);
    uint32_t s = 0;
    for (uint32_t i = b0; i < b1; ++i) s += c[i];
    uint32_t inc = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    if (t == 0) {
        uint32_t acc = 0;
        for (int k = 0; k < kCtaWarps; ++k) { const uint32_t v = wsum[k]; wsum[k] = acc; acc += v; }
    }
    __syncthreads();
    uint32_t run = inc - s + wsum[w];
    for (uint32_t i = b0; i < b1; ++i) { const uint32_t v = c[i]; c[i] = run; run += v; }
    __syncthreads();
}

template <typename SM>
__device__ void sort_span(SM &S, const int32_t *src, int32_t *dst, int m, int32_t lo, uint32_t range)
{
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    uint32_t nb = 1;
    while (nb * 4 <= (uint32_t)m && nb < SM::kBuckets) nb <<= 1;
    if (range == 0) range = 1;
    const uint32_t mul = bucket_mul(nb, range);
    for (uint32_t i = t; i <= nb; i += kCtaThreads) S.cnt[i] = 0;
    __syncthreads();
    for (int i = t; i < m; i += kCtaThreads) atomicAdd(&S.cnt[__umulhi((uint32_t)(src[i] - lo), mul)], 1u);
    __syncthreads();
    cta_exclusive_scan(S.cnt, nb, S.wsum);
    for (int i = t; i < m; i += kCtaThreads) {
        const uint32_t k = (uint32_t)(src[i] - lo);
        S.tmp[atomicAdd(&S.cnt[__umulhi(k, mul)], 1u)] = k;
    }
    __syncthreads();
    sort_buckets(S.tmp, S.cnt, nb, (uint32_t)w * 32, kCtaWarps * 32, lane);
    __syncthreads();
    for (int i = t; i < m; i += kCtaThreads) dst[i] = (int32_t)S.tmp[i] + lo;
    __syncthreads();
}

__global__ void __launch_bounds__(kCtaThreads) k_sort_cta_rows(const int32_t *__restrict__ rows,
                                                                const int32_t *__restrict__ cnt, int64_t n,
                                                                const int32_t *__restrict__ graph_of,
                                                                const int64_t *__restrict__ noff,
                                                                const int64_t *__restrict__ row_off,
                                                                int32_t *__restrict__ col_idx)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    SortSmem &S = *reinterpret_cast<SortSmem *>(smraw);
    const int64_t r = blockIdx.x;
    if (r >= *cnt) return;
    const int32_t id = rows[r];
    const int64_t base = row_off[id];
    const int d = (int)(row_off[id + 1] - base);
    sort_span(S, col_idx + base, col_idx + base, d, 0, row_range(n, graph_of, noff, id));
}

// --------------------------------------------------------------------------
// Big rows.
// --------------------------------------------------------------------------
struct BigRow { int64_t tmp_off; int64_t hist_off; int32_t nbk; int32_t id; int64_t ch_off; int64_t range; };
struct Item { int64_t src; int64_t dst; int32_t len; int32_t lo; uint32_t range; int32_t pad; };

constexpr int kBigChunk = 4096;   // entries of a big row one CTA histograms / scatters
constexpr int kBigSmemBk = 8192;  // id buckets a CTA aggregates in shared memory

// offsets of the big rows' ids (tmp), bucket counters (hist) and chunks: one
// CTA, chunked prefix sums over the rows
__global__ void __launch_bounds__(kSetupThreads) k_big_setup(const int32_t *__restrict__ rows, int n_big, int64_t n,
                                                    const int32_t *__restrict__ graph_of,
                                                    const int64_t *__restrict__ noff,
                                                    const int64_t *__restrict__ row_off, BigRow *__restrict__ br)
{
    __shared__ long long s_t[32], s_h[32], s_c[32];
    __shared__ long long carry_t, carry_h, carry_c;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    if (t == 0) { carry_t = 0; carry_h = 0; carry_c = 0; }
    __syncthreads();
    for (int k0 = 0; k0 < n_big; k0 += blockDim.x) {
        const int k = k0 + t;
        long long d = 0, h = 0, c = 0;
        int32_t id = 0, nbk = 0;
        if (k < n_big) {
            id = rows[k];
            d = row_off[id + 1] - row_off[id];
            nbk = 2;
            while ((long long)nbk * 4096 < d) nbk <<= 1;
            h = 2 * (long long)nbk;
            c = (d + kBigChunk - 1) / kBigChunk;
        }
        long long it = d, ih = h, ic = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long yt = __shfl_up_sync(0xffffffffu, it, o), yh = __shfl_up_sync(0xffffffffu, ih, o),
                            yc = __shfl_up_sync(0xffffffffu, ic, o);
            if (lane >= o) { it += yt; ih += yh; ic += yc; }
        }
        if (lane == 31) { s_t[w] = it; s_h[w] = ih; s_c[w] = ic; }
        __syncthreads();
        if (t == 0) {
            long long at = carry_t, ah = carry_h, ac = carry_c;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
                const long long vt = s_t[q], vh = s_h[q], vc = s_c[q];
                s_t[q] = at; s_h[q] = ah; s_c[q] = ac;
                at += vt; ah += vh; ac += vc;
            }
            carry_t = at;
            carry_h = ah;
            carry_c = ac;
        }
        __syncthreads();
        if (k < n_big)
            br[k] = BigRow{s_t[w] + it - d, s_h[w] + ih - h, nbk, id, s_c[w] + ic - c, row_range(n, graph_of, noff, id)};
        __syncthreads();
    }
}

// first key of id bucket i of a row with multiplier mul: the least v with
// umulhi(v, mul) >= i, i.e. ceil(i 2^32 / mul)
__device__ __forceinline__ int64_t bucket_lo(int64_t i, uint32_t mul)
{
    return (int64_t)((((uint64_t)i << 32) + mul - 1) / mul);
}

// the chunk of this CTA: its row (binary search over the rows' chunk offsets)
// and the entry range [c0, c1) inside the row
__device__ __forceinline__ bool big_chunk(const BigRow *br, int n_big, const int64_t *row_off, BigRow &R,
                                          int64_t &base, int64_t &c0, int64_t &c1)
{
    const int64_t c = blockIdx.x;
    int lo = 0, hi = n_big;  // last row with ch_off <= c
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (br[mid].ch_off <= c) lo = mid; else hi = mid;
    }
    R = br[lo];
    base = row_off[R.id];
    const int64_t len = row_off[R.id + 1] - base;
    c0 = (c - R.ch_off) * kBigChunk;
    c1 = min(len, c0 + kBigChunk);
    return c0 < len;
}

// Histogram of the id buckets of every big row, aggregated per chunk in
// shared memory.
__global__ void __launch_bounds__(256) k_big_hist(const BigRow *__restrict__ br, int n_big,
                                                  const int64_t *__restrict__ row_off, int64_t n,
                                                  const int32_t *__restrict__ col_idx, int32_t *__restrict__ hist)
{
    __shared__ uint32_t hs[kBigSmemBk];
    BigRow R;
    int64_t base, c0, c1;
    if (!big_chunk(br, n_big, row_off, R, base, c0, c1)) return;
    const uint32_t mul = bucket_mul((uint32_t)R.nbk, (uint32_t)R.range);
    int32_t *h = hist + R.hist_off;
    if (R.nbk > kBigSmemBk) {
        for (int64_t i = c0 + threadIdx.x; i < c1; i += blockDim.x)
            atomicAdd(&h[__umulhi((uint32_t)col_idx[base + i], mul)], 1);
        return;
    }
    for (int i = threadIdx.x; i < R.nbk; i += blockDim.x) hs[i] = 0;
    __syncthreads();
    for (int64_t i = c0 + threadIdx.x; i < c1; i += blockDim.x)
        atomicAdd(&hs[__umulhi((uint32_t)col_idx[base + i], mul)], 1u);
    __syncthreads();
    for (int i = threadIdx.x; i < R.nbk; i += blockDim.x)
        if (hs[i]) atomicAdd(&h[i], (int32_t)hs[i]);
}

// exclusive scan of one row's bucket counts into its cursor half; one item per
// non-empty bucket (oversized ones into the fallback list)
__global__ void k_big_scan(const BigRow *__restrict__ br, const int64_t *__restrict__ row_off, int64_t n,
                           int32_t *__restrict__ hist, Item *__restrict__ items, int32_t *__restrict__ n_items,
                           Item *__restrict__ slow, int32_t *__restrict__ n_slow)
{
    __shared__ int32_t buf[1024];
    __shared__ int32_t carry;
    const BigRow R = br[blockIdx.x];
    int32_t *h = hist + R.hist_off;
    int32_t *cur = h + R.nbk;
    const int64_t rbase = row_off[R.id];
    const uint32_t mul = bucket_mul((uint32_t)R.nbk, (uint32_t)R.range);
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int32_t t0 = 0; t0 < R.nbk; t0 += blockDim.x) {
        const int32_t i = t0 + threadIdx.x;
        const int32_t v = i < R.nbk ? h[i] : 0;
        buf[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < (int)blockDim.x; o <<= 1) {
            const int32_t y = threadIdx.x >= (unsigned)o ? buf[threadIdx.x - o] : 0;
            __syncthreads();
            buf[threadIdx.x] += y;
            __syncthreads();
        }
        if (i < R.nbk) {
            const int32_t st = carry + buf[threadIdx.x] - v;
            cur[i] = st;
            if (v > 0) {
                const int64_t lo = bucket_lo(i, mul), hi = min(R.range, bucket_lo(i + 1, mul));
                Item it{R.tmp_off + st, rbase + st, v, (int32_t)lo, (uint32_t)(hi - lo), 0};
                if (v <= kItemCap) items[atomicAdd(n_items, 1)] = it;
                else slow[atomicAdd(n_slow, 1)] = it;
            }
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry += buf[threadIdx.x];
        __syncthreads();
    }
}

// Scatter of every big row's ids into its id buckets (tmp): a chunk reserves
// its bucket ranges with one global atomic per non-empty bucket, then places
// its ids with shared-memory atomics.
__global__ void __launch_bounds__(256) k_big_scatter(const BigRow *__restrict__ br, int n_big,
                                                     const int64_t *__restrict__ row_off, int64_t n,
                                                     const int32_t *__restrict__ col_idx, int32_t *__restrict__ hist,
                                                     int32_t *__restrict__ tmp)
{
    __shared__ uint32_t hs[kBigSmemBk];
    BigRow R;
    int64_t base, c0, c1;
    if (!big_chunk(br, n_big, row_off, R, base, c0, c1)) return;
    const uint32_t mul = bucket_mul((uint32_t)R.nbk, (uint32_t)R.range);
    int32_t *cur = hist + R.hist_off + R.nbk;
    int32_t *t = tmp + R.tmp_off;
    if (R.nbk > kBigSmemBk) {
        for (int64_t i = c0 + threadIdx.x; i < c1; i += blockDim.x) {
            const int32_t v = col_idx[base + i];
            t[atomicAdd(&cur[__umulhi((uint32_t)v, mul)], 1)] = v;
        }
        return;
    }
    for (int i = threadIdx.x; i < R.nbk; i += blockDim.x) hs[i] = 0;
    __syncthreads();
    for (int64_t i = c0 + threadIdx.x; i < c1; i += blockDim.x)
        atomicAdd(&hs[__umulhi((uint32_t)col_idx[base + i], mul)], 1u);
    __syncthreads();
    for (int i = threadIdx.x; i < R.nbk; i += blockDim.x) {
        const uint32_t c = hs[i];
        if (c) hs[i] = (uint32_t)atomicAdd(&cur[i], (int32_t)c);
    }
    __syncthreads();
    for (int64_t i = c0 + threadIdx.x; i < c1; i += blockDim.x) {
        const int32_t v = col_idx[base + i];
        t[atomicAdd(&hs[__umulhi((uint32_t)v, mul)], 1u)] = v;
    }
}

__global__ void __launch_bounds__(kCtaThreads) k_sort_items(const Item *__restrict__ items,
                                                             const int32_t *__restrict__ n_items,
                                                             const int32_t *__restrict__ tmp,
                                                             int32_t *__restrict__ col_idx)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    ItemSmem &S = *reinterpret_cast<ItemSmem *>(smraw);
    const int32_t nit = *n_items;
    for (int32_t k = blockIdx.x; k < nit; k += gridDim.x) {
        const Item it = items[k];
        sort_span(S, tmp + it.src, col_idx + it.dst, it.len, it.lo, it.range);
    }
}

// Bitonic network over a span of any length in global memory (positions past
// the end act as +infinity and never move: the first step of every merge
// compares i with its mirror in the block, so all blocks sort ascending).
__global__ void __launch_bounds__(1024) k_sort_slow(const Item *__restrict__ items, const int32_t *__restrict__ n_items,
                                                    const int32_t *__restrict__ tmp, int32_t *__restrict__ col_idx)
{
    const int32_t nit = *n_items;
    for (int32_t k = blockIdx.x; k < nit; k += gridDim.x) {
        const Item it = items[k];
        int32_t *a = col_idx + it.dst;
        const int m = it.len;
        for (int i = threadIdx.x; i < m; i += blockDim.x) a[i] = tmp[it.src + i];
        __syncthreads();
        int M = 1;
        while (M < m) M <<= 1;
        for (int kk = 2; kk <= M; kk <<= 1) {
            for (int j = kk >> 1; j > 0; j >>= 1) {
                for (int i = threadIdx.x; i < M; i += blockDim.x) {
                    const int l = (j == (kk >> 1)) ? (i ^ (kk - 1)) : (i ^ j);
                    if (l > i && l < m) {
                        const int32_t x = a[i], y = a[l];
                        if (x > y) { a[i] = y; a[l] = x; }
                    }
                }
                __syncthreads();
            }
        }
    }
}

// One thread per entry of the three lists: its range by a search over the
// (few) bounds, then an append to that range's part of its class.
__global__ void k_split_lists(const int32_t *__restrict__ l0, const int32_t *__restrict__ l1,
                              const int32_t *__restrict__ l2, int32_t c0, int32_t c1, int32_t c2, int K,
                              const int64_t *__restrict__ bounds, const int64_t *__restrict__ row_off,
                              int32_t *__restrict__ sub, int32_t *__restrict__ sub_cnt, int64_t *__restrict__ sub_tot)
{
    const int64_t total = (int64_t)c0 + c1 + c2;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        int cls;
        int32_t id, cap;
        int64_t base;
        if (t < c0) {
            cls = 0; id = l0[t]; cap = c0; base = 0;
        } else if (t < (int64_t)c0 + c1) {
            cls = 1; id = l1[t - c0]; cap = c1; base = (int64_t)K * c0;
        } else {
            cls = 2; id = l2[t - c0 - c1]; cap = c2; base = (int64_t)K * (c0 + c1);
        }
        int k = 0;
        while (k + 1 < K && __ldg(bounds + k + 1) <= id) ++k;
        const int32_t slot = atomicAdd(&sub_cnt[3 * k + cls], 1);
        sub[base + (int64_t)k * cap + slot] = id;
        if (cls == 2) atomicAdd((unsigned long long *)&sub_tot[k], (unsigned long long)(row_off[id + 1] - row_off[id]));
    }
}

}  // namespace

cudaError_t launch_split_lists(const QueryBufs &b, const int32_t counts[3], int K, const int64_t *bounds,
                               const int64_t *row_off, int32_t *sub, int32_t *sub_cnt, int64_t *sub_tot,
                               cudaStream_t s)
{
    const int64_t total = (int64_t)counts[0] + counts[1] + counts[2];
    if (total == 0) return cudaSuccess;
    const unsigned g = (unsigned)std::min<int64_t>((total + 255) / 256, 152 * 8);
    k_split_lists<<<g, 256, 0, s>>>(b.rows[0], b.rows[1], b.rows[2], counts[0], counts[1], counts[2], K, bounds,
                                   row_off, sub, sub_cnt, sub_tot);
    return cudaGetLastError();
}

size_t sort_smem_bytes() { return sizeof(SortSmem); }

size_t big_sort_ws_bytes(int n_big, int64_t big_total)
{
    // BigRow descriptors, histograms + cursors, bucket items, fallback items, two counters
    const int64_t nbk_sum = 2 * (big_total / 4096 + 1) + 2 * (int64_t)n_big;
    return sizeof(BigRow) * (size_t)n_big + sizeof(int32_t) * 2 * (size_t)nbk_sum + sizeof(Item) * 2 * (size_t)nbk_sum +
           64;
}

int sort_launches(const int32_t counts[3])
{
    return (counts[0] > 0 ? 1 : 0) + (counts[1] > 0 ? 1 : 0) + (counts[2] > 0 ? 7 : 0);
}

cudaError_t launch_sort_rows(const Plan &p, const QueryBufs &b, const int32_t counts[3], int64_t big_total,
                             const int64_t *row_off, int32_t *col_idx, int32_t *tmp, void *ws, cudaStream_t s)
{
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_sort_cta_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(SortSmem));
        cudaFuncSetAttribute(k_sort_items, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(ItemSmem));
        attr = true;
    }
    if (counts[0] > 0)
        k_sort_warp<<<(unsigned)((counts[0] + kSortRowsPerBlock - 1) / kSortRowsPerBlock), kSortThreads, 0, s>>>(
            b.rows[0], b.list_cnt + 0, p.n, b.graph_of, b.noff, row_off, col_idx);
    if (counts[1] > 0)
        k_sort_cta_rows<<<(unsigned)counts[1], kCtaThreads, sizeof(SortSmem), s>>>(
            b.rows[1], b.list_cnt + 1, p.n, b.graph_of, b.noff, row_off, col_idx);
    if (counts[2] > 0) {
        const int n_big = counts[2];
        const int64_t nbk_sum = 2 * (big_total / 4096 + 1) + 2 * (int64_t)n_big;
        char *w = (char *)ws;
        BigRow *br = (BigRow *)w;
        w += sizeof(BigRow) * (size_t)n_big;
        int32_t *hist = (int32_t *)w;
        w += sizeof(int32_t) * 2 * (size_t)nbk_sum;
        Item *items = (Item *)w;
        w += sizeof(Item) * (size_t)nbk_sum;
        Item *slow = (Item *)w;
        w += sizeof(Item) * (size_t)nbk_sum;
        int32_t *ctr = (int32_t *)w;
        cudaMemsetAsync(hist, 0, sizeof(int32_t) * 2 * (size_t)nbk_sum, s);
        cudaMemsetAsync(ctr, 0, 2 * sizeof(int32_t), s);
        k_big_setup<<<1, kSetupThreads, 0, s>>>(b.rows[2], n_big, p.n, b.graph_of, b.noff, row_off, br);
        // chunks: sum over the rows of ceil(d / kBigChunk) <= big_total / kBigChunk + n_big
        const unsigned gc = (unsigned)(big_total / kBigChunk + n_big);
        k_big_hist<<<gc, 256, 0, s>>>(br, n_big, row_off, p.n, col_idx, hist);
        k_big_scan<<<n_big, 1024, 0, s>>>(br, row_off, p.n, hist, items, ctr, slow, ctr + 1);
        k_big_scatter<<<gc, 256, 0, s>>>(br, n_big, row_off, p.n, col_idx, hist, tmp);
        const unsigned gi = (unsigned)std::min<int64_t>(nbk_sum, 152 * 8);
        k_sort_items<<<gi, kCtaThreads, sizeof(ItemSmem), s>>>(items, ctr, tmp, col_idx);
        k_sort_slow<<<64, 1024, 0, s>>>(slow, ctr + 1, tmp, col_idx);
    }
    return cudaGetLastError();
}

}  // namespace hrg
