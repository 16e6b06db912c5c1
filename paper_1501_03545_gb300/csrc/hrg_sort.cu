// hrg_sort.cu -- ascending vertex ids inside every CSR row.
//
// The query traversal emits a row's neighbours in (band, angle) order.  The
// canonical CSR lists each row ascending, so rows longer than kRegRow (sorted
// in registers by the query itself) are sorted here:
//   * kRegRow < d <= kWarpRow:  one warp per row, bitonic sort in shared memory;
//   * kWarpRow < d <= kSmemRow: one CTA per row, stable LSD radix sort in
//     shared memory (8-bit digits, ranks within a warp from __match_any_sync);
//   * d > kSmemRow: the row's ids are split by value into buckets of expected
//     size <= 4096 (bucket k holds ids in [k n / nbk, (k+1) n / nbk)), every
//     bucket is sorted by the CTA radix sort; a bucket that still exceeds
//     kSmemRow (only for id-clustered injected point sets) is sorted by a
//     bitonic network in global memory.
#include <cstdio>
#include "hrg_internal.h"

namespace hrg {

namespace {

constexpr int kSortThreads = 256;
constexpr int kWarps = kSortThreads / 32;

__device__ __forceinline__ int bits_for(uint32_t range)
{
    return range <= 1 ? 1 : 32 - __clz(range - 1);
}

// --------------------------------------------------------------------------
// Warp bitonic sort of m (power of two) keys in shared memory.
// --------------------------------------------------------------------------
__device__ void warp_bitonic(int32_t *s, int m, int lane)
{
    for (int k = 2; k <= m; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = lane; i < m; i += 32) {
                const int l = i ^ j;
                if (l > i) {
                    const int32_t a = s[i], c = s[l];
                    if ((a > c) == ((i & k) == 0)) { s[i] = c; s[l] = a; }
                }
            }
            __syncwarp();
        }
    }
}

__global__ void __launch_bounds__(kSortThreads) k_sort_warp(const int32_t *__restrict__ rows, const int32_t *__restrict__ cnt,
                                                            const int64_t *__restrict__ row_off, int32_t *__restrict__ col_idx)
{
    __shared__ int32_t sm[kWarps][kWarpRow];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t r = (int64_t)blockIdx.x * kWarps + w;
    if (r >= *cnt) return;
    const int32_t id = rows[r];
    const int64_t base = row_off[id];
    const int d = (int)(row_off[id + 1] - base);
    int m = 32;
    while (m < d) m <<= 1;
    int32_t *s = sm[w];
    for (int i = lane; i < m; i += 32) s[i] = i < d ? col_idx[base + i] : 0x7fffffff;
    __syncwarp();
    warp_bitonic(s, m, lane);
    for (int i = lane; i < d; i += 32) col_idx[base + i] = s[i];
}

// --------------------------------------------------------------------------
// Stable CTA LSD radix sort of m <= kSmemRow unsigned keys in shared memory.
// keys/tmp: shared arrays of kSmemRow; cnt: [kWarps][256] shared counters.
// Returns the array that holds the sorted keys.
// --------------------------------------------------------------------------
__device__ uint32_t *cta_radix_sort(uint32_t *keys, uint32_t *tmp, uint32_t (*cnt)[256], uint32_t *dsum, int m,
                                    int bits)
{
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    int chunk = (m + kWarps - 1) / kWarps;
    chunk = (chunk + 31) & ~31;
    const int lo = w * chunk, hi = min(m, lo + chunk);
    uint32_t *src = keys, *dst = tmp;
    for (int shift = 0; shift < bits; shift += 8) {
        for (int i = threadIdx.x; i < kWarps * 256; i += kSortThreads) (&cnt[0][0])[i] = 0;
        __syncthreads();
        // per-warp digit counts
        for (int g = lo; g < hi; g += 32) {
            const int i = g + lane;
            const bool v = i < hi;
            const uint32_t d = v ? (src[i] >> shift) & 255u : 256u + lane;
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            if (v && (peers & lt) == 0) cnt[w][d] += __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        // offsets, digit-major then warp: thread t owns digit t
        {
            const int t = threadIdx.x;
            uint32_t tot = 0;
            for (int ww = 0; ww < kWarps; ++ww) tot += cnt[ww][t];
            // block exclusive scan of tot over the 256 digits
            uint32_t inc = tot;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
            }
            if (lane == 31) dsum[w] = inc;
            __syncthreads();
            if (t < 32) {
                const uint32_t v = t < kWarps ? dsum[t] : 0u;
                uint32_t vi = v;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, vi, o);
                    if (t >= o) vi += y;
                }
                if (t < kWarps) dsum[t] = vi - v;
            }
            __syncthreads();
            uint32_t run = inc - tot + dsum[w];
            for (int ww = 0; ww < kWarps; ++ww) {
                const uint32_t c = cnt[ww][t];
                cnt[ww][t] = run;
                run += c;
            }
        }
        __syncthreads();
        // stable scatter
        for (int g = lo; g < hi; g += 32) {
            const int i = g + lane;
            const bool v = i < hi;
            const uint32_t key = v ? src[i] : 0u;
            const uint32_t d = v ? (key >> shift) & 255u : 256u + lane;
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            uint32_t pos = 0;
            if (v) pos = cnt[w][d] + __popc(peers & lt);
            __syncwarp();
            if (v && (peers & lt) == 0) cnt[w][d] += __popc(peers);
            if (v) dst[pos] = key;
            __syncwarp();
        }
        __syncthreads();
        uint32_t *t2 = src;
        src = dst;
        dst = t2;
    }
    return src;
}

struct SortSmem {
    uint32_t keys[kSmemRow];
    uint32_t tmp[kSmemRow];
    uint32_t cnt[kWarps][256];
    uint32_t dsum[32];
};

__device__ void sort_span(SortSmem &S, const int32_t *src, int32_t *dst, int m, int32_t lo, int bits)
{
    for (int i = threadIdx.x; i < m; i += kSortThreads) S.keys[i] = (uint32_t)(src[i] - lo);
    __syncthreads();
    const uint32_t *out = cta_radix_sort(S.keys, S.tmp, S.cnt, S.dsum, m, bits);
    for (int i = threadIdx.x; i < m; i += kSortThreads) dst[i] = (int32_t)out[i] + lo;
    __syncthreads();
}

__global__ void __launch_bounds__(kSortThreads) k_sort_cta_rows(const int32_t *__restrict__ rows,
                                                                const int32_t *__restrict__ cnt, int64_t n,
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
    sort_span(S, col_idx + base, col_idx + base, d, 0, bits_for((uint32_t)n));
}

// --------------------------------------------------------------------------
// Big rows.
// --------------------------------------------------------------------------
struct BigRow { int64_t tmp_off; int64_t hist_off; int32_t nbk; int32_t id; };
struct Item { int64_t src; int64_t dst; int32_t len; int32_t lo; int32_t bits; int32_t pad; };

__global__ void k_big_setup(const int32_t *__restrict__ rows, int n_big, const int64_t *__restrict__ row_off,
                            BigRow *__restrict__ br)
{
    // serial prefix over the (few) big rows
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    int64_t toff = 0, hoff = 0;
    for (int k = 0; k < n_big; ++k) {
        const int32_t id = rows[k];
        const int64_t d = row_off[id + 1] - row_off[id];
        int32_t nbk = 2;
        while ((int64_t)nbk * 4096 < d) nbk <<= 1;
        br[k] = BigRow{toff, hoff, nbk, id};
        toff += d;
        hoff += 2 * (int64_t)nbk;
    }
}

__device__ __forceinline__ int32_t big_bucket(int32_t v, int32_t nbk, int64_t n)
{
    return (int32_t)(((int64_t)v * nbk) / n);
}

__global__ void k_big_hist(const BigRow *__restrict__ br, const int64_t *__restrict__ row_off, int64_t n,
                           const int32_t *__restrict__ col_idx, int32_t *__restrict__ hist)
{
    const BigRow R = br[blockIdx.x];
    const int64_t base = row_off[R.id], len = row_off[R.id + 1] - base;
    int32_t *h = hist + R.hist_off;
    for (int64_t i = (int64_t)blockIdx.y * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.y * blockDim.x)
        atomicAdd(&h[big_bucket(col_idx[base + i], R.nbk, n)], 1);
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
                const int32_t lo = (int32_t)(((int64_t)i * n + R.nbk - 1) / R.nbk);
                const int32_t hi = (int32_t)(((int64_t)(i + 1) * n + R.nbk - 1) / R.nbk);
                Item it{R.tmp_off + st, rbase + st, v, lo, bits_for((uint32_t)(hi - lo)), 0};
                if (v <= kSmemRow) items[atomicAdd(n_items, 1)] = it;
                else slow[atomicAdd(n_slow, 1)] = it;
            }
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry += buf[threadIdx.x];
        __syncthreads();
    }
}

__global__ void k_big_scatter(const BigRow *__restrict__ br, const int64_t *__restrict__ row_off, int64_t n,
                              const int32_t *__restrict__ col_idx, int32_t *__restrict__ hist,
                              int32_t *__restrict__ tmp)
{
    const BigRow R = br[blockIdx.x];
    const int64_t base = row_off[R.id], len = row_off[R.id + 1] - base;
    int32_t *cur = hist + R.hist_off + R.nbk;
    int32_t *t = tmp + R.tmp_off;
    for (int64_t i = (int64_t)blockIdx.y * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.y * blockDim.x) {
        const int32_t v = col_idx[base + i];
        t[atomicAdd(&cur[big_bucket(v, R.nbk, n)], 1)] = v;
    }
}

__global__ void __launch_bounds__(kSortThreads) k_sort_items(const Item *__restrict__ items,
                                                             const int32_t *__restrict__ n_items,
                                                             const int32_t *__restrict__ tmp,
                                                             int32_t *__restrict__ col_idx)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    SortSmem &S = *reinterpret_cast<SortSmem *>(smraw);
    const int32_t nit = *n_items;
    for (int32_t k = blockIdx.x; k < nit; k += gridDim.x) {
        const Item it = items[k];
        sort_span(S, tmp + it.src, col_idx + it.dst, it.len, it.lo, it.bits);
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

}  // namespace

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
        cudaFuncSetAttribute(k_sort_items, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(SortSmem));
        attr = true;
    }
    if (counts[0] > 0)
        k_sort_warp<<<(unsigned)((counts[0] + kWarps - 1) / kWarps), kSortThreads, 0, s>>>(b.rows[0], b.list_cnt + 0,
                                                                                        row_off, col_idx);
    if (counts[1] > 0)
        k_sort_cta_rows<<<(unsigned)counts[1], kSortThreads, sizeof(SortSmem), s>>>(b.rows[1], b.list_cnt + 1, p.n,
                                                                                 row_off, col_idx);
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
        k_big_setup<<<1, 1, 0, s>>>(b.rows[2], n_big, row_off, br);
        dim3 g(n_big, 64);
        k_big_hist<<<g, 256, 0, s>>>(br, row_off, p.n, col_idx, hist);
        k_big_scan<<<n_big, 1024, 0, s>>>(br, row_off, p.n, hist, items, ctr, slow, ctr + 1);
        k_big_scatter<<<g, 256, 0, s>>>(br, row_off, p.n, col_idx, hist, tmp);
        const unsigned gi = (unsigned)std::min<int64_t>(nbk_sum, 152 * 8);
        k_sort_items<<<gi, kSortThreads, sizeof(SortSmem), s>>>(items, ctr, tmp, col_idx);
        k_sort_slow<<<64, 1024, 0, s>>>(slow, ctr + 1, tmp, col_idx);
    }
    return cudaGetLastError();
}

}  // namespace hrg
