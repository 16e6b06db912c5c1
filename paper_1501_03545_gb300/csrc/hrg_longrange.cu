// hrg_longrange.cu -- random long-range edges added to a generated graph.
//
// Sec. 4.2 (and the appendix on additional random edges) adds 0.5 % of the
// edges between random vertex pairs, which shortens the diameter while the
// other properties stay close.  Pair k draws the Philox4x32-10 block at
// counter 2^63 + k, key = seed (the point draws use counters below 2^31),
// and maps each 64-bit half w to the vertex floor(w n / 2^64).  Self-pairs,
// pairs drawn twice and pairs already in the graph are dropped; the rest is
// merged into a new canonical CSR:
//   1. per vertex, the number of drawn partners (both endpoints of a pair);
//   2. scan; the partners listed per vertex;
//   3. per vertex (one thread: the lists hold ~2 count / n entries), the
//      list sorted, repeats and present neighbours dropped, the new degree;
//   4. scan of the new degrees (the caller's row offsets);
//   5. the old rows and the new partners merged: an old entry's place is its
//      row's new offset plus its index in the row plus the number of the
//      row's new partners below it; a new partner's, the new offset plus its
//      index plus the number of old entries below it (binary searches).  The
//      old entries are walked as one flat array in chunks of kRun per lane
//      (a warp finds its chunk's rows once), so a row of millions of entries
//      is spread over many warps.
#include <algorithm>
#include "hrg_common.cuh"
#include "hrg_graph_ops.h"
#include "hrg_graph_util.cuh"

namespace hrg {

namespace {

using namespace graph_util;

constexpr int kThreads = 256;
constexpr int kWarpsPerBlock = kThreads / 32;

__device__ __forceinline__ void random_pair(int64_t k, uint64_t seed, uint64_t n, int32_t &u, int32_t &v)
{
    const U4 w = philox_block((1ull << 63) | (uint64_t)k, seed);
    const uint64_t a = ((uint64_t)w.x << 32) | w.y, b = ((uint64_t)w.z << 32) | w.w;
    u = (int32_t)__umul64hi(a, n);
    v = (int32_t)__umul64hi(b, n);
}

__global__ void k_lr_count(int64_t n, int64_t count, uint64_t seed, int32_t *__restrict__ cnt)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count; k += stride) {
        int32_t u, v;
        random_pair(k, seed, (uint64_t)n, u, v);
        if (u == v) continue;
        atomicAdd(cnt + u, 1);
        atomicAdd(cnt + v, 1);
    }
}

__global__ void k_lr_fill(int64_t n, int64_t count, uint64_t seed, const int64_t *__restrict__ loff,
                          int32_t *__restrict__ cur, int32_t *__restrict__ list)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count; k += stride) {
        int32_t u, v;
        random_pair(k, seed, (uint64_t)n, u, v);
        if (u == v) continue;
        list[loff[u] + atomicAdd(cur + u, 1)] = v;
        list[loff[v] + atomicAdd(cur + v, 1)] = u;
    }
}

__device__ __forceinline__ bool in_sorted(const int32_t *__restrict__ a, int64_t len, int32_t x)
{
    const int64_t i = lower_bound(a, 0, len, x);
    return i < len && a[i] == x;
}

// one thread per vertex: its drawn partners sorted (insertion), repeats and
// present neighbours dropped, compacted; fin = partners kept, newdeg = d + fin
__global__ void k_lr_clean(int64_t n, const int64_t *__restrict__ row_off, const int32_t *__restrict__ col_idx,
                           const int64_t *__restrict__ loff, int32_t *__restrict__ list, int32_t *__restrict__ fin,
                           int32_t *__restrict__ newdeg)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        int32_t *L = list + loff[v];
        const int64_t c = loff[v + 1] - loff[v];
        for (int64_t i = 1; i < c; ++i) {
            const int32_t x = L[i];
            int64_t j = i;
            for (; j > 0 && L[j - 1] > x; --j) L[j] = L[j - 1];
            L[j] = x;
        }
        const int64_t rb = row_off[v], d = row_off[v + 1] - rb;
        int32_t kept = 0;
        for (int64_t i = 0; i < c; ++i) {
            const int32_t x = L[i];
            if (i > 0 && x == L[i - 1]) continue;
            if (in_sorted(col_idx + rb, d, x)) continue;
            L[kept++] = x;
        }
        fin[v] = kept;
        newdeg[v] = (int32_t)d + kept;
    }
}

constexpr int kRun = 32;  // old entries per lane of the flat merge

// old entries at their new places; warp chunk = 32 * kRun entries, lane run = kRun
__global__ void k_lr_merge_old(int64_t n, const int64_t *__restrict__ row_off, const int32_t *__restrict__ col_idx,
                               const int64_t *__restrict__ loff, const int32_t *__restrict__ list,
                               const int32_t *__restrict__ fin, const int64_t *__restrict__ row_off_out,
                               int32_t *__restrict__ col_out)
{
    const int lane = threadIdx.x & 31;
    const int64_t base = row_off[0], total = row_off[n] - base;
    const int64_t chunk = 32 * (int64_t)kRun;
    const int64_t nwarps = (int64_t)gridDim.x * kWarpsPerBlock;
    for (int64_t c0 = ((int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5)) * chunk; c0 < total;
         c0 += nwarps * chunk) {
        // rows of the chunk's first and last entries, once per warp
        int64_t v_lo = 0, v_hi = 0;
        if (lane == 0) v_lo = last_at_most(row_off, 0, n - 1, base + c0);
        if (lane == 31) v_hi = last_at_most(row_off, 0, n - 1, base + min(c0 + chunk, total) - 1);
        v_lo = __shfl_sync(0xffffffffu, v_lo, 0);
        v_hi = __shfl_sync(0xffffffffu, v_hi, 31);
        const int64_t p0 = c0 + (int64_t)lane * kRun;
        if (p0 >= total) continue;
        const int64_t p1 = min(p0 + (int64_t)kRun, total);
        int64_t v = last_at_most(row_off, v_lo, v_hi, base + p0);
        int64_t rb = row_off[v], re = row_off[v + 1];
        for (int64_t p = p0; p < p1; ++p) {
            const int64_t q = base + p;
            while (q >= re) {  // past the row's end (empty rows skipped)
                ++v;
                rb = re;
                re = row_off[v + 1];
            }
            const int32_t x = col_idx[q];
            const int64_t f = fin[v];
            const int64_t shift = f ? lower_bound(list + loff[v], 0, f, x) : 0;
            col_out[row_off_out[v] + (q - rb) + shift] = x;
        }
    }
}

// kept partners at their new places (one thread per vertex)
__global__ void k_lr_merge_new(int64_t n, const int64_t *__restrict__ row_off, const int32_t *__restrict__ col_idx,
                               const int64_t *__restrict__ loff, const int32_t *__restrict__ list,
                               const int32_t *__restrict__ fin, const int64_t *__restrict__ row_off_out,
                               int32_t *__restrict__ col_out)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const int64_t f = fin[v];
        if (f == 0) continue;
        const int32_t *O = col_idx + row_off[v];
        const int64_t d = row_off[v + 1] - row_off[v];
        const int32_t *Nw = list + loff[v];
        for (int64_t j = 0; j < f; ++j) {
            const int32_t y = Nw[j];
            col_out[row_off_out[v] + j + lower_bound(O, 0, d, y)] = y;
        }
    }
}

}  // namespace

cudaError_t launch_lr_count(int64_t n, int64_t count, uint64_t seed, int32_t *cnt, cudaStream_t s)
{
    k_lr_count<<<std::min(grid_for(count, kThreads * 4), 152u * 16u), kThreads, 0, s>>>(n, count, seed, cnt);
    return cudaGetLastError();
}

cudaError_t launch_lr_fill(int64_t n, int64_t count, uint64_t seed, const int64_t *loff, int32_t *cur, int32_t *list,
                           cudaStream_t s)
{
    k_lr_fill<<<std::min(grid_for(count, kThreads * 4), 152u * 16u), kThreads, 0, s>>>(n, count, seed, loff, cur,
                                                                                       list);
    return cudaGetLastError();
}

cudaError_t launch_lr_clean(int64_t n, const int64_t *row_off, const int32_t *col_idx, const int64_t *loff,
                            int32_t *list, int32_t *fin, int32_t *newdeg, cudaStream_t s)
{
    k_lr_clean<<<grid_for(n, kThreads * 4), kThreads, 0, s>>>(n, row_off, col_idx, loff, list, fin, newdeg);
    return cudaGetLastError();
}

cudaError_t launch_lr_merge(int64_t n, int64_t old_entries, const int64_t *row_off, const int32_t *col_idx,
                            const int64_t *loff, const int32_t *list, const int32_t *fin, const int64_t *row_off_out,
                            int32_t *col_out, cudaStream_t s)
{
    if (old_entries > 0)
        k_lr_merge_old<<<std::min(grid_for(old_entries, kThreads * kRun), 152u * 16u), kThreads, 0, s>>>(
            n, row_off, col_idx, loff, list, fin, row_off_out, col_out);
    k_lr_merge_new<<<grid_for(n, kThreads * 4), kThreads, 0, s>>>(n, row_off, col_idx, loff, list, fin, row_off_out,
                                                                 col_out);
    return cudaGetLastError();
}

}  // namespace hrg
