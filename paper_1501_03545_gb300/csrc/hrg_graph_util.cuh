// hrg_graph_util.cuh -- small helpers shared by the operations over a
// generated CSR (hrg_props.cu, hrg_longrange.cu, hrg_bfs.cu).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace hrg {
namespace graph_util {

// blocks for `items` at `per_block` items a block, at least 1, at most 2^20
inline unsigned grid_for(int64_t items, int per_block)
{
    int64_t g = (items + per_block - 1) / per_block;
    if (g < 1) g = 1;
    if (g > (1 << 20)) g = 1 << 20;
    return (unsigned)g;
}

// entries of the ascending a[lo, hi) below x: the first index with a[i] >= x
__device__ __forceinline__ int64_t lower_bound(const int32_t *__restrict__ a, int64_t lo, int64_t hi, int32_t x)
{
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (a[mid] < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// the last index i in [lo, hi] with off[i] <= q, for non-decreasing off with
// off[lo] <= q: the row (or list) that holds entry q when off are offsets,
// rows without entries skipped
__device__ __forceinline__ int64_t last_at_most(const int64_t *__restrict__ off, int64_t lo, int64_t hi, int64_t q)
{
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (off[mid] <= q) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace graph_util
}  // namespace hrg
