// hrg_bfs.cu -- breadth-first search over a generated graph.
//
// Sec. 4.1 measures the diameter (the longest shortest path) of the largest
// component; Sec. 4.2 reports that random long-range edges shorten it.  The
// search is level-synchronous: the frontier's degrees are scanned, and its
// edges are expanded in fixed chunks per thread (a thread finds the frontier
// vertex of its first edge by binary search and walks on), so that a hub of
// millions of neighbours is spread over many threads.  A vertex is claimed by
// the compare-and-swap that sets its distance; the claimant appends it to the
// next frontier.
#include <algorithm>
#include <climits>
#include "hrg_graph_ops.h"
#include "hrg_graph_util.cuh"

namespace hrg {

namespace {

using namespace graph_util;

constexpr int kThreads = 256;
constexpr int kEdgesPerThread = 16;

__global__ void k_bfs_init(int64_t n, int32_t *__restrict__ dist, const int64_t *__restrict__ row_off,
                           unsigned long long *__restrict__ best)
{
    // dist = -1; best = max over v of (degree << 31 | (2^31 - 1 - v)): the
    // highest degree, lowest id among ties
    unsigned long long b = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        dist[v] = -1;
        const unsigned long long d = (unsigned long long)(row_off[v + 1] - row_off[v]);
        const unsigned long long key = (d << 31) | (unsigned long long)(0x7fffffffLL - v);
        b = max(b, key);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) b = max(b, __shfl_down_sync(0xffffffffu, b, o));
    if ((threadIdx.x & 31) == 0 && b) atomicMax(best, b);
}

__global__ void k_bfs_seed(const unsigned long long *__restrict__ best, int64_t source, int32_t *__restrict__ dist,
                           int32_t *__restrict__ frontier, int64_t *__restrict__ source_out, int32_t *__restrict__ far)
{
    const int64_t s = source >= 0 ? source : 0x7fffffffLL - (int64_t)(*best & 0x7fffffffull);
    dist[s] = 0;
    frontier[0] = (int32_t)s;
    *source_out = s;
    *far = INT_MAX;
}

__global__ void k_bfs_frontier_deg(int32_t fsize, const int32_t *__restrict__ frontier,
                                   const int64_t *__restrict__ row_off, int32_t *__restrict__ fdeg)
{
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < fsize) {
        const int32_t u = frontier[i];
        fdeg[i] = (int32_t)(row_off[u + 1] - row_off[u]);
    }
}

__global__ void k_bfs_expand(int32_t level, int32_t fsize, const int32_t *__restrict__ frontier,
                             const int64_t *__restrict__ foff, const int64_t *__restrict__ row_off,
                             const int32_t *__restrict__ col_idx, int32_t *__restrict__ dist,
                             int32_t *__restrict__ next, int32_t *__restrict__ nnext)
{
    const int64_t E = foff[fsize];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x * kEdgesPerThread;
    for (int64_t e0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * kEdgesPerThread; e0 < E; e0 += stride) {
        const int64_t e1 = min(e0 + (int64_t)kEdgesPerThread, E);
        int32_t i = (int32_t)last_at_most(foff, 0, fsize - 1, e0);  // the frontier vertex of edge e0
        int64_t ib = foff[i], ie = foff[i + 1];
        int32_t u = frontier[i];
        int64_t rb = row_off[u];
        for (int64_t e = e0; e < e1; ++e) {
            while (e >= ie) {  // next frontier vertex (those of degree 0 skipped)
                ++i;
                ib = ie;
                ie = foff[i + 1];
                u = frontier[i];
                rb = row_off[u];
            }
            const int32_t w = col_idx[rb + (e - ib)];
            if (dist[w] < 0 && atomicCAS(dist + w, -1, level + 1) == -1) next[atomicAdd(nnext, 1)] = w;
        }
    }
}

// the lowest id at distance ecc
__global__ void k_bfs_far(int64_t n, const int32_t *__restrict__ dist, int32_t ecc, int32_t *__restrict__ far)
{
    int32_t f = INT_MAX;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        if (dist[v] == ecc) {
            f = (int32_t)v;
            break;  // ids only grow along a thread's walk
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) f = min(f, __shfl_down_sync(0xffffffffu, f, o));
    if ((threadIdx.x & 31) == 0 && f != INT_MAX) atomicMin(far, f);
}

}  // namespace

cudaError_t launch_bfs_init(int64_t n, int32_t *dist, const int64_t *row_off, unsigned long long *best,
                            cudaStream_t s)
{
    k_bfs_init<<<grid_for(n, kThreads * 4), kThreads, 0, s>>>(n, dist, row_off, best);
    return cudaGetLastError();
}

cudaError_t launch_bfs_seed(const unsigned long long *best, int64_t source, int32_t *dist, int32_t *frontier,
                            int64_t *source_out, int32_t *far, cudaStream_t s)
{
    k_bfs_seed<<<1, 1, 0, s>>>(best, source, dist, frontier, source_out, far);
    return cudaGetLastError();
}

cudaError_t launch_bfs_frontier_deg(int32_t fsize, const int32_t *frontier, const int64_t *row_off, int32_t *fdeg,
                                    cudaStream_t s)
{
    k_bfs_frontier_deg<<<grid_for(fsize, kThreads), kThreads, 0, s>>>(fsize, frontier, row_off, fdeg);
    return cudaGetLastError();
}

cudaError_t launch_bfs_expand(int32_t level, int32_t fsize, const int32_t *frontier, const int64_t *foff,
                              const int64_t *row_off, const int32_t *col_idx, int32_t *dist, int32_t *next,
                              int32_t *nnext, cudaStream_t s)
{
    // the frontier's edge count stays on the device (foff[fsize]): a
    // persistent grid walks however many there are
    k_bfs_expand<<<152 * 16, kThreads, 0, s>>>(level, fsize, frontier, foff, row_off, col_idx, dist, next, nnext);
    return cudaGetLastError();
}

cudaError_t launch_bfs_far(int64_t n, const int32_t *dist, int32_t ecc, int32_t *far, cudaStream_t s)
{
    k_bfs_far<<<grid_for(n, kThreads * 64), kThreads, 0, s>>>(n, dist, ecc, far);
    return cudaGetLastError();
}

}  // namespace hrg
