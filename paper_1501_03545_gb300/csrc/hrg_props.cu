// hrg_props.cu -- the graph properties of Sec. 4.1 over a generated CSR.
//
// Sec. 4.1 studies the degree distribution (a power law with exponent
// gamma = 2 alpha + 1, Sec. 2.1) and the clustering coefficient, defined
// there as the fraction of closed triangles among triads (paths of length
// two).  Over a canonical CSR (rows ascending, both directions of each edge):
//   * one pass over the row offsets: largest degree, triads
//     sum_v d_v (d_v - 1) / 2, and the two sums of the degree tail's discrete
//     maximum-likelihood exponent (Clauset, Shalizi and Newman, SIAM Review
//     51, 2009, Eq. 3.7): the count N of vertices with d >= d_min and
//     sum ln(d / (d_min - 1/2)), gamma = 1 + N / sum;
//   * a degree histogram (shared-memory bins for small degrees);
//   * triangles by the degree-ordered orientation: vertex v keeps its
//     neighbours ranked above it (rank = (degree, id)), N+(v), each at most
//     O(sqrt m) long; a triangle is found once, at its lowest-ranked corner u
//     and its middle corner v, as a common entry of N+(u) and N+(v).  One
//     warp per u, one lane per v in N+(u); the shorter list is searched in
//     the longer.  Every triangle adds one to the count of each corner
//     (local clustering t_v / (d_v (d_v - 1) / 2)).
#include <algorithm>
#include <cstdio>
#include "hrg_graph_ops.h"
#include "hrg_graph_util.cuh"

namespace hrg {

namespace {

using namespace graph_util;

constexpr int kThreads = 256;
constexpr int kWarpsPerBlock = kThreads / 32;
constexpr int kHistSmem = 2048;  // degrees below this are binned in shared memory first

// acc_i: [0] largest degree, [1] tail count, [2] triads; acc_d: [0] tail log sum
__global__ void k_degree_stats(int64_t n, const int64_t *__restrict__ row_off, int64_t d_min,
                               unsigned long long *__restrict__ acc_i, double *__restrict__ acc_d)
{
    unsigned long long mx = 0, tail = 0, triads = 0;
    double logs = 0.0;
    const double den = (double)d_min - 0.5;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const int64_t d = row_off[v + 1] - row_off[v];
        mx = max(mx, (unsigned long long)d);
        triads += (unsigned long long)(d * (d - 1) / 2);
        if (d >= d_min) {
            ++tail;
            logs += log((double)d / den);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_down_sync(0xffffffffu, mx, o));
    tail = warp_sum(tail);
    triads = warp_sum(triads);
    logs = warp_sum(logs);
    if ((threadIdx.x & 31) == 0) {
        if (mx) atomicMax(acc_i + 0, mx);
        if (tail) atomicAdd(acc_i + 1, tail);
        if (triads) atomicAdd(acc_i + 2, triads);
        if (tail) atomicAdd(acc_d, logs);
    }
}

__global__ void k_degree_hist(int64_t n, const int64_t *__restrict__ row_off, int64_t max_degree,
                              unsigned long long *__restrict__ hist, int *__restrict__ overflow)
{
    __shared__ unsigned int sh[kHistSmem];
    for (int k = threadIdx.x; k < kHistSmem; k += blockDim.x) sh[k] = 0;
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const int64_t d = row_off[v + 1] - row_off[v];
        if (d > max_degree) {
            atomicOr(overflow, 1);
        } else if (d < kHistSmem) {
            atomicAdd(&sh[d], 1u);
        } else {
            atomicAdd(hist + d, 1ull);
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kHistSmem; k += blockDim.x)
        if (sh[k]) atomicAdd(hist + k, (unsigned long long)sh[k]);
}

// N+(v): the neighbours w of v with (d_w, w) > (d_v, v), in id order.  One
// warp per vertex; FILL = false counts them, FILL = true writes them.
template <bool FILL>
__global__ void k_out_edges(int64_t n, const int64_t *__restrict__ row_off, const int32_t *__restrict__ col_idx,
                            int32_t *__restrict__ out_deg, const int64_t *__restrict__ out_off,
                            int32_t *__restrict__ out_col)
{
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * kWarpsPerBlock;
    for (int64_t v = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5); v < n; v += nwarps) {
        const int64_t base = row_off[v], d = row_off[v + 1] - base;
        int64_t pos = FILL ? out_off[v] : 0;
        int32_t cnt = 0;
        for (int64_t i0 = 0; i0 < d; i0 += 32) {
            const int64_t i = i0 + lane;
            bool up = false;
            int32_t w = 0;
            if (i < d) {
                w = col_idx[base + i];
                const int64_t dw = row_off[w + 1] - row_off[w];
                up = dw > d || (dw == d && w > v);
            }
            const unsigned m = __ballot_sync(0xffffffffu, up);
            if (FILL && up) out_col[pos + __popc(m & ((1u << lane) - 1u))] = w;
            pos += __popc(m);
            cnt += __popc(m);
        }
        if (!FILL && lane == 0) out_deg[v] = cnt;
    }
}

// Triangles: warp per u, lane per v in N+(u), |N+(u) ∩ N+(v)| by searching
// the shorter list's entries in the longer one (both ascending, so each
// search starts where the last one ended).  t (may be null) gets one per
// corner of every triangle.
__global__ void k_triangles(int64_t n, const int64_t *__restrict__ out_off, const int32_t *__restrict__ out_col,
                            unsigned long long *__restrict__ t, unsigned long long *__restrict__ total)
{
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * kWarpsPerBlock;
    unsigned long long found = 0;
    for (int64_t u = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5); u < n; u += nwarps) {
        const int64_t ab = out_off[u], a = out_off[u + 1] - ab;
        const int32_t *A = out_col + ab;
        unsigned long long tu = 0;
        for (int64_t j = lane; j < a; j += 32) {
            const int32_t v = A[j];
            const int64_t bb = out_off[v], b = out_off[v + 1] - bb;
            const int32_t *B = out_col + bb;
            const int32_t *S = a <= b ? A : B;
            const int32_t *L = a <= b ? B : A;
            const int64_t s = a <= b ? a : b, l = a <= b ? b : a;
            unsigned long long c = 0;
            int64_t p = 0;
            for (int64_t k = 0; k < s && p < l; ++k) {
                const int32_t x = S[k];
                p = lower_bound(L, p, l, x);
                if (p < l && L[p] == x) {
                    ++c;
                    if (t) atomicAdd(t + x, 1ull);
                    ++p;
                }
            }
            if (t && c) atomicAdd(t + v, c);
            tu += c;
        }
        tu = warp_sum(tu);
        if (lane == 0 && tu) {
            if (t) atomicAdd(t + u, tu);
            found += tu;
        }
    }
    if (lane == 0 && found) atomicAdd(total, found);
}

// sum over v of t_v / (d_v (d_v - 1) / 2), vertices of degree < 2 adding 0
__global__ void k_local_clustering(int64_t n, const int64_t *__restrict__ row_off,
                                   const unsigned long long *__restrict__ t, double *__restrict__ acc)
{
    double s = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const int64_t d = row_off[v + 1] - row_off[v];
        if (d >= 2) s += (double)t[v] / (double)(d * (d - 1) / 2);
    }
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0 && s != 0.0) atomicAdd(acc, s);
}

}  // namespace

cudaError_t launch_degree_stats(int64_t n, const int64_t *row_off, int64_t d_min, unsigned long long *acc_i,
                                double *acc_d, cudaStream_t s)
{
    k_degree_stats<<<grid_for(n, kThreads * 4), kThreads, 0, s>>>(n, row_off, d_min, acc_i, acc_d);
    return cudaGetLastError();
}

cudaError_t launch_degree_hist(int64_t n, const int64_t *row_off, int64_t max_degree, unsigned long long *hist,
                               int *overflow, cudaStream_t s)
{
    k_degree_hist<<<std::min(grid_for(n, kThreads * 16), 152u * 8u), kThreads, 0, s>>>(n, row_off, max_degree, hist,
                                                                                       overflow);
    return cudaGetLastError();
}

cudaError_t launch_out_edges(int64_t n, const int64_t *row_off, const int32_t *col_idx, int32_t *out_deg,
                             const int64_t *out_off, int32_t *out_col, bool fill, cudaStream_t s)
{
    const unsigned g = grid_for(n, kWarpsPerBlock * 4);
    if (fill) k_out_edges<true><<<g, kThreads, 0, s>>>(n, row_off, col_idx, out_deg, out_off, out_col);
    else k_out_edges<false><<<g, kThreads, 0, s>>>(n, row_off, col_idx, out_deg, out_off, out_col);
    return cudaGetLastError();
}

cudaError_t launch_triangles(int64_t n, const int64_t *out_off, const int32_t *out_col, unsigned long long *t,
                             unsigned long long *total, cudaStream_t s)
{
    k_triangles<<<grid_for(n, kWarpsPerBlock * 4), kThreads, 0, s>>>(n, out_off, out_col, t, total);
    return cudaGetLastError();
}

cudaError_t launch_local_clustering(int64_t n, const int64_t *row_off, const unsigned long long *t, double *acc,
                                    cudaStream_t s)
{
    k_local_clustering<<<grid_for(n, kThreads * 4), kThreads, 0, s>>>(n, row_off, t, acc);
    return cudaGetLastError();
}

}  // namespace hrg
