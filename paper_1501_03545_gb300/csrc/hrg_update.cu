// hrg_update.cu -- vertex movement: the graph after k vertices moved.
//
// The paper's conclusion names a dynamic model, vertices that move on the
// disk, as future work and leaves the movement open; here the moves are the
// caller's input (new coordinates of k vertices) and the result is the
// threshold graph (Sec. 2.1's edge rule) of the updated point set.  Because
// the edge rule is symmetric, only rows that hold a moved vertex change:
//   * a moved vertex u gets a fresh row: its new position is queried against
//     the band structure rebuilt from the updated points (hrg_query.cu,
//     k_move_query);
//   * a vertex w that stays loses the moved vertices of its old row (they
//     are exactly those whose old rows hold w) and gains the moved vertices
//     whose new rows hold it.
// So: count the removals (walking the moved vertices' old rows), the gains
// and the moved rows (the count pass of the moved queries), form the new
// degrees and row offsets; then copy every untouched row as one flat array,
// compact the rows that lost entries, let the moved queries write their rows
// and append themselves to the rows that gained them, and sort the rows that
// were written out of order (the moved rows and the rows that gained).
#include <algorithm>
#include "hrg_internal.h"
#include "hrg_graph_util.cuh"

namespace hrg {

namespace {

using namespace graph_util;

constexpr int kThreads = 256;
constexpr int kWarpsPerBlock = kThreads / 32;
constexpr int kRun = 32;  // old entries per lane of the flat copy

__device__ __forceinline__ bool is_moved(const uint32_t *__restrict__ moved, int64_t v)
{
    return (__ldg(moved + (v >> 5)) >> (v & 31)) & 1u;
}

// ids in [0, n) and distinct, coordinates in [0, R) x [0, 2pi): err |= 1 on
// a bad coordinate or id, 2 on a repeated id; moved bits set
__global__ void k_mv_check(int64_t n, int64_t k, double R, const int32_t *__restrict__ ids,
                           const double *__restrict__ r_new, const double *__restrict__ phi_new,
                           uint32_t *__restrict__ moved, int *__restrict__ err)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += stride) {
        const int32_t id = ids[i];
        const double r = r_new[i], ph = phi_new[i];
        if (id < 0 || id >= n || !(r >= 0.0 && r < R) || !(ph >= 0.0 && ph < kTwoPi)) {
            atomicOr(err, 1);
            continue;
        }
        const uint32_t bit = 1u << (id & 31);
        if (atomicOr(moved + (id >> 5), bit) & bit) atomicOr(err, 2);
    }
}

__global__ void k_mv_apply(int64_t k, const int32_t *__restrict__ ids, const double *__restrict__ r_new,
                           const double *__restrict__ phi_new, double *__restrict__ r, double *__restrict__ phi)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += stride) {
        const int32_t id = ids[i];
        r[id] = r_new[i];
        phi[id] = phi_new[i];
    }
}

// rem[w] += 1 for every vertex w that stays, per moved vertex in its old row
// (one warp per moved vertex)
__global__ void k_mv_removed(int64_t k, const int32_t *__restrict__ ids, const int64_t *__restrict__ row_off,
                             const int32_t *__restrict__ col_idx, const uint32_t *__restrict__ moved,
                             int32_t *__restrict__ rem)
{
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * kWarpsPerBlock;
    for (int64_t i = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5); i < k; i += nw) {
        const int32_t u = ids[i];
        const int64_t b = row_off[u], e = row_off[u + 1];
        for (int64_t q = b + lane; q < e; q += 32) {
            const int32_t w = col_idx[q];
            if (!is_moved(moved, w)) atomicAdd(rem + w, 1);
        }
    }
}

// list[...] += v for the lanes with f: one atomic per warp
__device__ __forceinline__ void warp_push(int32_t *list, int32_t *count, bool f, int32_t v)
{
    const int lane = threadIdx.x & 31;
    const unsigned m = __ballot_sync(0xffffffffu, f);
    if (m == 0) return;
    int32_t base = 0;
    if (lane == 0) base = atomicAdd(count, __popc(m));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (f) list[base + __popc(m & ((1u << lane) - 1u))] = v;
}

// New degrees.  A moved vertex: its fresh count (deg, from the count pass).
// A vertex that stays: old degree - removed + gained; keep[w] = old degree -
// removed, the start of its gained entries.  Rows that lost entries go to
// the compaction list (lists[3], count cnt[3]); rows written out of order
// (moved, or gained) with two or more entries to the sort lists by length
// (lists[0..2], cnt[0..2]; the longest ones' total in *big_total).
__global__ void k_mv_degrees(int64_t n, const int64_t *__restrict__ row_off, const uint32_t *__restrict__ moved,
                             const int32_t *__restrict__ rem, const int32_t *__restrict__ add,
                             int32_t *__restrict__ deg, int32_t *__restrict__ keep, MoveLists lists, int32_t *cnt,
                             unsigned long long *big_total)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t n_up = (n + 31) & ~(int64_t)31;  // whole warps (warp_push)
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n_up; v += stride) {
        bool compact = false, sort = false;
        int32_t d = 0;
        if (v < n) {
            if (is_moved(moved, v)) {
                d = deg[v];
                sort = d >= 2;
            } else {
                const int32_t od = (int32_t)(row_off[v + 1] - row_off[v]), rm = rem[v], ad = add[v];
                d = od - rm + ad;
                deg[v] = d;
                keep[v] = od - rm;
                compact = rm > 0;
                sort = ad > 0 && d >= 2;
            }
        }
        warp_push(lists.l[3], cnt + 3, compact, (int32_t)v);
        const int cls = d <= kWarpRow ? 0 : (d <= kSmemRow ? 1 : 2);
#pragma unroll
        for (int c = 0; c < 3; ++c) warp_push(lists.l[c], cnt + c, sort && cls == c, (int32_t)v);
        if (sort && cls == 2) atomicAdd(big_total, (unsigned long long)d);
    }
}

// Rows that neither moved nor lost an entry, copied as one flat array of the
// old entries (warp chunk = 32 kRun entries, lane run = kRun; the warp finds
// its chunk's rows once): entry q of row v goes to row_off_out[v] + (q - start).
__global__ void k_mv_copy(int64_t n, const int64_t *__restrict__ row_off, const int32_t *__restrict__ col_idx,
                          const uint32_t *__restrict__ moved, const int32_t *__restrict__ rem,
                          const int64_t *__restrict__ row_off_out, int32_t *__restrict__ col_out)
{
    const int lane = threadIdx.x & 31;
    const int64_t base = row_off[0], total = row_off[n] - base;
    const int64_t chunk = 32 * (int64_t)kRun;
    const int64_t nwarps = (int64_t)gridDim.x * kWarpsPerBlock;
    for (int64_t c0 = ((int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5)) * chunk; c0 < total;
         c0 += nwarps * chunk) {
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
        bool skip = is_moved(moved, v) || rem[v] > 0;
        int64_t dst = row_off_out[v] - rb;
        for (int64_t p = p0; p < p1; ++p) {
            const int64_t q = base + p;
            while (q >= re) {  // past the row's end (empty rows skipped)
                ++v;
                rb = re;
                re = row_off[v + 1];
                skip = is_moved(moved, v) || rem[v] > 0;
                dst = row_off_out[v] - rb;
            }
            if (!skip) col_out[dst + q] = col_idx[q];
        }
    }
}

// Rows that lost entries (and did not move): the old row without the moved
// vertices, order kept, at row_off_out[v] (one warp per row).
__global__ void k_mv_compact(const int32_t *__restrict__ rows, const int32_t *__restrict__ nrows,
                             const int64_t *__restrict__ row_off, const int32_t *__restrict__ col_idx,
                             const uint32_t *__restrict__ moved, const int64_t *__restrict__ row_off_out,
                             int32_t *__restrict__ col_out)
{
    const int lane = threadIdx.x & 31;
    const int32_t nr = *nrows;
    const int64_t nw = (int64_t)gridDim.x * kWarpsPerBlock;
    for (int64_t t = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5); t < nr; t += nw) {
        const int32_t v = rows[t];
        const int64_t b = row_off[v], e = row_off[v + 1];
        int64_t out = row_off_out[v];
        for (int64_t q0 = b; q0 < e; q0 += 32) {
            const int64_t q = q0 + lane;
            int32_t x = 0;
            bool keep = false;
            if (q < e) {
                x = col_idx[q];
                keep = !is_moved(moved, x);
            }
            const unsigned m = __ballot_sync(0xffffffffu, keep);
            if (keep) col_out[out + __popc(m & ((1u << lane) - 1u))] = x;
            out += __popc(m);
        }
    }
}

// the write pass gave every row that stays exactly the gains the count pass found
__global__ void k_mv_check_gains(int64_t n, const int32_t *__restrict__ cnt, const int32_t *__restrict__ cur,
                                 unsigned long long *err)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        if (cnt[v] != cur[v]) atomicOr(err, 1ull);
}

}  // namespace

cudaError_t launch_move_check(int64_t n, int64_t k, double R, const int32_t *ids, const double *r_new,
                              const double *phi_new, uint32_t *moved, int *err, cudaStream_t s)
{
    if (k <= 0) return cudaSuccess;
    k_mv_check<<<grid_for(k, kThreads), kThreads, 0, s>>>(n, k, R, ids, r_new, phi_new, moved, err);
    return cudaGetLastError();
}

cudaError_t launch_move_apply(int64_t k, const int32_t *ids, const double *r_new, const double *phi_new, double *r,
                              double *phi, cudaStream_t s)
{
    if (k <= 0) return cudaSuccess;
    k_mv_apply<<<grid_for(k, kThreads), kThreads, 0, s>>>(k, ids, r_new, phi_new, r, phi);
    return cudaGetLastError();
}

cudaError_t launch_move_removed(int64_t k, const int32_t *ids, const int64_t *row_off, const int32_t *col_idx,
                                const uint32_t *moved, int32_t *rem, cudaStream_t s)
{
    if (k <= 0) return cudaSuccess;
    k_mv_removed<<<grid_for(k, kWarpsPerBlock), kThreads, 0, s>>>(k, ids, row_off, col_idx, moved, rem);
    return cudaGetLastError();
}

cudaError_t launch_move_degrees(int64_t n, const int64_t *row_off, const uint32_t *moved, const int32_t *rem,
                                const int32_t *add, int32_t *deg, int32_t *keep, MoveLists lists, int32_t *cnt,
                                unsigned long long *big_total, cudaStream_t s)
{
    k_mv_degrees<<<std::min(grid_for(n, kThreads), 152u * 16u), kThreads, 0, s>>>(n, row_off, moved, rem, add, deg,
                                                                                   keep, lists, cnt, big_total);
    return cudaGetLastError();
}

cudaError_t launch_move_rows(int64_t n, const int64_t *row_off, const int32_t *col_idx, const uint32_t *moved,
                             const int32_t *rem, const int32_t *compact_rows, const int32_t *n_compact,
                             int32_t compact_count, const int64_t *row_off_out, int32_t *col_out, cudaStream_t s)
{
    k_mv_copy<<<152u * 16u, kThreads, 0, s>>>(n, row_off, col_idx, moved, rem, row_off_out, col_out);
    if (compact_count > 0)
        k_mv_compact<<<grid_for(compact_count, kWarpsPerBlock), kThreads, 0, s>>>(compact_rows, n_compact, row_off,
                                                                                  col_idx, moved, row_off_out,
                                                                                  col_out);
    return cudaGetLastError();
}

cudaError_t launch_move_check_gains(int64_t n, const int32_t *cnt, const int32_t *cur, unsigned long long *err,
                                    cudaStream_t s)
{
    k_mv_check_gains<<<std::min(grid_for(n, kThreads), 152u * 16u), kThreads, 0, s>>>(n, cnt, cur, err);
    return cudaGetLastError();
}

}  // namespace hrg
