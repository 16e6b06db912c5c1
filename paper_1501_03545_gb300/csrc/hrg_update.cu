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
// drop the moved vertices from the rows that lost them, let the moved queries write their rows
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
constexpr int kChunk = 4096;  // old entries a block copies at a time
constexpr int kChunkItems = kChunk / kThreads;

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
// removed, the start of its gained entries.  Rows written out of order
// (moved, or gained) with two or more entries go to the sort lists by length
// (lists[0..2], cnt[0..2]; the longest ones' total in *big_total).
__global__ void k_mv_degrees(int64_t n, const int64_t *__restrict__ row_off, const uint32_t *__restrict__ moved,
                             const int32_t *__restrict__ rem, const int32_t *__restrict__ add,
                             int32_t *__restrict__ deg, int32_t *__restrict__ keep, MoveLists lists, int32_t *cnt,
                             unsigned long long *big_total, int64_t chunks, uint8_t *__restrict__ dirty)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t n_up = (n + 31) & ~(int64_t)31;  // whole warps (warp_push)
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n_up; v += stride) {
        bool sort = false;
        int32_t d = 0;
        if (v < n) {
            bool changed = true;
            if (is_moved(moved, v)) {
                d = deg[v];
                sort = d >= 2;
            } else {
                const int32_t od = (int32_t)(row_off[v + 1] - row_off[v]), rm = rem[v], ad = add[v];
                d = od - rm + ad;
                deg[v] = d;
                keep[v] = od - rm;
                sort = ad > 0 && d >= 2;
                changed = rm > 0 || ad > 0;
            }
            if (changed) {
                // the chunks of the old flat array that hold this row's
                // entries, or its place if it had none, are not plain shifted copies
                const int64_t a = row_off[v] - row_off[0], b = row_off[v + 1] - row_off[0];
                const int64_t c1 = b > a ? (b - 1) / kChunk : a / kChunk;
                for (int64_t c = a / kChunk; c <= c1 && c < chunks; ++c) dirty[c] = 1;
            }
        }
        const int cls = d <= kWarpRow ? 0 : (d <= kSmemRow ? 1 : 2);
#pragma unroll
        for (int c = 0; c < 3; ++c) warp_push(lists.l[c], cnt + c, sort && cls == c, (int32_t)v);
        if (sort && cls == 2) atomicAdd(big_total, (unsigned long long)d);
    }
}

// The rows of the vertices that stay are copied as one flat array of the old
// entries, in chunks of kChunk entries per block (coalesced loads and
// stores).  The block stages the offsets of the chunk's rows in shared memory
// with each row's status (copied as it is; lost entries; moved, so not
// copied) and its shift to the new offsets; an entry's row comes from a
// binary search there.  Only the rows that lost entries look at their
// entries: those holding a moved vertex are dropped, and a kept entry moves
// down by the entries dropped before it in its row, K(q) - K(start of row),
// K the prefix count of dropped entries over the flat array, from the chunk
// totals (scanned) and the prefix inside the chunk.
constexpr int kChunkRows = 512;  // rows a block stages; a chunk over more rows searches global memory
enum : int8_t { ROW_COPY = 0, ROW_DROPS = 1, ROW_MOVED = 2 };

struct ChunkRows {
    int64_t v0, nv;                  // first row overlapping the chunk, rows staged (0: none, search globally)
    int32_t any_drops;               // a row of the chunk lost entries
    int64_t off[kChunkRows + 1];     // row_off[v0 .. v0 + nv]
    int64_t shift[kChunkRows];       // row_off_out[v] - row_off[v]
    int8_t state[kChunkRows];
    int32_t row[kChunk + kChunk / 32];  // staged row of every position (slot p + p/32: no bank conflicts)
};

__device__ __forceinline__ int slot(int64_t p) { return (int)(p + (p >> 5)); }

__device__ __forceinline__ int8_t row_state(const uint32_t *__restrict__ moved, const int32_t *__restrict__ rem,
                                            int64_t v)
{
    return is_moved(moved, v) ? ROW_MOVED : (rem[v] > 0 ? ROW_DROPS : ROW_COPY);
}

// Stages the chunk's rows.  The row of each position: every row that starts
// inside the chunk marks its first position (atomicMax: of several rows
// starting there, the empty ones first, the last one holds the entries),
// then a running maximum over the positions fills the rest.
__device__ __forceinline__ void chunk_rows(ChunkRows &S, int32_t *s_warp, int64_t n, int64_t c,
                                           const int64_t *__restrict__ chunk_row,
                                           const int64_t *__restrict__ row_off,
                                           const int64_t *__restrict__ row_off_out, const uint32_t *__restrict__ moved,
                                           const int32_t *__restrict__ rem, int64_t q0, int64_t q1)
{
    if (threadIdx.x == 0) {
        const int64_t v_lo = chunk_row[c], v_hi = chunk_row[c + 1];  // rows holding q0 and q1 (or the last row)
        S.v0 = v_lo;
        S.nv = v_hi - v_lo + 1 <= kChunkRows ? v_hi - v_lo + 1 : 0;
        S.any_drops = S.nv == 0;  // too many rows to stage: look at every entry
    }
    for (int p = threadIdx.x; p < kChunk + kChunk / 32; p += blockDim.x) S.row[p] = 0;
    __syncthreads();
    const int64_t nv = S.nv;
    if (nv == 0) return;
    bool drops = false;
    for (int64_t i = threadIdx.x; i <= nv; i += blockDim.x) {
        const int64_t v = S.v0 + i;
        const int64_t o = row_off[v];
        S.off[i] = o;
        if (i < nv) {
            S.shift[i] = row_off_out[v] - o;
            S.state[i] = row_state(moved, rem, v);
            drops |= S.state[i] == ROW_DROPS;
        }
    }
    __syncthreads();
    for (int64_t i = 1 + threadIdx.x; i < nv; i += blockDim.x) {
        const int64_t o = S.off[i];
        if (o >= q0 && o < q1) atomicMax(&S.row[slot(o - q0)], (int)i);
    }
    __syncthreads();
    // running maximum: thread t owns positions [kChunkItems t, kChunkItems (t + 1))
    {
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        const int p0 = threadIdx.x * kChunkItems;
        int m = 0;
#pragma unroll
        for (int j = 0; j < kChunkItems; ++j) m = max(m, S.row[slot(p0 + j)]);
        int inc = m;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc = max(inc, y);
        }
        const int below = __shfl_up_sync(0xffffffffu, inc, 1);
        if (lane == 31) s_warp[wid] = inc;
        __syncthreads();
        int run = lane > 0 ? below : 0;
        for (int w = 0; w < wid; ++w) run = max(run, s_warp[w]);
#pragma unroll
        for (int j = 0; j < kChunkItems; ++j) {
            run = max(run, S.row[slot(p0 + j)]);
            S.row[slot(p0 + j)] = run;
        }
    }
    if (__syncthreads_or(drops)) {
        if (threadIdx.x == 0) S.any_drops = 1;
    }
    __syncthreads();
}

// the staged index of the row holding flat position q (q inside the chunk),
// or the row itself (global search) when nothing is staged
__device__ __forceinline__ int64_t row_of(const ChunkRows &S, int64_t n, const int64_t *__restrict__ row_off, int64_t q,
                                          int64_t q0)
{
    if (S.nv == 0) return last_at_most(row_off, S.v0, n - 1, q);
    return S.row[slot(q - q0)];
}

// exclusive block prefix of 0/1 flags, kChunkItems per thread in the order
// j kThreads + t; returns the block total
__device__ __forceinline__ int32_t block_flag_prefix(const bool (&f)[kChunkItems], int32_t (&pre)[kChunkItems],
                                                     int32_t *s_warp)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < kChunkItems; ++j) {
        const unsigned m = __ballot_sync(0xffffffffu, f[j]);
        if (lane == 0) s_warp[j * kWarpsPerBlock + w] = __popc(m);
        pre[j] = __popc(m & ((1u << lane) - 1u));
    }
    __syncthreads();
    if (threadIdx.x < 32) {  // the warps' counts in flat order (j, w), scanned by warp 0
        constexpr int kCounts = kChunkItems * kWarpsPerBlock;  // 128
        int32_t a[kCounts / 32], run = 0;
#pragma unroll
        for (int i = 0; i < kCounts / 32; ++i) {
            a[i] = s_warp[threadIdx.x * (kCounts / 32) + i];
            run += a[i];
        }
        int32_t inc = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if ((int)threadIdx.x >= o) inc += y;
        }
        int32_t ex = inc - run;
#pragma unroll
        for (int i = 0; i < kCounts / 32; ++i) {
            s_warp[threadIdx.x * (kCounts / 32) + i] = ex;
            ex += a[i];
        }
        if (threadIdx.x == 31) s_warp[kCounts] = inc;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kChunkItems; ++j) pre[j] += s_warp[j * kWarpsPerBlock + w];
    const int32_t total = s_warp[kChunkItems * kWarpsPerBlock];
    __syncthreads();
    return total;
}

// the dropped entries of a chunk that has rows with lost entries: f[j] for
// its entries (an entry of such a row that holds a moved vertex), x[j] the ids
__device__ __forceinline__ void chunk_drops(const ChunkRows &S, int64_t n, const int64_t *__restrict__ row_off,
                                            const int32_t *__restrict__ col_idx, const uint32_t *__restrict__ moved,
                                            const int32_t *__restrict__ rem, int64_t q0, int64_t q1,
                                            bool (&f)[kChunkItems], int32_t (&x)[kChunkItems])
{
#pragma unroll
    for (int j = 0; j < kChunkItems; ++j) {
        const int64_t q = q0 + j * kThreads + threadIdx.x;
        f[j] = false;
        x[j] = 0;
        if (q >= q1) continue;
        x[j] = col_idx[q];
        const int64_t i = row_of(S, n, row_off, q, q0);
        const int8_t st = S.nv ? S.state[i] : row_state(moved, rem, i);
        f[j] = st == ROW_DROPS && is_moved(moved, x[j]);
    }
}

// chunk_row[c] = the row holding flat position row_off[0] + c kChunk (each
// chunk start lies in one non-empty row), chunk_row[chunks] = n - 1
__global__ void k_mv_chunk_rows(int64_t n, const int64_t *__restrict__ row_off, int64_t chunks,
                                int64_t *__restrict__ chunk_row)
{
    const int64_t base = row_off[0];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const int64_t a = row_off[v] - base, b = row_off[v + 1] - base;
        if (a == b) continue;
        for (int64_t c = (a + kChunk - 1) / kChunk; c * kChunk < b; ++c) chunk_row[c] = v;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) chunk_row[chunks] = n - 1;
}

// Pass 1: per chunk, the dropped entries (chunk_drop[c]), and for every row
// that lost entries and starts in the chunk, the dropped entries of the chunk
// before its start (start_drop[v]).
__global__ void __launch_bounds__(kThreads) k_mv_drop_count(int64_t n, const int64_t *__restrict__ chunk_row,
                                                           const uint8_t *__restrict__ dirty,
                                                           const int64_t *__restrict__ row_off,
                                                           const int32_t *__restrict__ col_idx,
                                                           const uint32_t *__restrict__ moved,
                                                           const int32_t *__restrict__ rem,
                                                           const int64_t *__restrict__ row_off_out,
                                                           int32_t *__restrict__ chunk_drop,
                                                           int32_t *__restrict__ start_drop)
{
    __shared__ int32_t s_warp[kChunkItems * kWarpsPerBlock + 1];
    __shared__ int16_t s_pre[kChunk];
    __shared__ ChunkRows S;
    const int64_t base = row_off[0], total = row_off[n] - base;
    const int64_t chunks = (total + kChunk - 1) / kChunk;
    for (int64_t c = blockIdx.x; c < chunks; c += gridDim.x) {
        if (!dirty[c]) {  // no changed row: nothing dropped
            if (threadIdx.x == 0) chunk_drop[c] = 0;
            continue;
        }
        const int64_t q0 = base + c * kChunk, q1 = min(q0 + kChunk, base + total);
        chunk_rows(S, s_warp, n, c, chunk_row, row_off, row_off_out, moved, rem, q0, q1);
        if (!S.any_drops) {  // uniform: nothing dropped here
            if (threadIdx.x == 0) chunk_drop[c] = 0;
            __syncthreads();
            continue;
        }
        bool f[kChunkItems];
        int32_t x[kChunkItems], pre[kChunkItems];
        chunk_drops(S, n, row_off, col_idx, moved, rem, q0, q1, f, x);
        const int32_t tot = block_flag_prefix(f, pre, s_warp);
        if (threadIdx.x == 0) chunk_drop[c] = tot;
#pragma unroll
        for (int j = 0; j < kChunkItems; ++j) s_pre[j * kThreads + threadIdx.x] = (int16_t)pre[j];
        __syncthreads();
        // the rows that lost entries and start in [q0, q1)
        if (S.nv > 0) {
            for (int64_t i = threadIdx.x; i < S.nv; i += blockDim.x)
                if (S.state[i] == ROW_DROPS && S.off[i] >= q0 && S.off[i] < q1)
                    start_drop[S.v0 + i] = s_pre[S.off[i] - q0];
        } else {
            for (int64_t v = S.v0 + threadIdx.x; v < n && row_off[v] < q1; v += blockDim.x)
                if (row_off[v] >= q0 && row_state(moved, rem, v) == ROW_DROPS) start_drop[v] = s_pre[row_off[v] - q0];
        }
        __syncthreads();
    }
}

// The chunks that hold no entry of a changed row (dirty[c] == 0): one shift
// for the whole chunk, a plain copy.
__global__ void __launch_bounds__(kThreads) k_mv_copy_clean(int64_t n, const int64_t *__restrict__ chunk_row,
                                                           const uint8_t *__restrict__ dirty,
                                                           const int64_t *__restrict__ row_off,
                                                           const int32_t *__restrict__ col_idx,
                                                           const int64_t *__restrict__ row_off_out,
                                                           int32_t *__restrict__ col_out)
{
    const int64_t base = row_off[0], total = row_off[n] - base;
    const int64_t chunks = (total + kChunk - 1) / kChunk;
    for (int64_t c = blockIdx.x; c < chunks; c += gridDim.x) {
        if (dirty[c]) continue;
        const int64_t v = chunk_row[c];
        const int64_t shift = row_off_out[v] - row_off[v];
        const int64_t q0 = base + c * kChunk, q1 = min(q0 + kChunk, base + total);
        int32_t x[kChunkItems];
#pragma unroll
        for (int j = 0; j < kChunkItems; ++j) {
            const int64_t q = q0 + j * kThreads + threadIdx.x;
            if (q < q1) x[j] = col_idx[q];
        }
#pragma unroll
        for (int j = 0; j < kChunkItems; ++j) {
            const int64_t q = q0 + j * kThreads + threadIdx.x;
            if (q < q1) col_out[q + shift] = x[j];
        }
    }
}

// Pass 2 (the chunk totals scanned into chunk_before): the copy of the
// chunks that hold a changed row.
__global__ void __launch_bounds__(kThreads, 3) k_mv_copy(int64_t n, const int64_t *__restrict__ chunk_row,
                                                        const uint8_t *__restrict__ dirty,
                                                        const int64_t *__restrict__ row_off,
                                                     const int32_t *__restrict__ col_idx,
                                                     const uint32_t *__restrict__ moved,
                                                     const int32_t *__restrict__ rem,
                                                     const int64_t *__restrict__ chunk_before,
                                                     const int32_t *__restrict__ start_drop,
                                                     const int64_t *__restrict__ row_off_out,
                                                     int32_t *__restrict__ col_out)
{
    __shared__ int32_t s_warp[kChunkItems * kWarpsPerBlock + 1];
    __shared__ ChunkRows S;
    const int64_t base = row_off[0], total = row_off[n] - base;
    const int64_t chunks = (total + kChunk - 1) / kChunk;
    for (int64_t c = blockIdx.x; c < chunks; c += gridDim.x) {
        if (!dirty[c]) continue;  // k_mv_copy_clean's
        const int64_t q0 = base + c * kChunk, q1 = min(q0 + kChunk, base + total);
        chunk_rows(S, s_warp, n, c, chunk_row, row_off, row_off_out, moved, rem, q0, q1);
        if (!S.any_drops) {  // uniform: every staged row is copied or skipped whole
#pragma unroll 4
            for (int j = 0; j < kChunkItems; ++j) {
                const int64_t q = q0 + j * kThreads + threadIdx.x;
                if (q >= q1) continue;
                const int64_t i = row_of(S, n, row_off, q, q0);
                if (S.state[i] == ROW_COPY) col_out[q + S.shift[i]] = col_idx[q];
            }
            __syncthreads();
            continue;
        }
        bool f[kChunkItems];
        int32_t x[kChunkItems], pre[kChunkItems];
        chunk_drops(S, n, row_off, col_idx, moved, rem, q0, q1, f, x);
        block_flag_prefix(f, pre, s_warp);
        const int64_t kc = chunk_before[c];
#pragma unroll
        for (int j = 0; j < kChunkItems; ++j) {
            const int64_t q = q0 + j * kThreads + threadIdx.x;
            if (q >= q1 || f[j]) continue;
            const int64_t i = row_of(S, n, row_off, q, q0);
            const int64_t v = S.nv ? S.v0 + i : i;
            const int8_t st = S.nv ? S.state[i] : row_state(moved, rem, v);
            if (st == ROW_MOVED) continue;
            const int64_t rb = S.nv ? S.off[i] : row_off[v];
            int64_t dst = (S.nv ? S.shift[i] : row_off_out[v] - rb) + q;
            if (st == ROW_DROPS) {  // dropped entries of the row before q: K(q) - K(rb)
                const int64_t cb = (rb - base) / kChunk;
                dst -= (kc + pre[j]) - (chunk_before[cb] + start_drop[v]);
            }
            col_out[dst] = x[j];
        }
        __syncthreads();
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


// workspace of the copy: chunk_drop int32[chunks + 1], chunk_before and
// chunk_row int64[chunks + 1], dirty uint8[chunks + 1], the scan's
size_t move_rows_ws_bytes(int64_t entries)
{
    const int64_t chunks = (entries + kChunk - 1) / kChunk;
    return (4 + 8 + 8 + 1) * (size_t)(chunks + 1) + 2048 + scan_workspace_bytes(chunks + 1);
}

struct MoveRowsWs {
    int32_t *chunk_drop;
    int64_t *chunk_before, *chunk_row;
    uint8_t *dirty;
    void *scan;
};

static MoveRowsWs carve(void *ws, int64_t chunks)
{
    MoveRowsWs m;
    char *w = (char *)ws;
    auto take = [&](size_t bytes) {
        char *p = w;
        w = (char *)(((uintptr_t)(w + bytes) + 255) & ~(uintptr_t)255);
        return p;
    };
    m.chunk_drop = (int32_t *)take(4 * (size_t)(chunks + 1));
    m.chunk_before = (int64_t *)take(8 * (size_t)(chunks + 1));
    m.chunk_row = (int64_t *)take(8 * (size_t)(chunks + 1));
    m.dirty = (uint8_t *)take((size_t)(chunks + 1));
    m.scan = (void *)w;
    return m;
}

cudaError_t launch_move_degrees(int64_t n, int64_t entries, const int64_t *row_off, const uint32_t *moved,
                                const int32_t *rem, const int32_t *add, int32_t *deg, int32_t *keep, MoveLists lists,
                                int32_t *cnt, unsigned long long *big_total, void *ws, cudaStream_t s)
{
    const int64_t chunks = (entries + kChunk - 1) / kChunk;
    MoveRowsWs m = carve(ws, chunks);
    cudaError_t e = cudaMemsetAsync(m.dirty, 0, (size_t)(chunks + 1), s);
    if (e != cudaSuccess) return e;
    k_mv_degrees<<<std::min(grid_for(n, kThreads), 152u * 16u), kThreads, 0, s>>>(
        n, row_off, moved, rem, add, deg, keep, lists, cnt, big_total, chunks, m.dirty);
    return cudaGetLastError();
}

cudaError_t launch_move_rows(int64_t n, int64_t entries, const int64_t *row_off, const int32_t *col_idx,
                             const uint32_t *moved, const int32_t *rem, int32_t *start_drop, void *ws,
                             const int64_t *row_off_out, int32_t *col_out, cudaStream_t s)
{
    if (entries <= 0) return cudaSuccess;
    const int64_t chunks = (entries + kChunk - 1) / kChunk;
    MoveRowsWs m = carve(ws, chunks);
    k_mv_chunk_rows<<<std::min(grid_for(n, kThreads), 152u * 16u), kThreads, 0, s>>>(n, row_off, chunks,
                                                                                     m.chunk_row);
    const unsigned g = (unsigned)std::min<int64_t>(chunks, 1u << 20);
    k_mv_drop_count<<<g, kThreads, 0, s>>>(n, m.chunk_row, m.dirty, row_off, col_idx, moved, rem, row_off_out,
                                           m.chunk_drop, start_drop);
    cudaError_t e = scan_i32_to_i64(m.chunk_drop, m.chunk_before, chunks, m.scan, s);
    if (e != cudaSuccess) return e;
    k_mv_copy_clean<<<std::min<unsigned>(g, 152u * 16u), kThreads, 0, s>>>(n, m.chunk_row, m.dirty, row_off, col_idx,
                                                                          row_off_out, col_out);
    k_mv_copy<<<g, kThreads, 0, s>>>(n, m.chunk_row, m.dirty, row_off, col_idx, moved, rem, m.chunk_before,
                                     start_drop, row_off_out, col_out);
    return cudaGetLastError();
}

cudaError_t launch_move_check_gains(int64_t n, const int32_t *cnt, const int32_t *cur, unsigned long long *err,
                                    cudaStream_t s)
{
    k_mv_check_gains<<<std::min(grid_for(n, kThreads), 152u * 16u), kThreads, 0, s>>>(n, cnt, cur, err);
    return cudaGetLastError();
}

}  // namespace hrg
