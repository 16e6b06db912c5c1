// hrg_internal.h -- launchers shared between the generator's translation units.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "hrg_common.cuh"

namespace hrg {

// ---- points (hrg_points.cu) ----
// The sampler's table of 2^63 / F_j, log F_j 2^64 and ln 2 2^64 (acosh_fix);
// once per device.
cudaError_t upload_log_table();
// Sampler of Algorithm 1 (angle and radius draws, Eq. (1)): writes r, phi in
// vertex-id order, and with them every point's angular bucket (gbuf), its
// rank inside the bucket (slot; order inside a bucket is unspecified), the
// bucket occupancy (cnt, zeroed by the caller) and the exact per-band counts
// (band_cnt, zeroed by the caller) under the plan's bucket layout.
cudaError_t launch_sample_bucket(const Plan &p, uint64_t seed, double *r, double *phi, int32_t *gbuf, int32_t *slot,
                                 int32_t *cnt, int64_t *band_cnt, cudaStream_t s);
// Per-band point counts of an injected point set.
cudaError_t launch_count_bands(const Plan &p, const double *r, const double *phi, int64_t *band_cnt, cudaStream_t s);
// The same bucket data for an injected point set: angular-bucket id of every
// point (gbuf, id order), bucket occupancy (cnt) and the point's rank inside
// its bucket (slot).
cudaError_t launch_bucket_hist(const Plan &p, const double *r, const double *phi, int32_t *gbuf, int32_t *slot,
                               int32_t *cnt, cudaStream_t s);
// Structure-of-arrays in bucket order (point i at start[gbuf[i]] + slot[i]):
// fixed-point angle, FP32 scaled exps + id; optionally the FP64 data of the
// plain double-precision path.  pos_of[i] receives point i's position.  With
// rec (PointRec[n] scratch) non-null, angle and exps travel as one record per
// position and a second kernel splits them (FP32 path; pms64 must be null).
struct __align__(32) PointRec { PMS q; uint64_t A; uint64_t pad; };
static_assert(sizeof(PointRec) == 32, "one record is one 32-byte sector");
cudaError_t launch_scatter_soa(const Plan &p, const int32_t *gbuf, const int32_t *slot, const int32_t *start,
                               const double *r, const double *phi, PointRec *rec, uint64_t *A, PMS *pms,
                               PMS64 *pms64, int32_t *pos_of, cudaStream_t s);

// Batches: plans[NG] in device memory, graph g owning positions and global
// ids [plans[g].id_off, plans[g].id_off + plans[g].n).
cudaError_t launch_graph_of(const Plan *plans, int NG, int32_t *graph_of, cudaStream_t s);
cudaError_t launch_sample_bucket_batch(const Plan *plans, const int32_t *graph_of, int64_t N, double *r, double *phi,
                                       int32_t *gbuf, int32_t *slot, int32_t *cnt, cudaStream_t s);
cudaError_t launch_scatter_soa_batch(const Plan *plans, const int32_t *graph_of, int64_t N, const int32_t *gbuf,
                                     const int32_t *slot, const int32_t *start, const double *r, const double *phi,
                                     PointRec *rec, uint64_t *A, PMS *pms, PMS64 *pms64, int32_t *pos_of,
                                     cudaStream_t s);
// hub queries of every graph: fill=false counts them (hub_cnt[NG]) and scans
// into hub_off[NG+1]; fill=true writes their positions into hub_pos
cudaError_t launch_hub_list(const Plan *plans, int NG, const int32_t *start, int32_t *hub_cnt, int32_t *hub_off,
                            int32_t *hub_pos, void *ws, cudaStream_t s, bool fill);

// Exclusive prefix sums with the total stored at out[N].
size_t scan_workspace_bytes(int64_t N);
int scan_launches(int64_t N);  // kernels one scan of length N launches
cudaError_t scan_i32_to_i32(const int32_t *in, int32_t *out, int64_t N, void *ws, cudaStream_t s);
cudaError_t scan_i32_to_i64(const int32_t *in, int64_t *out, int64_t N, void *ws, cudaStream_t s);

// ---- queries (hrg_query.cu) and row sorts (hrg_sort.cu) ----
constexpr int kRegRow = 32;       // rows up to this are sorted in registers by the write pass
constexpr int kKeepRow = 256;     // rows up to this are kept by the count pass (no second traversal)
constexpr int kCopySortRow = 128; // kept rows up to this are sorted by the copy, longer ones by the row sort
constexpr int kWarpRow = 1024;    // rows up to this: one warp, bucket sort in shared memory
constexpr int kSmemRow = 12288;   // rows up to this: one CTA, bucket sort in shared memory

// Up to 64 ids sorted ascending by a bitonic network over a warp's registers:
// element i in lane i mod 32 (register a for i < 32, b for i >= 32), pads
// 0x7fffffff.  Partners j < 32 apart are exchanged by shuffles, the pair 32
// apart sits inside a lane; the lower index of a pair keeps the minimum when
// its block sorts ascending.
__device__ __forceinline__ void warp_bitonic64(int32_t &a, int32_t &b, int lane)
{
#pragma unroll
    for (int k = 2; k <= 64; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j == 32) {  // k = 64: every block ascending
                const int32_t lo = min(a, b), hi = max(a, b);
                a = lo;
                b = hi;
            } else {
                const int32_t pa = __shfl_xor_sync(0xffffffffu, a, j), pb = __shfl_xor_sync(0xffffffffu, b, j);
                const bool lower = (lane & j) == 0;
                const bool up_a = (lane & k) == 0, up_b = ((lane + 32) & k) == 0;
                a = (lower == up_a) ? min(a, pa) : max(a, pa);
                b = (lower == up_b) ? min(b, pb) : max(b, pb);
            }
        }
    }
}

// Up to 32 R ids sorted the same way with R registers a lane (R = 2, 4, 8):
// element i = lane + 32 r in v[r].  Partners 32 or more apart sit inside a
// lane (registers r and r | j/32), nearer ones are exchanged by shuffles.
template <int R>
__device__ __forceinline__ void warp_bitonic_regs(int32_t (&v)[R], int lane)
{
#pragma unroll
    for (int k = 2; k <= 32 * R; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= 32) {
                const int rj = j >> 5;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    if (r & rj) continue;  // r is the lower index of the pair (r, r | rj)
                    const bool up = ((lane + 32 * r) & k) == 0;
                    const int32_t lo = min(v[r], v[r | rj]), hi = max(v[r], v[r | rj]);
                    v[r] = up ? lo : hi;
                    v[r | rj] = up ? hi : lo;
                }
            } else {
                const bool lower = (lane & j) == 0;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int32_t p = __shfl_xor_sync(0xffffffffu, v[r], j);
                    const bool up = ((lane + 32 * r) & k) == 0;
                    v[r] = (lower == up) ? min(v[r], p) : max(v[r], p);
                }
            }
        }
    }
}

__device__ __forceinline__ void warp_bitonic128(int32_t (&v)[4], int lane) { warp_bitonic_regs<4>(v, lane); }

struct QueryBufs {
    const uint64_t *A;        // [n] fixed-point angles, bucket order
    const PMS *pms;           // [n] FP32 scaled exps + id
    const PMS64 *pms64;       // [n] FP64 data (plain path) or null
    const int32_t *start;     // [G+1] first position of each bucket
    const double *r;          // [n] id order (FP64 recheck)
    const double *phi;        // [n] id order
    int32_t *deg;             // [n] id order
    unsigned long long *stats;  // [8] counters: candidates, rechecks, edges, ..., [7] error flag
    int32_t *rows[3];         // ids of rows to sort: (kRegRow, kWarpRow], (kWarpRow, kSmemRow], > kSmemRow
    int32_t *list_cnt;        // [16] lengths: [0..2] the three sort lists, [3] heavy segments,
                              //     [4..7] rim rows to traverse again
    const int32_t *pos_of;    // [n] by vertex id: its position in the band structure
    int32_t *relist[4];       // [n] each: positions of rim queries the write pass traverses again, by
                              //     length: up to 64, 128, 256 entries, longer
    int64_t *big_total;       // [1] sum of degrees of the longest rows
    int4 *heavy;              // [heavy_cap] (query position, 2*band+part, begin, end) of long hub ranges
    int32_t heavy_cap;
    int32_t *cursor;          // [p_hub] write cursor of each hub row's heavy segments
    int32_t *warp_cnt;        // [p_hub] entries a hub query's own warp found (count pass)
    int32_t *seg_cnt;         // [heavy_cap] entries found in each heavy segment (count pass)
    int32_t *col_out;         // CSR neighbour ids being written (write pass only)
    // hub entries pooled by the count pass (null pool: not pooled)
    int32_t *pool;            // [pool_cap] the ids found for hub rows, in runs of one query each
    int4 *runs;               // [run_cap] (hub query, entries, pool offset lo, hi) of every run
    unsigned long long *pool_cur;  // [1] runs reserved << 40 | pool entries reserved (above the caps: overflow)
    int64_t pool_cap;         // below 2^40
    int32_t run_cap;          // below 2^24
    int32_t *small;           // [small_cap] rim rows of up to kKeepRow entries kept by the count pass
    int32_t *small_off;       // [n] by position: start of the kept row in small, -1 if none
    unsigned long long *small_cursor;  // [1] bump allocator over small
    int64_t small_cap;
    // batches of graphs (null / 0 for a single graph)
    const Plan *plans;        // [NG] the graphs' plans in device memory
    const int32_t *graph_of;  // [N] graph of every position (= of every global id)
    const int64_t *sec_off;   // [NG+1] first global rim sector of each graph
    const int32_t *hub_pos;   // [hub queries] position of each hub query
    const int64_t *noff;      // [NG+1] first global id of each graph
    int32_t NG;
    int64_t n_sectors;        // rim sectors over all graphs
};

constexpr int kHeavy = 8192;      // hub ranges longer than this are split into chunks for whole CTAs

// Degrees of hub-band vertices (one warp each, long ranges as CTA chunks).
// deg must be zero for them beforehand.
cudaError_t launch_count_hub(const Plan &p, const QueryBufs &b, bool fp64_only, int32_t p_hub, cudaStream_t s);
// Degrees of rim-band vertices (one CTA per angular sector, one thread per vertex).
cudaError_t launch_count_rim(const Plan &p, const QueryBufs &b, bool fp64_only, cudaStream_t s);
// Same traversals, writing neighbour ids into col_idx[row_off[id] ..]; hub
// rows are written in no particular order (sorted later): the query's warp
// first, then its heavy segments, each at an offset reserved with one atomic.
// The hub rows of ids [lo, hi) from the pooled runs (one atomic per run on
// the row's cursor, cursor zeroed by the caller); check: then every hub row's
// cursor checked against its degree (after the last range).
cudaError_t launch_copy_hub(const QueryBufs &b, int32_t p_hub, int32_t n_runs, const int64_t *row_off,
                            int32_t *col_idx, int64_t lo, int64_t hi, bool check, cudaStream_t s);
cudaError_t launch_write_hub(const Plan &p, const QueryBufs &b, bool fp64_only, int32_t p_hub,
                             const int64_t *row_off, int32_t *col_idx, cudaStream_t s);
// Rim rows of ids [lo, hi) (lo a multiple of 32): kept rows are copied
// (those of up to kCopySortRow entries sorted on the way), the others
// traversed again.
cudaError_t launch_write_rim(const Plan &p, const QueryBufs &b, bool fp64_only, const int64_t *row_off,
                             int32_t *col_idx, int64_t lo, int64_t hi, cudaStream_t s);
int query_launches(const Plan &p, int32_t p_hub, bool write);
// Moved vertices of a dynamic update: one CTA per id in ids[k] queries its
// position in the band structure.  Count (write = false): deg[u] = new
// degree, add[w] += 1 for each neighbour w whose bit in moved is clear.
// Write: u's row (unsorted) at row_off_out[u]; u into each such w's row at
// row_off_out[w] + keep[w] + (slot from add[w], zeroed by the caller).
cudaError_t launch_move_query(const Plan &p, const QueryBufs &b, bool fp64_only, bool write, int64_t k,
                              const int32_t *ids, const uint32_t *moved, int32_t *deg, int32_t *add,
                              const int32_t *keep, const int64_t *row_off_out, int32_t *col_out, cudaStream_t s);

// ---- vertex movement (hrg_update.cu) ----
// moved: one bit per vertex (zeroed by the caller); err |= 1 for an id or a
// coordinate out of range, 2 for a repeated id.
cudaError_t launch_move_check(int64_t n, int64_t k, double R, const int32_t *ids, const double *r_new,
                              const double *phi_new, uint32_t *moved, int *err, cudaStream_t s);
cudaError_t launch_move_apply(int64_t k, const int32_t *ids, const double *r_new, const double *phi_new, double *r,
                              double *phi, cudaStream_t s);
// rem[w] += moved vertices in the old row of w (w not moved; rem zeroed by the caller)
cudaError_t launch_move_removed(int64_t k, const int32_t *ids, const int64_t *row_off, const int32_t *col_idx,
                                const uint32_t *moved, int32_t *rem, cudaStream_t s);
// new degrees (deg: moved rows' counts in, all new degrees out), keep[w] =
// old degree - removed; l[0..2]: rows to sort by length class as for the
// row sort (counts cnt[0..2] zeroed by the caller)
struct MoveLists { int32_t *l[3]; };
// (ws: move_rows_ws_bytes(entries), kept until launch_move_rows; entries =
// old entries from row_off[0]: the chunks of the flat copy that hold a changed
// row are marked there)
cudaError_t launch_move_degrees(int64_t n, int64_t entries, const int64_t *row_off, const uint32_t *moved,
                                const int32_t *rem, const int32_t *add, int32_t *deg, int32_t *keep, MoveLists lists,
                                int32_t *cnt, unsigned long long *big_total, void *ws, cudaStream_t s);
// the rows of the vertices that stay, copied as one flat array of the old
// entries (entries old entries from row_off[0]) without the moved vertices;
// start_drop: int32[n] scratch, ws: move_rows_ws_bytes(entries)
size_t move_rows_ws_bytes(int64_t entries);
cudaError_t launch_move_rows(int64_t n, int64_t entries, const int64_t *row_off, const int32_t *col_idx,
                             const uint32_t *moved, const int32_t *rem, int32_t *start_drop, void *ws,
                             const int64_t *row_off_out, int32_t *col_out, cudaStream_t s);
cudaError_t launch_move_check_gains(int64_t n, const int32_t *cnt, const int32_t *cur, unsigned long long *err,
                                    cudaStream_t s);

// Sort rows longer than kRegRow; tmp holds big_total ids, ws big_sort_ws_bytes.
size_t sort_smem_bytes();
size_t big_sort_ws_bytes(int n_big, int64_t big_total);
int sort_launches(const int32_t counts[3]);
cudaError_t launch_sort_rows(const Plan &p, const QueryBufs &b, const int32_t counts[3], int64_t big_total,
                             const int64_t *row_off, int32_t *col_idx, int32_t *tmp, void *ws, cudaStream_t s);
// The three sort lists split by id range: range k = [bounds[k], bounds[k+1])
// of K ranges.  Class c's rows of range k go to sub + off_c + k cap_c (off_c
// = K (cap_0 + ... + cap_{c-1}), cap_c = counts[c]), their number to
// sub_cnt[3 k + c] and, for class 2, their degree sum to sub_tot[k]
// (sub_cnt and sub_tot zeroed by the caller).
cudaError_t launch_split_lists(const QueryBufs &b, const int32_t counts[3], int K, const int64_t *bounds,
                               const int64_t *row_off, int32_t *sub, int32_t *sub_cnt, int64_t *sub_tot,
                               cudaStream_t s);

}  // namespace hrg
