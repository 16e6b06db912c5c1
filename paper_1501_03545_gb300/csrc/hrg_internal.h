// hrg_internal.h -- launchers shared between the generator's translation units.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "hrg_common.cuh"

namespace hrg {

// ---- points (hrg_points.cu) ----
// Sampler of Algorithm 1 (angle and radius draws, Eq. (1)): writes r, phi in
// vertex-id order and the per-band point counts.
cudaError_t launch_sample(const Plan &p, uint64_t seed, double *r, double *phi, int64_t *band_cnt, cudaStream_t s);
// Per-band point counts of an injected point set.
cudaError_t launch_count_bands(const Plan &p, const double *r, const double *phi, int64_t *band_cnt, cudaStream_t s);
// Angular-bucket id of every point (gbuf, id order) and bucket occupancy.
cudaError_t launch_bucket_hist(const Plan &p, const double *r, const double *phi, int32_t *gbuf, int32_t *cnt,
                               cudaStream_t s);
// perm[start[g] ..] = ids of bucket g (order inside a bucket unspecified).
cudaError_t launch_bucket_scatter(const Plan &p, const int32_t *gbuf, const int32_t *start, int32_t *cnt,
                                  int32_t *perm, cudaStream_t s);
// Structure-of-arrays in bucket order: fixed-point angle, FP32 scaled exps
// + id; optionally the FP64 data of the plain double-precision path.
cudaError_t launch_build_soa(const Plan &p, const int32_t *perm, const double *r, const double *phi, uint64_t *A,
                             PMS *pms, PMS64 *pms64, cudaStream_t s);

// Exclusive prefix sums with the total stored at out[N].
size_t scan_workspace_bytes(int64_t N);
int scan_launches(int64_t N);  // kernels one scan of length N launches
cudaError_t scan_i32_to_i32(const int32_t *in, int32_t *out, int64_t N, void *ws, cudaStream_t s);
cudaError_t scan_i32_to_i64(const int32_t *in, int64_t *out, int64_t N, void *ws, cudaStream_t s);

// ---- queries (hrg_query.cu) ----
struct QueryBufs {
    const uint64_t *A;        // [n] fixed-point angles, bucket order
    const PMS *pms;           // [n] FP32 scaled exps + id
    const PMS64 *pms64;       // [n] FP64 data (plain path) or null
    const int32_t *start;     // [G+1] first position of each bucket
    const double *r;          // [n] id order (FP64 recheck)
    const double *phi;        // [n] id order
    int32_t *deg;             // [n] id order
    unsigned long long *stats;  // [8] counters (see HRG_STAT_*)
    int32_t *mid_rows;        // list of (id) rows with 32 < deg <= kSmemRow
    int32_t *big_rows;        // list of (id) rows with deg > kSmemRow
    int32_t *list_cnt;        // [2] lengths of the two lists
    int64_t *big_total;       // [1] sum of degrees of big rows
};

constexpr int kRegRow = 32;       // rows up to this are sorted in registers
constexpr int kSmemRow = 12288;   // rows up to this are sorted in shared memory

// Degrees of all vertices: queries at sorted positions [0, p_hub) (hub bands)
// run one CTA each, the rest one thread each.
cudaError_t launch_count_split(const Plan &p, const QueryBufs &b, bool fp64_only, int32_t p_hub, cudaStream_t s);
// Same traversal, writing neighbour ids into col_idx[row_off[id] ..].
cudaError_t launch_write_split(const Plan &p, const QueryBufs &b, bool fp64_only, int32_t p_hub,
                               const int64_t *row_off, int32_t *col_idx, cudaStream_t s);
// Sort rows longer than kRegRow (mid rows in shared memory, big rows by id
// buckets through tmp[big_total]).
size_t big_sort_hist_words(int64_t n, int n_big);
cudaError_t launch_sort_rows(const Plan &p, const QueryBufs &b, int n_mid, int n_big, const int64_t *row_off,
                             int32_t *col_idx, int32_t *tmp, int64_t tmp_len, int32_t *bucket_ws,
                             int64_t bucket_ws_len, cudaStream_t s);

}  // namespace hrg
