// hrg_graph_ops.h -- launchers of the operations over a generated CSR:
// the graph properties of Sec. 4.1 (hrg_props.cu) and the random long-range
// edges of Sec. 4.2 (hrg_longrange.cu).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace hrg {

// ---- graph properties of Sec. 4.1 over a canonical CSR ----
// acc_i[0..2] += largest degree (max), tail count, triads; acc_d[0] += tail log sum.
cudaError_t launch_degree_stats(int64_t n, const int64_t *row_off, int64_t d_min, unsigned long long *acc_i,
                                double *acc_d, cudaStream_t s);
// hist[d] += vertices of degree d (hist zeroed by the caller); *overflow set if a degree exceeds max_degree.
cudaError_t launch_degree_hist(int64_t n, const int64_t *row_off, int64_t max_degree, unsigned long long *hist,
                               int *overflow, cudaStream_t s);
// The neighbours ranked above each vertex (rank = (degree, id)): counts (fill = false) or lists (fill = true).
cudaError_t launch_out_edges(int64_t n, const int64_t *row_off, const int32_t *col_idx, int32_t *out_deg,
                             const int64_t *out_off, int32_t *out_col, bool fill, cudaStream_t s);
// *total += triangles; t[v] += triangles at v (t may be null).
cudaError_t launch_triangles(int64_t n, const int64_t *out_off, const int32_t *out_col, unsigned long long *t,
                             unsigned long long *total, cudaStream_t s);
// *acc += sum over v of t_v / (d_v (d_v - 1) / 2).
cudaError_t launch_local_clustering(int64_t n, const int64_t *row_off, const unsigned long long *t, double *acc,
                                    cudaStream_t s);

// ---- random long-range edges (hrg_longrange.cu), pair k from Philox at counter 2^63 + k ----
// cnt[v] += drawn partners of v (cnt zeroed by the caller).
cudaError_t launch_lr_count(int64_t n, int64_t count, uint64_t seed, int32_t *cnt, cudaStream_t s);
// list[loff[v] + ...] = the partners of v (cur zeroed by the caller).
cudaError_t launch_lr_fill(int64_t n, int64_t count, uint64_t seed, const int64_t *loff, int32_t *cur, int32_t *list,
                           cudaStream_t s);
// Partner lists sorted, repeats and present neighbours dropped: fin[v] kept, newdeg[v] = d_v + fin[v].
cudaError_t launch_lr_clean(int64_t n, const int64_t *row_off, const int32_t *col_idx, const int64_t *loff,
                            int32_t *list, int32_t *fin, int32_t *newdeg, cudaStream_t s);
// New rows: old rows (old_entries = row_off[n] - row_off[0]) and kept partners merged, at row_off_out.
cudaError_t launch_lr_merge(int64_t n, int64_t old_entries, const int64_t *row_off, const int32_t *col_idx,
                            const int64_t *loff, const int32_t *list, const int32_t *fin, const int64_t *row_off_out,
                            int32_t *col_out, cudaStream_t s);

// ---- breadth-first search (hrg_bfs.cu) ----
// dist[v] = -1; *best = max over v of (degree << 31 | (2^31 - 1 - v)) (best zeroed by the caller).
cudaError_t launch_bfs_init(int64_t n, int32_t *dist, const int64_t *row_off, unsigned long long *best,
                            cudaStream_t s);
// The source (or, for source < 0, the vertex *best names) at distance 0, alone in frontier; *far = INT_MAX.
cudaError_t launch_bfs_seed(const unsigned long long *best, int64_t source, int32_t *dist, int32_t *frontier,
                            int64_t *source_out, int32_t *far, cudaStream_t s);
cudaError_t launch_bfs_frontier_deg(int32_t fsize, const int32_t *frontier, const int64_t *row_off, int32_t *fdeg,
                                    cudaStream_t s);
// One level: the vertices first reached from the frontier get level + 1 and join next (*nnext counts them).
cudaError_t launch_bfs_expand(int32_t level, int32_t fsize, const int32_t *frontier, const int64_t *foff,
                              const int64_t *row_off, const int32_t *col_idx, int32_t *dist, int32_t *next,
                              int32_t *nnext, cudaStream_t s);
// *far = min(*far, the lowest id at distance ecc).
cudaError_t launch_bfs_far(int64_t n, const int32_t *dist, int32_t ecc, int32_t *far, cudaStream_t s);

}  // namespace hrg
