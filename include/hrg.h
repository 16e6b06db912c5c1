/*
 * hrg.h -- C ABI of the GB300 generator of threshold random hyperbolic graphs.
 *
 * Model (von Looz, Meyerhenke, Prutkin, Staudt, "Fast generation of complex
 * networks with underlying hyperbolic geometry", Sec. 2.1): n points on a
 * hyperbolic disk of radius R with curvature -1; angle uniform on [0, 2pi),
 * radius with density alpha sinh(alpha r) / (cosh(alpha R) - 1) (Eq. (1));
 * two points are adjacent exactly when their hyperbolic distance is below R.
 * The problem statement of Algorithm 1 is (n, average degree, alpha) -> graph;
 * this library adds a seed and returns the points and the graph:
 *
 *   (n, alpha, kbar, seed) -> r[n], phi[n] (FP64, vertex-id order)
 *                           + CSR: row_off[n+1] (int64), col_idx[2m] (int32)
 *
 * Conventions
 *   - Vertex i is the i-th draw: its uniforms are the Philox4x32-10 block at
 *     counter (i, 0, 0) under key = seed (low word, high word); the top 53
 *     bits of the first and second 64-bit halves give u_phi and u_r;
 *     phi = u_phi * 2pi and r = acosh(1 + u_r (cosh(alpha R) - 1)) / alpha.
 *   - The CSR holds each undirected edge in both rows, no self-loops, every
 *     row strictly ascending.  2m = row_off[n].
 *   - All device pointers are plain CUDA device addresses on the context's
 *     device; host pointers are ordinary (preferably pinned) host memory.
 *   - Every call returns an int status; HRG_OK is 0.  No call throws.  On a
 *     non-OK status the outputs are undefined and hrg_last_error() explains.
 *   - Buffers passed in are owned by the caller.  The library owns the
 *     workspace inside a context; one job may be in flight per context.
 */
#ifndef HRG_H
#define HRG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    HRG_OK = 0,
    HRG_EINVAL = 1,    /* invalid parameter (see each call)                  */
    HRG_ENOMEM = 2,    /* device or pinned host allocation failed            */
    HRG_EOVERFLOW = 3, /* output larger than the caller's capacity / index type */
    HRG_ECUDA = 4,     /* a CUDA runtime error; message in hrg_last_error()  */
    HRG_ESTATE = 5,    /* call out of order (e.g. finish without begin)      */
    HRG_EINTERNAL = 6, /* a device-side consistency check failed             */
    HRG_ETIMEOUT = 7   /* hrg_server_wait: the request is not done yet       */
};

/* Flags of hrg_params.flags */
#define HRG_FLAG_FP64_ONLY 0x1u /* decide every candidate pair in FP64 (the plain path) */

typedef struct hrg_params {
    int64_t n;          /* number of vertices, 2 <= n < 2^31                        */
    double alpha;       /* radial dispersion, alpha > 1/2 (power-law regime, Sec. 2.1) */
    double avg_degree;  /* target average degree kbar, 0 < kbar < n-1               */
    uint64_t seed;      /* Philox key                                                */
    double R_override;  /* > 0: use this disk radius instead of solving Eq. (22)     */
    uint32_t flags;     /* HRG_FLAG_*                                                */
    int32_t bands;      /* 0: automatic; else number of radial bands (1..64)         */
    int32_t hub_candidates; /* 0: automatic (512); vertices whose band's inner radius
                               expects more candidates are queried one warp each     */
    int32_t reserved;
} hrg_params;

typedef struct hrg_stats {
    double R;                    /* radius used                                      */
    int64_t n_entries;           /* 2m, directed CSR entries                         */
    uint64_t candidates;         /* candidate pairs tested in the count pass        */
    uint64_t rechecks;           /* pairs re-decided in FP64 in the count pass      */
    int32_t bands;               /* radial bands                                    */
    int32_t hub_bands;           /* innermost bands queried by whole thread blocks  */
    int64_t buckets;             /* angular buckets over all bands                  */
    int32_t hub_queries;         /* vertices in the hub bands                       */
    int32_t mid_rows;            /* rows sorted in shared memory                    */
    int32_t big_rows;            /* rows sorted by id buckets                       */
    int32_t reserved;
    float mu;                    /* relative half-width of the FP32 undecided band  */
    /* device time of each stage in ms (CUDA events on the job's stream), valid
     * after hrg_generate_finish: [0] sampling, [1] band structure (band counts
     * read-back, bucket counting sort, structure-of-arrays), [2] degree count
     * of hub-band vertices, [3] degree count of rim-band vertices, [4] row
     * offsets, [5] neighbour write of hub-band vertices, [6] neighbour write of
     * rim-band vertices, [7] row sort */
    float stage_ms[8];
    int32_t launches;            /* kernels this library launched for the job       */
    /* the tie band: candidate pairs whose FP64 value cosh d lies within
     * 1e-12 cosh R of cosh R (relative), each pair counted once.  Two
     * correct FP64 evaluations of such a pair may decide it differently, so
     * it is the only place an exact comparison may differ; expected ~0. */
    uint64_t ties;
    /* fallbacks of the count pass (they change the speed, never the graph):
     * rim rows it found no room to keep (the write pass traverses them
     * again), hub rows traversed again because the pool of hub ids or its run
     * table overflowed (0 when the pool held them all), and count passes run
     * again because the list of long hub ranges overflowed */
    int64_t rows_no_room;
    int32_t hub_rows_retraversed;
    int32_t heavy_retries;
    /* id ranges the neighbour write ran in: 1, or (hrg_generate_host, graphs
     * of 2^26 entries or more) up to 8, each range's ids going back to the
     * host while the next is written and sorted; stage_ms[5..7] are then
     * sums over the ranges */
    int32_t write_chunks;
    /* hrg_generate_host only (else -1): ms from the first device-to-host copy
     * (the points, as soon as they are sampled) to the end of the last */
    float d2h_ms;
} hrg_stats;

typedef struct hrg_ctx hrg_ctx;
typedef struct hrg_job hrg_job;

/*
 * hrg_solve_radius -- Appendix B.1 / Algorithm 1 first line.
 * Solves Krioukov et al.'s Eq. (22) (zeta = 1, middle term read as
 * (pi-1)/alpha) for R: returns the largest double R on the decreasing branch
 * of the expression with kbar(R) >= avg_degree.
 * Errors: HRG_EINVAL if n < 2, alpha <= 1/2, avg_degree <= 0,
 * avg_degree >= n-1, or avg_degree above the expression's maximum.
 * Pure host computation; needs no context or device.
 */
int hrg_solve_radius(int64_t n, double alpha, double avg_degree, double *R_out);

/* Expected average degree of Eq. (22) at radius R (zeta = 1). Host only. */
double hrg_expected_degree(int64_t n, double alpha, double R);

/*
 * hrg_create / hrg_destroy -- a context bound to one CUDA device.  The context
 * owns a grow-only device workspace reused across calls; destroy frees it.
 * A generation's workspace (beside the caller's outputs) comes to about 250
 * bytes per vertex of the graph or batch, plus 64 MB, plus 4 bytes per entry
 * of the rows longer than 12288 entries (their sort buffer); less per vertex
 * above n = 6.7e7, where the buffer of kept rows stops growing at 2^31 ids
 * (~200 bytes at n = 1e8).
 * Errors: HRG_EINVAL (null out), HRG_ECUDA (device cannot be selected).
 */
int hrg_create(hrg_ctx **out, int device);
int hrg_destroy(hrg_ctx *ctx);

/* Device bytes the context's workspace holds now (it grows as jobs need it
 * and stays until hrg_release_workspace or hrg_destroy).  Host only.
 * Errors: HRG_EINVAL (null argument). */
int hrg_workspace_bytes(const hrg_ctx *ctx, int64_t *bytes);

/* Frees the context's workspace; the next job allocates what it needs again.
 * Errors: HRG_EINVAL, HRG_ESTATE (a job is open), HRG_ECUDA. */
int hrg_release_workspace(hrg_ctx *ctx);

/*
 * hrg_generate_begin -- sampling, band structure, degree count, row offsets
 * (Algorithm 1 except the edge insertion).
 *   p            parameters (copied)
 *   stream       cudaStream_t (as void*), 0 for the legacy stream
 *   r_out        device double[n]  radii, vertex-id order          (caller owned)
 *   phi_out      device double[n]  angles in [0, 2pi), id order    (caller owned)
 *   row_off_out  device int64[n+1] CSR row offsets                 (caller owned)
 *   job          receives the job handle (owned by the context)
 *   n_entries    receives 2m, the length col_idx must have
 * The call synchronizes the stream twice (band counts, total).  The outputs
 * are complete when it returns.
 * Errors: HRG_EINVAL (bad parameters, null pointers), HRG_ENOMEM, HRG_ECUDA,
 * HRG_ESTATE (a job of this context is still open).
 */
int hrg_generate_begin(hrg_ctx *ctx, const hrg_params *p, void *stream, double *r_out, double *phi_out,
                       int64_t *row_off_out, hrg_job **job, int64_t *n_entries);

/*
 * hrg_generate_from_points_begin -- as hrg_generate_begin for an injected
 * point set (used for special geometries and tests): r[n] (0 <= r), phi[n]
 * (0 <= phi < 2pi) are the caller's device arrays in id order and are only
 * read; R is the disk radius.  Same outputs and errors.
 */
int hrg_generate_from_points_begin(hrg_ctx *ctx, int64_t n, double R, const double *r, const double *phi,
                                   uint32_t flags, int32_t bands, void *stream, int64_t *row_off_out,
                                   hrg_job **job, int64_t *n_entries);

/*
 * hrg_generate_batch_begin -- as hrg_generate_begin for `count` independent
 * graphs generated together: every stage runs once over all of them (one
 * kernel launch per stage for the whole batch), so thousands of small graphs
 * cost about as much as one graph of their total size.
 *   count        1 <= count <= 2^24
 *   items        host hrg_params[count]; each item as in hrg_generate_begin
 *                (its flags are ignored: the batch's `flags` apply to all)
 *   r_out, phi_out   device double[N], N = sum of items[g].n (< 2^31)
 *   row_off_out  device int64[N+1]
 * Layout: graph g owns positions [off_g, off_g + n_g) of r_out, phi_out and
 * the rows [off_g, off_g + n_g) of one concatenated CSR, off_g = n_0 + ... +
 * n_{g-1}.  Its vertex i is Philox counter i under key items[g].seed (the
 * points equal those of a single-graph call with the same parameters), and
 * its rows hold LOCAL vertex ids in [0, n_g), ascending; row_off is global
 * (graph g's entries are col_idx[row_off[off_g] .. row_off[off_g + n_g])).
 * The band layout of each graph is planned from its expected band counts
 * (Eq. (1)), so it can differ from a single-graph call's; the graph cannot.
 * Finish with hrg_generate_finish; hrg_job_stats then reports totals
 * (R, bands and mu of graph 0).
 * Errors: as hrg_generate_begin; an invalid item returns HRG_EINVAL naming
 * the item in hrg_last_error().
 */
int hrg_generate_batch_begin(hrg_ctx *ctx, int32_t count, const hrg_params *items, uint32_t flags, void *stream,
                             double *r_out, double *phi_out, int64_t *row_off_out, hrg_job **job,
                             int64_t *n_entries);

/*
 * hrg_update_begin -- vertex movement.  The paper's conclusion names a
 * dynamic model, in which vertices move and the incremental quadtree follows
 * them, as future work, and defines no movement law; so the moves are an
 * input: vertex ids[i] moves to (r_new[i], phi_new[i]).  The result is the
 * threshold graph (Sec. 2.1's edge rule) of the updated point set -- the
 * graph hrg_generate_from_points_begin builds from it -- as a canonical CSR
 * (rows ascending, symmetric, no self-loops).  Finish with
 * hrg_generate_finish(job, col_idx_out), col_idx_out of *n_entries entries.
 *   n, R        the graph's vertex count (1 <= n < 2^31) and disk radius
 *   r, phi      device double[n]: the current points (caller owned), changed
 *               in place to the updated ones once the moves are accepted
 *   row_off, col_idx  device: the current canonical CSR of (r, phi) (read;
 *               both must stay untouched until finish; row_off[0] may be
 *               non-zero)
 *   k           0 <= k <= n moved vertices; ids device int32[k], distinct,
 *               in [0, n); r_new, phi_new device double[k], 0 <= r_new < R,
 *               0 <= phi_new < 2pi
 *   flags       HRG_FLAG_FP64_ONLY as for generation; bands as for
 *               hrg_generate_from_points_begin
 *   row_off_out device int64[n+1] (caller owned): the new row offsets, from 0
 * Work: the band structure is rebuilt from the updated points (no sampling);
 * only the k moved vertices are queried; every other row changes only by the
 * moved vertices it loses (those in its old row) and gains (those whose new
 * row holds it), so untouched rows are copied and the rest compacted or
 * merged.  The call synchronizes the stream (read-backs of the check and of
 * the totals).  hrg_job_stats reports the moved queries' candidates,
 * rechecks and ties; its stage times are [0] band counts, [1] band
 * structure, [2] moved vertices counted, [3] removals and degrees, [4] row
 * offsets, [5] moved rows written, [6] other rows copied, [7] row sort.
 * Errors: HRG_EINVAL (sizes, null pointers, an id out of range or repeated, a
 * coordinate outside [0, R) x [0, 2pi) -- then r and phi are unchanged),
 * HRG_ESTATE, HRG_ENOMEM, HRG_ECUDA.
 */
int hrg_update_begin(hrg_ctx *ctx, int64_t n, double R, double *r, double *phi, const int64_t *row_off,
                     const int32_t *col_idx, int64_t k, const int32_t *ids, const double *r_new,
                     const double *phi_new, uint32_t flags, int32_t bands, void *stream, int64_t *row_off_out,
                     hrg_job **job, int64_t *n_entries);

/*
 * hrg_generate_finish -- the edge insertion of Algorithm 1: writes the
 * neighbour ids of every vertex into col_idx_out (device int32[n_entries],
 * caller owned) at the offsets produced by begin, each row ascending.
 * Synchronizes the stream before returning and checks the device-side
 * consistency flag.  The job stays open for hrg_job_stats until released.
 * Errors: HRG_ESTATE (job already finished/released), HRG_ENOMEM, HRG_ECUDA,
 * HRG_EINTERNAL (count and write passes disagreed).
 */
int hrg_generate_finish(hrg_job *job, int32_t *col_idx_out);

/*
 * hrg_set_limits -- capacities of the buffers the count pass fills for the
 * write pass, for a context's later jobs (0 or a null lim: automatic).  A
 * smaller buffer means less workspace and more work, never another graph:
 *   row_buffer_ids  ids of the buffer of kept rim rows (automatic: 32 per
 *                   vertex, below 2^31); rows that find no room are
 *                   traversed again by the write pass (rows_no_room)
 *   hub_pool_ids    ids of the pool of hub-row entries (automatic: 8 per
 *                   vertex + 2^24), below 2^40; hub_runs: entries of its run
 *                   table (automatic from the pool size), below 2^24.  When
 *                   either overflows, the write pass traverses every hub row
 *                   again (hub_rows_retraversed)
 *   heavy_segments  first capacity of the list of long hub ranges (automatic:
 *                   max(2^16, n/64)); when it overflows the count pass runs
 *                   once more with room for all (heavy_retries)
 *   workspace_bytes the most device memory the context's workspace may hold
 *                   (0: no cap); a call that would need more returns
 *                   HRG_ENOMEM, as when the device itself has no room, and
 *                   the context stays usable (a smaller graph, a higher cap
 *                   or hrg_release_workspace, which gives back what the
 *                   context holds, lets the next call run)
 * Errors: HRG_EINVAL (negative or oversized value), HRG_ESTATE (a job is open).
 */
typedef struct hrg_limits {
    int64_t row_buffer_ids;
    int64_t hub_pool_ids;
    int32_t hub_runs;
    int32_t heavy_segments;
    int64_t workspace_bytes;
} hrg_limits;

int hrg_set_limits(hrg_ctx *ctx, const hrg_limits *lim);

/* Statistics of a job (after begin; candidate counts from the count pass). */
int hrg_job_stats(const hrg_job *job, hrg_stats *out);

/* Closes the job so the context can run the next one. */
int hrg_job_release(hrg_job *job);

/*
 * hrg_generate -- begin + finish on device buffers in one call.
 * col_capacity is the length of col_idx_out; when 2m exceeds it the call
 * returns HRG_EOVERFLOW with *n_entries set and col_idx_out untouched.
 */
int hrg_generate(hrg_ctx *ctx, const hrg_params *p, void *stream, double *r_out, double *phi_out,
                 int64_t *row_off_out, int32_t *col_idx_out, int64_t col_capacity, int64_t *n_entries,
                 hrg_stats *stats_out);

/*
 * hrg_generate_host -- the whole generator with HOST output buffers: the
 * library generates into context-owned device memory and copies r, phi,
 * row_off and col_idx back (r_host double[n], phi_host double[n],
 * row_off_host int64[n+1], col_idx_host int32[col_capacity]).  Host buffers
 * registered with cudaHostRegister (or pinned) copy at full link speed.
 * The context generates on a stream of its own and copies on a second one:
 * r and phi as soon as the sampler has written them, row_off once the
 * degrees are counted, and, for graphs of 2^26 entries or more, the
 * neighbour ids in up to 8 id ranges, each as soon as its rows are written
 * and sorted while the next range is (stats_out->write_chunks, d2h_ms).
 * The call returns when every copy is complete; the host buffers must not be
 * read before.
 * Errors as hrg_generate.
 */
int hrg_generate_host(hrg_ctx *ctx, const hrg_params *p, double *r_host, double *phi_host, int64_t *row_off_host,
                      int32_t *col_idx_host, int64_t col_capacity, int64_t *n_entries, hrg_stats *stats_out);

/*
 * hrg_row_offsets_noalloc -- CSR row offsets from vertex degrees with no
 * device allocation.  The paper has no counterpart; this is a service entry
 * for callers that are not allowed to allocate GPU memory: code that runs
 * inside a host framework which owns every device byte through its own pool,
 * or a serving loop with a fixed memory budget where an allocation (which may
 * also synchronize the device) is not permitted.
 *   deg      device int32[n], degrees in vertex-id order        (caller owned, read)
 *   n        0 <= n <= 2^28
 *   row_off  device int64[n+1]; row_off[i] = deg[0] + ... + deg[i-1],
 *            row_off[n] = the total                             (caller owned)
 *   stream   cudaStream_t (as void*), 0 for the legacy stream; the call is
 *            asynchronous on it
 * Scratch: a 1 MiB array compiled into the library as device memory, held by
 * every device that loads the library until the process exits.  The first
 * call on a device looks up that array's device address (with the device
 * current), so make the first call on each device before any stream capture.
 * The library caches that address per device for the life of the process; a
 * cudaDeviceReset invalidates it, so do not call this entry point on a device
 * after resetting it.
 * All calls share the array: calls whose executions overlap on the GPU (on
 * different streams, or from different threads) race and corrupt each other's
 * results; serialize them.
 * Errors: HRG_EINVAL (n outside [0, 2^28], null pointer), HRG_ECUDA (address
 * lookup or launch failed).  Calls no cudaMalloc/cudaFree.
 */
int hrg_row_offsets_noalloc(const int32_t *deg, int64_t n, int64_t *row_off, void *stream);

/*
 * Graph properties of Sec. 4.1, computed on the device over a canonical CSR
 * (rows ascending, both directions of every edge, no self-loops: the
 * generator's output).  Sec. 4.1 studies the degree distribution (a power law
 * with exponent gamma = 2 alpha + 1, Sec. 2.1) and the clustering
 * coefficient, which it defines as the fraction of closed triangles among
 * triads (paths of length two).
 *   row_off  device int64[n+1]; the ids of vertex v's neighbours are
 *            col_idx[row_off[v] .. row_off[v+1]) (row_off[0] need not be 0)
 *   col_idx  device int32, ids in [0, n)            (read only; may be null
 *            without HRG_PROPS_TRIANGLES)
 *   d_min    >= 1: the tail used for gamma
 *   flags    HRG_PROPS_TRIANGLES to count triangles (degree-ordered
 *            orientation; workspace ~ 16 B per vertex + 4 B per edge)
 *   stream   cudaStream_t (as void*); the call returns with *out filled
 * gamma is the discrete maximum-likelihood approximation of Clauset,
 * Shalizi and Newman (SIAM Review 51, 2009, Eq. 3.7):
 * 1 + tail_count / tail_log_sum.  Undefined values are NaN (gamma without a
 * tail, clustering without triads, both clusterings without
 * HRG_PROPS_TRIANGLES, where triangles is -1).
 * Errors: HRG_EINVAL (n outside [0, 2^31), d_min < 1, null pointer, unknown
 * flag), HRG_ENOMEM, HRG_ECUDA.
 */
#define HRG_PROPS_TRIANGLES 0x1u

typedef struct hrg_props {
    int64_t n;                    /* vertices                                           */
    int64_t entries;              /* directed CSR entries, 2m                          */
    int64_t max_degree;
    int64_t d_min;                /* tail threshold used for gamma                     */
    int64_t tail_count;           /* vertices of degree >= d_min                       */
    double tail_log_sum;          /* sum over them of ln(d / (d_min - 1/2))            */
    double gamma;                 /* 1 + tail_count / tail_log_sum                     */
    int64_t triads;               /* sum over v of d_v (d_v - 1) / 2                   */
    int64_t triangles;            /* closed triangles, each counted once               */
    double clustering;            /* 3 triangles / triads (Sec. 4.1)                   */
    double avg_local_clustering;  /* mean over all v of t_v / (d_v (d_v - 1) / 2), t_v
                                     the triangles at v; vertices of degree < 2 add 0  */
} hrg_props;

int hrg_graph_props(hrg_ctx *ctx, int64_t n, const int64_t *row_off, const int32_t *col_idx, int64_t d_min,
                    uint32_t flags, void *stream, hrg_props *out);

/*
 * hrg_degree_histogram -- hist[d] = vertices of degree d, d = 0..max_degree,
 * of the CSR given by row_off (as for hrg_graph_props).
 *   hist     device int64[max_degree + 1] (caller owned, overwritten)
 * The call returns when hist is complete.
 * Errors: HRG_EINVAL (a degree above max_degree -- hist then holds the
 * others --, null pointer, n outside [0, 2^31), max_degree < 0), HRG_ECUDA.
 */
int hrg_degree_histogram(hrg_ctx *ctx, int64_t n, const int64_t *row_off, int64_t max_degree, int64_t *hist,
                         void *stream);

/*
 * hrg_add_random_edges -- the graph with random long-range edges (Sec. 4.2
 * and its appendix: adding 0.5 % of the edges at random shortens the
 * diameter while the other properties stay close).  Pair k = 0..count-1 draws
 * the Philox4x32-10 block at counter 2^63 + k (words (k_lo, k_hi + 2^31, 0,
 * 0); the point draws use counters below 2^31), key (seed_lo, seed_hi), and
 * takes the vertices u = floor(w0 n / 2^64), v = floor(w1 n / 2^64) of its
 * two 64-bit halves w0 = (x0 << 32) | x1, w1 = (x2 << 32) | x3.  Self-pairs,
 * pairs drawn twice and pairs already present are dropped; the rest become
 * undirected edges.  The paper's 0.5 % is count = ceil(0.005 m).
 *   row_off, col_idx   device, the input CSR as for hrg_graph_props (read)
 *   row_off_out        device int64[n+1] (caller owned): the new offsets, from 0
 *   col_idx_out        device int32[col_capacity] (caller owned); 2m + 2 count
 *                      always suffices
 *   *entries_out       the new 2m; *added_out (may be null) the added edges
 *   stream             cudaStream_t (as void*); the call returns when done
 * The output is again canonical: rows ascending, symmetric, no self-loops.
 * Errors: HRG_EINVAL (n outside [0, 2^31), count outside [0, 2^30], null
 * pointer), HRG_EOVERFLOW (*entries_out above col_capacity: row_off_out is
 * written, col_idx_out untouched), HRG_ENOMEM, HRG_ECUDA.
 */
int hrg_add_random_edges(hrg_ctx *ctx, int64_t n, const int64_t *row_off, const int32_t *col_idx, int64_t count,
                         uint64_t seed, void *stream, int64_t *row_off_out, int32_t *col_idx_out,
                         int64_t col_capacity, int64_t *entries_out, int64_t *added_out);

/*
 * hrg_bfs -- breadth-first search over a CSR (as for hrg_graph_props), for
 * the diameter of Sec. 4.1 (the longest shortest path) that Sec. 4.2's
 * long-range edges shorten.
 *   source   vertex to start from, or -1 for the vertex of highest degree
 *            (lowest id among ties)
 *   dist     device int32[n] (caller owned): hops from the source, -1 where
 *            unreached
 *   *ecc_out the source's eccentricity in its component; *reached_out
 *            (may be null) the component's size; *far_out (may be null) the
 *            lowest id at distance ecc; *source_out (may be null) the source
 *   stream   cudaStream_t (as void*); the call returns when done (one
 *            read-back per level)
 * Errors: HRG_EINVAL (n outside [1, 2^31), source >= n, null pointer),
 * HRG_ENOMEM, HRG_ECUDA.
 */
int hrg_bfs(hrg_ctx *ctx, int64_t n, const int64_t *row_off, const int32_t *col_idx, int64_t source, void *stream,
            int32_t *dist, int32_t *ecc_out, int64_t *reached_out, int64_t *far_out, int64_t *source_out);

/*
 * hrg_diameter_bounds -- lower <= diameter <= upper for the component of the
 * highest-degree vertex, by repeated double sweeps: a search from root r
 * gives ecc(r) <= diameter <= 2 ecc(r); the first root is the vertex of
 * highest degree (lowest id among ties), each next root the previous search's
 * farthest vertex (lowest id among ties), at most `sweeps` searches (1..64),
 * stopping when the farthest vertex is the root.  *component (may be null)
 * is the component's size; roots (host int64[sweeps], may be null) receives
 * the roots used, -1 after the last.
 * Errors as hrg_bfs, and HRG_EINVAL for sweeps outside [1, 64].
 */
int hrg_diameter_bounds(hrg_ctx *ctx, int64_t n, const int64_t *row_off, const int32_t *col_idx, int32_t sweeps,
                        void *stream, int32_t *lower, int32_t *upper, int64_t *component, int64_t *roots);

/*
 * Request server -- generation requests of different sizes and parameters on
 * one GPU with continuous batching.  The paper has no serving layer; this is
 * the request loop around Algorithm 1 for callers that submit many graphs.
 *
 * hrg_server_create starts `slots` worker threads (1..64), each with its own
 * context (whose workspace, band structures included, stays resident across
 * requests) and stream.  A free worker admits the queued requests in arrival
 * order while the device bytes they add fit in mem_budget_bytes (<= 0: 70 %
 * of the device's free memory at create): their outputs, and the growth of
 * the worker's workspace beyond what it already holds (estimated; measured
 * once the batch is done, and counted as long as the workspace stays).  A
 * worker that finds the next request too large while idle frees its own
 * workspace first.  It generates the admitted requests together as one
 * batch (hrg_generate_batch_begin);
 * requests arriving meanwhile join the next batch.  Batches of different
 * workers run concurrently on the device.  Results do not depend on the
 * batching: each equals hrg_generate of the same parameters.
 * Errors: HRG_EINVAL (bad slots / out), HRG_ECUDA (device, memory query).
 */
typedef struct hrg_server hrg_server;

typedef struct hrg_result {
    int32_t status;         /* HRG_OK or the batch's error code                     */
    int32_t batch_size;     /* requests generated together with this one           */
    int64_t n;              /* vertices                                            */
    int64_t n_entries;      /* 2m                                                  */
    /* device pointers owned by the server until hrg_server_release:
     * r[n], phi[n] in vertex-id order; row_off[n+1]; the neighbour ids of
     * vertex i are col_idx[row_off[i] .. row_off[i+1]) (row_off[0] is in general
     * not 0: col_idx is shared with the other requests of the batch), local
     * ids in [0, n), ascending */
    const double *r, *phi;
    const int64_t *row_off;
    const int32_t *col_idx;
    /* seconds since hrg_server_create: submitted, admitted to a batch, done */
    double submit_s, start_s, done_s;
} hrg_result;

typedef struct hrg_server_counters {
    int64_t completed;         /* requests finished (any status)              */
    int64_t batches;           /* batches generated                           */
    int64_t batched_requests;  /* requests over all batches                   */
    int64_t queued;            /* requests waiting for admission               */
    int64_t max_running;       /* most batches in flight at once              */
    int64_t in_use_bytes;      /* device bytes counted against the budget: the
                                  workers' resident workspaces (measured), the
                                  outputs of unreleased requests and the
                                  estimated workspace growth of running batches */
    int64_t peak_in_use_bytes; /* maximum of in_use_bytes                     */
    int64_t budget_bytes;
    int64_t resident_bytes;    /* the workers' workspaces, measured after each batch */
} hrg_server_counters;

int hrg_server_create(hrg_server **out, int device, int32_t slots, int64_t mem_budget_bytes);

/* Queue a request (parameters as hrg_generate_begin; flags ignored).
 * Errors: HRG_EINVAL (invalid parameters, no radius), HRG_ENOMEM (the
 * request alone exceeds the memory budget). */
int hrg_server_submit(hrg_server *s, const hrg_params *p, int64_t *ticket);

/* Wait up to timeout_s seconds (< 0: no limit) for a request; fills *out and
 * returns its status, or HRG_ETIMEOUT.  HRG_EINVAL for an unknown ticket. */
int hrg_server_wait(hrg_server *s, int64_t ticket, double timeout_s, hrg_result *out);

/* Give a finished request's device buffers back (they are freed when every
 * request of the batch has been released).  HRG_ESTATE if not finished. */
int hrg_server_release(hrg_server *s, int64_t ticket);

int hrg_server_stats(hrg_server *s, hrg_server_counters *out);
const char *hrg_server_last_error(hrg_server *s);

/* Cancels queued requests (status HRG_ESTATE), waits for running batches,
 * frees every result not yet released and the workers' contexts. */
int hrg_server_destroy(hrg_server *s);

/* Message of the last error on this context (never null). */
const char *hrg_last_error(const hrg_ctx *ctx);

/* Library version string. */
const char *hrg_version(void);

#ifdef __cplusplus
}
#endif

#endif /* HRG_H */
