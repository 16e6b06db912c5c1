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
    HRG_EINTERNAL = 6  /* a device-side consistency check failed             */
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
 * Errors: HRG_EINVAL (null out), HRG_ECUDA (device cannot be selected).
 */
int hrg_create(hrg_ctx **out, int device);
int hrg_destroy(hrg_ctx *ctx);

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
 * hrg_generate_finish -- the edge insertion of Algorithm 1: writes the
 * neighbour ids of every vertex into col_idx_out (device int32[n_entries],
 * caller owned) at the offsets produced by begin, each row ascending.
 * Synchronizes the stream before returning and checks the device-side
 * consistency flag.  The job stays open for hrg_job_stats until released.
 * Errors: HRG_ESTATE (job already finished/released), HRG_ENOMEM, HRG_ECUDA,
 * HRG_EINTERNAL (count and write passes disagreed).
 */
int hrg_generate_finish(hrg_job *job, int32_t *col_idx_out);

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
 * All calls share the array: calls whose executions overlap on the GPU (on
 * different streams, or from different threads) race and corrupt each other's
 * results; serialize them.
 * Errors: HRG_EINVAL (n outside [0, 2^28], null pointer), HRG_ECUDA (address
 * lookup or launch failed).  Calls no cudaMalloc/cudaFree.
 */
int hrg_row_offsets_noalloc(const int32_t *deg, int64_t n, int64_t *row_off, void *stream);

/* Message of the last error on this context (never null). */
const char *hrg_last_error(const hrg_ctx *ctx);

/* Library version string. */
const char *hrg_version(void);

#ifdef __cplusplus
}
#endif

#endif /* HRG_H */
