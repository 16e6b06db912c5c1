// hrg_points.cu -- point sampling and the angle-sorted radial-band structure.
//
// Algorithm 1 draws every point, maps it to the Poincare disk and inserts it
// into a polar quadtree.  Here the points stay in native coordinates and the
// quadtree is replaced by B radial bands, each cut into 2^g equal angular
// buckets (g chosen so a bucket holds about one point).  A counting sort by
// (band, bucket) gives every band as a contiguous, angle-bucketed array; the
// bucket start table doubles as the angular index used by the queries.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include "hrg_internal.h"

namespace hrg {

namespace {

constexpr int kThreads = 256;
constexpr int kSampleGrid = 152 * 16;  // persistent grid of the samplers (each CTA loads the log table once)
constexpr int kSplitGrid = 152 * 8;    // persistent: the split reads the records front to back

// 2^63 / F_j, log F_j 2^64 (F_j = 1 + j/128) and ln 2 2^64 (log_fix); filled
// once per device
constexpr int kLogTab = 257;
__device__ uint64_t g_log_tab[kLogTab];

__device__ __forceinline__ void load_log_tab(uint64_t *s_tab)
{
    for (int k = threadIdx.x; k < kLogTab; k += blockDim.x) s_tab[k] = g_log_tab[k];
    __syncthreads();
}

inline int grid_for(int64_t n, int threads, int per_thread = 1)
{
    int64_t g = (n + (int64_t)threads * per_thread - 1) / ((int64_t)threads * per_thread);
    if (g < 1) g = 1;
    if (g > (1 << 20)) g = 1 << 20;
    return (int)g;
}

// per-band counts: shared-memory histogram, one global atomic per band per block
__device__ __forceinline__ void band_hist_flush(const Plan &p, int *sh, int64_t *band_cnt)
{
    __syncthreads();
    for (int k = threadIdx.x; k < p.B; k += blockDim.x)
        if (sh[k]) atomicAdd((unsigned long long *)&band_cnt[k], (unsigned long long)sh[k]);
}

// Algorithm 1's two draws: phi uniform on [0, 2pi) and r with density
// Eq. (1), by the inverse CDF r = acosh(1 + u (cosh(alpha R) - 1)) / alpha.
// Uniforms come from Philox4x32-10 at counter = vertex id, key = seed.
// The bucket layout of a sampled graph is planned before the draws (from the
// expected band counts), so the same pass files every point under its
// (band, angular bucket): gbuf, the bucket occupancy cnt, the point's rank in
// its bucket (slot) and the exact per-band counts.  The sampler is bound by
// the FP64 pipe, the bucket atomics by memory latency: together they overlap.
__global__ void k_sample_bucket(Plan p, uint64_t seed, double *__restrict__ r_out, double *__restrict__ phi_out,
                                int32_t *__restrict__ gbuf, int32_t *__restrict__ slot, int32_t *__restrict__ cnt,
                                int64_t *__restrict__ band_cnt)
{
    __shared__ uint64_t s_tab[kLogTab];
    __shared__ int sh[HRG_MAX_BANDS];
    for (int k = threadIdx.x; k < HRG_MAX_BANDS; k += blockDim.x) sh[k] = 0;
    load_log_tab(s_tab);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p.n; i += stride) {
        const U4 w = philox_block((uint64_t)i, seed);
        const double k_phi = top53(w.x, w.y);
        const double k_r = top53(w.z, w.w);
        const double ph = __dmul_rn(k_phi, kTwoPiScaled);  // = u_phi 2pi, rounded once
        const double rr = radius_of(k_r, p.big53, p.inv_alpha, s_tab);
        phi_out[i] = ph;
        r_out[i] = rr;
        const int band = band_of(p, rr);
        const int64_t g = bucket_of(p, band, sampled_angle_key(w));
        gbuf[i] = (int32_t)g;
        slot[i] = atomicAdd(&cnt[g], 1);
        atomicAdd(&sh[band], 1);
    }
    band_hist_flush(p, sh, band_cnt);
}

__global__ void k_count_bands(Plan p, const double *__restrict__ r, int64_t *__restrict__ band_cnt)
{
    __shared__ int sh[HRG_MAX_BANDS];
    for (int k = threadIdx.x; k < HRG_MAX_BANDS; k += blockDim.x) sh[k] = 0;
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p.n; i += stride)
        atomicAdd(&sh[band_of(p, r[i])], 1);
    band_hist_flush(p, sh, band_cnt);
}

// Bucket of every point of an injected point set (gbuf, id order), bucket
// occupancy, and the point's rank inside its bucket (slot: the count it found
// there).
__global__ void k_bucket_hist(Plan p, const double *__restrict__ r, const double *__restrict__ phi,
                              int32_t *__restrict__ gbuf, int32_t *__restrict__ slot, int32_t *__restrict__ cnt)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p.n; i += stride) {
        const int band = band_of(p, r[i]);
        const int64_t g = bucket_of(p, band, angle_key(phi[i]));
        gbuf[i] = (int32_t)g;
        slot[i] = atomicAdd(&cnt[g], 1);
    }
}

// Structure of arrays in (band, bucket) order, written from id order: point i
// goes to position k = start[gbuf[i]] + slot[i], recorded in pos_of[i].  The
// positions are random, so an 8-byte angle and a 16-byte {P, M, S, id} stored
// there would each be a partial 32-byte sector, which DRAM reads and writes
// back.  With rec non-null the two go out as one 32-byte record per position
// instead (a whole sector), and k_split separates the records sequentially;
// the plain FP64 path stores its three arrays directly.
__device__ __forceinline__ void place_point(const Plan &p, int64_t i, const int32_t *__restrict__ gbuf,
                                            const int32_t *__restrict__ slot, const int32_t *__restrict__ start,
                                            const double *__restrict__ r, const double *__restrict__ phi,
                                            PointRec *__restrict__ rec, uint64_t *__restrict__ A,
                                            PMS *__restrict__ pms, PMS64 *__restrict__ pms64,
                                            int32_t *__restrict__ pos_of)
{
    const int64_t k = (int64_t)__ldg(start + gbuf[i]) + slot[i];
    pos_of[i] = (int32_t)k;
    const double rr = r[i], ph = phi[i];
    const PMS q = scaled_exps(p, rr, (int32_t)i);
    const uint64_t a = angle_key(ph);
    if (rec) {
        int4 *dst = reinterpret_cast<int4 *>(rec + k);
        dst[0] = *reinterpret_cast<const int4 *>(&q);
        dst[1] = make_int4((int)(uint32_t)a, (int)(uint32_t)(a >> 32), 0, 0);
    } else {
        A[k] = a;
        pms[k] = q;
        if (pms64) pms64[k] = scaled_exps64(p, rr, ph);
    }
}

__global__ void k_scatter_soa(Plan p, const int32_t *__restrict__ gbuf, const int32_t *__restrict__ slot,
                              const int32_t *__restrict__ start, const double *__restrict__ r,
                              const double *__restrict__ phi, PointRec *__restrict__ rec, uint64_t *__restrict__ A,
                              PMS *__restrict__ pms, PMS64 *__restrict__ pms64, int32_t *__restrict__ pos_of)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p.n; i += stride)
        place_point(p, i, gbuf, slot, start, r, phi, rec, A, pms, pms64, pos_of);
}

// the records, in position order, into the angle and {P, M, S, id} arrays
__global__ void k_split(int64_t N, const PointRec *__restrict__ rec, uint64_t *__restrict__ A, PMS *__restrict__ pms)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += stride) {
        const int4 *src = reinterpret_cast<const int4 *>(rec + k);
        const int4 lo = __ldcs(src), hi = __ldcs(src + 1);
        reinterpret_cast<int4 *>(pms)[k] = lo;
        A[k] = ((uint64_t)(uint32_t)hi.y << 32) | (uint32_t)hi.x;
    }
}

// ---------------------------------------------------------------------------
// Batches of graphs.  Graph g owns positions and global ids [off_g, off_g +
// n_g); graph_of[] maps either back to g.  Each kernel is the single-graph
// kernel above with the plan looked up per point.
// ---------------------------------------------------------------------------
__global__ void k_graph_of(const Plan *__restrict__ plans, int32_t *__restrict__ graph_of)
{
    const int g = blockIdx.x;
    const int64_t off = plans[g].id_off, n = plans[g].n;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) graph_of[off + i] = g;
}

__global__ void k_sample_bucket_batch(const Plan *__restrict__ plans, const int32_t *__restrict__ graph_of,
                                      int64_t N, double *__restrict__ r_out, double *__restrict__ phi_out,
                                      int32_t *__restrict__ gbuf, int32_t *__restrict__ slot,
                                      int32_t *__restrict__ cnt)
{
    __shared__ uint64_t s_tab[kLogTab];
    load_log_tab(s_tab);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
        const Plan &p = plans[__ldg(graph_of + i)];
        const U4 w = philox_block((uint64_t)(i - p.id_off), p.seed);
        const double k_phi = top53(w.x, w.y);
        const double k_r = top53(w.z, w.w);
        const double ph = __dmul_rn(k_phi, kTwoPiScaled);  // = u_phi 2pi, rounded once
        const double rr = radius_of(k_r, p.big53, p.inv_alpha, s_tab);
        phi_out[i] = ph;
        r_out[i] = rr;
        const int64_t g = bucket_of(p, band_of(p, rr), sampled_angle_key(w));
        gbuf[i] = (int32_t)g;
        slot[i] = atomicAdd(&cnt[g], 1);
    }
}

__global__ void k_scatter_soa_batch(const Plan *__restrict__ plans, const int32_t *__restrict__ graph_of, int64_t N,
                                    const int32_t *__restrict__ gbuf, const int32_t *__restrict__ slot,
                                    const int32_t *__restrict__ start, const double *__restrict__ r,
                                    const double *__restrict__ phi, PointRec *__restrict__ rec,
                                    uint64_t *__restrict__ A, PMS *__restrict__ pms, PMS64 *__restrict__ pms64,
                                    int32_t *__restrict__ pos_of)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride)
        place_point(plans[__ldg(graph_of + i)], i, gbuf, slot, start, r, phi, rec, A, pms, pms64, pos_of);
}

// hub queries of graph g: its positions before its first rim-band bucket
__global__ void k_hub_count(const Plan *__restrict__ plans, int NG, const int32_t *__restrict__ start,
                            int32_t *__restrict__ hub_cnt)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= NG) return;
    const Plan &p = plans[g];
    hub_cnt[g] = __ldg(start + p.base[p.hub_bands]) - p.id_off;
}

__global__ void k_hub_fill(const Plan *__restrict__ plans, const int32_t *__restrict__ hub_off,
                           int32_t *__restrict__ hub_pos)
{
    const int g = blockIdx.x;
    const int32_t o = hub_off[g], c = hub_off[g + 1] - o, first = plans[g].id_off;
    for (int32_t t = threadIdx.x; t < c; t += blockDim.x) hub_pos[o + t] = first + t;
}

// ---------------------------------------------------------------------------
// Exclusive scan: tiles of kTile elements; tile sums scanned recursively.
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int64_t kTile = (int64_t)kScanThreads * kScanItems;

template <typename T>
__device__ __forceinline__ T block_exclusive_scan(T v, T *warp_tot, T *total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_tot[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        T t = lane < nw ? warp_tot[lane] : T(0);
        T ti = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, ti, o);
            if (lane >= o) ti += y;
        }
        if (lane < nw) warp_tot[lane] = ti - t;
        if (lane == nw - 1) *total = ti;
    }
    __syncthreads();
    const T res = inc - v + warp_tot[wid];
    __syncthreads();
    return res;
}

template <typename Tin, typename Tacc>
__global__ void k_scan_reduce(const Tin *__restrict__ in, int64_t N, Tacc *__restrict__ sums)
{
    __shared__ Tacc wt[32];
    __shared__ Tacc tot;
    const int64_t base = (int64_t)blockIdx.x * kTile;
    Tacc s = 0;
    for (int j = 0; j < kScanItems; ++j) {
        const int64_t i = base + (int64_t)j * kScanThreads + threadIdx.x;
        if (i < N) s += (Tacc)in[i];
    }
    block_exclusive_scan<Tacc>(s, wt, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// Down-sweep of one tile.  The tile moves through shared memory twice so
// that every global load and store of a warp touches consecutive addresses
// while each thread scans kScanItems consecutive elements: loaded in the
// order j kScanThreads + t, read back as t kScanItems + j, the results
// written in place and stored in the first order.  Slot p + p/32 keeps the
// per-thread reads free of bank conflicts.
__device__ __forceinline__ int scan_slot(int p) { return p + (p >> 5); }

template <typename Tin, typename Tout, typename Tacc>
__global__ void __launch_bounds__(kScanThreads) k_scan_down(const Tin *__restrict__ in, int64_t N,
                                                            const Tacc *__restrict__ offs, Tout *__restrict__ out,
                                                            bool write_total)
{
    __shared__ Tacc wt[32];
    __shared__ Tacc tot;
    __shared__ Tacc buf[kTile + kTile / 32];
    const int64_t base = (int64_t)blockIdx.x * kTile;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        const int p = j * kScanThreads + threadIdx.x;
        const int64_t i = base + p;
        buf[scan_slot(p)] = i < N ? (Tacc)in[i] : Tacc(0);
    }
    __syncthreads();
    Tacc s = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) s += buf[scan_slot(threadIdx.x * kScanItems + j)];
    Tacc run = block_exclusive_scan<Tacc>(s, wt, &tot) + (offs ? offs[blockIdx.x] : Tacc(0));
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        const int k = scan_slot(threadIdx.x * kScanItems + j);
        const Tacc x = buf[k];
        buf[k] = run;
        run += x;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        const int p = j * kScanThreads + threadIdx.x;
        const int64_t i = base + p;
        if (i < N) out[i] = (Tout)buf[scan_slot(p)];
    }
    if (write_total && blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1) out[N] = (Tout)run;
}

template <typename Tin, typename Tout>
cudaError_t scan_impl(const Tin *in, Tout *out, int64_t N, int64_t *ws, cudaStream_t s)
{
    const int64_t tiles = (N + kTile - 1) / kTile;
    if (N <= 0) {
        return cudaMemsetAsync(out, 0, sizeof(Tout), s);
    }
    if (tiles == 1) {
        k_scan_down<Tin, Tout, int64_t><<<1, kScanThreads, 0, s>>>(in, N, nullptr, out, true);
        return cudaGetLastError();
    }
    int64_t *sums = ws;
    int64_t *sums_scan = ws + tiles;
    k_scan_reduce<Tin, int64_t><<<(unsigned)tiles, kScanThreads, 0, s>>>(in, N, sums);
    cudaError_t e = scan_impl<int64_t, int64_t>(sums, sums_scan, tiles, ws + 2 * tiles + 1, s);
    if (e != cudaSuccess) return e;
    k_scan_down<Tin, Tout, int64_t><<<(unsigned)tiles, kScanThreads, 0, s>>>(in, N, sums_scan, out, true);
    return cudaGetLastError();
}

}  // namespace

int scan_launches(int64_t N)
{
    int k = 1;
    int64_t m = N;
    while (m > kTile) {
        m = (m + kTile - 1) / kTile;
        k += 2;
    }
    return k;
}

size_t scan_workspace_bytes(int64_t N)
{
    size_t words = 0;
    int64_t m = N;
    while (m > kTile) {
        const int64_t t = (m + kTile - 1) / kTile;
        words += 2 * t + 1;
        m = t;
    }
    return (words + 8) * sizeof(int64_t);
}

cudaError_t scan_i32_to_i32(const int32_t *in, int32_t *out, int64_t N, void *ws, cudaStream_t s)
{
    return scan_impl<int32_t, int32_t>(in, out, N, (int64_t *)ws, s);
}

cudaError_t scan_i32_to_i64(const int32_t *in, int64_t *out, int64_t N, void *ws, cudaStream_t s)
{
    return scan_impl<int32_t, int64_t>(in, out, N, (int64_t *)ws, s);
}

cudaError_t launch_sample_bucket(const Plan &p, uint64_t seed, double *r, double *phi, int32_t *gbuf, int32_t *slot,
                                 int32_t *cnt, int64_t *band_cnt, cudaStream_t s)
{
    k_sample_bucket<<<std::min(grid_for(p.n, kThreads, 4), kSampleGrid), kThreads, 0, s>>>(p, seed, r, phi, gbuf, slot,
                                                                                           cnt, band_cnt);
    return cudaGetLastError();
}

cudaError_t launch_count_bands(const Plan &p, const double *r, const double *, int64_t *band_cnt, cudaStream_t s)
{
    k_count_bands<<<grid_for(p.n, kThreads, 4), kThreads, 0, s>>>(p, r, band_cnt);
    return cudaGetLastError();
}

cudaError_t launch_bucket_hist(const Plan &p, const double *r, const double *phi, int32_t *gbuf, int32_t *slot,
                               int32_t *cnt, cudaStream_t s)
{
    k_bucket_hist<<<grid_for(p.n, kThreads, 4), kThreads, 0, s>>>(p, r, phi, gbuf, slot, cnt);
    return cudaGetLastError();
}

cudaError_t launch_scatter_soa(const Plan &p, const int32_t *gbuf, const int32_t *slot, const int32_t *start,
                               const double *r, const double *phi, PointRec *rec, uint64_t *A, PMS *pms,
                               PMS64 *pms64, int32_t *pos_of, cudaStream_t s)
{
    k_scatter_soa<<<grid_for(p.n, kThreads, 4), kThreads, 0, s>>>(p, gbuf, slot, start, r, phi, rec, A, pms, pms64,
                                                                   pos_of);
    if (rec) k_split<<<std::min(grid_for(p.n, kThreads, 4), kSplitGrid), kThreads, 0, s>>>(p.n, rec, A, pms);
    return cudaGetLastError();
}

namespace {

typedef unsigned __int128 u128;

// floor(a b / 2^127) for a, b < 2^127 (numbers below 1 in Q127), from 64-bit
// limbs: exact integer arithmetic, the same on every host
u128 mul_q127(u128 a, u128 b)
{
    const uint64_t a0 = (uint64_t)a, a1 = (uint64_t)(a >> 64), b0 = (uint64_t)b, b1 = (uint64_t)(b >> 64);
    const u128 t0 = (u128)a0 * b0, t1 = (u128)a1 * b0, t2 = (u128)a0 * b1, t3 = (u128)a1 * b1;
    const u128 mid = (t0 >> 64) + (uint64_t)t1 + (uint64_t)t2;
    const u128 hi = t3 + (t1 >> 64) + (t2 >> 64) + (mid >> 64);
    return (hi << 1) | ((uint64_t)mid >> 63);
}

// log(num / den) 2^64, rounded, for 1 <= num / den <= 2: 2 atanh(u) with
// u = (num - den) / (num + den) <= 1/3 by its series u + u^3/3 + ... in
// Q127 (each step truncates below 2^-126; the terms fall by u^2 <= 1/9)
uint64_t log_ratio_q64(unsigned num, unsigned den)
{
    const u128 u = (((u128)(num - den) << 120) / (num + den)) << 7;
    const u128 u2 = mul_q127(u, u);
    u128 sum = 0, term = u;
    for (unsigned k = 1; term != 0; k += 2) {
        sum += term / k;
        term = mul_q127(term, u2);
    }
    return (uint64_t)((sum + ((u128)1 << 61)) >> 62);  // 2 sum 2^64 / 2^127, rounded
}

}  // namespace

cudaError_t upload_log_table()
{
    uint64_t tab[kLogTab];
    for (unsigned j = 0; j < 128; ++j) {
        tab[j] = (uint64_t)(((u128)1 << 70) / (128 + j));  // floor(2^63 / F_j), F_j = (128 + j) / 128
        tab[128 + j] = log_ratio_q64(128 + j, 128);
    }
    tab[256] = log_ratio_q64(2, 1);
    return cudaMemcpyToSymbol(g_log_tab, tab, sizeof tab);
}

cudaError_t launch_graph_of(const Plan *plans, int NG, int32_t *graph_of, cudaStream_t s)
{
    k_graph_of<<<NG, 256, 0, s>>>(plans, graph_of);
    return cudaGetLastError();
}

cudaError_t launch_sample_bucket_batch(const Plan *plans, const int32_t *graph_of, int64_t N, double *r, double *phi,
                                       int32_t *gbuf, int32_t *slot, int32_t *cnt, cudaStream_t s)
{
    k_sample_bucket_batch<<<std::min(grid_for(N, kThreads, 4), kSampleGrid), kThreads, 0, s>>>(plans, graph_of, N, r,
                                                                                               phi, gbuf, slot, cnt);
    return cudaGetLastError();
}

cudaError_t launch_scatter_soa_batch(const Plan *plans, const int32_t *graph_of, int64_t N, const int32_t *gbuf,
                                     const int32_t *slot, const int32_t *start, const double *r, const double *phi,
                                     PointRec *rec, uint64_t *A, PMS *pms, PMS64 *pms64, int32_t *pos_of,
                                     cudaStream_t s)
{
    k_scatter_soa_batch<<<grid_for(N, kThreads, 4), kThreads, 0, s>>>(plans, graph_of, N, gbuf, slot, start, r, phi,
                                                                       rec, A, pms, pms64, pos_of);
    if (rec) k_split<<<std::min(grid_for(N, kThreads, 4), kSplitGrid), kThreads, 0, s>>>(N, rec, A, pms);
    return cudaGetLastError();
}

cudaError_t launch_hub_list(const Plan *plans, int NG, const int32_t *start, int32_t *hub_cnt, int32_t *hub_off,
                            int32_t *hub_pos, void *ws, cudaStream_t s, bool fill)
{
    if (!fill) {
        k_hub_count<<<(NG + 255) / 256, 256, 0, s>>>(plans, NG, start, hub_cnt);
        return scan_i32_to_i32(hub_cnt, hub_off, NG, ws, s);
    }
    k_hub_fill<<<NG, 256, 0, s>>>(plans, hub_off, hub_pos);
    return cudaGetLastError();
}

}  // namespace hrg
