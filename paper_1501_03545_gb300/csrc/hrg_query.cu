// hrg_query.cu -- the neighbourhood queries of Algorithm 1.
//
// Algorithm 1 runs, for every vertex v in parallel, a range query for the
// hyperbolic circle of radius R around v and adds (v, w) for every w inside.
// Here a query visits every radial band, bounds its admissible angle by the
// closed-form window at the band's inner radius, reads the angular buckets
// the window touches, and decides each candidate with
//   * an FP32 test of the scaled predicate with an undecided band of
//     relative half-width mu, and an FP64 recheck of the pairs inside it, or
//   * the FP64 predicate on every candidate (the plain double path).
// The same traversal runs twice: once to count degrees, once to write the
// neighbour ids into the caller's CSR (rows longer than kRegRow are sorted
// afterwards by hrg_sort.cu).
//
// Two work mappings:
//   * rim bands (most vertices, small windows): one CTA per angular sector,
//     one thread per query, all bands of the sector together so that the
//     band data near the sector is read once per sector;
//   * hub bands (few vertices, wide windows): one warp per query; lane j
//     sets up band j's window, then all lanes stride over each band's
//     candidates.
#include <cstdio>
#include "hrg_internal.h"

namespace hrg {

namespace {

enum { ST_CAND = 0, ST_RECHECK = 1, ST_EDGES = 2, ST_ERR = 7 };

// Candidate positions of a query in band j: up to two ranges [s0,e0) [s1,e1)
struct Ranges { int32_t s0, e0, s1, e1; uint64_t W; };

__device__ __forceinline__ Ranges band_ranges(const Plan &p, const int32_t *__restrict__ start, const PMS &q,
                                              uint64_t Aq, int j)
{
    // four table reads, always issued (no branch on their values), so the
    // reads of several bands can be in flight together
    Ranges rg;
    const int64_t b0 = p.base[j];
    const int g = p.gbits[j];
    const int64_t G = (int64_t)1 << g;  // buckets of band j
    const uint64_t W = window_halfwidth(p, q, j);
    rg.W = W;
    int64_t i0 = 0, i1 = G, i2 = 0, i3 = 0;
    if (W != kFullCircle && g != 0) {
        const uint64_t lo = Aq - W, hi = Aq + W;
        const int64_t bl = (int64_t)(lo >> (64 - g)), bh = (int64_t)(hi >> (64 - g));
        i0 = bl;
        if (lo <= hi) {
            i1 = bh + 1;
        } else {  // the window wraps through angle 0
            i3 = bh + 1;
        }
    }
    rg.s0 = __ldg(start + b0 + i0);
    rg.e0 = __ldg(start + b0 + i1);
    rg.s1 = __ldg(start + b0 + i2);
    rg.e1 = __ldg(start + b0 + i3);
    return rg;
}

__device__ __forceinline__ bool within(uint64_t Aq, uint64_t Ac, uint64_t W)
{
    const uint64_t d = Ac - Aq;
    const uint64_t ad = (int64_t)d < 0 ? (0ull - d) : d;
    return ad <= W;
}

// Decide candidate c (position cpos, data already loaded) for query q.
template <bool F64>
__device__ __forceinline__ bool decide_loaded(const Plan &p, const QueryBufs &b, const PMS &q, const PMS64 &q64,
                                              uint64_t Aq, uint64_t Ac, const PMS &cc, int32_t cpos, uint64_t W,
                                              unsigned &n_cand, unsigned &n_re)
{
    if (W != kFullCircle && !within(Aq, Ac, W)) return false;
    ++n_cand;
    if (F64) {
        const PMS64 c64 = b.pms64[cpos];
        return edge_pms64(p, q64, c64);
    } else {
        const float v = lhs32(q, cc, (int64_t)(Ac - Aq));
        if (v < p.rhs32 * (1.0f - p.mu)) return true;
        if (v > p.rhs32 * (1.0f + p.mu)) return false;
        ++n_re;
        return edge64(__ldg(b.r + q.id), __ldg(b.phi + q.id), __ldg(b.r + cc.id), __ldg(b.phi + cc.id), p.coshR);
    }
}

__device__ __forceinline__ void add_stats(unsigned long long *stats, unsigned n_cand, unsigned n_re, unsigned n_edge)
{
    unsigned long long a = n_cand, r = n_re, e = n_edge;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        r += __shfl_down_sync(0xffffffffu, r, o);
        e += __shfl_down_sync(0xffffffffu, e, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (a) atomicAdd(&stats[ST_CAND], a);
        if (r) atomicAdd(&stats[ST_RECHECK], r);
        if (e) atomicAdd(&stats[ST_EDGES], e);
    }
}

// rows longer than kRegRow go to one of three sort lists
__device__ __forceinline__ void classify_row(const QueryBufs &b, int32_t id, int32_t d)
{
    if (d <= kRegRow) return;
    const int cls = d <= kWarpRow ? 0 : (d <= kSmemRow ? 1 : 2);
    const int k = atomicAdd(&b.list_cnt[cls], 1);
    b.rows[cls][k] = id;
    if (cls == 2) atomicAdd((unsigned long long *)b.big_total, (unsigned long long)d);
}

// Bitonic sorting network over v[0..N) with compile-time indices (the array
// stays in registers); the pad value 0x7fffffff sorts to the end.
template <int N>
__device__ __forceinline__ void bitonic_regs(int32_t (&v)[kRegRow])
{
#pragma unroll
    for (int k = 2; k <= N; k <<= 1)
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1)
#pragma unroll
            for (int i = 0; i < N; ++i) {
                const int l = i ^ j;
                if (l > i) {
                    const int32_t a = v[i], c = v[l];
                    if ((i & k) == 0) { v[i] = min(a, c); v[l] = max(a, c); }
                    else { v[i] = max(a, c); v[l] = min(a, c); }
                }
            }
}

// ---------------------------------------------------------------------------
// One query, one thread (rim bands).  Rows of up to kRegRow entries are kept
// sorted in registers.  The count pass stores such a row in the row buffer
// (b.small) and records where (b.small_off[position]); the write pass then
// copies it instead of traversing the query again.  Longer rows, and rows
// that did not fit in the buffer, are traversed again by the write pass.
// ---------------------------------------------------------------------------
template <bool F64, bool WRITE>
__device__ __forceinline__ void thread_query(const Plan &p, const QueryBufs &b, int32_t qp, bool active,
                                             const int64_t *__restrict__ row_off, int32_t *__restrict__ col_idx,
                                             unsigned &n_cand, unsigned &n_re, unsigned &n_edge)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    PMS q{};
    int64_t base = 0;
    int32_t deg = 0;
    int32_t stored = -1;
    if (active) {
        q = b.pms[qp];
        if (WRITE) {
            base = row_off[q.id];
            deg = (int32_t)(row_off[q.id + 1] - base);
            stored = b.small_off[qp];
        }
    }
    if (WRITE && active && stored >= 0) {
        // the count pass kept this row (unsorted): sort it in registers, store it
        int32_t v[kRegRow];
#pragma unroll
        for (int k = 0; k < kRegRow; ++k) v[k] = k < deg ? b.small[stored + k] : 0x7fffffff;
        if (deg > 16) bitonic_regs<32>(v);
        else if (deg > 8) bitonic_regs<16>(v);
        else if (deg > 4) bitonic_regs<8>(v);
        else if (deg > 1) bitonic_regs<4>(v);
#pragma unroll
        for (int k = 0; k < kRegRow; ++k)
            if (k < deg) col_idx[base + k] = v[k];
        return;
    }
    int32_t buf[kRegRow];
    int32_t cnt = 0;
    if (active) {
        const uint64_t Aq = b.A[qp];
        PMS64 q64{};
        if (F64) q64 = b.pms64[qp];
        for (int j = 0; j < p.B; ++j) {
            const Ranges rg = band_ranges(p, b.start, q, Aq, j);
            for (int part = 0; part < 2; ++part) {
                const int32_t s = part ? rg.s1 : rg.s0, e = part ? rg.e1 : rg.e0;
                for (int32_t c = s; c < e; ++c) {
                    if (c == qp) continue;
                    const uint64_t Ac = __ldg(b.A + c);
                    if (rg.W != kFullCircle && !within(Aq, Ac, rg.W)) continue;
                    const PMS cc = b.pms[c];
                    if (decide_loaded<F64>(p, b, q, q64, Aq, Ac, cc, c, kFullCircle, n_cand, n_re)) {
                        if (WRITE) {
                            if (cnt < kRegRow) {  // insertion into the sorted list (rows not kept)
                                int32_t k = cnt;
                                while (k > 0 && buf[k - 1] > cc.id) { buf[k] = buf[k - 1]; --k; }
                                buf[k] = cc.id;
                            }
                            if (deg > kRegRow && cnt < deg) col_idx[base + cnt] = cc.id;
                        } else if (cnt < kRegRow) {
                            buf[cnt] = cc.id;  // count pass: kept unsorted
                        }
                        ++cnt;
                    }
                }
            }
        }
    }
    if (WRITE) {
        if (active) {
            if (cnt != deg) atomicOr((unsigned long long *)&b.stats[ST_ERR], 1ull);
            if (deg <= kRegRow)
                for (int32_t k = 0; k < cnt && k < deg; ++k) col_idx[base + k] = buf[k];
        }
    } else {
        // keep rows of up to kRegRow entries: warp-aggregated reservation in b.small
        const bool keep = active && cnt <= kRegRow && cnt > 0;
        int32_t want = keep ? cnt : 0;
        int32_t incl = want;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const int32_t tot = __shfl_sync(0xffffffffu, incl, 31);
        long long wbase = 0;
        if (lane == 31 && tot > 0) wbase = atomicAdd((unsigned long long *)b.small_cursor, (unsigned long long)tot);
        wbase = __shfl_sync(0xffffffffu, wbase, 31);
        (void)lt;
        if (active) {
            const long long pos = wbase + incl - want;
            int32_t off = -1;
            if (keep && pos + cnt <= b.small_cap) {
                for (int32_t k = 0; k < cnt; ++k) b.small[pos + k] = buf[k];
                off = (int32_t)pos;
            }
            b.small_off[qp] = off;
            b.deg[q.id] = cnt;
            classify_row(b, q.id, cnt);
        }
    }
    if (active) n_edge += cnt;
}

// One CTA per angular sector: the queries of all rim bands whose angle lies
// in the sector.  Sector s of band j is the bucket range
// [s << (g_j - sbits), (s + 1) << (g_j - sbits)) (every band has g_j >= sbits).
template <bool F64, bool WRITE>
__global__ void __launch_bounds__(256) k_rim_sector(Plan p, QueryBufs b, const int64_t *__restrict__ row_off,
                                                    int32_t *__restrict__ col_idx)
{
    __shared__ int32_t s_beg[HRG_MAX_BANDS];
    __shared__ int32_t s_pre[HRG_MAX_BANDS + 1];
    const int64_t sector = blockIdx.x;
    if (threadIdx.x < HRG_MAX_BANDS) {
        const int j = threadIdx.x;
        int32_t s = 0, e = 0;
        if (j >= p.hub_bands && j < p.B) {
            const int sh = p.gbits[j] - p.sbits;
            const int64_t b0 = p.base[j] + (sector << sh);
            s = __ldg(b.start + b0);
            e = __ldg(b.start + b0 + ((int64_t)1 << sh));
        }
        s_beg[j] = s;
        s_pre[j + 1] = e - s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        s_pre[0] = 0;
        for (int j = 0; j < HRG_MAX_BANDS; ++j) s_pre[j + 1] += s_pre[j];
    }
    __syncthreads();
    const int32_t total = s_pre[HRG_MAX_BANDS];
    unsigned n_cand = 0, n_re = 0, n_edge = 0;
    int j = 0;
    // warp-uniform loop (the count pass reserves buffer space per warp)
    for (int32_t t0 = threadIdx.x & ~31; t0 < total; t0 += blockDim.x) {
        const int32_t t = t0 + (threadIdx.x & 31);
        const bool active = t < total;
        int32_t qp = 0;
        if (active) {
            while (t >= s_pre[j + 1]) ++j;  // t only grows, so j only moves forward
            qp = s_beg[j] + (t - s_pre[j]);
        }
        thread_query<F64, WRITE>(p, b, qp, active, row_off, col_idx, n_cand, n_re, n_edge);
    }
    if (!WRITE) add_stats(b.stats, n_cand, n_re, n_edge);
}

// ---------------------------------------------------------------------------
// Hub bands.  One warp per query: lane j sets up band j's window, then all
// lanes stride over each band's range, two candidates per lane in flight.
// Ranges longer than kHeavy are cut into chunks (count pass) and processed by
// whole CTAs (k_hub_heavy), so no single warp walks millions of candidates.
// Degrees accumulate with atomics; rows are written through a per-row cursor
// in no particular order and sorted afterwards.
// ---------------------------------------------------------------------------
__device__ __forceinline__ Ranges shfl_ranges(const Ranges &r, int src)
{
    Ranges o;
    o.s0 = __shfl_sync(0xffffffffu, r.s0, src);
    o.e0 = __shfl_sync(0xffffffffu, r.e0, src);
    o.s1 = __shfl_sync(0xffffffffu, r.s1, src);
    o.e1 = __shfl_sync(0xffffffffu, r.e1, src);
    o.W = __shfl_sync(0xffffffffu, r.W, src);
    return o;
}

// warp-aggregated write of this lane's edge (if any) into a hub row
__device__ __forceinline__ void warp_emit(const QueryBufs &b, int32_t qp, int64_t base, int32_t deg, bool e,
                                          int32_t id, unsigned lt, int lane)
{
    const unsigned m = __ballot_sync(0xffffffffu, e);
    if (m == 0) return;
    int32_t slot = 0;
    if (lane == 0) slot = atomicAdd(&b.cursor[qp], __popc(m));
    slot = __shfl_sync(0xffffffffu, slot, 0);
    if (e) {
        const int32_t pos = slot + __popc(m & lt);
        if (pos < deg) b.col_out[base + pos] = id;
    }
}

template <bool F64, bool WRITE>
__global__ void __launch_bounds__(256) k_hub_warp(Plan p, QueryBufs b, int32_t p_hub,
                                                  const int64_t *__restrict__ row_off)
{
    const int32_t qp = (int32_t)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (qp >= p_hub) return;  // uniform per warp
    const PMS q = b.pms[qp];
    const uint64_t Aq = b.A[qp];
    PMS64 q64{};
    if (F64) q64 = b.pms64[qp];
    const Ranges empty{0, 0, 0, 0, kFullCircle};
    const Ranges rA = lane < p.B ? band_ranges(p, b.start, q, Aq, lane) : empty;
    const Ranges rB = lane + 32 < p.B ? band_ranges(p, b.start, q, Aq, lane + 32) : empty;
    int64_t base = 0;
    int32_t deg = 0;
    if (WRITE) {
        base = row_off[q.id];
        deg = (int32_t)(row_off[q.id + 1] - base);
    }
    const unsigned lt = (1u << lane) - 1u;
    unsigned n_cand = 0, n_re = 0;
    int32_t mine = 0;
    for (int j = 0; j < p.B; ++j) {
        const Ranges rg = shfl_ranges(j < 32 ? rA : rB, j & 31);
        for (int part = 0; part < 2; ++part) {
            const int32_t s = part ? rg.s1 : rg.s0, e = part ? rg.e1 : rg.e0;
            if (e - s > kHeavy) {
                if (!WRITE) {
                    const int32_t nch = (e - s + kHeavy - 1) / kHeavy;
                    for (int32_t k = lane; k < nch; k += 32) {
                        const int32_t idx = atomicAdd(&b.list_cnt[3], 1);
                        if (idx < b.heavy_cap)
                            b.heavy[idx] = make_int4(qp, 2 * j + part, s + k * kHeavy, min(e, s + (k + 1) * kHeavy));
                    }
                }
                continue;
            }
            for (int32_t c0 = s; c0 < e; c0 += 64) {
                const int32_t ca = c0 + lane, cb = c0 + 32 + lane;
                const bool va = ca < e && ca != qp, vb = cb < e && cb != qp;
                uint64_t Aa = 0, Ab = 0;
                PMS pa{}, pb{};
                if (va) { Aa = __ldg(b.A + ca); pa = b.pms[ca]; }
                if (vb) { Ab = __ldg(b.A + cb); pb = b.pms[cb]; }
                const bool ea = va && decide_loaded<F64>(p, b, q, q64, Aq, Aa, pa, ca, rg.W, n_cand, n_re);
                const bool eb = vb && decide_loaded<F64>(p, b, q, q64, Aq, Ab, pb, cb, rg.W, n_cand, n_re);
                if (WRITE) {
                    warp_emit(b, qp, base, deg, ea, pa.id, lt, lane);
                    warp_emit(b, qp, base, deg, eb, pb.id, lt, lane);
                } else {
                    mine += (int)ea + (int)eb;
                }
            }
        }
    }
    if (!WRITE) {
        int32_t d = mine;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
        if (lane == 0 && d) atomicAdd(&b.deg[q.id], d);
        add_stats(b.stats, n_cand, n_re, lane == 0 ? (unsigned)d : 0u);
    }
}

// One CTA per chunk of a long hub range.
template <bool F64, bool WRITE>
__global__ void __launch_bounds__(256) k_hub_heavy(Plan p, QueryBufs b, const int64_t *__restrict__ row_off)
{
    __shared__ int32_t s_red[8];
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int32_t nseg = min(*((volatile int32_t *)&b.list_cnt[3]), b.heavy_cap);
    unsigned n_cand = 0, n_re = 0, n_edge = 0;
    for (int32_t k = blockIdx.x; k < nseg; k += gridDim.x) {
        const int4 sg = b.heavy[k];
        const int32_t qp = sg.x;
        const int j = sg.y >> 1;
        const PMS q = b.pms[qp];
        const uint64_t Aq = b.A[qp];
        PMS64 q64{};
        if (F64) q64 = b.pms64[qp];
        const uint64_t W = window_halfwidth(p, q, j);
        int64_t base = 0;
        int32_t deg = 0;
        if (WRITE) {
            base = row_off[q.id];
            deg = (int32_t)(row_off[q.id + 1] - base);
        }
        int32_t mine = 0;
        for (int32_t c0 = sg.z; c0 < sg.w; c0 += blockDim.x) {  // uniform trip count per warp
            const int32_t c = c0 + threadIdx.x;
            const bool v = c < sg.w && c != qp;
            uint64_t Ac = 0;
            PMS pc{};
            if (v) { Ac = __ldg(b.A + c); pc = b.pms[c]; }
            const bool e = v && decide_loaded<F64>(p, b, q, q64, Aq, Ac, pc, c, W, n_cand, n_re);
            if (WRITE) warp_emit(b, qp, base, deg, e, pc.id, lt, lane);
            else mine += (int)e;
        }
        if (!WRITE) {
            int32_t d = mine;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
            if (lane == 0) s_red[threadIdx.x >> 5] = d;
            __syncthreads();
            if (threadIdx.x == 0) {
                int32_t t = 0;
                for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_red[w];
                if (t) atomicAdd(&b.deg[q.id], t);
                n_edge += t;
            }
            __syncthreads();
        }
    }
    if (!WRITE) add_stats(b.stats, n_cand, n_re, n_edge);
}

// hub rows are written out of order: every one with two or more entries is sorted
__global__ void k_hub_classify(QueryBufs b, int32_t p_hub)
{
    const int64_t qp = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (qp >= p_hub) return;
    const int32_t id = b.pms[qp].id;
    const int32_t d = b.deg[id];
    if (d < 2) return;
    const int cls = d <= kWarpRow ? 0 : (d <= kSmemRow ? 1 : 2);
    const int k = atomicAdd(&b.list_cnt[cls], 1);
    b.rows[cls][k] = id;
    if (cls == 2) atomicAdd((unsigned long long *)b.big_total, (unsigned long long)d);
}

__global__ void k_hub_check(QueryBufs b, int32_t p_hub)
{
    const int64_t qp = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (qp >= p_hub) return;
    if (b.cursor[qp] != b.deg[b.pms[qp].id]) atomicOr((unsigned long long *)&b.stats[ST_ERR], 1ull);
}

constexpr unsigned kHeavyGrid = 152 * 8;

}  // namespace

int query_launches(const Plan &p, int32_t p_hub, bool write)
{
    return (p_hub > 0 ? 3 : 0) + (p.hub_bands < p.B ? 1 : 0);
}

cudaError_t launch_count_hub(const Plan &p, const QueryBufs &b, bool fp64_only, int32_t p_hub, cudaStream_t s)
{
    if (p_hub <= 0) return cudaSuccess;
    const unsigned g = (unsigned)(((int64_t)p_hub * 32 + 255) / 256);
    if (fp64_only) {
        k_hub_warp<true, false><<<g, 256, 0, s>>>(p, b, p_hub, nullptr);
        k_hub_heavy<true, false><<<kHeavyGrid, 256, 0, s>>>(p, b, nullptr);
    } else {
        k_hub_warp<false, false><<<g, 256, 0, s>>>(p, b, p_hub, nullptr);
        k_hub_heavy<false, false><<<kHeavyGrid, 256, 0, s>>>(p, b, nullptr);
    }
    k_hub_classify<<<(unsigned)((p_hub + 255) / 256), 256, 0, s>>>(b, p_hub);
    return cudaGetLastError();
}

cudaError_t launch_write_hub(const Plan &p, const QueryBufs &b, bool fp64_only, int32_t p_hub,
                             const int64_t *row_off, int32_t *col_idx, cudaStream_t s)
{
    if (p_hub <= 0) return cudaSuccess;
    QueryBufs bw = b;
    bw.col_out = col_idx;
    const unsigned g = (unsigned)(((int64_t)p_hub * 32 + 255) / 256);
    if (fp64_only) {
        k_hub_warp<true, true><<<g, 256, 0, s>>>(p, bw, p_hub, row_off);
        k_hub_heavy<true, true><<<kHeavyGrid, 256, 0, s>>>(p, bw, row_off);
    } else {
        k_hub_warp<false, true><<<g, 256, 0, s>>>(p, bw, p_hub, row_off);
        k_hub_heavy<false, true><<<kHeavyGrid, 256, 0, s>>>(p, bw, row_off);
    }
    k_hub_check<<<(unsigned)((p_hub + 255) / 256), 256, 0, s>>>(bw, p_hub);
    return cudaGetLastError();
}

cudaError_t launch_count_rim(const Plan &p, const QueryBufs &b, bool fp64_only, cudaStream_t s)
{
    if (p.hub_bands >= p.B) return cudaSuccess;
    const unsigned sectors = 1u << p.sbits;
    if (fp64_only) k_rim_sector<true, false><<<sectors, 256, 0, s>>>(p, b, nullptr, nullptr);
    else k_rim_sector<false, false><<<sectors, 256, 0, s>>>(p, b, nullptr, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_write_rim(const Plan &p, const QueryBufs &b, bool fp64_only, const int64_t *row_off,
                             int32_t *col_idx, cudaStream_t s)
{
    if (p.hub_bands >= p.B) return cudaSuccess;
    const unsigned sectors = 1u << p.sbits;
    if (fp64_only) k_rim_sector<true, true><<<sectors, 256, 0, s>>>(p, b, row_off, col_idx);
    else k_rim_sector<false, true><<<sectors, 256, 0, s>>>(p, b, row_off, col_idx);
    return cudaGetLastError();
}

}  // namespace hrg
