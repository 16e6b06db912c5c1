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
// The count pass counts degrees and keeps what it finds where that is cheap:
// rim rows of up to kKeepRow ids in a row buffer, hub rows in a pool of runs.
// The write pass copies those into the caller's CSR and traverses only the
// longer rim rows again (and the hub rows if the pool overflowed); rows not
// sorted on the way are sorted afterwards by hrg_sort.cu.
//
// Two work mappings:
//   * rim bands (most vertices, small windows): one CTA per angular sector,
//     one thread per query, all bands of the sector together so that the
//     band data near the sector is read once per sector;
//   * hub bands (few vertices, wide windows): one warp per query; lane j
//     sets up band j's window, then all lanes stride over each band's
//     candidates.
#include <algorithm>
#include <cstdio>
#include "hrg_internal.h"

namespace hrg {

namespace {

enum { ST_CAND = 0, ST_RECHECK = 1, ST_EDGES = 2, ST_TIES = 3, ST_NOROOM = 4, ST_ERR = 7 };



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
        if (lo <= hi) {
            i0 = bl;
            i1 = bh + 1;
        } else if (bh < bl) {  // the window wraps through angle 0
            i0 = bl;
            i3 = bh + 1;
        }  // else it wraps and leaves a gap inside one bucket: the whole band, once
    }
    rg.s0 = __ldg(start + b0 + i0);
    rg.e0 = __ldg(start + b0 + i1);
    rg.s1 = __ldg(start + b0 + i2);
    rg.e1 = __ldg(start + b0 + i3);
    return rg;
}

// Candidate positions in band j of every query whose fixed-point angle lies
// in [Amin, Amax] (no wrap: one angular sector) and whose window is at most
// W: the buckets of [Amin - W, Amax + W], one or two ranges, or the whole
// band.
__device__ __forceinline__ Ranges span_ranges(const Plan &p, const int32_t *__restrict__ start, uint64_t Amin,
                                              uint64_t Amax, uint64_t W, int j)
{
    Ranges rg;
    const int64_t b0 = p.base[j];
    const int g = p.gbits[j];
    const int64_t G = (int64_t)1 << g;
    rg.W = W;
    int64_t i0 = 0, i1 = G, i2 = 0, i3 = 0;
    const uint64_t span = Amax - Amin;
    if (W != kFullCircle && g != 0 && W < (~0ull - span) / 2) {
        const uint64_t lo = Amin - W, hi = Amax + W;
        const int64_t bl = (int64_t)(lo >> (64 - g)), bh = (int64_t)(hi >> (64 - g));
        if (lo <= hi) {
            i0 = bl;
            i1 = bh + 1;
        } else if (bh < bl) {  // through angle 0
            i0 = bl;
            i3 = bh + 1;
        }  // else the gap lies inside one bucket: the whole band
    }
    rg.s0 = __ldg(start + b0 + i0);
    rg.e0 = __ldg(start + b0 + i1);
    rg.s1 = __ldg(start + b0 + i2);
    rg.e1 = __ldg(start + b0 + i3);
    return rg;
}

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

__device__ __forceinline__ bool within(uint64_t Aq, uint64_t Ac, uint64_t W)
{
    const uint64_t d = Ac - Aq;
    const uint64_t ad = (int64_t)d < 0 ? (0ull - d) : d;
    return ad <= W;
}

// Decide candidate c (position cpos, data already loaded) for query q.
// n_re counts the FP64 rechecks in its low 24 bits and, above them, the
// pairs of the tie band (each pair once: from its smaller id); one counter
// keeps the register budget of the hot loop.
constexpr unsigned kTieUnit = 1u << 24;
// tie_side: whether this side of the pair counts it (one of the two sides).
template <bool F64>
__device__ __forceinline__ bool decide_pair(const Plan &p, const QueryBufs &b, const PMS &q, const PMS64 &q64,
                                            uint64_t Aq, uint64_t Ac, const PMS &cc, int32_t cpos, uint64_t W,
                                            unsigned &n_cand, unsigned &n_re, bool tie_side)
{
    if (W != kFullCircle && !within(Aq, Ac, W)) return false;
    ++n_cand;
    if (F64) {
        const PMS64 c64 = b.pms64[cpos];
        const double v = lhs_pms64(q64, c64);
        const long long vb = __double_as_longlong(v);
        if (vb > p.tie_lo && vb < p.tie_hi && tie_side) n_re += kTieUnit;
        return v < p.rhs64;
    } else {
        const float v = lhs32(q, cc, (int64_t)(Ac - Aq));
        if (v < p.rhs32 * (1.0f - p.mu)) return true;
        if (v > p.rhs32 * (1.0f + p.mu)) return false;
        const double d = cosh_dist64(__ldg(b.r + q.id), __ldg(b.phi + q.id), __ldg(b.r + cc.id), __ldg(b.phi + cc.id));
        n_re += 1u + ((fabs(d - p.coshR) < kTieBand * p.coshR && tie_side) ? kTieUnit : 0u);
        return d < p.coshR;
    }
}

// every vertex queries: the pair counts from its smaller id
template <bool F64>
__device__ __forceinline__ bool decide_loaded(const Plan &p, const QueryBufs &b, const PMS &q, const PMS64 &q64,
                                              uint64_t Aq, uint64_t Ac, const PMS &cc, int32_t cpos, uint64_t W,
                                              unsigned &n_cand, unsigned &n_re)
{
    return decide_pair<F64>(p, b, q, q64, Aq, Ac, cc, cpos, W, n_cand, n_re, q.id < cc.id);
}

__device__ __forceinline__ void add_stats(unsigned long long *stats, unsigned n_cand, unsigned n_re, unsigned n_edge)
{
    unsigned long long a = n_cand, r = n_re & (kTieUnit - 1u), e = n_edge, t = n_re / kTieUnit;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        r += __shfl_down_sync(0xffffffffu, r, o);
        e += __shfl_down_sync(0xffffffffu, e, o);
        t += __shfl_down_sync(0xffffffffu, t, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (a) atomicAdd(&stats[ST_CAND], a);
        if (r) atomicAdd(&stats[ST_RECHECK], r);
        if (e) atomicAdd(&stats[ST_EDGES], e);
        if (t) atomicAdd(&stats[ST_TIES], t);
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

// list[...] += v for the lanes with e: one atomic per warp
__device__ __forceinline__ void warp_append(int32_t *list, int32_t *count, bool e, int32_t v, int lane)
{
    const unsigned m = __ballot_sync(0xffffffffu, e);
    if (m == 0) return;
    int32_t base = 0;
    if (lane == 0) base = atomicAdd(count, __popc(m));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (e) list[base + __popc(m & ((1u << lane) - 1u))] = v;
}

constexpr int kRimThreads = 128;

// ---------------------------------------------------------------------------
// One query, one thread (rim bands).  The count pass stores a row of up to
// kKeepRow entries in the row buffer (b.small) and records where
// (b.small_off[position]); the write pass then copies it instead of
// traversing the query again (k_rim_copy), sorting rows of up to
// kCopySortRow entries on the way (longer kept rows go to the row sort).
// Longer rows, and rows that did not fit in the buffer, are traversed again
// by the write pass, which keeps rows of up to kRegRow entries sorted in
// registers.
// ---------------------------------------------------------------------------
// The traversal.  Count pass: every query of the sector, all lanes of the
// warp together (warp-collective operations); write pass: only queries whose
// row was not kept (no warp-collective operations there, so the write pass
// may call it for any subset of lanes).
template <bool F64, bool WRITE>
__device__ __forceinline__ void thread_query(const Plan &p, const QueryBufs &b, int32_t qp, bool active,
                                             const int64_t *__restrict__ row_off,
                                             int32_t *__restrict__ col_idx, unsigned &n_cand, unsigned &n_re,
                                             unsigned &n_edge)
{
    const int lane = threadIdx.x & 31;
    PMS q{};
    int64_t base = 0;
    int32_t deg = 0;
    if (active) {
        q = b.pms[qp];
        if (WRITE) {
            base = row_off[q.id];
            deg = (int32_t)(row_off[q.id + 1] - base);
        }
    }
    int32_t buf[kKeepRow];
    int32_t cnt = 0;
    if (!WRITE) {
        // Count pass (all lanes of the warp here): the hub bands for the
        // warp's queries together.  Their windows shrink as the query moves
        // out, so the window at the warp's smallest radius, widened by the
        // warp's angular span, holds every candidate of every lane; lane h
        // finds band h's range, then all lanes walk each range (the same
        // candidate for all lanes: one load) and decide it for their own
        // query by the predicate alone.
        const int H = p.hub_bands;
        if (H > p.first_band && __any_sync(0xffffffffu, active)) {
            const uint64_t Aq = active ? b.A[qp] : 0ull;
            PMS64 q64{};
            if (F64 && active) q64 = b.pms64[qp];
            const unsigned pkey = active ? __float_as_uint(q.P) : 0xFFFFFFFFu;  // P > 0: bits order like values
            const unsigned pmin = __reduce_min_sync(0xffffffffu, pkey);
            const int src = __ffs(__ballot_sync(0xffffffffu, pkey == pmin)) - 1;
            PMS qm;
            qm.P = __shfl_sync(0xffffffffu, q.P, src);
            qm.M = __shfl_sync(0xffffffffu, q.M, src);
            qm.S = __shfl_sync(0xffffffffu, q.S, src);
            qm.id = 0;
            uint64_t amin = active ? Aq : ~0ull, amax = active ? Aq : 0ull;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const uint64_t x = __shfl_xor_sync(0xffffffffu, amin, o), y = __shfl_xor_sync(0xffffffffu, amax, o);
                amin = min(amin, x);
                amax = max(amax, y);
            }
            for (int h0 = 0; h0 < H; h0 += 32) {
                const int hl = h0 + lane;
                Ranges mine{0, 0, 0, 0, 0};
                if (hl < H && hl >= p.first_band)
                    mine = span_ranges(p, b.start, amin, amax, window_halfwidth(p, qm, hl), hl);
                // the candidates of all these bands as one list: lane h's
                // ranges hold items [excl, incl) of it
                const int32_t n0 = max(0, mine.e0 - mine.s0), nh = n0 + max(0, mine.e1 - mine.s1);
                int32_t incl = nh;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += y;
                }
                const int32_t total = __shfl_sync(0xffffffffu, incl, 31);
                for (int32_t i0 = 0; i0 < total; i0 += 32) {
                    // lane l loads item i0 + l: its band lane is the first with incl > item
                    const int32_t it = i0 + lane;
                    int own = 0;
#pragma unroll
                    for (int step = 16; step > 0; step >>= 1) {
                        const int32_t v = __shfl_sync(0xffffffffu, incl, own + step - 1);
                        if (v <= it) own += step;
                    }
                    own = min(own, 31);
                    const int32_t o_incl = __shfl_sync(0xffffffffu, incl, own);
                    const int32_t o_n = __shfl_sync(0xffffffffu, nh, own);
                    const int32_t o_n0 = __shfl_sync(0xffffffffu, n0, own);
                    const int32_t o_s0 = __shfl_sync(0xffffffffu, mine.s0, own);
                    const int32_t o_s1 = __shfl_sync(0xffffffffu, mine.s1, own);
                    const int32_t pos = it - (o_incl - o_n);
                    const int32_t cp = pos < o_n0 ? o_s0 + pos : o_s1 + (pos - o_n0);
                    uint64_t Al = 0;
                    PMS pl{};
                    if (it < total) {
                        Al = __ldg(b.A + cp);
                        pl = b.pms[cp];
                    }
                    const int m = min(32, total - i0);
                    for (int k = 0; k < m; ++k) {  // warp-uniform: every lane decides item i0 + k
                        PMS cc;
                        cc.P = __shfl_sync(0xffffffffu, pl.P, k);
                        cc.M = __shfl_sync(0xffffffffu, pl.M, k);
                        cc.S = __shfl_sync(0xffffffffu, pl.S, k);
                        cc.id = __shfl_sync(0xffffffffu, pl.id, k);
                        const uint64_t Ac = __shfl_sync(0xffffffffu, Al, k);
                        const int32_t c = __shfl_sync(0xffffffffu, cp, k);
                        if (!active) continue;
                        if (!decide_loaded<F64>(p, b, q, q64, Aq, Ac, cc, c, kFullCircle, n_cand, n_re)) continue;
                        if (cnt < kKeepRow) buf[cnt] = cc.id;
                        ++cnt;
                    }
                }
            }
        }
    }
    if (active) {
        const uint64_t Aq = b.A[qp];
        PMS64 q64{};
        if (F64) q64 = b.pms64[qp];
        // bands before first_band hold no point; the count pass has done the hub bands
        for (int j = WRITE ? p.first_band : max(p.first_band, p.hub_bands); j < p.B; ++j) {
            const Ranges rg = band_ranges(p, b.start, q, Aq, j);
            for (int part = 0; part < 2; ++part) {
                const int32_t s = part ? rg.s1 : rg.s0, e = part ? rg.e1 : rg.e0;
                // the next candidate's data is loaded one iteration ahead
                uint64_t An = 0;
                PMS cn{};
                if (s < e) {
                    An = __ldg(b.A + s);
                    cn = b.pms[s];
                }
                for (int32_t c = s; c < e; ++c) {
                    const uint64_t Ac = An;
                    const PMS cc = cn;
                    if (c + 1 < e) {
                        An = __ldg(b.A + c + 1);
                        cn = b.pms[c + 1];
                    }
                    if (c == qp) continue;
                    if (rg.W != kFullCircle && !within(Aq, Ac, rg.W)) continue;
                    if (!decide_loaded<F64>(p, b, q, q64, Aq, Ac, cc, c, kFullCircle, n_cand, n_re)) continue;
                    const int32_t id = cc.id;
                    if (WRITE) {
                        if (cnt < kRegRow) {  // insertion into the sorted list (rows not kept)
                            int32_t k = cnt;
                            for (; k > 0 && buf[k - 1] > id; --k) buf[k] = buf[k - 1];
                            buf[k] = id;
                        }
                        if (deg > kRegRow && cnt < deg) col_idx[base + cnt] = id - p.id_off;
                    } else if (cnt < kKeepRow) {
                        buf[cnt] = id;  // count pass: kept unsorted
                    }
                    ++cnt;
                }
            }
        }
    }
    if (WRITE) {
        if (active) {
            if (cnt != deg) atomicOr((unsigned long long *)&b.stats[ST_ERR], 1ull);
            if (deg <= kRegRow)
                for (int32_t k = 0; k < cnt && k < deg; ++k) col_idx[base + k] = buf[k] - p.id_off;
        }
    } else {
        // keep rows of up to kKeepRow entries: warp-aggregated reservation in b.small
        const bool keep = active && cnt <= kKeepRow && cnt > 0;
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
        int32_t off = -1;
        if (active) {
            const long long pos = wbase + incl - want;
            if (keep && pos + cnt <= b.small_cap) {
                for (int32_t k = 0; k < cnt; ++k) b.small[pos + k] = buf[k];
                off = (int32_t)pos;
            } else if (keep) {
                atomicAdd(&b.stats[ST_NOROOM], 1ull);  // kept nowhere: the write pass traverses it again
            }
            b.small_off[qp] = off;
            b.deg[q.id] = cnt;
            if (off < 0 || cnt > kCopySortRow) classify_row(b, q.id, cnt);  // the rest is sorted by k_rim_copy
        }
        // the write pass's work list: rows to traverse again, by length (a
        // warp then walks rows of similar length); kept rows are found by id
        const int rc = cnt <= 64 ? 0 : (cnt <= 128 ? 1 : (cnt <= 256 ? 2 : 3));
#pragma unroll
        for (int c = 0; c < 4; ++c)
            warp_append(b.relist[c], &b.list_cnt[4 + c], active && off < 0 && cnt > 0 && rc == c, qp, lane);
    }
    if (active) n_edge += cnt;
}

// One CTA per angular sector: the queries of all rim bands whose angle lies
// in the sector.  Sector s of band j is the bucket range
// [s << (g_j - sbits), (s + 1) << (g_j - sbits)) (every band has g_j >= sbits).
template <bool F64>
__device__ __forceinline__ void rim_sector(const Plan &p, const QueryBufs &b, int64_t sector)
{
    __shared__ int32_t s_beg[HRG_MAX_BANDS];
    __shared__ int32_t s_pre[HRG_MAX_BANDS + 1];
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
    __shared__ int32_t s_next;
    if (threadIdx.x == 0) {
        s_pre[0] = 0;
        for (int j = 0; j < HRG_MAX_BANDS; ++j) s_pre[j + 1] += s_pre[j];
        s_next = blockDim.x;
    }
    __syncthreads();
    const int32_t total = s_pre[HRG_MAX_BANDS];
    unsigned n_cand = 0, n_re = 0, n_edge = 0;
    int j = 0;
    // Warp-uniform loop (the count pass reserves buffer space per warp):
    // warp w takes the 32 queries from 32 w first, then the next 32 not yet
    // taken, so the warps of the block finish together although their
    // queries' costs differ (the block's slot on the SM is free only when its
    // last warp is done).
    for (int32_t t0 = threadIdx.x & ~31; t0 < total;) {
        const int32_t t = t0 + (threadIdx.x & 31);
        const bool active = t < total;
        int32_t qp = 0;
        if (active) {
            while (t >= s_pre[j + 1]) ++j;  // t only grows, so j only moves forward
            qp = s_beg[j] + (t - s_pre[j]);
        }
        thread_query<F64, false>(p, b, qp, active, nullptr, nullptr, n_cand, n_re, n_edge);
        int32_t nx = 0;
        if ((threadIdx.x & 31) == 0) nx = atomicAdd(&s_next, 32);
        t0 = __shfl_sync(0xffffffffu, nx, 0);
    }
    add_stats(b.stats, n_cand, n_re, n_edge);
}

// Write pass of the rim rows kept by the count pass, in vertex-id order: warp
// w takes the ids [32 t, 32 t + 32) for t = w, w + (all warps), ..., lane l
// the id 32 t + l.  A row whose position has a kept row (small_off >= 0, at
// most kKeepRow entries) is read from the row buffer, sorted and stored at
// its row offset.  Consecutive rows thus fill col_idx front to back in whole
// sectors; the scattered accesses are reads of the row buffer instead.  Rows
// of up to kRegRow entries: every lane loads its own row into registers (all
// loads of the warp in flight together), sorts it with the network that fits
// the longest of them and leaves it in the warp's shared-memory tile, which
// the warp stores row by row (coalesced).  Longer kept rows are handled one
// at a time by the whole warp: sorted across its registers up to
// kCopySortRow entries (two ids a lane up to 64, four beyond), copied as kept
// above that (the row sort orders them).
constexpr int kCopyWarps = 8;
static_assert(kCopySortRow <= 128, "kept rows are sorted in at most four registers a lane");

template <int N>
__device__ __forceinline__ void sort_tile_row(int32_t (*T)[kRegRow + 1], const int32_t *__restrict__ src, int lane,
                                              int32_t deg, int32_t off)
{
    int32_t v[kRegRow];
#pragma unroll
    for (int j = 0; j < N; ++j) v[j] = j < deg ? __ldg(src + j) : 0x7fffffff;
    bitonic_regs<N>(v);
#pragma unroll
    for (int j = 0; j < N; ++j)
        if (j < deg) T[lane][j] = v[j] - off;
}

// Ids [lo, hi) only (lo a multiple of 32).
template <bool BATCH>
__global__ void __launch_bounds__(32 * kCopyWarps) k_rim_copy(Plan p, QueryBufs b, const int64_t *__restrict__ row_off,
                                                              int32_t *__restrict__ col_idx, int64_t lo, int64_t hi)
{
    __shared__ int32_t tile[kCopyWarps][kRegRow][kRegRow + 1];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int32_t(*T)[kRegRow + 1] = tile[w];
    const int64_t n = hi, groups = (hi + 31) >> 5;
    const int64_t nwarps = (int64_t)gridDim.x * kCopyWarps;
    for (int64_t t = (lo >> 5) + (int64_t)blockIdx.x * kCopyWarps + w; t < groups; t += nwarps) {
        const int64_t id = (t << 5) + lane;
        int32_t stored = -1, deg = 0, off = 0;
        int64_t base = 0;
        if (id < n) {
            stored = b.small_off[__ldg(b.pos_of + id)];
            if (stored >= 0) {
                base = row_off[id];
                deg = (int32_t)(row_off[id + 1] - base);
                off = BATCH ? b.plans[__ldg(b.graph_of + id)].id_off : p.id_off;
            }
        }
        const int32_t dt = (stored >= 0 && deg <= kRegRow) ? deg : 0;  // rows of the tile
        const int32_t dmax = (int32_t)__reduce_max_sync(0xffffffffu, (unsigned)dt);
        if (dmax > 0) {
            const int32_t *src = b.small + (dt > 0 ? stored : 0);
            if (dmax <= 4) sort_tile_row<4>(T, src, lane, dt, off);
            else if (dmax <= 8) sort_tile_row<8>(T, src, lane, dt, off);
            else if (dmax <= 16) sort_tile_row<16>(T, src, lane, dt, off);
            else sort_tile_row<32>(T, src, lane, dt, off);
            __syncwarp();
            for (int i = 0; i < 32; ++i) {
                const int64_t bi = __shfl_sync(0xffffffffu, base, i);
                const int32_t di = __shfl_sync(0xffffffffu, dt, i);
                if (lane < di) col_idx[bi + lane] = T[i][lane];
            }
            __syncwarp();
        }
        // kept rows of kRegRow < d <= kKeepRow entries: one at a time
        unsigned longer = __ballot_sync(0xffffffffu, stored >= 0 && deg > kRegRow);
        while (longer) {
            const int i = __ffs(longer) - 1;
            longer &= longer - 1;
            const int32_t si = __shfl_sync(0xffffffffu, stored, i), di = __shfl_sync(0xffffffffu, deg, i);
            const int32_t oi = __shfl_sync(0xffffffffu, off, i);
            const int64_t bi = __shfl_sync(0xffffffffu, base, i);
            if (di > kCopySortRow) {  // copied as kept; the row sort orders it
                for (int32_t t = lane; t < di; t += 32) col_idx[bi + t] = b.small[si + t] - oi;
                continue;
            }
            if (di > 64) {  // four ids a lane
                int32_t v[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) v[r] = lane + 32 * r < di ? b.small[si + lane + 32 * r] : 0x7fffffff;
                warp_bitonic128(v, lane);
#pragma unroll
                for (int r = 0; r < 4; ++r)
                    if (lane + 32 * r < di) col_idx[bi + lane + 32 * r] = v[r] - oi;
                continue;
            }
            int32_t x = lane < di ? b.small[si + lane] : 0x7fffffff;
            int32_t y = lane + 32 < di ? b.small[si + lane + 32] : 0x7fffffff;
            warp_bitonic64(x, y, lane);
            if (lane < di) col_idx[bi + lane] = x - oi;
            if (lane + 32 < di) col_idx[bi + lane + 32] = y - oi;
        }
    }
}

// Rows the count pass did not keep (longer than kRegRow, or no room): the
// traversal again, one thread per row, all such rows side by side.
// Rows of ids [lo, hi) only.
template <bool F64, bool BATCH>
__global__ void __launch_bounds__(256) k_rim_relist(Plan p, QueryBufs b, const int64_t *__restrict__ row_off,
                                                    int32_t *__restrict__ col_idx, int64_t lo, int64_t hi)
{
    const int cls = blockIdx.y;
    const int32_t nr = *((volatile int32_t *)&b.list_cnt[4 + cls]);
    const int32_t *relist = b.relist[cls];
    unsigned n_cand = 0, n_re = 0, n_edge = 0;
    const bool all = lo == 0 && hi >= p.n;
    for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < nr; k += gridDim.x * blockDim.x) {
        const int32_t qp = relist[k];
        if (!all) {
            const int32_t id = b.pms[qp].id;
            if (id < lo || id >= hi) continue;
        }
        if (BATCH)
            thread_query<F64, true>(b.plans[__ldg(b.graph_of + qp)], b, qp, true, row_off, col_idx, n_cand, n_re,
                                    n_edge);
        else
            thread_query<F64, true>(p, b, qp, true, row_off, col_idx, n_cand, n_re, n_edge);
    }
}

// the graph of global item k of a batch: the last g with off[g] <= k
__device__ __forceinline__ int graph_search(const int64_t *__restrict__ off, int NG, int64_t k)
{
    int lo = 0, hi = NG;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(off + mid) <= k) lo = mid; else hi = mid;
    }
    return lo;
}

// Count pass.  One graph: block x is sector x.  A batch: block x is global
// sector x; the sector table gives its graph.  Eight blocks of four warps per
// SM leave 64 registers a thread, room for the candidate prefetch; small
// blocks free their SM slot soon after their sector's last query.
template <bool F64, bool BATCH>
__global__ void __launch_bounds__(kRimThreads, 8) k_rim_sector(Plan p, QueryBufs b)
{
    if (BATCH) {
        const int g = graph_search(b.sec_off, b.NG, blockIdx.x);
        rim_sector<F64>(b.plans[g], b, (int64_t)blockIdx.x - __ldg(b.sec_off + g));
    } else {
        rim_sector<F64>(p, b, blockIdx.x);
    }
}

// ---------------------------------------------------------------------------
// Hub bands.  One warp per query: lane j sets up band j's window, then all
// lanes stride over each band's range, two candidates per lane in flight.
// Ranges longer than kHeavy are cut into chunks (count pass) and processed by
// whole CTAs (k_hub_heavy), so no single warp walks millions of candidates.
// Degrees accumulate with atomics; rows are written through a per-row cursor
// in no particular order and sorted afterwards.  The count pass also keeps
// the ids it finds: a warp gathers them in shared memory (kHubStage) and, when
// that fills, reserves a run of the global pool with one atomic and copies
// them there, tagged with the query; a heavy chunk flushes its (at most
// kHeavy) ids once.  The write pass then copies the runs into the rows
// (k_hub_copy) instead of deciding the candidates again; only when the pool
// overflowed does it traverse them again.
// ---------------------------------------------------------------------------
constexpr int kHubStage = 1024;
constexpr int kHubPer = 2;  // candidates a lane per step of a hub query's walk
constexpr int kPoolRunShift = 40;  // pool_cur[0] = runs << 40 | entries: one atomic reserves both

// a run of `fill` ids: (pool offset, run index), or false when the pool or
// the run table overflowed (the host then traverses the hub rows again)
__device__ __forceinline__ bool pool_reserve(const QueryBufs &b, int32_t fill, unsigned long long &off,
                                             unsigned long long &run)
{
    const unsigned long long old = atomicAdd(&b.pool_cur[0], (1ull << kPoolRunShift) | (unsigned long long)fill);
    off = old & ((1ull << kPoolRunShift) - 1);
    run = old >> kPoolRunShift;
    return off + (unsigned long long)fill <= (unsigned long long)b.pool_cap && run < (unsigned long long)b.run_cap;
}

// ids buf[0, fill) of hub query qi into a run of the pool (whole warp)
__device__ __forceinline__ void pool_flush(const QueryBufs &b, int32_t qi, const int32_t *buf, int32_t fill, int lane)
{
    if (fill == 0) return;
    unsigned long long off = 0, run = 0;
    int ok = 0;
    if (lane == 0) ok = pool_reserve(b, fill, off, run);
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (!ok) return;
    off = __shfl_sync(0xffffffffu, off, 0);
    for (int32_t k = lane; k < fill; k += 32) b.pool[off + k] = buf[k];
    if (lane == 0) b.runs[run] = make_int4(qi, fill, (int)(uint32_t)off, (int)(uint32_t)(off >> 32));
}

// write of this lane's edge (if any) at the warp's running offset pos of a
// hub row: no atomics, the warp owns [base, base + its count)
__device__ __forceinline__ void warp_put(int32_t *__restrict__ out, int64_t base, int32_t lim, int32_t &pos, bool e,
                                         int32_t id, unsigned lt)
{
    const unsigned m = __ballot_sync(0xffffffffu, e);
    if (e) {
        const int32_t k = pos + __popc(m & lt);
        if (k < lim) out[base + k] = id;
    }
    pos += __popc(m);
}

// Hub query number qi at position qp (the same for a single graph; the hub
// list of a batch maps one to the other).
template <bool F64, bool WRITE>
__device__ __forceinline__ void hub_query(const Plan &p, const QueryBufs &b, int32_t qi, int32_t qp,
                                          const int64_t *__restrict__ row_off, int32_t *stage)
{
    const int lane = threadIdx.x & 31;
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
    int32_t pos = 0;                               // write pass: entries this warp has written
    const int32_t lim = WRITE ? b.warp_cnt[qi] : 0;  // ... and must write
    const bool pooled = !WRITE && b.pool != nullptr;
    int32_t fill = 0;                              // count pass: ids gathered in stage (warp-uniform)
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
                            b.heavy[idx] = make_int4(qi, 2 * j + part, s + k * kHeavy, min(e, s + (k + 1) * kHeavy));
                    }
                }
                continue;
            }
            // kHubPer candidates a lane per step, their loads in flight together
            for (int32_t c0 = s; c0 < e; c0 += 32 * kHubPer) {
                bool v[kHubPer], ed[kHubPer];
                uint64_t Ac[kHubPer];
                PMS pc[kHubPer];
#pragma unroll
                for (int u = 0; u < kHubPer; ++u) {
                    const int32_t c = c0 + 32 * u + lane;
                    v[u] = c < e && c != qp;
                    Ac[u] = 0;
                    pc[u] = PMS{};
                    if (v[u]) {
                        Ac[u] = __ldg(b.A + c);
                        pc[u] = b.pms[c];
                    }
                }
#pragma unroll
                for (int u = 0; u < kHubPer; ++u)
                    ed[u] = v[u] && decide_loaded<F64>(p, b, q, q64, Aq, Ac[u], pc[u], c0 + 32 * u + lane, rg.W,
                                                       n_cand, n_re);
                if (WRITE) {
#pragma unroll
                    for (int u = 0; u < kHubPer; ++u) warp_put(b.col_out, base, lim, pos, ed[u], pc[u].id - p.id_off, lt);
                } else {
                    unsigned m[kHubPer];
                    int32_t add = 0;
#pragma unroll
                    for (int u = 0; u < kHubPer; ++u) {
                        mine += (int)ed[u];
                        m[u] = __ballot_sync(0xffffffffu, ed[u]);
                        add += __popc(m[u]);
                    }
                    if (pooled) {
                        if (fill + add > kHubStage) {
                            __syncwarp();
                            pool_flush(b, qi, stage, fill, lane);
                            __syncwarp();
                            fill = 0;
                        }
#pragma unroll
                        for (int u = 0; u < kHubPer; ++u) {
                            if (ed[u]) stage[fill + __popc(m[u] & lt)] = pc[u].id - p.id_off;
                            fill += __popc(m[u]);
                        }
                    }
                }
            }
        }
    }
    if (!WRITE) {
        if (pooled) {
            __syncwarp();
            pool_flush(b, qi, stage, fill, lane);
        }
        int32_t d = mine;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
        if (lane == 0) {
            b.warp_cnt[qi] = d;
            if (d) atomicAdd(&b.deg[q.id], d);
        }
        add_stats(b.stats, n_cand, n_re, lane == 0 ? (unsigned)d : 0u);
    } else if (lane == 0 && (pos != lim || lim > deg)) {
        atomicOr((unsigned long long *)&b.stats[ST_ERR], 1ull);
    }
    (void)deg;
}

template <bool F64, bool WRITE, bool BATCH>
__global__ void __launch_bounds__(256) k_hub_warp(Plan p, QueryBufs b, int32_t p_hub,
                                                  const int64_t *__restrict__ row_off)
{
    __shared__ int32_t s_stage[WRITE ? 1 : 8][WRITE ? 1 : kHubStage];  // count pass: one stage per warp
    const int32_t qi = (int32_t)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    if (qi >= p_hub) return;  // uniform per warp
    int32_t *stage = WRITE ? nullptr : s_stage[WRITE ? 0 : (threadIdx.x >> 5)];
    if (BATCH) {
        const int32_t qp = __ldg(b.hub_pos + qi);
        hub_query<F64, WRITE>(b.plans[__ldg(b.graph_of + qp)], b, qi, qp, row_off, stage);
    } else {
        hub_query<F64, WRITE>(p, b, qi, qi, row_off, stage);
    }
}

// One chunk (segment k) of a long hub range, by the whole CTA.  The count
// pass records the chunk's edges (seg_cnt[k]); the write pass reserves that
// many entries of the row with one atomic and places them by warp.
template <bool F64, bool WRITE>
__device__ __forceinline__ void heavy_chunk(const Plan &p, const QueryBufs &b, int32_t k, const int4 sg, int32_t qp,
                                            const int64_t *__restrict__ row_off, int32_t *s_red, int32_t *s_ids,
                                            unsigned &n_cand, unsigned &n_re, unsigned &n_edge)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int32_t qi = sg.x;
    const int j = sg.y >> 1;
    const PMS q = b.pms[qp];
    const uint64_t Aq = b.A[qp];
    PMS64 q64{};
    if (F64) q64 = b.pms64[qp];
    const uint64_t W = window_halfwidth(p, q, j);
    int64_t base = 0;
    int32_t lim = 0;
    if (WRITE) {
        // s_red[0]: first entry of this chunk in the row, s_red[1]: entries placed
        if (threadIdx.x == 0) {
            const int32_t cnt = b.seg_cnt[k];
            s_red[0] = b.warp_cnt[qi] + atomicAdd(&b.cursor[qi], cnt);
            s_red[1] = 0;
            s_red[2] = cnt;
        }
        __syncthreads();
        base = row_off[q.id] + s_red[0];
        lim = s_red[2];
    }
    int32_t mine = 0;
    const bool pooled = !WRITE && b.pool != nullptr;
    if (pooled) {  // s_red[8]: ids gathered in s_ids (at most kHeavy: one per candidate)
        if (threadIdx.x == 0) s_red[8] = 0;
        __syncthreads();
    }
    for (int32_t c0 = sg.z; c0 < sg.w; c0 += blockDim.x) {  // uniform trip count per warp
        const int32_t c = c0 + threadIdx.x;
        const bool v = c < sg.w && c != qp;
        uint64_t Ac = 0;
        PMS pc{};
        if (v) { Ac = __ldg(b.A + c); pc = b.pms[c]; }
        const bool e = v && decide_loaded<F64>(p, b, q, q64, Aq, Ac, pc, c, W, n_cand, n_re);
        if (pooled) {
            const unsigned m = __ballot_sync(0xffffffffu, e);
            if (m) {
                int32_t off = 0;
                if (lane == 0) off = atomicAdd(&s_red[8], __popc(m));
                off = __shfl_sync(0xffffffffu, off, 0) + __popc(m & lt);
                if (e) s_ids[off] = pc.id - p.id_off;
            }
        }
        if (WRITE) {
            const unsigned m = __ballot_sync(0xffffffffu, e);
            if (m) {
                int32_t off = 0;
                if (lane == 0) off = atomicAdd(&s_red[1], __popc(m));
                off = __shfl_sync(0xffffffffu, off, 0) + __popc(m & lt);
                if (e && off < lim) b.col_out[base + off] = pc.id - p.id_off;
            }
        } else {
            mine += (int)e;
        }
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
            b.seg_cnt[k] = t;
            if (t) atomicAdd(&b.deg[q.id], t);
            n_edge += t;
            // the chunk's ids: one run of the pool (s_red[9..11]: offset lo, hi, keep)
            const int32_t fill = pooled ? s_red[8] : 0;
            s_red[11] = 0;
            if (fill > 0) {
                unsigned long long off, run;
                if (pool_reserve(b, fill, off, run)) {
                    b.runs[run] = make_int4(qi, fill, (int)(uint32_t)off, (int)(uint32_t)(off >> 32));
                    s_red[9] = (int32_t)(uint32_t)off;
                    s_red[10] = (int32_t)(uint32_t)(off >> 32);
                    s_red[11] = fill;
                }
            }
        }
        __syncthreads();
        if (s_red[11] > 0) {
            const unsigned long long off =
                ((unsigned long long)(uint32_t)s_red[10] << 32) | (unsigned long long)(uint32_t)s_red[9];
            for (int32_t t = threadIdx.x; t < s_red[11]; t += blockDim.x) b.pool[off + t] = s_ids[t];
        }
        __syncthreads();
    } else {
        __syncthreads();
        if (threadIdx.x == 0 && s_red[1] != lim) atomicOr((unsigned long long *)&b.stats[ST_ERR], 1ull);
        __syncthreads();
    }
}

// One CTA per chunk of a long hub range.
template <bool F64, bool WRITE, bool BATCH>
__global__ void __launch_bounds__(256) k_hub_heavy(Plan p, QueryBufs b, const int64_t *__restrict__ row_off)
{
    __shared__ int32_t s_red[12];
    __shared__ int32_t s_ids[WRITE ? 1 : kHeavy];  // count pass: the chunk's ids for the pool
    const int32_t nseg = min(*((volatile int32_t *)&b.list_cnt[3]), b.heavy_cap);
    unsigned n_cand = 0, n_re = 0, n_edge = 0;
    for (int32_t k = blockIdx.x; k < nseg; k += gridDim.x) {
        const int4 sg = b.heavy[k];
        if (BATCH) {
            const int32_t qp = __ldg(b.hub_pos + sg.x);
            heavy_chunk<F64, WRITE>(b.plans[__ldg(b.graph_of + qp)], b, k, sg, qp, row_off, s_red, s_ids, n_cand,
                                    n_re, n_edge);
        } else {
            heavy_chunk<F64, WRITE>(p, b, k, sg, sg.x, row_off, s_red, s_ids, n_cand, n_re, n_edge);
        }
    }
    if (!WRITE) add_stats(b.stats, n_cand, n_re, n_edge);
}

__device__ __forceinline__ int32_t hub_position(const QueryBufs &b, int32_t qi)
{
    return b.hub_pos ? __ldg(b.hub_pos + qi) : qi;
}

// hub rows are written out of order: every one with two or more entries is sorted
__global__ void k_hub_classify(QueryBufs b, int32_t p_hub)
{
    const int64_t qi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (qi >= p_hub) return;
    const int32_t id = b.pms[hub_position(b, (int32_t)qi)].id;
    const int32_t d = b.deg[id];
    if (d < 2) return;
    const int cls = d <= kWarpRow ? 0 : (d <= kSmemRow ? 1 : 2);
    const int k = atomicAdd(&b.list_cnt[cls], 1);
    b.rows[cls][k] = id;
    if (cls == 2) atomicAdd((unsigned long long *)b.big_total, (unsigned long long)d);
}

__global__ void k_hub_check(QueryBufs b, int32_t p_hub)
{
    const int64_t qi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (qi >= p_hub) return;
    if (b.warp_cnt[qi] + b.cursor[qi] != b.deg[b.pms[hub_position(b, (int32_t)qi)].id])
        atomicOr((unsigned long long *)&b.stats[ST_ERR], 1ull);
}

// Write pass from the pool: one warp per run; its place in the row comes from
// one atomic on the row's cursor.
// Runs of the rows of ids [lo, hi) only.
__global__ void __launch_bounds__(256) k_hub_copy(QueryBufs b, int32_t n_runs, const int64_t *__restrict__ row_off,
                                                  int32_t *__restrict__ col_out, int64_t lo, int64_t hi)
{
    const int lane = threadIdx.x & 31;
    const int32_t nwarps = (int32_t)(gridDim.x * (blockDim.x >> 5));
    for (int32_t k = (int32_t)(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)); k < n_runs; k += nwarps) {
        const int4 run = b.runs[k];
        const int32_t qi = run.x, cnt = run.y;
        const unsigned long long off = ((unsigned long long)(uint32_t)run.w << 32) | (unsigned long long)(uint32_t)run.z;
        int64_t dst = -1;
        if (lane == 0) {
            const int32_t id = b.pms[hub_position(b, qi)].id;
            if (id >= lo && id < hi) dst = row_off[id] + atomicAdd(&b.cursor[qi], cnt);
        }
        dst = __shfl_sync(0xffffffffu, dst, 0);
        if (dst < 0) continue;
        for (int32_t t = lane; t < cnt; t += 32) col_out[dst + t] = b.pool[off + t];
    }
}

// every pooled hub row complete: its cursor equals its degree
__global__ void k_hub_check_pooled(QueryBufs b, int32_t p_hub)
{
    const int64_t qi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (qi >= p_hub) return;
    if (b.cursor[qi] != b.deg[b.pms[hub_position(b, (int32_t)qi)].id])
        atomicOr((unsigned long long *)&b.stats[ST_ERR], 1ull);
}

constexpr unsigned kHeavyGrid = 152 * 16;

template <bool F64, bool WRITE, bool BATCH>
static void hub_launch(const Plan &p, const QueryBufs &b, int32_t p_hub, const int64_t *row_off, cudaStream_t s)
{
    const unsigned g = (unsigned)(((int64_t)p_hub * 32 + 255) / 256);
    k_hub_warp<F64, WRITE, BATCH><<<g, 256, 0, s>>>(p, b, p_hub, row_off);
    k_hub_heavy<F64, WRITE, BATCH><<<kHeavyGrid, 256, 0, s>>>(p, b, row_off);
}

template <bool WRITE>
static void hub_dispatch(const Plan &p, const QueryBufs &b, bool fp64_only, int32_t p_hub, const int64_t *row_off,
                         cudaStream_t s)
{
    const bool batch = b.plans != nullptr;
    if (fp64_only) {
        if (batch) hub_launch<true, WRITE, true>(p, b, p_hub, row_off, s);
        else hub_launch<true, WRITE, false>(p, b, p_hub, row_off, s);
    } else {
        if (batch) hub_launch<false, WRITE, true>(p, b, p_hub, row_off, s);
        else hub_launch<false, WRITE, false>(p, b, p_hub, row_off, s);
    }
}

constexpr unsigned kRimWriteGrid = 152 * 16;

static void rim_count_dispatch(const Plan &p, const QueryBufs &b, bool fp64_only, unsigned sectors, cudaStream_t s)
{
    const bool batch = b.plans != nullptr;
    if (fp64_only) {
        if (batch) k_rim_sector<true, true><<<sectors, kRimThreads, 0, s>>>(p, b);
        else k_rim_sector<true, false><<<sectors, kRimThreads, 0, s>>>(p, b);
    } else {
        if (batch) k_rim_sector<false, true><<<sectors, kRimThreads, 0, s>>>(p, b);
        else k_rim_sector<false, false><<<sectors, kRimThreads, 0, s>>>(p, b);
    }
}

static void rim_write_dispatch(const Plan &p, const QueryBufs &b, bool fp64_only, const int64_t *row_off,
                               int32_t *col_idx, int64_t lo, int64_t hi, cudaStream_t s)
{
    const bool batch = b.plans != nullptr;
    const unsigned cg = kRimWriteGrid / 2;
    const dim3 rg(kRimWriteGrid / 4, 4);
    if (batch) k_rim_copy<true><<<cg, 32 * kCopyWarps, 0, s>>>(p, b, row_off, col_idx, lo, hi);
    else k_rim_copy<false><<<cg, 32 * kCopyWarps, 0, s>>>(p, b, row_off, col_idx, lo, hi);
    if (fp64_only) {
        if (batch) k_rim_relist<true, true><<<rg, 256, 0, s>>>(p, b, row_off, col_idx, lo, hi);
        else k_rim_relist<true, false><<<rg, 256, 0, s>>>(p, b, row_off, col_idx, lo, hi);
    } else {
        if (batch) k_rim_relist<false, true><<<rg, 256, 0, s>>>(p, b, row_off, col_idx, lo, hi);
        else k_rim_relist<false, false><<<rg, 256, 0, s>>>(p, b, row_off, col_idx, lo, hi);
    }
}

// ---------------------------------------------------------------------------
// Moved vertices of a dynamic update (hrg_update_begin): one CTA per moved
// vertex u queries its new position against the rebuilt band structure (all
// points at their current coordinates), every thread striding over each
// band's window.  Count pass: u's new degree into deg[u], and add[w] += 1 for
// every neighbour w that did not move (w gains u).  Write pass: u's row,
// unsorted, at row_off_out[u], and u itself into each such w's row after
// w's kept entries (keep[w]) at the slot add[w] hands out.  moved is a bit
// per vertex.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool moved_bit(const uint32_t *__restrict__ moved, int32_t v)
{
    return (__ldg(moved + (v >> 5)) >> (v & 31)) & 1u;
}

template <bool F64, bool WRITE>
__global__ void __launch_bounds__(256) k_move_query(Plan p, QueryBufs b, int64_t k, const int32_t *__restrict__ ids,
                                                    const uint32_t *__restrict__ moved, int32_t *__restrict__ deg,
                                                    int32_t *__restrict__ add, const int32_t *__restrict__ keep,
                                                    const int64_t *__restrict__ row_off_out, int32_t *col_out)
{
    __shared__ int32_t s_cnt;
    __shared__ int32_t s_red[8];
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    unsigned n_cand = 0, n_re = 0, n_edge = 0;
    for (int64_t i = blockIdx.x; i < k; i += gridDim.x) {
        const int32_t u = __ldg(ids + i);
        const int32_t qp = __ldg(b.pos_of + u);
        const PMS q = b.pms[qp];
        const uint64_t Aq = b.A[qp];
        PMS64 q64{};
        if (F64) q64 = b.pms64[qp];
        int64_t base = 0;
        if (WRITE) base = row_off_out[u];
        if (threadIdx.x == 0) s_cnt = 0;
        __syncthreads();
        int32_t mine = 0;
        for (int j = p.first_band; j < p.B; ++j) {
            const Ranges rg = band_ranges(p, b.start, q, Aq, j);
            for (int part = 0; part < 2; ++part) {
                const int32_t s = part ? rg.s1 : rg.s0, e = part ? rg.e1 : rg.e0;
                for (int32_t c0 = s; c0 < e; c0 += blockDim.x) {  // uniform trip count per warp
                    const int32_t c = c0 + (int32_t)threadIdx.x;
                    const bool v = c < e && c != qp;
                    uint64_t Ac = 0;
                    PMS pc{};
                    bool other_moved = false;
                    if (v) {
                        Ac = __ldg(b.A + c);
                        pc = b.pms[c];
                        other_moved = moved_bit(moved, pc.id);
                    }
                    // a pair with a vertex that stays is queried from this side only
                    const bool ed = v && decide_pair<F64>(p, b, q, q64, Aq, Ac, pc, c, rg.W, n_cand, n_re,
                                                          !other_moved || u < pc.id);
                    const bool stays = ed && !other_moved;
                    if (!WRITE) {
                        mine += (int)ed;
                        if (stays) atomicAdd(add + pc.id, 1);
                    } else {
                        const unsigned m = __ballot_sync(0xffffffffu, ed);
                        if (m) {
                            int32_t off = 0;
                            if (lane == 0) off = atomicAdd(&s_cnt, __popc(m));
                            off = __shfl_sync(0xffffffffu, off, 0) + __popc(m & lt);
                            if (ed) col_out[base + off] = pc.id;
                        }
                        if (stays) {
                            const int32_t w = pc.id;
                            col_out[row_off_out[w] + __ldg(keep + w) + atomicAdd(add + w, 1)] = u;
                        }
                    }
                }
            }
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
                deg[u] = t;
                n_edge += t;
            }
        } else {
            __syncthreads();
            if (threadIdx.x == 0 && (int64_t)s_cnt != row_off_out[u + 1] - base)
                atomicOr((unsigned long long *)&b.stats[ST_ERR], 1ull);
        }
        __syncthreads();
    }
    if (!WRITE) add_stats(b.stats, n_cand, n_re, n_edge);
}

}  // namespace

int query_launches(const Plan &p, int32_t p_hub, bool write)
{
    return (p_hub > 0 ? 3 : 0) + (p.hub_bands < p.B ? (write ? 2 : 1) : 0);
}

cudaError_t launch_count_hub(const Plan &p, const QueryBufs &b, bool fp64_only, int32_t p_hub, cudaStream_t s)
{
    if (p_hub <= 0) return cudaSuccess;
    hub_dispatch<false>(p, b, fp64_only, p_hub, nullptr, s);
    k_hub_classify<<<(unsigned)((p_hub + 255) / 256), 256, 0, s>>>(b, p_hub);
    return cudaGetLastError();
}

cudaError_t launch_copy_hub(const QueryBufs &b, int32_t p_hub, int32_t n_runs, const int64_t *row_off,
                            int32_t *col_idx, int64_t lo, int64_t hi, bool check, cudaStream_t s)
{
    if (p_hub <= 0) return cudaSuccess;
    if (n_runs > 0) k_hub_copy<<<kRimWriteGrid / 2, 256, 0, s>>>(b, n_runs, row_off, col_idx, lo, hi);
    if (check) k_hub_check_pooled<<<(unsigned)((p_hub + 255) / 256), 256, 0, s>>>(b, p_hub);
    return cudaGetLastError();
}

cudaError_t launch_write_hub(const Plan &p, const QueryBufs &b, bool fp64_only, int32_t p_hub,
                             const int64_t *row_off, int32_t *col_idx, cudaStream_t s)
{
    if (p_hub <= 0) return cudaSuccess;
    QueryBufs bw = b;
    bw.col_out = col_idx;
    hub_dispatch<true>(p, bw, fp64_only, p_hub, row_off, s);
    k_hub_check<<<(unsigned)((p_hub + 255) / 256), 256, 0, s>>>(bw, p_hub);
    return cudaGetLastError();
}

cudaError_t launch_move_query(const Plan &p, const QueryBufs &b, bool fp64_only, bool write, int64_t k,
                              const int32_t *ids, const uint32_t *moved, int32_t *deg, int32_t *add,
                              const int32_t *keep, const int64_t *row_off_out, int32_t *col_out, cudaStream_t s)
{
    if (k <= 0) return cudaSuccess;
    const unsigned g = (unsigned)std::min<int64_t>(k, 152 * 8);
    if (fp64_only) {
        if (write) k_move_query<true, true><<<g, 256, 0, s>>>(p, b, k, ids, moved, deg, add, keep, row_off_out, col_out);
        else k_move_query<true, false><<<g, 256, 0, s>>>(p, b, k, ids, moved, deg, add, keep, row_off_out, col_out);
    } else {
        if (write) k_move_query<false, true><<<g, 256, 0, s>>>(p, b, k, ids, moved, deg, add, keep, row_off_out, col_out);
        else k_move_query<false, false><<<g, 256, 0, s>>>(p, b, k, ids, moved, deg, add, keep, row_off_out, col_out);
    }
    return cudaGetLastError();
}

cudaError_t launch_count_rim(const Plan &p, const QueryBufs &b, bool fp64_only, cudaStream_t s)
{
    if (b.plans == nullptr && p.hub_bands >= p.B) return cudaSuccess;
    const unsigned sectors = b.plans ? (unsigned)b.n_sectors : 1u << p.sbits;
    if (sectors == 0) return cudaSuccess;
    rim_count_dispatch(p, b, fp64_only, sectors, s);
    return cudaGetLastError();
}

cudaError_t launch_write_rim(const Plan &p, const QueryBufs &b, bool fp64_only, const int64_t *row_off,
                             int32_t *col_idx, int64_t lo, int64_t hi, cudaStream_t s)
{
    if (b.plans == nullptr && p.hub_bands >= p.B) return cudaSuccess;
    if (b.plans != nullptr && b.n_sectors == 0) return cudaSuccess;
    rim_write_dispatch(p, b, fp64_only, row_off, col_idx, lo, hi, s);
    return cudaGetLastError();
}

}  // namespace hrg
