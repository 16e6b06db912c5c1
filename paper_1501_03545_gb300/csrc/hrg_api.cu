// hrg_api.cu -- the C ABI (include/hrg.h): contexts, jobs, workspace, plan.
#include <algorithm>
#include <cmath>
#include <nvtx3/nvToolsExt.h>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "../../include/hrg.h"
#include "hrg_internal.h"
#include "hrg_graph_ops.h"

using namespace hrg;

// ---------------------------------------------------------------------------
// Eq. (22) of Krioukov et al. (Appendix B.1), zeta = 1.  The expression is
//   kbar(R) = (2/pi) xi^2 n [ e^{-R/2} + e^{-alpha R} ( (alpha R / 2) c - 1 ) ],
//   xi = alpha / (alpha - 1/2),  c = (pi/4) alpha^-2 - (pi - 1) alpha^-1 + pi - 2.
// ---------------------------------------------------------------------------
static double eq22(double n, double alpha, double R)
{
    const double pi = 3.141592653589793;
    const double xi = alpha / (alpha - 0.5);
    const double ia = 1.0 / alpha;
    const double c = (pi / 4.0) * ia * ia - (pi - 1.0) * ia + (pi - 2.0);
    return (2.0 / pi) * xi * xi * n * (std::exp(-R / 2.0) + std::exp(-alpha * R) * (alpha * (R / 2.0) * c - 1.0));
}

extern "C" double hrg_expected_degree(int64_t n, double alpha, double R) { return eq22((double)n, alpha, R); }

// The expression rises from 0 at R = 0 to one maximum and then decays; the
// radius of a sparse graph lies on the decaying side.  Golden-section search
// brackets the maximum, then bisection finds the largest double R with
// kbar(R) >= target (it stops when the midpoint coincides with an end).
extern "C" int hrg_solve_radius(int64_t n, double alpha, double avg_degree, double *R_out)
{
    if (!R_out || n < 2 || !(alpha > 0.5) || !(avg_degree > 0.0) || !(avg_degree < (double)(n - 1)))
        return HRG_EINVAL;
    const double nn = (double)n;
    // coarse scan for the maximum on (0, 24], then golden-section search in
    // the two cells around the best point
    double best = -1e300, at = 0.0;
    for (int i = 1; i <= 96; ++i) {
        const double R = 0.25 * i;
        const double k = eq22(nn, alpha, R);
        if (k > best) { best = k; at = R; }
    }
    double a = std::max(0.0, at - 0.25), b = at + 0.25;
    const double gr = 0.6180339887498949;
    double x1 = b - gr * (b - a), x2 = a + gr * (b - a);
    double f1 = eq22(nn, alpha, x1), f2 = eq22(nn, alpha, x2);
    for (int it = 0; it < 90; ++it) {
        if (f1 < f2) { a = x1; x1 = x2; f1 = f2; x2 = a + gr * (b - a); f2 = eq22(nn, alpha, x2); }
        else { b = x2; x2 = x1; f2 = f1; x1 = b - gr * (b - a); f1 = eq22(nn, alpha, x1); }
    }
    const double peak = 0.5 * (a + b);
    if (eq22(nn, alpha, peak) < avg_degree) return HRG_EINVAL;
    double lo = peak, hi = peak + 1.0;
    while (eq22(nn, alpha, hi) >= avg_degree) {
        hi = peak + 2.0 * (hi - peak);
        if (hi > 1e7) return HRG_EINVAL;
    }
    for (;;) {
        const double mid = lo + 0.5 * (hi - lo);
        if (!(mid > lo && mid < hi)) break;
        if (eq22(nn, alpha, mid) >= avg_degree) lo = mid; else hi = mid;
    }
    *R_out = lo;
    return HRG_OK;
}

extern "C" const char *hrg_version(void) { return "hrg-gb300 0.1 (sm_103a)"; }

// ---------------------------------------------------------------------------
// Context and workspace.
// ---------------------------------------------------------------------------
struct DevBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
};

struct hrg_job {
    hrg_ctx *ctx = nullptr;
    Plan plan{};
    bool fp64 = false;
    bool sampled = false;  // points drawn by the generator (else injected)
    bool hub_pooled = false;  // the count pass kept every hub entry: the write pass copies them
    int32_t hub_runs = 0;
    int32_t heavy_retries = 0;  // count passes repeated for lack of room in the list of long hub ranges
    int32_t write_chunks = 1;   // id ranges of the write pass (hrg_generate_host)
    bool open = false;
    bool finished = false;
    int32_t p_hub = 0;
    int32_t lists[3] = {0, 0, 0};
    int64_t big_total = 0;
    int64_t n_entries = 0;
    uint64_t stats[8] = {};
    float stage_ms[8] = {};
    const double *r = nullptr, *phi = nullptr;
    int64_t *row_off = nullptr;
    cudaStream_t stream = nullptr;
    QueryBufs qb{};
    int32_t batch = 0;       // graphs of a batch job (0: a single graph)
    int64_t batch_G = 0;     // buckets over all graphs of a batch
    // vertex movement (hrg_update_begin): the old CSR, the moves and the
    // per-vertex bookkeeping between the two passes
    bool update = false;
    const int64_t *old_off = nullptr;
    const int32_t *old_col = nullptr;
    int64_t moves = 0;
    const int32_t *move_ids = nullptr;
    uint32_t *moved = nullptr;
    int32_t *rem = nullptr, *gain = nullptr, *gain_cur = nullptr, *keep = nullptr;
    int64_t old_entries = 0;
};

// The write pass of hrg_generate_host runs in up to kMaxChunks id ranges, so
// that each range's neighbour ids go back to the host while the next range
// is written and sorted.
constexpr int kMaxChunks = 8;

struct hrg_ctx {
    int device = 0;
    std::string err;
    // workspace slots
    enum { W_BANDCNT, W_GBUF, W_CNT, W_START, W_SLOT, W_A, W_PMS, W_PMS64, W_DEG, W_STATS, W_LIST0, W_LIST1,
           W_LIST2, W_LISTCNT, W_BIGTOT, W_SCAN, W_TMP, W_BUCKET, W_OUT_R, W_OUT_PHI, W_OUT_OFF, W_OUT_COL,
           W_HEAVY, W_CURSOR, W_SMALL, W_SMALLOFF, W_SMALLCUR, W_PLANS, W_NOFF, W_SOFF, W_GRAPHOF, W_HUBCNT,
           W_HUBOFF, W_HUBPOS, W_WARPCNT, W_SEGCNT, W_POSOF, W_RELIST0, W_RELIST1, W_RELIST2, W_RELIST3,
           W_PACC, W_POUTDEG, W_POUTOFF, W_POUTCOL, W_PTRI, W_PSCAN, W_LRCNT, W_LROFF, W_LRLIST, W_LRFIN,
           W_LRDEG, W_HPOOL, W_HRUNS, W_HPCUR, W_BFSF0, W_BFSF1, W_BFSDEG, W_BFSOFF, W_BFSACC, W_BFSDIST,
           W_MVBITS, W_MVREM, W_MVADD, W_MVCUR, W_MVKEEP, W_MVERR, W_MVSTART, W_MVWS, W_CHUNK, W_COUNT };
    DevBuf ws[W_COUNT];
    void *pinned = nullptr;  // small pinned staging area for read-backs
    cudaEvent_t ev[10] = {};  // stage boundaries of the current job
    bool nvtx_open = false;   // a stage's NVTX range is open on the host thread (stage_mark)
    cudaStream_t work = nullptr, copy = nullptr;  // hrg_generate_host: generation and read-back streams
    // hrg_generate_host: [0] points sampled, [1] [2] first and last read-back
    // on the copy stream, then four per range of the chunked write pass
    cudaEvent_t hev[3 + 4 * kMaxChunks] = {};
    hrg_job job;
    hrg_limits lim{};  // capacities of the count pass's buffers (0: automatic)
    std::vector<Plan> batch_plans;  // host plans of the current batch
    std::vector<int64_t> batch_noff, batch_soff;
};

static int set_err(hrg_ctx *c, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return code;
}

#define CK(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return set_err(ctx, HRG_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                           __FILE__, __LINE__);                                                    \
    } while (0)

// Kept-row buffer of the rim count pass: room for 32 entries per vertex.  The
// scatter's 32-byte point records use it before the count pass.
static int64_t small_capacity(int64_t n) { return std::min<int64_t>(32 * n + 1024, 0x7fff0000LL); }
// Stage boundary k of a job: the CUDA event that times the stages, and an
// NVTX range on the host thread around the launches of the stage that starts
// there (for profilers that record NVTX; a no-op otherwise).
static cudaError_t stage_mark(hrg_ctx *ctx, int k, cudaStream_t st)
{
    static const char *const names[10] = {"hrg sample",    "hrg bands", "hrg count hub", "hrg count rim",
                                          "hrg offsets",   nullptr,     "hrg write",     "hrg write rim",
                                          "hrg row sort",  nullptr};
    if (ctx->nvtx_open) nvtxRangePop();
    ctx->nvtx_open = names[k] != nullptr;
    if (ctx->nvtx_open) nvtxRangePushA(names[k]);
    return cudaEventRecord(ctx->ev[k], st);
}

static size_t small_bytes(int64_t n)
{
    return std::max(sizeof(int32_t) * (size_t)small_capacity(n), sizeof(PointRec) * (size_t)n);
}

static int ensure(hrg_ctx *ctx, int slot, size_t bytes, void **out)
{
    DevBuf &b = ctx->ws[slot];
    if (bytes == 0) bytes = 16;
    if (b.bytes < bytes) {
        if (b.ptr) cudaFree(b.ptr);
        b.ptr = nullptr;
        b.bytes = 0;
        size_t want = bytes + bytes / 8;  // grow with some slack
        if (ctx->lim.workspace_bytes > 0) {  // the caller's cap on the whole workspace
            size_t held = 0;
            for (const auto &o : ctx->ws) held += o.bytes;
            const size_t cap = (size_t)ctx->lim.workspace_bytes;
            if (held + bytes > cap)
                return set_err(ctx, HRG_ENOMEM, "workspace of %zu bytes would exceed its cap of %zu", held + bytes,
                               cap);
            if (held + want > cap) want = bytes;
        }
        cudaError_t e = cudaMalloc(&b.ptr, want);
        if (e != cudaSuccess) {
            cudaGetLastError();
            e = cudaMalloc(&b.ptr, bytes);
            if (e != cudaSuccess) {
                cudaGetLastError();
                b.ptr = nullptr;
                return set_err(ctx, HRG_ENOMEM, "device allocation of %zu bytes failed", bytes);
            }
            b.bytes = bytes;
        } else {
            b.bytes = want;
        }
    }
    *out = b.ptr;
    return HRG_OK;
}

extern "C" int hrg_create(hrg_ctx **out, int device)
{
    if (!out) return HRG_EINVAL;
    *out = nullptr;
    hrg_ctx *ctx = new hrg_ctx();
    ctx->device = device;
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) {
        delete ctx;
        return HRG_ECUDA;
    }
    e = upload_log_table();
    if (e != cudaSuccess) {
        delete ctx;
        return HRG_ECUDA;
    }
    e = cudaMallocHost(&ctx->pinned, 4096);
    if (e != cudaSuccess) {
        delete ctx;
        return HRG_ENOMEM;
    }
    for (auto &ev : ctx->ev) {
        if (cudaEventCreate(&ev) != cudaSuccess) {
            cudaFreeHost(ctx->pinned);
            delete ctx;
            return HRG_ECUDA;
        }
    }
    *out = ctx;
    return HRG_OK;
}

extern "C" int hrg_destroy(hrg_ctx *ctx)
{
    if (!ctx) return HRG_EINVAL;
    cudaSetDevice(ctx->device);
    for (auto &b : ctx->ws)
        if (b.ptr) cudaFree(b.ptr);
    if (ctx->pinned) cudaFreeHost(ctx->pinned);
    if (ctx->work) cudaStreamDestroy(ctx->work);
    if (ctx->copy) cudaStreamDestroy(ctx->copy);
    for (auto &ev : ctx->ev)
        if (ev) cudaEventDestroy(ev);
    for (auto &ev : ctx->hev)
        if (ev) cudaEventDestroy(ev);
    delete ctx;
    return HRG_OK;
}

extern "C" int hrg_workspace_bytes(const hrg_ctx *ctx, int64_t *bytes)
{
    if (!ctx || !bytes) return HRG_EINVAL;
    int64_t t = 0;
    for (const auto &b : ctx->ws) t += (int64_t)b.bytes;
    *bytes = t;
    return HRG_OK;
}

extern "C" int hrg_release_workspace(hrg_ctx *ctx)
{
    if (!ctx) return HRG_EINVAL;
    if (ctx->job.open) return set_err(ctx, HRG_ESTATE, "a job of this context is still open");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return set_err(ctx, HRG_ECUDA, "cudaSetDevice failed");
    for (auto &b : ctx->ws) {
        if (b.ptr) cudaFree(b.ptr);
        b.ptr = nullptr;
        b.bytes = 0;
    }
    return HRG_OK;
}

extern "C" int hrg_set_limits(hrg_ctx *ctx, const hrg_limits *lim)
{
    if (!ctx) return HRG_EINVAL;
    if (ctx->job.open) return set_err(ctx, HRG_ESTATE, "a job of this context is still open");
    hrg_limits l{};
    if (lim) l = *lim;
    if (l.row_buffer_ids < 0 || l.hub_pool_ids < 0 || l.hub_pool_ids >= (1LL << 40) || l.hub_runs < 0 ||
        l.hub_runs >= (1 << 24) || l.heavy_segments < 0 || l.workspace_bytes < 0)
        return set_err(ctx, HRG_EINVAL, "limits out of range");
    ctx->lim = l;
    return HRG_OK;
}

extern "C" const char *hrg_last_error(const hrg_ctx *ctx)
{
    if (!ctx) return "null context";
    return ctx->err.c_str();
}

// ---------------------------------------------------------------------------
// Plan.
// ---------------------------------------------------------------------------
static float f32(double x) { return (float)x; }

// Band layout before the band counts are known.
static void plan_bands(Plan &p, int64_t n, double R, double alpha, int bands)
{
    memset(&p, 0, sizeof p);
    p.n = n;
    p.R = R;
    p.coshR = std::cosh(R);
    p.alpha = alpha;
    p.big = std::cosh(alpha * R) - 1.0;
    p.big53 = std::ldexp(p.big, -53);
    p.inv_alpha = 1.0 / alpha;
    p.half_R = 0.5 * R;
    p.half_R_hi = (float)p.half_R;
    p.half_R_lo = (float)(p.half_R - (double)p.half_R_hi);
    int B = bands > 0 ? bands : (int)std::ceil(R / 1.7);
    if (B < 1) B = 1;
    if (B > HRG_MAX_BANDS) B = HRG_MAX_BANDS;
    p.B = B;
    p.inv_width = (double)B / R;
    for (int k = 0; k < B; ++k) p.band_lo[k] = R * (double)k / (double)B;
    p.band_lo[B] = INFINITY;
    for (int k = 0; k < B; ++k) {
        const double b = p.band_lo[k];
        p.Pb[k] = f32(std::exp(b - 0.5 * R));
        p.Mb[k] = f32(std::exp(-b - 0.5 * R));
        p.Sb[k] = f32(2.0 * std::exp(-0.5 * R) * std::sinh(b));
    }
    p.rhs64 = 1.0 + std::exp(-2.0 * R);
    p.rhs32 = f32(p.rhs64);
    const double tie_lo = p.rhs64 - 1e-12 * p.rhs64, tie_hi = p.rhs64 + 1e-12 * p.rhs64;
    memcpy(&p.tie_lo, &tie_lo, 8);
    memcpy(&p.tie_hi, &tie_hi, 8);
    // Undecided band of the FP32 filter, relative to 1 + e^{-2R}.  The FP32
    // value P_a M_b + P_b M_a + S_a S_b s^2 has non-negative terms, each
    // within ~30 u (u = 2^-24) of its exact value: P, M within 3 u, S within
    // 5 u, s = sin(dphi/2) within ~7 u (dA pi / 2^64 within 3 ulp, the sine's
    // series and its evaluation), a few roundings; so the sum is within
    // ~2e-6 relative.  The fixed-point angle difference dA is within 2^13
    // units (2.8e-15 rad) of the FP64 angles' difference; that moves the
    // third term by S_a S_b |dphi| 1.4e-15, and with S_a S_b dphi^2 / 4 <= 1
    // near the threshold and S <= e^{R/2}, by at most 2.8e-15 e^{R/2}.  mu
    // takes 2e-4 (100 times the first) plus 8e-15 e^{R/2} (almost 3 times the
    // second); pairs outside [1 - mu, 1 + mu] are then decided as the exact
    // predicate decides them, those inside are decided again in FP64.
    p.mu = f32(2e-4 + 8e-15 * std::exp(0.5 * R));
}

// Angular buckets and hub bands once the band counts are known.
static void plan_buckets(Plan &p, const int64_t *cnt, int32_t *p_hub, double hub_cand)
{
    // 2^sbits angular sectors of about 1024 points each; every band gets at
    // least one bucket per sector so sectors are bucket-aligned in each band
    int sb = 0;
    while (sb < 20 && ((int64_t)1024 << (sb + 1)) <= p.n) ++sb;
    p.sbits = sb;
    int64_t G = 0;
    for (int k = 0; k < p.B; ++k) {
        // about one point per bucket; twice as many buckets in bands of more
        // than 2^16 points, where a rim window's bucket range then carries
        // fewer points outside the window (the candidates the window test rejects)
        int g = 0;
        while (g < 40 && ((int64_t)1 << (g + 1)) <= cnt[k]) ++g;
        if (cnt[k] > ((int64_t)1 << 16)) ++g;
        if (g < sb) g = sb;
        p.gbits[k] = g;
        p.base[k] = G;
        G += (int64_t)1 << g;
    }
    p.base[p.B] = G;
    p.G = G;
    // hub bands: expected candidates of a query at the band's inner radius
    // above hub_cand (sum over bands of count * window / pi)
    int hub = 0;
    for (int i = 0; i < p.B; ++i) {
        const double rq = p.band_lo[i];
        double cand = 0.0;
        for (int j = 0; j < p.B; ++j) {
            const double b = p.band_lo[j];
            double frac;
            if (rq + b <= p.R || rq == 0.0 || b == 0.0) frac = 1.0;
            else {
                double x = (p.coshR - std::cosh(rq - b)) / (2.0 * std::sinh(rq) * std::sinh(b));
                x = std::min(1.0, std::max(0.0, x));
                frac = 2.0 * std::asin(std::sqrt(x)) / 3.141592653589793;
            }
            cand += frac * (double)cnt[j];
        }
        if (cand > hub_cand) hub = i + 1; else break;
    }
    p.hub_bands = hub;
    int64_t ph = 0;
    for (int k = 0; k < hub; ++k) ph += cnt[k];
    *p_hub = (int32_t)ph;
}

// Degree count and row offsets over the structure in J.qb (A, pms, pms64,
// start and, for batches, the batch tables already set): positions and
// global ids [0, n).
static int count_and_offsets(hrg_ctx *ctx, hrg_job &J, int64_t n, cudaStream_t st, int64_t *row_off_out,
                             int64_t *n_entries)
{
    QueryBufs &b = J.qb;
    void *deg, *stats, *lists[3], *listcnt, *bigtot, *scanws;
    int rc;
    if ((rc = ensure(ctx, hrg_ctx::W_DEG, sizeof(int32_t) * n, &deg))) return rc;
    if ((rc = ensure(ctx, hrg_ctx::W_STATS, sizeof(uint64_t) * 8, &stats))) return rc;
    for (int k = 0; k < 3; ++k)
        if ((rc = ensure(ctx, hrg_ctx::W_LIST0 + k, sizeof(int32_t) * n, &lists[k]))) return rc;
    if ((rc = ensure(ctx, hrg_ctx::W_LISTCNT, sizeof(int32_t) * 16, &listcnt))) return rc;
    if ((rc = ensure(ctx, hrg_ctx::W_BIGTOT, sizeof(int64_t), &bigtot))) return rc;
    if ((rc = ensure(ctx, hrg_ctx::W_SCAN, scan_workspace_bytes(n), &scanws))) return rc;
    void *relist[4];
    for (int k = 0; k < 4; ++k)
        if ((rc = ensure(ctx, hrg_ctx::W_RELIST0 + k, sizeof(int32_t) * n, &relist[k]))) return rc;
    const Plan &p = J.plan;
    b.r = J.r;
    b.phi = J.phi;
    b.deg = (int32_t *)deg;
    b.stats = (unsigned long long *)stats;
    for (int k = 0; k < 3; ++k) b.rows[k] = (int32_t *)lists[k];
    b.list_cnt = (int32_t *)listcnt;
    for (int k = 0; k < 4; ++k) b.relist[k] = (int32_t *)relist[k];
    b.big_total = (int64_t *)bigtot;
    // heavy hub segments (long hub ranges cut into CTA chunks) and hub row cursors
    void *heavy = nullptr, *cursor = nullptr, *wcnt = nullptr, *scnt = nullptr;
    int64_t heavy_cap = ctx->lim.heavy_segments > 0 ? ctx->lim.heavy_segments : std::max<int64_t>(1 << 16, n / 64);
    if (J.p_hub > 0) {
        if ((rc = ensure(ctx, hrg_ctx::W_CURSOR, sizeof(int32_t) * J.p_hub, &cursor))) return rc;
        if ((rc = ensure(ctx, hrg_ctx::W_WARPCNT, sizeof(int32_t) * J.p_hub, &wcnt))) return rc;
    }
    b.cursor = (int32_t *)cursor;
    b.warp_cnt = (int32_t *)wcnt;
    // rim rows of up to kKeepRow entries kept by the count pass (room for 32
    // entries per vertex, below 2^31 in all; rows that find none are
    // traversed again)
    void *small = nullptr, *small_off = nullptr, *small_cur = nullptr;
    const int64_t small_cap =
        ctx->lim.row_buffer_ids > 0 ? std::min(ctx->lim.row_buffer_ids, small_capacity(n)) : small_capacity(n);
    if ((rc = ensure(ctx, hrg_ctx::W_SMALL, small_bytes(n), &small))) return rc;
    if ((rc = ensure(ctx, hrg_ctx::W_SMALLOFF, sizeof(int32_t) * n, &small_off))) return rc;
    if ((rc = ensure(ctx, hrg_ctx::W_SMALLCUR, sizeof(unsigned long long), &small_cur))) return rc;
    b.small = (int32_t *)small;
    b.small_off = (int32_t *)small_off;
    b.small_cursor = (unsigned long long *)small_cur;
    b.small_cap = small_cap;

    // the hub rows' ids, kept by the count pass in runs (room for 8 per vertex:
    // on overflow the write pass traverses the hub rows again instead)
    void *pool = nullptr, *runs = nullptr, *pool_cur = nullptr;
    const int64_t pool_cap = ctx->lim.hub_pool_ids > 0 ? ctx->lim.hub_pool_ids : 8 * n + (1 << 24);
    if (J.p_hub > 0) {
        if ((rc = ensure(ctx, hrg_ctx::W_HPOOL, sizeof(int32_t) * pool_cap, &pool))) return rc;
        if ((rc = ensure(ctx, hrg_ctx::W_HPCUR, sizeof(unsigned long long), &pool_cur))) return rc;
    }
    char *hp = (char *)ctx->pinned;
    for (int attempt = 0;; ++attempt) {
        if ((rc = ensure(ctx, hrg_ctx::W_HEAVY, sizeof(int4) * heavy_cap, &heavy))) return rc;
        if ((rc = ensure(ctx, hrg_ctx::W_SEGCNT, sizeof(int32_t) * heavy_cap, &scnt))) return rc;
        b.heavy = (int4 *)heavy;
        b.seg_cnt = (int32_t *)scnt;
        b.heavy_cap = (int32_t)heavy_cap;
        // a warp's runs hold at least 1024 - 64 ids, except its last one and one per heavy chunk
        const int64_t run_cap = ctx->lim.hub_runs > 0
                                    ? ctx->lim.hub_runs
                                    : std::min<int64_t>(pool_cap / 512 + J.p_hub + heavy_cap + 1024, (1 << 24) - 1);
        if (J.p_hub > 0) {
            if ((rc = ensure(ctx, hrg_ctx::W_HRUNS, sizeof(int4) * run_cap, &runs))) return rc;
            CK(cudaMemsetAsync(pool_cur, 0, sizeof(unsigned long long), st));
        }
        b.pool = (int32_t *)pool;
        b.runs = (int4 *)runs;
        b.pool_cur = (unsigned long long *)pool_cur;
        b.pool_cap = pool_cap;
        b.run_cap = (int32_t)run_cap;
        CK(cudaMemsetAsync(stats, 0, sizeof(uint64_t) * 8, st));
        CK(cudaMemsetAsync(listcnt, 0, sizeof(int32_t) * 16, st));
        CK(cudaMemsetAsync(bigtot, 0, sizeof(int64_t), st));
        CK(cudaMemsetAsync(deg, 0, sizeof(int32_t) * n, st));
        CK(cudaMemsetAsync(small_cur, 0, sizeof(unsigned long long), st));
        CK(cudaMemsetAsync(small_off, 0xFF, sizeof(int32_t) * n, st));  // -1: no kept row (hub positions too)
        CK(launch_count_hub(p, b, J.fp64, J.p_hub, st));
        CK(stage_mark(ctx, 3, st));
        CK(launch_count_rim(p, b, J.fp64, st));
        CK(stage_mark(ctx, 4, st));

        // 4. row offsets; the totals, the list lengths (the heavy hub
        // segments among them) and the counters come back together
        CK(scan_i32_to_i64((int32_t *)deg, row_off_out, n, scanws, st));
        CK(stage_mark(ctx, 5, st));
        CK(cudaMemcpyAsync(hp + 0, row_off_out + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(hp + 8, listcnt, sizeof(int32_t) * 4, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(hp + 24, bigtot, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(hp + 64, stats, sizeof(uint64_t) * 8, cudaMemcpyDeviceToHost, st));
        if (pool_cur) CK(cudaMemcpyAsync(hp + 128, pool_cur, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        J.hub_pooled = false;
        J.hub_runs = 0;
        if (pool_cur) {
            uint64_t pc;
            memcpy(&pc, hp + 128, 8);
            const uint64_t entries = pc & ((1ull << 40) - 1), nruns = pc >> 40;
            J.hub_pooled = entries <= (uint64_t)pool_cap && nruns <= (uint64_t)b.run_cap;
            J.hub_runs = J.hub_pooled ? (int32_t)nruns : 0;
        }
        int32_t heavy_found;
        memcpy(&heavy_found, hp + 8 + 12, 4);
        if (J.p_hub == 0 || heavy_found <= heavy_cap) break;
        // the heavy hub segments did not fit: the degrees are incomplete, so
        // grow the list and count again
        if (attempt > 0 || heavy_found > (1 << 30)) return set_err(ctx, HRG_EINTERNAL, "heavy segment list overflow");
        heavy_cap = (int64_t)heavy_found + heavy_found / 8 + 1024;
        J.heavy_retries = attempt + 1;
    }
    memcpy(&J.n_entries, hp + 0, 8);
    memcpy(J.lists, hp + 8, 12);
    memcpy(&J.big_total, hp + 24, 8);
    memcpy(J.stats, hp + 64, 64);
    J.open = true;
    *n_entries = J.n_entries;
    return HRG_OK;
}

static void expected_band_counts(const Plan &p, int64_t *cnt)
{
    // radial CDF of Eq. (1): F(r) = (cosh(alpha r) - 1) / (cosh(alpha R) - 1)
    double prev = 0.0;
    for (int k = 0; k < p.B; ++k) {
        const double hi = (k + 1 < p.B) ? (std::cosh(p.alpha * p.band_lo[k + 1]) - 1.0) / p.big : 1.0;
        cnt[k] = (int64_t)std::llround((double)p.n * std::max(0.0, hi - prev));
        prev = hi;
    }
}

// hrg_generate_host: the sampled points go back to these host buffers on
// the copy stream as soon as the sampler has written them.
struct HostPoints {
    double *r_host, *phi_host;
    cudaStream_t copy;
    cudaEvent_t sampled, copy_start;
};

static int begin_common(hrg_ctx *ctx, hrg_job &J, bool sampled, const hrg_params *prm, int64_t n, double R,
                        double alpha, const double *r_in, const double *phi_in, double *r_out, double *phi_out,
                        uint32_t flags, int32_t bands, cudaStream_t st, int64_t *row_off_out, int64_t *n_entries,
                        bool count_pass = true, const HostPoints *hpts = nullptr)
{
    if (cudaSetDevice(ctx->device) != cudaSuccess) return set_err(ctx, HRG_ECUDA, "cudaSetDevice failed");
    J = hrg_job();
    J.ctx = ctx;
    J.stream = st;
    J.fp64 = (flags & HRG_FLAG_FP64_ONLY) != 0 || R > 80.0;
    J.sampled = sampled;
    J.row_off = row_off_out;
    Plan &p = J.plan;
    plan_bands(p, n, R, alpha, bands);

    void *band_cnt, *gbuf, *slot, *A, *pms, *pms64 = nullptr, *scanws, *pos_of;
    int rc;
    if ((rc = ensure(ctx, hrg_ctx::W_BANDCNT, sizeof(int64_t) * HRG_MAX_BANDS, &band_cnt))) return rc;
    if ((rc = ensure(ctx, hrg_ctx::W_POSOF, sizeof(int32_t) * n, &pos_of))) return rc;
    if ((rc = ensure(ctx, hrg_ctx::W_GBUF, sizeof(int32_t) * n, &gbuf))) return rc;
    if ((rc = ensure(ctx, hrg_ctx::W_SLOT, sizeof(int32_t) * n, &slot))) return rc;
    if ((rc = ensure(ctx, hrg_ctx::W_A, sizeof(uint64_t) * n, &A))) return rc;
    if ((rc = ensure(ctx, hrg_ctx::W_PMS, sizeof(PMS) * n, &pms))) return rc;
    if (J.fp64 && (rc = ensure(ctx, hrg_ctx::W_PMS64, sizeof(PMS64) * n, &pms64))) return rc;

    // 1. points and their (band, angular bucket).  A sampled graph's bucket
    // layout is planned from the expected band counts (Eq. (1)) and filled by
    // the sampler itself; an injected point set's from its actual counts.
    const double hub_cand = (prm && prm->hub_candidates > 0) ? (double)prm->hub_candidates : 512.0;
    int64_t cnt_copy[HRG_MAX_BANDS];
    int64_t *h_cnt = (int64_t *)ctx->pinned;
    void *cnt = nullptr, *start = nullptr;
    scanws = nullptr;
    // bucket occupancy and start tables once the layout is known
    auto bucket_tables = [&]() -> int {
        plan_buckets(p, cnt_copy, &J.p_hub, hub_cand);
        const size_t scan_bytes = std::max(scan_workspace_bytes(p.G), scan_workspace_bytes(n));
        int e;
        if ((e = ensure(ctx, hrg_ctx::W_CNT, sizeof(int32_t) * p.G, &cnt))) return e;
        if ((e = ensure(ctx, hrg_ctx::W_START, sizeof(int32_t) * (p.G + 1), &start))) return e;
        if ((e = ensure(ctx, hrg_ctx::W_SCAN, scan_bytes, &scanws))) return e;
        return HRG_OK;
    };
    CK(stage_mark(ctx, 0, st));
    CK(cudaMemsetAsync(band_cnt, 0, sizeof(int64_t) * HRG_MAX_BANDS, st));
    if (sampled) {
        expected_band_counts(p, cnt_copy);
        if ((rc = bucket_tables())) return rc;
        CK(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * p.G, st));
        CK(launch_sample_bucket(p, prm->seed, r_out, phi_out, (int32_t *)gbuf, (int32_t *)slot, (int32_t *)cnt,
                                (int64_t *)band_cnt, st));
        J.r = r_out;
        J.phi = phi_out;
        CK(stage_mark(ctx, 1, st));
        if (hpts) {
            CK(cudaEventRecord(hpts->sampled, st));
            CK(cudaStreamWaitEvent(hpts->copy, hpts->sampled, 0));
            CK(cudaEventRecord(hpts->copy_start, hpts->copy));
            CK(cudaMemcpyAsync(hpts->r_host, r_out, sizeof(double) * n, cudaMemcpyDeviceToHost, hpts->copy));
            CK(cudaMemcpyAsync(hpts->phi_host, phi_out, sizeof(double) * n, cudaMemcpyDeviceToHost, hpts->copy));
        }
        CK(cudaMemcpyAsync(h_cnt, band_cnt, sizeof(int64_t) * p.B, cudaMemcpyDeviceToHost, st));
    } else {
        CK(launch_count_bands(p, r_in, phi_in, (int64_t *)band_cnt, st));
        J.r = r_in;
        J.phi = phi_in;
        CK(cudaMemcpyAsync(h_cnt, band_cnt, sizeof(int64_t) * p.B, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        memcpy(cnt_copy, h_cnt, sizeof(int64_t) * p.B);
        CK(stage_mark(ctx, 1, st));
        if ((rc = bucket_tables())) return rc;
        CK(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * p.G, st));
        CK(launch_bucket_hist(p, J.r, J.phi, (int32_t *)gbuf, (int32_t *)slot, (int32_t *)cnt, st));
    }

    // 2. counting sort by (band, angular bucket)
    CK(scan_i32_to_i32((int32_t *)cnt, (int32_t *)start, p.G, scanws, st));
    void *recs = nullptr;  // the FP32 path's point records (in the kept-row buffer, idle until the count pass)
    if (!pms64 && (rc = ensure(ctx, hrg_ctx::W_SMALL, small_bytes(n), &recs))) return rc;
    CK(launch_scatter_soa(p, (int32_t *)gbuf, (int32_t *)slot, (int32_t *)start, J.r, J.phi, (PointRec *)recs,
                          (uint64_t *)A, (PMS *)pms, (PMS64 *)pms64, (int32_t *)pos_of, st));
    CK(stage_mark(ctx, 2, st));
    // the exact band counts (read back behind the scan and the scatter): hub
    // queries and empty innermost bands
    if (sampled) {
        CK(cudaStreamSynchronize(st));
        memcpy(cnt_copy, h_cnt, sizeof(int64_t) * p.B);
    }
    J.p_hub = 0;
    for (int k = 0; k < p.hub_bands; ++k) J.p_hub += (int32_t)cnt_copy[k];
    while (p.first_band < p.B - 1 && cnt_copy[p.first_band] == 0) ++p.first_band;

    // 3. degrees, 4. row offsets
    QueryBufs &b = J.qb;
    b = QueryBufs{};
    b.A = (uint64_t *)A;
    b.pms = (PMS *)pms;
    b.pms64 = (PMS64 *)pms64;
    b.start = (int32_t *)start;
    b.pos_of = (int32_t *)pos_of;
    if (!count_pass) return HRG_OK;  // the band structure only (vertex movement)
    return count_and_offsets(ctx, J, n, st, row_off_out, n_entries);
}

static int check_params(hrg_ctx *ctx, const hrg_params *p, double *R)
{
    if (!p) return set_err(ctx, HRG_EINVAL, "null params");
    if (p->n < 2 || p->n > 0x7fffffffLL) return set_err(ctx, HRG_EINVAL, "n must be in [2, 2^31)");
    if (!(p->alpha > 0.5)) return set_err(ctx, HRG_EINVAL, "alpha must exceed 1/2");
    if (p->bands < 0 || p->bands > HRG_MAX_BANDS) return set_err(ctx, HRG_EINVAL, "bands must be in [0, 64]");
    if (p->R_override > 0.0) {
        *R = p->R_override;
        return HRG_OK;
    }
    if (hrg_solve_radius(p->n, p->alpha, p->avg_degree, R) != HRG_OK)
        return set_err(ctx, HRG_EINVAL, "no radius for n=%lld alpha=%g avg_degree=%g (Eq. (22))",
                       (long long)p->n, p->alpha, p->avg_degree);
    return HRG_OK;
}

static int generate_begin(hrg_ctx *ctx, const hrg_params *p, void *stream, double *r_out, double *phi_out,
                          int64_t *row_off_out, hrg_job **job, int64_t *n_entries, const HostPoints *hpts)
{
    if (!ctx) return HRG_EINVAL;
    if (!job || !n_entries || !r_out || !phi_out || !row_off_out) return set_err(ctx, HRG_EINVAL, "null argument");
    if (ctx->job.open) return set_err(ctx, HRG_ESTATE, "a job of this context is still open");
    double R;
    int rc = check_params(ctx, p, &R);
    if (rc) return rc;
    rc = begin_common(ctx, ctx->job, true, p, p->n, R, p->alpha, nullptr, nullptr, r_out, phi_out, p->flags,
                      p->bands, (cudaStream_t)stream, row_off_out, n_entries, true, hpts);
    if (rc) {
        ctx->job.open = false;
        return rc;
    }
    *job = &ctx->job;
    return HRG_OK;
}

extern "C" int hrg_generate_begin(hrg_ctx *ctx, const hrg_params *p, void *stream, double *r_out, double *phi_out,
                                  int64_t *row_off_out, hrg_job **job, int64_t *n_entries)
{
    return generate_begin(ctx, p, stream, r_out, phi_out, row_off_out, job, n_entries, nullptr);
}

extern "C" int hrg_generate_from_points_begin(hrg_ctx *ctx, int64_t n, double R, const double *r, const double *phi,
                                              uint32_t flags, int32_t bands, void *stream, int64_t *row_off_out,
                                              hrg_job **job, int64_t *n_entries)
{
    if (!ctx) return HRG_EINVAL;
    if (!job || !n_entries || !r || !phi || !row_off_out) return set_err(ctx, HRG_EINVAL, "null argument");
    if (ctx->job.open) return set_err(ctx, HRG_ESTATE, "a job of this context is still open");
    if (n < 1 || n > 0x7fffffffLL) return set_err(ctx, HRG_EINVAL, "n must be in [1, 2^31)");
    if (!(R > 0.0) || !std::isfinite(R)) return set_err(ctx, HRG_EINVAL, "R must be positive and finite");
    if (bands < 0 || bands > HRG_MAX_BANDS) return set_err(ctx, HRG_EINVAL, "bands must be in [0, 64]");
    int rc = begin_common(ctx, ctx->job, false, nullptr, n, R, 1.0, r, phi, nullptr, nullptr, flags, bands,
                          (cudaStream_t)stream, row_off_out, n_entries);
    if (rc) {
        ctx->job.open = false;
        return rc;
    }
    *job = &ctx->job;
    return HRG_OK;
}

// ---------------------------------------------------------------------------
// Batches: many independent graphs through one pass of every stage.  Graph g
// owns positions, global ids and CSR rows [off_g, off_g + n_g) with off the
// prefix sum of the n's; its buckets follow those of graph g-1.  The band
// layout of each graph is planned from the expected band counts of Eq. (1)
// (n times the radial CDF mass of the band), so planning needs no read-back.
// ---------------------------------------------------------------------------
extern "C" int hrg_generate_batch_begin(hrg_ctx *ctx, int32_t count, const hrg_params *items, uint32_t flags,
                                        void *stream, double *r_out, double *phi_out, int64_t *row_off_out,
                                        hrg_job **job, int64_t *n_entries)
{
    if (!ctx) return HRG_EINVAL;
    if (!items || !job || !n_entries || !r_out || !phi_out || !row_off_out)
        return set_err(ctx, HRG_EINVAL, "null argument");
    if (count < 1 || count > (1 << 24)) return set_err(ctx, HRG_EINVAL, "count must be in [1, 2^24]");
    if (ctx->job.open) return set_err(ctx, HRG_ESTATE, "a job of this context is still open");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return set_err(ctx, HRG_ECUDA, "cudaSetDevice failed");
    cudaStream_t st = (cudaStream_t)stream;
    hrg_job &J = ctx->job;
    J = hrg_job();
    J.ctx = ctx;
    J.stream = st;
    J.row_off = row_off_out;
    J.batch = count;

    // plans on the host
    std::vector<Plan> &plans = ctx->batch_plans;
    std::vector<int64_t> &noff = ctx->batch_noff, &soff = ctx->batch_soff;
    plans.resize(count);
    noff.assign(count + 1, 0);
    soff.assign(count + 1, 0);
    // each graph's own plan, in parallel over host threads (the radius solve
    // and the band layout are independent per graph)
    std::vector<double> radius(count, 0.0);
    std::vector<char> bad(count, 0);
    auto plan_range = [&](int32_t g0, int32_t g1) {
        for (int32_t g = g0; g < g1; ++g) {
            const hrg_params &it = items[g];
            double R = it.R_override;
            if (it.n < 2 || it.n > 0x7fffffffLL || !(it.alpha > 0.5) || it.bands < 0 || it.bands > HRG_MAX_BANDS ||
                (!(R > 0.0) && hrg_solve_radius(it.n, it.alpha, it.avg_degree, &R) != HRG_OK)) {
                bad[g] = 1;
                continue;
            }
            radius[g] = R;
            Plan &p = plans[g];
            plan_bands(p, it.n, R, it.alpha, it.bands);
            int64_t cnt[HRG_MAX_BANDS];
            expected_band_counts(p, cnt);
            int32_t ph = 0;
            plan_buckets(p, cnt, &ph, it.hub_candidates > 0 ? (double)it.hub_candidates : 512.0);
        }
    };
    const int nt = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)std::thread::hardware_concurrency(), 32,
                                                                 (int64_t)count / 64 + 1}));
    if (nt == 1) {
        plan_range(0, count);
    } else {
        std::vector<std::thread> pool;
        for (int t = 0; t < nt; ++t)
            pool.emplace_back(plan_range, (int32_t)((int64_t)count * t / nt), (int32_t)((int64_t)count * (t + 1) / nt));
        for (auto &th : pool) th.join();
    }
    // the batch layout, in order
    int64_t N = 0, G = 0, S = 0;
    bool fp64 = (flags & HRG_FLAG_FP64_ONLY) != 0;
    for (int32_t g = 0; g < count; ++g) {
        if (bad[g]) {
            double R;
            const int rc = check_params(ctx, &items[g], &R);
            return set_err(ctx, rc ? rc : HRG_EINVAL, "item %d: %s", g, ctx->err.c_str());
        }
        fp64 = fp64 || radius[g] > 80.0;
        Plan &p = plans[g];
        noff[g] = N;
        soff[g] = S;
        p.id_off = (int32_t)N;
        p.seed = items[g].seed;
        for (int k = 0; k <= p.B; ++k) p.base[k] += G;
        N += p.n;
        G += p.G;
        if (p.hub_bands < p.B) S += (int64_t)1 << p.sbits;
        if (N > 0x7fffffffLL || G > 0x7fffffffLL) return set_err(ctx, HRG_EINVAL, "batch larger than 2^31 points");
    }
    noff[count] = N;
    soff[count] = S;
    J.fp64 = fp64;
    J.plan = plans[0];
    J.plan.n = N;
    J.batch_G = G;

    // device tables
    void *d_plans, *d_noff, *d_soff, *graph_of, *gbuf, *slot, *A, *pms, *pms64 = nullptr, *cnt, *start, *scanws, *pos_of;
    void *hub_cnt, *hub_off, *hub_pos = nullptr;
    int rc;
    if ((rc = ensure(ctx, hrg_ctx::W_PLANS, sizeof(Plan) * count, &d_plans))) return rc;
    if ((rc = ensure(ctx, hrg_ctx::W_NOFF, sizeof(int64_t) * (count + 1), &d_noff))) return rc;
    if ((rc = ensure(ctx, hrg_ctx::W_SOFF, sizeof(int64_t) * (count + 1), &d_soff))) return rc;
    if ((rc = ensure(ctx, hrg_ctx::W_GRAPHOF, sizeof(int32_t) * N, &graph_of))) return rc;
    if ((rc = ensure(ctx, hrg_ctx::W_POSOF, sizeof(int32_t) * N, &pos_of))) return rc;
    if ((rc = ensure(ctx, hrg_ctx::W_GBUF, sizeof(int32_t) * N, &gbuf))) return rc;
    if ((rc = ensure(ctx, hrg_ctx::W_SLOT, sizeof(int32_t) * N, &slot))) return rc;
    if ((rc = ensure(ctx, hrg_ctx::W_A, sizeof(uint64_t) * N, &A))) return rc;
    if ((rc = ensure(ctx, hrg_ctx::W_PMS, sizeof(PMS) * N, &pms))) return rc;
    if (fp64 && (rc = ensure(ctx, hrg_ctx::W_PMS64, sizeof(PMS64) * N, &pms64))) return rc;
    if ((rc = ensure(ctx, hrg_ctx::W_CNT, sizeof(int32_t) * G, &cnt))) return rc;
    if ((rc = ensure(ctx, hrg_ctx::W_START, sizeof(int32_t) * (G + 1), &start))) return rc;
    if ((rc = ensure(ctx, hrg_ctx::W_HUBCNT, sizeof(int32_t) * (count + 1), &hub_cnt))) return rc;
    if ((rc = ensure(ctx, hrg_ctx::W_HUBOFF, sizeof(int32_t) * (count + 1), &hub_off))) return rc;
    const size_t scan_bytes = std::max(std::max(scan_workspace_bytes(G), scan_workspace_bytes(N)),
                                       scan_workspace_bytes(count));
    if ((rc = ensure(ctx, hrg_ctx::W_SCAN, scan_bytes, &scanws))) return rc;
    CK(cudaMemcpyAsync(d_plans, plans.data(), sizeof(Plan) * count, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(d_noff, noff.data(), sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(d_soff, soff.data(), sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice, st));

    // 1. points
    const Plan *P = (const Plan *)d_plans;
    CK(stage_mark(ctx, 0, st));
    CK(launch_graph_of(P, count, (int32_t *)graph_of, st));
    CK(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * G, st));
    CK(launch_sample_bucket_batch(P, (int32_t *)graph_of, N, r_out, phi_out, (int32_t *)gbuf, (int32_t *)slot,
                                  (int32_t *)cnt, st));
    J.r = r_out;
    J.phi = phi_out;
    CK(stage_mark(ctx, 1, st));

    // 2. counting sort by (graph, band, angular bucket); hub query list
    CK(scan_i32_to_i32((int32_t *)cnt, (int32_t *)start, G, scanws, st));
    void *recs = nullptr;  // the FP32 path's point records (in the kept-row buffer, idle until the count pass)
    if (!pms64 && (rc = ensure(ctx, hrg_ctx::W_SMALL, small_bytes(N), &recs))) return rc;
    CK(launch_scatter_soa_batch(P, (int32_t *)graph_of, N, (int32_t *)gbuf, (int32_t *)slot, (int32_t *)start, r_out,
                                phi_out, (PointRec *)recs, (uint64_t *)A, (PMS *)pms, (PMS64 *)pms64,
                                (int32_t *)pos_of, st));
    CK(launch_hub_list(P, count, (int32_t *)start, (int32_t *)hub_cnt, (int32_t *)hub_off, nullptr, scanws, st,
                       false));
    int32_t *hh = (int32_t *)ctx->pinned;
    CK(cudaMemcpyAsync(hh, (int32_t *)hub_off + count, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    J.p_hub = *hh;
    if (J.p_hub > 0) {
        if ((rc = ensure(ctx, hrg_ctx::W_HUBPOS, sizeof(int32_t) * J.p_hub, &hub_pos))) return rc;
        CK(launch_hub_list(P, count, (int32_t *)start, (int32_t *)hub_cnt, (int32_t *)hub_off, (int32_t *)hub_pos,
                           scanws, st, true));
    }
    CK(stage_mark(ctx, 2, st));

    // 3. degrees, 4. row offsets
    QueryBufs &b = J.qb;
    b = QueryBufs{};
    b.A = (uint64_t *)A;
    b.pms = (PMS *)pms;
    b.pms64 = (PMS64 *)pms64;
    b.start = (int32_t *)start;
    b.pos_of = (int32_t *)pos_of;
    b.plans = P;
    b.graph_of = (int32_t *)graph_of;
    b.sec_off = (int64_t *)d_soff;
    b.hub_pos = (int32_t *)hub_pos;
    b.noff = (int64_t *)d_noff;
    b.NG = count;
    b.n_sectors = S;
    rc = count_and_offsets(ctx, J, N, st, row_off_out, n_entries);
    if (rc) {
        J.open = false;
        return rc;
    }
    *job = &J;
    return HRG_OK;
}

// ---------------------------------------------------------------------------
// Vertex movement (kernels in hrg_update.cu and hrg_query.cu).  Begin: the
// moves checked and applied, the band structure rebuilt from the updated
// points, the moved vertices counted, the removals and gains of the other
// rows counted, new degrees and row offsets.  Finish (update_finish): the
// rows written and the rows written out of order sorted.
// ---------------------------------------------------------------------------
static void job_stage_times(hrg_ctx *ctx, hrg_job *job)
{
    const int pairs[8][2] = {{0, 1}, {1, 2}, {2, 3}, {3, 4}, {4, 5}, {6, 7}, {7, 8}, {8, 9}};
    for (int k = 0; k < 8; ++k) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, ctx->ev[pairs[k][0]], ctx->ev[pairs[k][1]]) != cudaSuccess) {
            cudaGetLastError();
            ms = -1.0f;
        }
        job->stage_ms[k] = ms;
    }
}

extern "C" int hrg_update_begin(hrg_ctx *ctx, int64_t n, double R, double *r, double *phi, const int64_t *row_off,
                                const int32_t *col_idx, int64_t k, const int32_t *ids, const double *r_new,
                                const double *phi_new, uint32_t flags, int32_t bands, void *stream,
                                int64_t *row_off_out, hrg_job **job, int64_t *n_entries)
{
    if (!ctx) return HRG_EINVAL;
    if (!r || !phi || !row_off || !row_off_out || !job || !n_entries) return set_err(ctx, HRG_EINVAL, "null argument");
    if (n < 1 || n > 0x7fffffffLL) return set_err(ctx, HRG_EINVAL, "n must be in [1, 2^31)");
    if (k < 0 || k > n) return set_err(ctx, HRG_EINVAL, "k must be in [0, n]");
    if (k > 0 && (!ids || !r_new || !phi_new)) return set_err(ctx, HRG_EINVAL, "null move arrays");
    if (!(R > 0.0) || !std::isfinite(R)) return set_err(ctx, HRG_EINVAL, "R must be positive and finite");
    if (bands < 0 || bands > HRG_MAX_BANDS) return set_err(ctx, HRG_EINVAL, "bands must be in [0, 64]");
    if (ctx->job.open) return set_err(ctx, HRG_ESTATE, "a job of this context is still open");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return set_err(ctx, HRG_ECUDA, "cudaSetDevice failed");
    cudaStream_t st = (cudaStream_t)stream;
    char *hp = (char *)ctx->pinned;
    CK(cudaMemcpyAsync(hp, row_off, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(hp + 8, row_off + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    int64_t o0, on;
    memcpy(&o0, hp, 8);
    memcpy(&on, hp + 8, 8);
    if (on > o0 && !col_idx) return set_err(ctx, HRG_EINVAL, "null col_idx");

    void *moved, *rem, *gain, *cur, *keep, *err;
    int rc;
    const int64_t words = (n + 31) / 32;
    if ((rc = ensure(ctx, hrg_ctx::W_MVBITS, sizeof(uint32_t) * words, &moved))) return rc;
    if ((rc = ensure(ctx, hrg_ctx::W_MVREM, sizeof(int32_t) * n, &rem))) return rc;
    if ((rc = ensure(ctx, hrg_ctx::W_MVADD, sizeof(int32_t) * n, &gain))) return rc;
    if ((rc = ensure(ctx, hrg_ctx::W_MVCUR, sizeof(int32_t) * n, &cur))) return rc;
    if ((rc = ensure(ctx, hrg_ctx::W_MVKEEP, sizeof(int32_t) * n, &keep))) return rc;
    if ((rc = ensure(ctx, hrg_ctx::W_MVERR, 64, &err))) return rc;
    CK(cudaMemsetAsync(moved, 0, sizeof(uint32_t) * words, st));
    CK(cudaMemsetAsync(err, 0, 64, st));
    // 0. the moves: checked first, so that the points stay as they were on an error
    CK(launch_move_check(n, k, R, ids, r_new, phi_new, (uint32_t *)moved, (int *)err, st));
    CK(cudaMemcpyAsync(hp, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    int bad;
    memcpy(&bad, hp, 4);
    if (bad & 1) return set_err(ctx, HRG_EINVAL, "a moved id outside [0, n) or a coordinate outside [0, R) x [0, 2pi)");
    if (bad & 2) return set_err(ctx, HRG_EINVAL, "a vertex is moved twice");
    CK(launch_move_apply(k, ids, r_new, phi_new, r, phi, st));

    // 1-2. the band structure of the updated points
    hrg_job &J = ctx->job;
    rc = begin_common(ctx, J, false, nullptr, n, R, 1.0, r, phi, nullptr, nullptr, flags, bands, st, row_off_out,
                      n_entries, false);
    if (rc) {
        J.open = false;
        return rc;
    }
    J.update = true;
    J.old_off = row_off;
    J.old_col = col_idx;
    J.moves = k;
    J.move_ids = ids;
    J.moved = (uint32_t *)moved;
    J.rem = (int32_t *)rem;
    J.gain = (int32_t *)gain;
    J.gain_cur = (int32_t *)cur;
    J.keep = (int32_t *)keep;

    // 3. counts: the moved rows, the gains and the removals of the others
    QueryBufs &b = J.qb;
    void *deg, *stats, *lists[3], *listcnt, *bigtot, *scanws;
    if ((rc = ensure(ctx, hrg_ctx::W_DEG, sizeof(int32_t) * n, &deg))) return rc;
    if ((rc = ensure(ctx, hrg_ctx::W_STATS, sizeof(uint64_t) * 8, &stats))) return rc;
    for (int c = 0; c < 3; ++c)
        if ((rc = ensure(ctx, hrg_ctx::W_LIST0 + c, sizeof(int32_t) * n, &lists[c]))) return rc;
    if ((rc = ensure(ctx, hrg_ctx::W_LISTCNT, sizeof(int32_t) * 16, &listcnt))) return rc;
    if ((rc = ensure(ctx, hrg_ctx::W_BIGTOT, sizeof(int64_t), &bigtot))) return rc;
    if ((rc = ensure(ctx, hrg_ctx::W_SCAN, scan_workspace_bytes(n), &scanws))) return rc;
    b.r = r;
    b.phi = phi;
    b.deg = (int32_t *)deg;
    b.stats = (unsigned long long *)stats;
    for (int c = 0; c < 3; ++c) b.rows[c] = (int32_t *)lists[c];
    b.list_cnt = (int32_t *)listcnt;
    b.big_total = (int64_t *)bigtot;
    CK(cudaMemsetAsync(stats, 0, sizeof(uint64_t) * 8, st));
    CK(cudaMemsetAsync(listcnt, 0, sizeof(int32_t) * 16, st));
    CK(cudaMemsetAsync(bigtot, 0, sizeof(int64_t), st));
    CK(cudaMemsetAsync(rem, 0, sizeof(int32_t) * n, st));
    CK(cudaMemsetAsync(gain, 0, sizeof(int32_t) * n, st));
    const Plan &p = J.plan;
    CK(launch_move_query(p, b, J.fp64, false, k, ids, (uint32_t *)moved, (int32_t *)deg, (int32_t *)gain, nullptr,
                         nullptr, nullptr, st));
    CK(stage_mark(ctx, 3, st));
    CK(launch_move_removed(k, ids, row_off, col_idx, (uint32_t *)moved, (int32_t *)rem, st));
    MoveLists ml{{(int32_t *)lists[0], (int32_t *)lists[1], (int32_t *)lists[2]}};
    void *rows_ws;
    if ((rc = ensure(ctx, hrg_ctx::W_MVWS, move_rows_ws_bytes(on - o0), &rows_ws))) return rc;
    CK(launch_move_degrees(n, on - o0, row_off, (uint32_t *)moved, (int32_t *)rem, (int32_t *)gain, (int32_t *)deg,
                           (int32_t *)keep, ml, (int32_t *)listcnt, (unsigned long long *)bigtot, rows_ws, st));
    CK(stage_mark(ctx, 4, st));
    // 4. row offsets
    CK(scan_i32_to_i64((int32_t *)deg, row_off_out, n, scanws, st));
    CK(stage_mark(ctx, 5, st));
    CK(cudaMemcpyAsync(hp + 0, row_off_out + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(hp + 8, listcnt, sizeof(int32_t) * 4, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(hp + 24, bigtot, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(hp + 64, stats, sizeof(uint64_t) * 8, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    memcpy(&J.n_entries, hp + 0, 8);
    memcpy(J.lists, hp + 8, 12);
    memcpy(&J.big_total, hp + 24, 8);
    J.old_entries = on - o0;
    memcpy(J.stats, hp + 64, 64);
    J.open = true;
    *n_entries = J.n_entries;
    *job = &J;
    return HRG_OK;
}

static int update_finish(hrg_job *job, int32_t *col_out)
{
    hrg_ctx *ctx = job->ctx;
    cudaStream_t st = job->stream;
    const Plan &p = job->plan;
    const int64_t n = p.n;
    CK(stage_mark(ctx, 6, st));
    CK(cudaMemsetAsync(job->gain_cur, 0, sizeof(int32_t) * n, st));
    CK(launch_move_query(p, job->qb, job->fp64, true, job->moves, job->move_ids, job->moved, nullptr, job->gain_cur,
                         job->keep, job->row_off, col_out, st));
    CK(stage_mark(ctx, 7, st));
    {
        void *start_drop, *ws;
        int rc;
        if ((rc = ensure(ctx, hrg_ctx::W_MVSTART, sizeof(int32_t) * n, &start_drop))) return rc;
        if ((rc = ensure(ctx, hrg_ctx::W_MVWS, move_rows_ws_bytes(job->old_entries), &ws))) return rc;  // held since begin
        CK(launch_move_rows(n, job->old_entries, job->old_off, job->old_col, job->moved, job->rem,
                            (int32_t *)start_drop, ws, job->row_off, col_out, st));
    }
    CK(stage_mark(ctx, 8, st));
    if (job->lists[0] > 0 || job->lists[1] > 0 || job->lists[2] > 0) {
        void *tmp = nullptr, *bws = nullptr;
        int rc;
        if (job->lists[2] > 0) {
            if ((rc = ensure(ctx, hrg_ctx::W_TMP, sizeof(int32_t) * job->big_total, &tmp))) return rc;
            if ((rc = ensure(ctx, hrg_ctx::W_BUCKET, big_sort_ws_bytes(job->lists[2], job->big_total), &bws)))
                return rc;
        }
        CK(launch_sort_rows(p, job->qb, job->lists, job->big_total, job->row_off, col_out, (int32_t *)tmp, bws, st));
    }
    CK(stage_mark(ctx, 9, st));
    CK(launch_move_check_gains(n, job->gain, job->gain_cur, job->qb.stats + 7, st));
    uint64_t *hs = (uint64_t *)ctx->pinned;
    CK(cudaMemcpyAsync(hs, job->qb.stats + 7, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    job->finished = true;
    job_stage_times(ctx, job);
    if (hs[0] != 0) return set_err(ctx, HRG_EINTERNAL, "count and write passes of the update disagree");
    return HRG_OK;
}

// hrg_generate_host: the neighbour ids go back to this host buffer, range by
// range, on the copy stream.
struct HostCol {
    int32_t *col_host;
    cudaStream_t copy;
};

// Ranges of the chunked write pass: about 2e8 entries each, at most
// kMaxChunks, and none below 2^26 entries in all (a single range then).
static int write_chunks(const hrg_job *job)
{
    if (!job->hub_pooled || job->batch || job->n_entries < ((int64_t)1 << 26)) return 1;
    return (int)std::min<int64_t>(kMaxChunks, std::max<int64_t>(2, job->n_entries / 200000000));
}

static int finish_impl(hrg_job *job, int32_t *col_idx_out, const HostCol *hc)
{
    hrg_ctx *ctx = job->ctx;
    if (job->update) return update_finish(job, col_idx_out);
    cudaStream_t st = job->stream;
    const Plan &p = job->plan;
    const int64_t n = p.n;
    const int K = hc ? write_chunks(job) : 1;
    job->write_chunks = K;
    int rc;
    void *tmp = nullptr, *bws = nullptr;
    if (job->lists[2] > 0) {
        if ((rc = ensure(ctx, hrg_ctx::W_TMP, sizeof(int32_t) * job->big_total, &tmp))) return rc;
        if ((rc = ensure(ctx, hrg_ctx::W_BUCKET, big_sort_ws_bytes(job->lists[2], job->big_total), &bws))) return rc;
    }
    // Range k holds the ids [bounds[k], bounds[k+1]) (multiples of 32) and the
    // entries [offs[k], offs[k+1]); the sort lists are split by range.
    int64_t bounds[kMaxChunks + 1], offs[kMaxChunks + 1];
    int32_t sub_cnt[3 * kMaxChunks] = {};
    int64_t sub_tot[kMaxChunks] = {};
    int32_t *sub = nullptr, *dsub_cnt = nullptr;
    if (K > 1) {
        for (int k = 0; k < K; ++k) bounds[k] = ((n * k / K) >> 5) << 5;
        bounds[K] = n;
        const int64_t lsum = (int64_t)job->lists[0] + job->lists[1] + job->lists[2];
        const size_t b_bounds = 64 * 2, b_cnt = 256, b_tot = 64 * 2;
        void *w;
        if ((rc = ensure(ctx, hrg_ctx::W_CHUNK, b_bounds + b_cnt + b_tot + sizeof(int32_t) * (K * lsum + 1), &w)))
            return rc;
        int64_t *dbounds = (int64_t *)w;
        dsub_cnt = (int32_t *)((char *)w + b_bounds);
        int64_t *dsub_tot = (int64_t *)((char *)w + b_bounds + b_cnt);
        sub = (int32_t *)((char *)w + b_bounds + b_cnt + b_tot);
        char *hp = (char *)ctx->pinned;
        memcpy(hp, bounds, sizeof(int64_t) * (K + 1));
        CK(cudaMemcpyAsync(dbounds, hp, sizeof(int64_t) * (K + 1), cudaMemcpyHostToDevice, st));
        CK(cudaMemsetAsync(dsub_cnt, 0, b_cnt + b_tot, st));
        CK(launch_split_lists(job->qb, job->lists, K, dbounds, job->row_off, sub, dsub_cnt, dsub_tot, st));
        CK(cudaMemcpyAsync(hp + 256, dsub_cnt, sizeof(int32_t) * 3 * K, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(hp + 512, dsub_tot, sizeof(int64_t) * K, cudaMemcpyDeviceToHost, st));
        for (int k = 0; k <= K; ++k)
            CK(cudaMemcpyAsync(hp + 768 + 8 * k, job->row_off + bounds[k], sizeof(int64_t), cudaMemcpyDeviceToHost,
                               st));
        CK(cudaStreamSynchronize(st));
        memcpy(sub_cnt, hp + 256, sizeof(int32_t) * 3 * K);
        memcpy(sub_tot, hp + 512, sizeof(int64_t) * K);
        memcpy(offs, hp + 768, sizeof(int64_t) * (K + 1));
    } else {
        bounds[0] = 0;
        bounds[1] = n;
        offs[0] = 0;
        offs[1] = job->n_entries;
        for (int c = 0; c < 3; ++c) sub_cnt[c] = job->lists[c];
        sub_tot[0] = job->big_total;
    }
    cudaEvent_t *cev = ctx->hev + 3;
    CK(stage_mark(ctx, 6, st));
    if (job->p_hub > 0) CK(cudaMemsetAsync(job->qb.cursor, 0, sizeof(int32_t) * job->p_hub, st));
    for (int k = 0; k < K; ++k) {
        const int64_t lo = bounds[k], hi = bounds[k + 1];
        if (K > 1) CK(cudaEventRecord(cev[4 * k + 0], st));
        if (job->hub_pooled)
            CK(launch_copy_hub(job->qb, job->p_hub, job->hub_runs, job->row_off, col_idx_out, lo, hi, k == K - 1,
                               st));
        else
            CK(launch_write_hub(p, job->qb, job->fp64, job->p_hub, job->row_off, col_idx_out, st));
        CK(K > 1 ? cudaEventRecord(cev[4 * k + 1], st) : stage_mark(ctx, 7, st));
        CK(launch_write_rim(p, job->qb, job->fp64, job->row_off, col_idx_out, lo, hi, st));
        CK(K > 1 ? cudaEventRecord(cev[4 * k + 2], st) : stage_mark(ctx, 8, st));
        const int32_t *cnt = sub_cnt + 3 * k;
        if (cnt[0] > 0 || cnt[1] > 0 || cnt[2] > 0) {
            QueryBufs bc = job->qb;
            if (K > 1) {
                int64_t off = 0;
                for (int c = 0; c < 3; ++c) {
                    bc.rows[c] = sub + off + (int64_t)k * job->lists[c];
                    off += (int64_t)K * job->lists[c];
                }
                bc.list_cnt = dsub_cnt + 3 * k;
            }
            CK(launch_sort_rows(p, bc, cnt, sub_tot[k], job->row_off, col_idx_out, (int32_t *)tmp, bws, st));
        }
        if (K > 1) CK(cudaEventRecord(cev[4 * k + 3], st));
        if (hc && offs[k + 1] > offs[k]) {
            cudaEvent_t done = K > 1 ? cev[4 * k + 3] : ctx->hev[0];
            if (K == 1) CK(cudaEventRecord(done, st));
            CK(cudaStreamWaitEvent(hc->copy, done, 0));
            CK(cudaMemcpyAsync(hc->col_host + offs[k], col_idx_out + offs[k], sizeof(int32_t) * (offs[k + 1] - offs[k]),
                               cudaMemcpyDeviceToHost, hc->copy));
        }
    }
    CK(stage_mark(ctx, 9, st));
    uint64_t *hs = (uint64_t *)ctx->pinned;
    CK(cudaMemcpyAsync(hs, job->qb.stats + 7, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    job->finished = true;
    auto elapsed = [](cudaEvent_t a, cudaEvent_t b) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
            cudaGetLastError();
            ms = -1.0f;
        }
        return ms;
    };
    const int pairs[5][2] = {{0, 1}, {1, 2}, {2, 3}, {3, 4}, {4, 5}};
    for (int k = 0; k < 5; ++k) job->stage_ms[k] = elapsed(ctx->ev[pairs[k][0]], ctx->ev[pairs[k][1]]);
    if (K > 1) {
        // the write stages summed over the ranges
        for (int j = 0; j < 3; ++j) {
            float t = 0.0f;
            for (int k = 0; k < K; ++k) t += elapsed(cev[4 * k + j], cev[4 * k + j + 1]);
            job->stage_ms[5 + j] = t;
        }
    } else {
        job->stage_ms[5] = elapsed(ctx->ev[6], ctx->ev[7]);
        job->stage_ms[6] = elapsed(ctx->ev[7], ctx->ev[8]);
        job->stage_ms[7] = elapsed(ctx->ev[8], ctx->ev[9]);
    }
    if (hs[0] != 0) return set_err(ctx, HRG_EINTERNAL, "count and write passes disagree on a row");
    return HRG_OK;
}

extern "C" int hrg_generate_finish(hrg_job *job, int32_t *col_idx_out)
{
    if (!job || !job->ctx) return HRG_EINVAL;
    hrg_ctx *ctx = job->ctx;
    if (!job->open || job->finished) return set_err(ctx, HRG_ESTATE, "job is not open");
    if (!col_idx_out && job->n_entries > 0) return set_err(ctx, HRG_EINVAL, "null col_idx");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return set_err(ctx, HRG_ECUDA, "cudaSetDevice failed");
    return finish_impl(job, col_idx_out, nullptr);
}

extern "C" int hrg_job_stats(const hrg_job *job, hrg_stats *out)
{
    if (!job || !out) return HRG_EINVAL;
    memset(out, 0, sizeof *out);
    out->R = job->plan.R;
    out->n_entries = job->n_entries;
    out->candidates = job->stats[0];
    out->rechecks = job->stats[1];
    out->bands = job->plan.B;
    out->hub_bands = job->plan.hub_bands;
    out->buckets = job->plan.G;
    out->hub_queries = job->p_hub;
    out->mid_rows = job->lists[0] + job->lists[1];
    out->big_rows = job->lists[2];
    out->mu = job->plan.mu;
    for (int k = 0; k < 8; ++k) out->stage_ms[k] = job->stage_ms[k];
    out->write_chunks = job->write_chunks;
    out->d2h_ms = -1.0f;
    out->ties = job->stats[3];
    out->rows_no_room = (int64_t)job->stats[4];
    out->hub_rows_retraversed = (job->p_hub > 0 && !job->hub_pooled) ? job->p_hub : 0;
    out->heavy_retries = job->heavy_retries;
    if (job->update) {
        // check, apply, band counts, bucket histogram, bucket scan, scatter
        // (records + split, 2; the FP64 path 1), moved count, removals,
        // degrees, row-offset scan; write: moved rows, dropped-entry count,
        // its scan and the copy, row sorts, gain check
        const int scatter = job->fp64 ? 1 : 2;
        int L = (job->moves > 0 ? 2 : 0) + 2 + scan_launches(job->plan.G) + scatter + (job->moves > 0 ? 2 : 0) + 1 +
                scan_launches(job->plan.n);
        const int64_t chunks = (job->old_entries + 4095) / 4096;
        if (job->finished)
            L += (job->moves > 0 ? 1 : 0) + (job->old_entries > 0 ? 4 + scan_launches(chunks) : 0) +
                 sort_launches(job->lists) + 1;
        out->launches = L;
        out->hub_rows_retraversed = 0;
        out->hub_queries = 0;
        return HRG_OK;
    }
    // kernels launched: points with their buckets (1; an injected point set:
    // band counts + bucket histogram, 2), bucket scan, structure-of-arrays
    // scatter (records + split, 2; the FP64 path 1), count (hub 3, rim 1),
    // row-offset scan, write (hub 3, rim 1), row sorts (warp 1, CTA 1, big 7)
    const int64_t n = job->plan.n;
    const int scatter = job->fp64 ? 1 : 2;
    int L;
    if (job->batch) {
        // graph map, points with their buckets, bucket scan, structure-of-arrays
        // scatter, hub count + scan (+ fill), count, row-offset scan
        L = 1 + 1 + scan_launches(job->batch_G) + scatter + 1 + scan_launches(job->batch) +
            (job->p_hub > 0 ? 1 : 0) + (job->p_hub > 0 ? 3 : 0) + (job->qb.n_sectors > 0 ? 1 : 0) + scan_launches(n);
        if (job->finished)
            L += (job->p_hub > 0 ? (job->hub_pooled ? (job->hub_runs > 0 ? 2 : 1) : 3) : 0) +
                 (job->qb.n_sectors > 0 ? 2 : 0) + sort_launches(job->lists);
        out->launches = L;
        out->buckets = job->batch_G;
        return HRG_OK;
    }
    L = (job->sampled ? 1 : 2) + scan_launches(job->plan.G) + scatter + query_launches(job->plan, job->p_hub, false) +
        scan_launches(n);
    if (job->finished) {
        L += query_launches(job->plan, job->p_hub, true) + sort_launches(job->lists);
        if (job->p_hub > 0 && job->hub_pooled) L -= job->hub_runs > 0 ? 1 : 2;  // copy + check instead of 3
    }
    out->launches = L;
    return HRG_OK;
}

extern "C" int hrg_job_release(hrg_job *job)
{
    if (!job || !job->ctx) return HRG_EINVAL;
    job->open = false;
    job->finished = false;
    return HRG_OK;
}

extern "C" int hrg_generate(hrg_ctx *ctx, const hrg_params *p, void *stream, double *r_out, double *phi_out,
                            int64_t *row_off_out, int32_t *col_idx_out, int64_t col_capacity, int64_t *n_entries,
                            hrg_stats *stats_out)
{
    hrg_job *job = nullptr;
    int64_t ne = 0;
    int rc = hrg_generate_begin(ctx, p, stream, r_out, phi_out, row_off_out, &job, &ne);
    if (rc) return rc;
    if (n_entries) *n_entries = ne;
    if (ne > col_capacity) {
        if (stats_out) hrg_job_stats(job, stats_out);
        hrg_job_release(job);
        return set_err(ctx, HRG_EOVERFLOW, "graph has %lld entries, capacity %lld", (long long)ne,
                       (long long)col_capacity);
    }
    rc = hrg_generate_finish(job, col_idx_out);
    if (stats_out) hrg_job_stats(job, stats_out);
    hrg_job_release(job);
    return rc;
}

extern "C" int hrg_generate_host(hrg_ctx *ctx, const hrg_params *p, double *r_host, double *phi_host,
                                 int64_t *row_off_host, int32_t *col_idx_host, int64_t col_capacity,
                                 int64_t *n_entries, hrg_stats *stats_out)
{
    if (!ctx) return HRG_EINVAL;
    if (!p || !r_host || !phi_host || !row_off_host || !n_entries) return set_err(ctx, HRG_EINVAL, "null argument");
    if (p->n < 2 || p->n > 0x7fffffffLL) return set_err(ctx, HRG_EINVAL, "n must be in [2, 2^31)");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return set_err(ctx, HRG_ECUDA, "cudaSetDevice failed");
    if (!ctx->work) CK(cudaStreamCreateWithFlags(&ctx->work, cudaStreamNonBlocking));
    if (!ctx->copy) CK(cudaStreamCreateWithFlags(&ctx->copy, cudaStreamNonBlocking));
    for (auto &ev : ctx->hev)
        if (!ev) CK(cudaEventCreate(&ev));
    const int64_t n = p->n;
    void *dr, *dphi, *doff, *dcol;
    int rc;
    if ((rc = ensure(ctx, hrg_ctx::W_OUT_R, sizeof(double) * n, &dr))) return rc;
    if ((rc = ensure(ctx, hrg_ctx::W_OUT_PHI, sizeof(double) * n, &dphi))) return rc;
    if ((rc = ensure(ctx, hrg_ctx::W_OUT_OFF, sizeof(int64_t) * (n + 1), &doff))) return rc;
    hrg_job *job = nullptr;
    int64_t ne = 0;
    cudaStream_t st = ctx->work, cp = ctx->copy;
    // the points go back while the graph is generated (from the sampler
    // on), the row offsets once they are known, the neighbour ids range by
    // range as the write pass finishes each
    const HostPoints hpts{r_host, phi_host, cp, ctx->hev[0], ctx->hev[1]};
    rc = generate_begin(ctx, p, st, (double *)dr, (double *)dphi, (int64_t *)doff, &job, &ne, &hpts);
    if (rc) {
        cudaStreamSynchronize(cp);
        return rc;
    }
    *n_entries = ne;
    if (ne > col_capacity || (ne > 0 && !col_idx_host)) {
        if (stats_out) hrg_job_stats(job, stats_out);
        hrg_job_release(job);
        cudaStreamSynchronize(cp);
        return set_err(ctx, HRG_EOVERFLOW, "graph has %lld entries, capacity %lld", (long long)ne,
                       (long long)col_capacity);
    }
    if ((rc = ensure(ctx, hrg_ctx::W_OUT_COL, sizeof(int32_t) * (ne > 0 ? ne : 1), &dcol))) {
        hrg_job_release(job);
        cudaStreamSynchronize(cp);
        return rc;
    }
    // begin has synchronized the generation stream: the row offsets are final
    CK(cudaMemcpyAsync(row_off_host, doff, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost, cp));
    const HostCol hcol{col_idx_host, cp};
    rc = finish_impl(job, (int32_t *)dcol, &hcol);
    CK(cudaEventRecord(ctx->hev[2], cp));
    const cudaError_t ce = cudaStreamSynchronize(cp);
    if (stats_out) {
        hrg_job_stats(job, stats_out);
        float ms = -1.0f;
        if (ce == cudaSuccess && cudaEventElapsedTime(&ms, ctx->hev[1], ctx->hev[2]) != cudaSuccess) {
            cudaGetLastError();
            ms = -1.0f;
        }
        stats_out->d2h_ms = ms;
    }
    hrg_job_release(job);
    if (rc) return rc;
    if (ce != cudaSuccess) return set_err(ctx, HRG_ECUDA, "read-back failed: %s", cudaGetErrorString(ce));
    return HRG_OK;
}

// ---------------------------------------------------------------------------
// Graph properties of Sec. 4.1 (kernels in hrg_props.cu).
// ---------------------------------------------------------------------------
extern "C" int hrg_graph_props(hrg_ctx *ctx, int64_t n, const int64_t *row_off, const int32_t *col_idx,
                               int64_t d_min, uint32_t flags, void *stream, hrg_props *out)
{
    if (!ctx) return HRG_EINVAL;
    if (!out) return set_err(ctx, HRG_EINVAL, "null out");
    if (n < 0 || n > 0x7fffffffLL) return set_err(ctx, HRG_EINVAL, "n must be in [0, 2^31)");
    if (n > 0 && !row_off) return set_err(ctx, HRG_EINVAL, "null row_off");
    if (d_min < 1) return set_err(ctx, HRG_EINVAL, "d_min must be at least 1");
    if (flags & ~HRG_PROPS_TRIANGLES) return set_err(ctx, HRG_EINVAL, "unknown flags");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return set_err(ctx, HRG_ECUDA, "cudaSetDevice failed");
    cudaStream_t st = (cudaStream_t)stream;
    memset(out, 0, sizeof *out);
    out->n = n;
    out->d_min = d_min;
    out->triangles = -1;
    out->gamma = out->clustering = out->avg_local_clustering = std::nan("");
    if (n == 0) return HRG_OK;
    int rc;
    void *acc;
    if ((rc = ensure(ctx, hrg_ctx::W_PACC, 64, &acc))) return rc;
    unsigned long long *ai = (unsigned long long *)acc;  // [0] max degree [1] tail [2] triads [3] triangles
    double *ad = (double *)((char *)acc + 32);           // [0] tail log sum [1] local clustering sum
    CK(cudaMemsetAsync(acc, 0, 64, st));
    CK(launch_degree_stats(n, row_off, d_min, ai, ad, st));
    char *hp = (char *)ctx->pinned;
    CK(cudaMemcpyAsync(hp, acc, 64, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(hp + 64, row_off, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(hp + 72, row_off + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    unsigned long long hi[4];
    double hd[2];
    int64_t o0, on;
    memcpy(hi, hp, 32);
    memcpy(hd, hp + 32, 16);
    memcpy(&o0, hp + 64, 8);
    memcpy(&on, hp + 72, 8);
    out->entries = on - o0;
    out->max_degree = (int64_t)hi[0];
    out->tail_count = (int64_t)hi[1];
    out->triads = (int64_t)hi[2];
    out->tail_log_sum = hd[0];
    if (out->tail_count > 0) out->gamma = 1.0 + (double)out->tail_count / out->tail_log_sum;
    if (!(flags & HRG_PROPS_TRIANGLES)) return HRG_OK;
    if (out->entries > 0 && !col_idx) return set_err(ctx, HRG_EINVAL, "null col_idx");

    // the neighbours ranked above each vertex, then the triangles
    void *odeg, *ooff, *ocol, *tri, *scanws;
    if ((rc = ensure(ctx, hrg_ctx::W_POUTDEG, sizeof(int32_t) * n, &odeg))) return rc;
    if ((rc = ensure(ctx, hrg_ctx::W_POUTOFF, sizeof(int64_t) * (n + 1), &ooff))) return rc;
    if ((rc = ensure(ctx, hrg_ctx::W_PTRI, sizeof(unsigned long long) * n, &tri))) return rc;
    if ((rc = ensure(ctx, hrg_ctx::W_PSCAN, scan_workspace_bytes(n), &scanws))) return rc;
    CK(launch_out_edges(n, row_off, col_idx, (int32_t *)odeg, nullptr, nullptr, false, st));
    CK(scan_i32_to_i64((const int32_t *)odeg, (int64_t *)ooff, n, scanws, st));
    CK(cudaMemcpyAsync(hp + 80, (int64_t *)ooff + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    int64_t m_up;
    memcpy(&m_up, hp + 80, 8);
    if ((rc = ensure(ctx, hrg_ctx::W_POUTCOL, sizeof(int32_t) * (m_up > 0 ? m_up : 1), &ocol))) return rc;
    CK(cudaMemsetAsync(tri, 0, sizeof(unsigned long long) * n, st));
    CK(launch_out_edges(n, row_off, col_idx, nullptr, (const int64_t *)ooff, (int32_t *)ocol, true, st));
    CK(launch_triangles(n, (const int64_t *)ooff, (const int32_t *)ocol, (unsigned long long *)tri, ai + 3, st));
    CK(launch_local_clustering(n, row_off, (const unsigned long long *)tri, ad + 1, st));
    CK(cudaMemcpyAsync(hp, acc, 64, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    memcpy(hi, hp, 32);
    memcpy(hd, hp + 32, 16);
    out->triangles = (int64_t)hi[3];
    if (out->triads > 0) out->clustering = 3.0 * (double)out->triangles / (double)out->triads;
    out->avg_local_clustering = hd[1] / (double)n;
    return HRG_OK;
}

extern "C" int hrg_degree_histogram(hrg_ctx *ctx, int64_t n, const int64_t *row_off, int64_t max_degree,
                                    int64_t *hist, void *stream)
{
    if (!ctx) return HRG_EINVAL;
    if (n < 0 || n > 0x7fffffffLL) return set_err(ctx, HRG_EINVAL, "n must be in [0, 2^31)");
    if ((n > 0 && !row_off) || !hist) return set_err(ctx, HRG_EINVAL, "null argument");
    if (max_degree < 0) return set_err(ctx, HRG_EINVAL, "max_degree must be >= 0");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return set_err(ctx, HRG_ECUDA, "cudaSetDevice failed");
    cudaStream_t st = (cudaStream_t)stream;
    int rc;
    void *acc;
    if ((rc = ensure(ctx, hrg_ctx::W_PACC, 64, &acc))) return rc;
    CK(cudaMemsetAsync(hist, 0, sizeof(int64_t) * (max_degree + 1), st));
    CK(cudaMemsetAsync(acc, 0, sizeof(int), st));
    if (n > 0)
        CK(launch_degree_hist(n, row_off, max_degree, (unsigned long long *)hist, (int *)acc, st));
    int *hflag = (int *)ctx->pinned;
    CK(cudaMemcpyAsync(hflag, acc, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (*hflag) return set_err(ctx, HRG_EINVAL, "a degree exceeds max_degree = %lld", (long long)max_degree);
    return HRG_OK;
}

// ---------------------------------------------------------------------------
// Random long-range edges of Sec. 4.2 (kernels in hrg_longrange.cu).
// ---------------------------------------------------------------------------
extern "C" int hrg_add_random_edges(hrg_ctx *ctx, int64_t n, const int64_t *row_off, const int32_t *col_idx,
                                    int64_t count, uint64_t seed, void *stream, int64_t *row_off_out,
                                    int32_t *col_idx_out, int64_t col_capacity, int64_t *entries_out,
                                    int64_t *added_out)
{
    if (!ctx) return HRG_EINVAL;
    if (n < 0 || n > 0x7fffffffLL) return set_err(ctx, HRG_EINVAL, "n must be in [0, 2^31)");
    if (count < 0 || count > (1LL << 30)) return set_err(ctx, HRG_EINVAL, "count must be in [0, 2^30]");
    if (!row_off || !row_off_out || !entries_out) return set_err(ctx, HRG_EINVAL, "null argument");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return set_err(ctx, HRG_ECUDA, "cudaSetDevice failed");
    cudaStream_t st = (cudaStream_t)stream;
    char *hp = (char *)ctx->pinned;
    CK(cudaMemcpyAsync(hp, row_off, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(hp + 8, row_off + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    int64_t o0, on;
    memcpy(&o0, hp, 8);
    memcpy(&on, hp + 8, 8);
    if (on > o0 && !col_idx) return set_err(ctx, HRG_EINVAL, "null col_idx");
    if (n == 0) {
        CK(cudaMemsetAsync(row_off_out, 0, sizeof(int64_t), st));
        CK(cudaStreamSynchronize(st));
        *entries_out = 0;
        if (added_out) *added_out = 0;
        return HRG_OK;
    }
    int rc;
    void *cnt, *loff, *list, *fin, *ndeg, *scanws;
    if ((rc = ensure(ctx, hrg_ctx::W_LRCNT, sizeof(int32_t) * n, &cnt))) return rc;
    if ((rc = ensure(ctx, hrg_ctx::W_LROFF, sizeof(int64_t) * (n + 1), &loff))) return rc;
    if ((rc = ensure(ctx, hrg_ctx::W_LRLIST, sizeof(int32_t) * (2 * count > 0 ? 2 * count : 1), &list))) return rc;
    if ((rc = ensure(ctx, hrg_ctx::W_LRFIN, sizeof(int32_t) * n, &fin))) return rc;
    if ((rc = ensure(ctx, hrg_ctx::W_LRDEG, sizeof(int32_t) * n, &ndeg))) return rc;
    if ((rc = ensure(ctx, hrg_ctx::W_PSCAN, scan_workspace_bytes(n), &scanws))) return rc;
    // partners of every vertex, listed
    CK(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * n, st));
    if (count > 0) CK(launch_lr_count(n, count, seed, (int32_t *)cnt, st));
    CK(scan_i32_to_i64((const int32_t *)cnt, (int64_t *)loff, n, scanws, st));
    CK(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * n, st));
    if (count > 0) CK(launch_lr_fill(n, count, seed, (const int64_t *)loff, (int32_t *)cnt, (int32_t *)list, st));
    // new degrees and row offsets
    CK(launch_lr_clean(n, row_off, col_idx, (const int64_t *)loff, (int32_t *)list, (int32_t *)fin, (int32_t *)ndeg,
                       st));
    CK(scan_i32_to_i64((const int32_t *)ndeg, row_off_out, n, scanws, st));
    CK(cudaMemcpyAsync(hp + 16, row_off_out + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    int64_t ne;
    memcpy(&ne, hp + 16, 8);
    *entries_out = ne;
    if (added_out) *added_out = (ne - (on - o0)) / 2;
    if (ne > col_capacity || (ne > 0 && !col_idx_out))
        return set_err(ctx, HRG_EOVERFLOW, "graph with the added edges has %lld entries, capacity %lld",
                       (long long)ne, (long long)col_capacity);
    CK(launch_lr_merge(n, on - o0, row_off, col_idx, (const int64_t *)loff, (const int32_t *)list,
                       (const int32_t *)fin, row_off_out, col_idx_out, st));
    CK(cudaStreamSynchronize(st));
    return HRG_OK;
}

// ---------------------------------------------------------------------------
// Breadth-first search and diameter bounds (Sec. 4.1, Sec. 4.2; kernels in
// hrg_bfs.cu).
// ---------------------------------------------------------------------------
extern "C" int hrg_bfs(hrg_ctx *ctx, int64_t n, const int64_t *row_off, const int32_t *col_idx, int64_t source,
                       void *stream, int32_t *dist, int32_t *ecc_out, int64_t *reached_out, int64_t *far_out,
                       int64_t *source_out)
{
    if (!ctx) return HRG_EINVAL;
    if (n < 1 || n > 0x7fffffffLL) return set_err(ctx, HRG_EINVAL, "n must be in [1, 2^31)");
    if (source >= n) return set_err(ctx, HRG_EINVAL, "source must be < n");
    if (!row_off || !dist || !ecc_out) return set_err(ctx, HRG_EINVAL, "null argument");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return set_err(ctx, HRG_ECUDA, "cudaSetDevice failed");
    cudaStream_t st = (cudaStream_t)stream;
    char *hp = (char *)ctx->pinned;
    CK(cudaMemcpyAsync(hp, row_off, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(hp + 8, row_off + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    int64_t o0, on;
    memcpy(&o0, hp, 8);
    memcpy(&on, hp + 8, 8);
    if (on > o0 && !col_idx) return set_err(ctx, HRG_EINVAL, "null col_idx");
    int rc;
    void *f0, *f1, *fdeg, *foff, *acc, *scanws;
    if ((rc = ensure(ctx, hrg_ctx::W_BFSF0, sizeof(int32_t) * n, &f0))) return rc;
    if ((rc = ensure(ctx, hrg_ctx::W_BFSF1, sizeof(int32_t) * n, &f1))) return rc;
    if ((rc = ensure(ctx, hrg_ctx::W_BFSDEG, sizeof(int32_t) * n, &fdeg))) return rc;
    if ((rc = ensure(ctx, hrg_ctx::W_BFSOFF, sizeof(int64_t) * (n + 1), &foff))) return rc;
    if ((rc = ensure(ctx, hrg_ctx::W_BFSACC, 64, &acc))) return rc;
    if ((rc = ensure(ctx, hrg_ctx::W_PSCAN, scan_workspace_bytes(n), &scanws))) return rc;
    unsigned long long *best = (unsigned long long *)acc;        // [0]
    int32_t *nnext = (int32_t *)((char *)acc + 8);               // [8]
    int32_t *far = (int32_t *)((char *)acc + 12);                // [12]
    int64_t *src = (int64_t *)((char *)acc + 16);                // [16]
    CK(cudaMemsetAsync(acc, 0, 64, st));
    CK(launch_bfs_init(n, dist, row_off, best, st));
    CK(launch_bfs_seed(best, source, dist, (int32_t *)f0, src, far, st));
    int32_t *cur = (int32_t *)f0, *nxt = (int32_t *)f1;
    int32_t fsize = 1, level = 0;
    int64_t reached = 1;
    for (;;) {
        CK(launch_bfs_frontier_deg(fsize, cur, row_off, (int32_t *)fdeg, st));
        CK(scan_i32_to_i64((const int32_t *)fdeg, (int64_t *)foff, fsize, scanws, st));
        CK(cudaMemsetAsync(nnext, 0, sizeof(int32_t), st));
        CK(launch_bfs_expand(level, fsize, cur, (const int64_t *)foff, row_off, col_idx, dist, nxt, nnext, st));
        CK(cudaMemcpyAsync(hp + 16, nnext, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        int32_t got;
        memcpy(&got, hp + 16, 4);
        if (got == 0) break;
        reached += got;
        fsize = got;
        ++level;
        std::swap(cur, nxt);
    }
    CK(launch_bfs_far(n, dist, level, far, st));
    CK(cudaMemcpyAsync(hp + 24, acc, 24, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    int32_t hfar;
    int64_t hsrc;
    memcpy(&hfar, hp + 24 + 12, 4);
    memcpy(&hsrc, hp + 24 + 16, 8);
    *ecc_out = level;
    if (reached_out) *reached_out = reached;
    if (far_out) *far_out = hfar;
    if (source_out) *source_out = hsrc;
    return HRG_OK;
}

extern "C" int hrg_diameter_bounds(hrg_ctx *ctx, int64_t n, const int64_t *row_off, const int32_t *col_idx,
                                   int32_t sweeps, void *stream, int32_t *lower, int32_t *upper,
                                   int64_t *component, int64_t *roots)
{
    if (!ctx) return HRG_EINVAL;
    if (n < 1 || n > 0x7fffffffLL) return set_err(ctx, HRG_EINVAL, "n must be in [1, 2^31)");
    if (sweeps < 1 || sweeps > 64) return set_err(ctx, HRG_EINVAL, "sweeps must be in [1, 64]");
    if (!lower || !upper) return set_err(ctx, HRG_EINVAL, "null argument");
    int rc;
    void *dist;
    if ((rc = ensure(ctx, hrg_ctx::W_BFSDIST, sizeof(int32_t) * n, &dist))) return rc;
    int64_t root = -1;
    int32_t lo = 0, hi = INT32_MAX;
    int64_t size = 0;
    if (roots)
        for (int32_t k = 0; k < sweeps; ++k) roots[k] = -1;
    for (int32_t k = 0; k < sweeps; ++k) {
        int32_t ecc;
        int64_t reached, far, src;
        if ((rc = hrg_bfs(ctx, n, row_off, col_idx, root, stream, (int32_t *)dist, &ecc, &reached, &far, &src)))
            return rc;
        if (roots) roots[k] = src;
        size = reached;
        lo = std::max(lo, ecc);
        hi = std::min(hi, 2 * ecc);
        if (far == src) break;
        root = far;
    }
    *lower = lo;
    *upper = hi;
    if (component) *component = size;
    return HRG_OK;
}
