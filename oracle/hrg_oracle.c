/*
 * hrg_oracle.c -- CPU oracle for the threshold random hyperbolic graph (RHG).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * restatement of what the generator computes.  Only the test-suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load it.  It shares no
 * code, header, table or helper with the CUDA library; the two meet only
 * through seeded parameters.
 *
 * What it follows (von Looz, Meyerhenke, Prutkin, Staudt, "Fast generation of
 * complex networks with underlying hyperbolic geometry"):
 *   - Sec. 2.1: points on the disk D_R with curvature -1 (zeta fixed to 1);
 *     angle uniform on [0, 2pi), radius with the density of Eq. (1); an edge
 *     joins u and v exactly when their hyperbolic distance is below R.
 *   - Appendix B.1: R is the solution of Krioukov et al.'s Eq. (22) for the
 *     requested average degree, found by binary search.
 *   - Algorithm 1: every vertex collects all points inside the hyperbolic
 *     circle of radius R around it; each undirected edge appears in both
 *     rows; a vertex is not its own neighbour.
 *
 * Readings taken where the paper is silent or garbled (all listed in the
 * design notes of the repository):
 *   - Eq. (22): the middle term reads (pi-1)*(zeta/alpha), not (pi-1)*xi/alpha;
 *     "\frac{zeta}{alpha}^2" reads (zeta/alpha)^2.
 *   - The binary search brackets R on the decreasing branch of Eq. (22), right
 *     of its single maximum, and returns the largest R with kbar(R) >= target.
 *   - Random numbers: Philox4x32-10 (Salmon et al., SC'11), key = seed,
 *     counter = (vertex id, 0, 0); uniforms from the top 53 bits of each
 *     64-bit half of the output block.
 *   - Predicate: cosh d = cosh(r1-r2) + 2 sinh r1 sinh r2 sin^2(dphi/2), the
 *     hyperbolic law of cosines rewritten so that both terms are positive;
 *     edge iff cosh d < cosh R (strict).
 *   - Tie band: pairs whose |cosh d - cosh R| < 1e-12 cosh R are reported so
 *     a comparison can exclude them.
 *
 * Build: gcc -O2 -fno-fast-math -ffp-contract=off -fopenmp -fPIC -shared
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_TWO_PI 6.283185307179586 /* the double nearest 2*pi */
#define ORC_PI 3.141592653589793

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, Sec. 4).                */
/* One round multiplies counter words 0 and 2 by two fixed odd constants,   */
/* swaps the halves of the products into the four words and mixes the key  */
/* in; the key advances by two Weyl constants between rounds.               */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ------------------------------------------------------------------------ */
/* Eq. (22) of Krioukov et al. as restated in Appendix B.1, zeta = 1:        */
/*   kbar = (2/pi) xi^2 n ( e^{-R/2} + e^{-alpha R} ( alpha R/2 (            */
/*          pi/4 (1/alpha)^2 - (pi-1)(1/alpha) + (pi-2) ) - 1 ) ),           */
/*   xi = alpha / (alpha - 1/2).                                             */
/* ------------------------------------------------------------------------ */
double orc_expected_degree(double n, double alpha, double R)
{
    double xi = alpha / (alpha - 0.5);
    double inner = (ORC_PI / 4.0) * (1.0 / alpha) * (1.0 / alpha)
                 - (ORC_PI - 1.0) * (1.0 / alpha)
                 + (ORC_PI - 2.0);
    double bracket = exp(-R / 2.0) + exp(-alpha * R) * (alpha * (R / 2.0) * inner - 1.0);
    return (2.0 / ORC_PI) * xi * xi * n * bracket;
}

/* Appendix B.1 binary search.  Returns 0 on success, -1 on invalid input.
 * The expression rises from 0 to one maximum and then decays, so the search
 * runs on [R_peak, R_hi] with kbar(R_peak) >= target > kbar(R_hi). */
int orc_solve_radius(int64_t n, double alpha, double kbar, double *R_out)
{
    if (!(n >= 2) || !(alpha > 0.5) || !(kbar > 0.0) || !(kbar < (double)(n - 1)))
        return -1;
    double nn = (double)n;
    /* locate the maximum: coarse grid, then ternary refinement */
    double best_R = 0.0, best_k = -INFINITY;
    for (int i = 1; i <= 4000; ++i) {
        double R = 0.005 * i; /* (0, 20] */
        double k = orc_expected_degree(nn, alpha, R);
        if (k > best_k) { best_k = k; best_R = R; }
    }
    double a = best_R - 0.005, b = best_R + 0.005;
    if (a < 0.0) a = 0.0;
    for (int it = 0; it < 200; ++it) {
        double m1 = a + (b - a) / 3.0, m2 = b - (b - a) / 3.0;
        if (orc_expected_degree(nn, alpha, m1) < orc_expected_degree(nn, alpha, m2)) a = m1; else b = m2;
    }
    double R_peak = 0.5 * (a + b);
    if (orc_expected_degree(nn, alpha, R_peak) < kbar) return -1;
    double step = 1.0, R_hi = R_peak + step;
    while (orc_expected_degree(nn, alpha, R_hi) >= kbar) {
        step *= 2.0;
        R_hi = R_peak + step;
        if (step > 1e6) return -1;
    }
    double lo = R_peak, hi = R_hi;
    for (;;) {
        double mid = lo + 0.5 * (hi - lo);
        if (mid <= lo || mid >= hi) break;
        if (orc_expected_degree(nn, alpha, mid) >= kbar) lo = mid; else hi = mid;
    }
    *R_out = lo;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Sampling (Algorithm 1, the two "draw" steps; radial density Eq. (1)).     */
/* Inverse transform: the CDF of Eq. (1) is (cosh(alpha r)-1)/(cosh(alpha R) */
/* -1), so r = acosh(1 + u (cosh(alpha R) - 1)) / alpha.                      */
/* ------------------------------------------------------------------------ */
void orc_uniforms(uint64_t seed, int64_t id, double *u_phi, double *u_r)
{
    uint32_t ctr[4] = {(uint32_t)((uint64_t)id & 0xffffffffu), (uint32_t)((uint64_t)id >> 32), 0u, 0u};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t x[4];
    orc_philox4x32_10(ctr, key, x);
    uint64_t a = ((uint64_t)x[0] << 32) | (uint64_t)x[1];
    uint64_t b = ((uint64_t)x[2] << 32) | (uint64_t)x[3];
    *u_phi = (double)(a >> 11) * 0x1.0p-53;
    *u_r = (double)(b >> 11) * 0x1.0p-53;
}

void orc_sample(int64_t n, double alpha, double R, uint64_t seed, double *r, double *phi)
{
    double big = cosh(alpha * R) - 1.0;
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double up, ur;
        orc_uniforms(seed, i, &up, &ur);
        phi[i] = up * ORC_TWO_PI;
        r[i] = acosh(1.0 + ur * big) / alpha;
    }
}

/* ------------------------------------------------------------------------ */
/* Predicate.  Hyperbolic law of cosines in native polar coordinates:        */
/*   cosh d = cosh r1 cosh r2 - sinh r1 sinh r2 cos(dphi)                     */
/*          = cosh(r1 - r2) + 2 sinh r1 sinh r2 sin^2(dphi/2).                */
/* The second form has only non-negative terms.                              */
/* ------------------------------------------------------------------------ */
double orc_cosh_dist(double r1, double phi1, double r2, double phi2)
{
    double s = sin((phi1 - phi2) / 2.0);
    return cosh(r1 - r2) + 2.0 * sinh(r1) * sinh(r2) * (s * s);
}

/* textbook form, for cross-checks at small R only */
double orc_cosh_dist_textbook(double r1, double phi1, double r2, double phi2)
{
    return cosh(r1) * cosh(r2) - sinh(r1) * sinh(r2) * cos(phi1 - phi2);
}

/* Eq. (2): Poincare metric between two points of the unit disk, after the
 * mapping of Appendix B.2, r_E = sqrt((cosh r - 1)/(cosh r + 1)).  Returns
 * cosh of the distance.  Valid only where 1 - r_E^2 is not rounded away. */
double orc_cosh_dist_poincare(double r1, double phi1, double r2, double phi2)
{
    double e1 = sqrt((cosh(r1) - 1.0) / (cosh(r1) + 1.0));
    double e2 = sqrt((cosh(r2) - 1.0) / (cosh(r2) + 1.0));
    double x1 = e1 * cos(phi1), y1 = e1 * sin(phi1);
    double x2 = e2 * cos(phi2), y2 = e2 * sin(phi2);
    double dx = x1 - x2, dy = y1 - y2;
    double num = dx * dx + dy * dy;
    return 1.0 + 2.0 * num / ((1.0 - e1 * e1) * (1.0 - e2 * e2));
}

/* Proposition 1: the hyperbolic circle of radius R around (phi_h, r_h) is the
 * Euclidean circle with centre (phi_h, 2 r_e/(ab+2)) and radius
 * sqrt(centre^2 - (2 r_e^2 - ab)/(ab+2)), a = cosh R - 1, b = 1 - r_e^2, where
 * r_e is the Poincare radius of the query.  Returns 1 when the second point
 * lies strictly inside. */
int orc_in_circle_prop1(double R, double rq, double phiq, double rc, double phic)
{
    double eq = sqrt((cosh(rq) - 1.0) / (cosh(rq) + 1.0));
    double ec = sqrt((cosh(rc) - 1.0) / (cosh(rc) + 1.0));
    double a = cosh(R) - 1.0, b = 1.0 - eq * eq;
    double cen = 2.0 * eq / (a * b + 2.0);
    double rad2 = cen * cen - (2.0 * eq * eq - a * b) / (a * b + 2.0);
    double cx = cen * cos(phiq), cy = cen * sin(phiq);
    double px = ec * cos(phic), py = ec * sin(phic);
    double dx = px - cx, dy = py - cy;
    return (dx * dx + dy * dy) < rad2;
}

/* ------------------------------------------------------------------------ */
/* Brute force (the plain definition): all pairs i<j, edge iff cosh d <     */
/* cosh R, both directions stored, rows ascending.                           */
/* ------------------------------------------------------------------------ */
static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* deg[n] out; returns the number of directed entries. */
int64_t orc_brute_degrees(int64_t n, const double *r, const double *phi, double R, int64_t *deg)
{
    double cR = cosh(R);
    int64_t total = 0;
    #pragma omp parallel for schedule(dynamic, 64) reduction(+ : total)
    for (int64_t i = 0; i < n; ++i) {
        int64_t d = 0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            if (orc_cosh_dist(r[i], phi[i], r[j], phi[j]) < cR) ++d;
        }
        deg[i] = d;
        total += d;
    }
    return total;
}

/* row_off[n+1] given (from the degrees), fills col_idx. */
void orc_brute_fill(int64_t n, const double *r, const double *phi, double R,
                    const int64_t *row_off, int32_t *col_idx)
{
    double cR = cosh(R);
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        int64_t k = row_off[i];
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            if (orc_cosh_dist(r[i], phi[i], r[j], phi[j]) < cR) col_idx[k++] = (int32_t)j;
        }
    }
}

/* Rows of selected vertices by scanning all n points (the definition, one
 * row at a time, for sampled checks at sizes where all pairs are too many).
 * First call with rows == NULL fills cnt[]; second call fills rows at off[]. */
void orc_brute_rows(int64_t n, const double *r, const double *phi, double R, int64_t nq, const int64_t *qids,
                    int64_t *cnt, const int64_t *off, int32_t *rows)
{
    double cR = cosh(R);
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t t = 0; t < nq; ++t) {
        int64_t i = qids[t], k = 0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            if (orc_cosh_dist(r[i], phi[i], r[j], phi[j]) < cR) {
                if (rows) rows[off[t] + k] = (int32_t)j;
                ++k;
            }
        }
        if (!rows) cnt[t] = k;
    }
}

/* Tie band: pairs i<j with |cosh d - cosh R| < tol * cosh R.  Writes up to
 * cap pairs (2 ints each) and returns how many exist. */
int64_t orc_brute_ties(int64_t n, const double *r, const double *phi, double R, double tol,
                       int64_t cap, int64_t *pairs)
{
    double cR = cosh(R);
    int64_t cnt = 0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j) {
            double v = orc_cosh_dist(r[i], phi[i], r[j], phi[j]);
            if (fabs(v - cR) < tol * cR) {
                if (cnt < cap) { pairs[2 * cnt] = i; pairs[2 * cnt + 1] = j; }
                ++cnt;
            }
        }
    return cnt;
}

/* ------------------------------------------------------------------------ */
/* CPU band algorithm.  Radial shells of width 1 (the last one shorter),    */
/* each sorted by angle.  A query in shell-less form: for every shell with  */
/* inner radius b, every neighbour c satisfies |dphi| <= theta(r_q, b),     */
/* since the admissible angle shrinks as r_c grows; theta comes from        */
/* sin^2(theta/2) = (cosh R - cosh(r_q - b)) / (2 sinh r_q sinh b), padded.  */
/* Candidates found by binary search on the shell's sorted angles are then   */
/* decided by the exact predicate above.                                     */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t n;
    double R, cR;
    int nshell;
    double *inner;      /* [nshell] inner radius */
    int64_t *start;     /* [nshell+1] */
    double *phi;        /* [n] sorted by (shell, phi) */
    double *r;          /* [n] */
    int32_t *id;        /* [n] */
} orc_bands;

typedef struct { double phi; double r; int32_t id; int shell; } orc_pt;

static int cmp_pt(const void *a, const void *b)
{
    const orc_pt *x = (const orc_pt *)a, *y = (const orc_pt *)b;
    if (x->shell != y->shell) return x->shell < y->shell ? -1 : 1;
    if (x->phi != y->phi) return x->phi < y->phi ? -1 : 1;
    return (x->id > y->id) - (x->id < y->id);
}

void *orc_bands_build(int64_t n, const double *r, const double *phi, double R)
{
    orc_bands *B = (orc_bands *)calloc(1, sizeof(orc_bands));
    B->n = n; B->R = R; B->cR = cosh(R);
    B->nshell = (int)ceil(R);
    if (B->nshell < 1) B->nshell = 1;
    B->inner = (double *)malloc(sizeof(double) * B->nshell);
    for (int k = 0; k < B->nshell; ++k) B->inner[k] = (double)k;
    orc_pt *pts = (orc_pt *)malloc(sizeof(orc_pt) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) {
        int s = (int)floor(r[i]);
        if (s < 0) s = 0;
        if (s >= B->nshell) s = B->nshell - 1;
        pts[i].phi = phi[i]; pts[i].r = r[i]; pts[i].id = (int32_t)i; pts[i].shell = s;
    }
    qsort(pts, (size_t)n, sizeof(orc_pt), cmp_pt);
    B->start = (int64_t *)calloc((size_t)B->nshell + 1, sizeof(int64_t));
    B->phi = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    B->r = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    B->id = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) {
        B->phi[i] = pts[i].phi; B->r[i] = pts[i].r; B->id[i] = pts[i].id;
        B->start[pts[i].shell + 1]++;
    }
    for (int k = 0; k < B->nshell; ++k) B->start[k + 1] += B->start[k];
    free(pts);
    return B;
}

void orc_bands_free(void *h)
{
    orc_bands *B = (orc_bands *)h;
    if (!B) return;
    free(B->inner); free(B->start); free(B->phi); free(B->r); free(B->id); free(B);
}

/* first index in [lo,hi) with phi >= x */
static int64_t lower_phi(const double *p, int64_t lo, int64_t hi, double x)
{
    while (lo < hi) {
        int64_t m = lo + (hi - lo) / 2;
        if (p[m] < x) lo = m + 1; else hi = m;
    }
    return lo;
}

/* half-width of the angular window of query radius rq in a shell whose
 * inner radius is b; returns pi when the whole shell may be adjacent. */
static double shell_window(double R, double cR, double rq, double b)
{
    if (rq + b <= R) return ORC_PI;
    double den = 2.0 * sinh(rq) * sinh(b);
    double num = cR - cosh(rq - b);
    double x = num / den;
    x = x * (1.0 + 1e-9) + 4e-16 * cR / den;
    if (x >= 1.0) return ORC_PI;
    if (x <= 0.0) x = 0.0;
    double t = 2.0 * asin(sqrt(x));
    t = t * (1.0 + 1e-9) + 1e-15;
    return t < ORC_PI ? t : ORC_PI;
}

/* Visits the candidates of query q (vertex id) in the windows of every
 * shell.  With ties == NULL: counts the neighbours, storing them into out[]
 * (sorted) when out != NULL.  With ties != NULL: windows are computed for the
 * widened radius Rw and every candidate c with id > qid whose predicate value
 * lies within tol * cosh R of cosh R is appended to ties (up to cap pairs);
 * returns the number of such pairs. */
static int64_t band_query(const orc_bands *B, double rq, double phiq, int32_t qid, int32_t *out,
                          double Rw, double tol, int64_t cap, int64_t *ties)
{
    int64_t d = 0;
    double cRw = cosh(Rw);
    for (int k = 0; k < B->nshell; ++k) {
        int64_t s = B->start[k], e = B->start[k + 1];
        if (s == e) continue;
        double th = shell_window(Rw, cRw, rq, B->inner[k]);
        int64_t ranges[2][2];
        int nr = 0;
        if (th >= ORC_PI) {
            ranges[0][0] = s; ranges[0][1] = e; nr = 1;
        } else {
            double lo = phiq - th, hi = phiq + th;
            if (lo < 0.0) {
                ranges[nr][0] = lower_phi(B->phi, s, e, lo + ORC_TWO_PI); ranges[nr][1] = e; ++nr;
                ranges[nr][0] = s; ranges[nr][1] = lower_phi(B->phi, s, e, nextafter(hi, INFINITY)); ++nr;
            } else if (hi >= ORC_TWO_PI) {
                ranges[nr][0] = lower_phi(B->phi, s, e, lo); ranges[nr][1] = e; ++nr;
                ranges[nr][0] = s; ranges[nr][1] = lower_phi(B->phi, s, e, nextafter(hi - ORC_TWO_PI, INFINITY)); ++nr;
            } else {
                ranges[nr][0] = lower_phi(B->phi, s, e, lo);
                ranges[nr][1] = lower_phi(B->phi, s, e, nextafter(hi, INFINITY));
                ++nr;
            }
            /* th < pi, so the two pieces of a wrapped window are disjoint */
        }
        for (int t = 0; t < nr; ++t)
            for (int64_t c = ranges[t][0]; c < ranges[t][1]; ++c) {
                if (B->id[c] == qid) continue;
                double v = orc_cosh_dist(rq, phiq, B->r[c], B->phi[c]);
                if (ties) {
                    if (B->id[c] > qid && fabs(v - B->cR) < tol * B->cR) {
                        if (d < cap) { ties[2 * d] = qid; ties[2 * d + 1] = B->id[c]; }
                        ++d;
                    }
                } else if (v < B->cR) {
                    if (out) out[d] = B->id[c];
                    ++d;
                }
            }
    }
    if (!ties && out && d > 1) qsort(out, (size_t)d, sizeof(int32_t), cmp_i32);
    return d;
}

/* degrees of all vertices (id order); returns the number of directed entries */
int64_t orc_bands_degrees(void *h, const double *r, const double *phi, int64_t *deg)
{
    orc_bands *B = (orc_bands *)h;
    int64_t total = 0;
    #pragma omp parallel for schedule(dynamic, 256) reduction(+ : total)
    for (int64_t i = 0; i < B->n; ++i) {
        deg[i] = band_query(B, r[i], phi[i], (int32_t)i, NULL, B->R, 0.0, 0, NULL);
        total += deg[i];
    }
    return total;
}

void orc_bands_fill(void *h, const double *r, const double *phi, const int64_t *row_off, int32_t *col_idx)
{
    orc_bands *B = (orc_bands *)h;
    #pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < B->n; ++i)
        band_query(B, r[i], phi[i], (int32_t)i, col_idx + row_off[i], B->R, 0.0, 0, NULL);
}

/* rows of selected vertices: counts first (rows == NULL), then rows */
void orc_bands_rows(void *h, const double *r, const double *phi, int64_t nq, const int64_t *qids,
                    int64_t *cnt, const int64_t *off, int32_t *rows)
{
    orc_bands *B = (orc_bands *)h;
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t t = 0; t < nq; ++t) {
        int64_t i = qids[t];
        if (rows) band_query(B, r[i], phi[i], (int32_t)i, rows + off[t], B->R, 0.0, 0, NULL);
        else cnt[t] = band_query(B, r[i], phi[i], (int32_t)i, NULL, B->R, 0.0, 0, NULL);
    }
}

/* Tie band over the candidates of windows widened to the radius Rw with
 * cosh Rw = (1 + 2 tol) cosh R, which contain every pair within the
 * tolerance.  Queries run in parallel; each thread keeps the pairs it finds
 * in a list of its own, and the lists are joined and sorted, so the result
 * is the (i, j)-ordered list whatever the thread count.  Writes up to cap
 * pairs (i<j) and returns how many exist. */
int orc_num_threads(void);
typedef struct { int64_t *p; int64_t len, cap; } orc_pairlist;

static void pairlist_add(orc_pairlist *L, const int64_t *pairs, int64_t k)
{
    if (L->len + k > L->cap) {
        int64_t c = L->cap ? 2 * L->cap : 64;
        while (c < L->len + k) c *= 2;
        L->p = (int64_t *)realloc(L->p, sizeof(int64_t) * 2 * (size_t)c);
        L->cap = c;
    }
    memcpy(L->p + 2 * L->len, pairs, sizeof(int64_t) * 2 * (size_t)k);
    L->len += k;
}

static int cmp_pair(const void *a, const void *b)
{
    const int64_t *x = (const int64_t *)a, *y = (const int64_t *)b;
    if (x[0] != y[0]) return x[0] < y[0] ? -1 : 1;
    return (x[1] > y[1]) - (x[1] < y[1]);
}

int64_t orc_bands_ties(void *h, const double *r, const double *phi, double tol, int64_t cap, int64_t *pairs)
{
    orc_bands *B = (orc_bands *)h;
    double Rw = acosh(B->cR * (1.0 + 2.0 * tol));
    int nt = orc_num_threads();
    orc_pairlist *lists = (orc_pairlist *)calloc((size_t)nt, sizeof(orc_pairlist));
    #pragma omp parallel
    {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        int64_t room = 64;
        int64_t *buf = (int64_t *)malloc(sizeof(int64_t) * 2 * (size_t)room);
        #pragma omp for schedule(dynamic, 256)
        for (int64_t i = 0; i < B->n; ++i) {
            int64_t got = band_query(B, r[i], phi[i], (int32_t)i, NULL, Rw, tol, room, buf);
            if (got > room) { /* more than fit: ask again with room for all */
                room = got;
                buf = (int64_t *)realloc(buf, sizeof(int64_t) * 2 * (size_t)room);
                got = band_query(B, r[i], phi[i], (int32_t)i, NULL, Rw, tol, room, buf);
            }
            if (got > 0) pairlist_add(&lists[t], buf, got);
        }
        free(buf);
    }
    int64_t cnt = 0;
    for (int t = 0; t < nt; ++t) cnt += lists[t].len;
    int64_t *all = (int64_t *)malloc(sizeof(int64_t) * 2 * (size_t)(cnt > 0 ? cnt : 1));
    int64_t k = 0;
    for (int t = 0; t < nt; ++t) {
        if (lists[t].len) memcpy(all + 2 * k, lists[t].p, sizeof(int64_t) * 2 * (size_t)lists[t].len);
        k += lists[t].len;
        free(lists[t].p);
    }
    free(lists);
    qsort(all, (size_t)cnt, sizeof(int64_t) * 2, cmp_pair);
    int64_t w = cnt < cap ? cnt : cap;
    if (w > 0) memcpy(pairs, all, sizeof(int64_t) * 2 * (size_t)w);
    free(all);
    return cnt;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/* ---------------------------------------------------------------------------
 * Graph properties of Sec. 4.1 over a canonical CSR (rows ascending, both
 * directions of every edge).
 *   - Degree tail: the power-law exponent by the discrete maximum-likelihood
 *     approximation of Clauset, Shalizi and Newman (SIAM Review 51, 2009,
 *     Eq. 3.7): gamma = 1 + N / sum ln(d / (d_min - 1/2)) over the N
 *     vertices of degree d >= d_min.  Returned as its two sums.
 *   - Triads: paths of length two, sum over v of d_v (d_v - 1) / 2.
 *   - Triangles: vertex triples u < v < w with all three edges, each counted
 *     once, found by walking N(u) and N(v) together above v; per-vertex
 *     counts (each triangle at its three corners) for local clustering.
 * The clustering coefficient of Sec. 4.1 is the fraction of closed triads:
 * 3 triangles / triads.
 * ------------------------------------------------------------------------- */
void orc_degree_stats(int64_t n, const int64_t *row_off, int64_t d_min, int64_t *out_i, double *out_d)
{
    int64_t max_d = 0, tail = 0, triads = 0;
    double logs = 0.0;
    for (int64_t v = 0; v < n; ++v) {
        const int64_t d = row_off[v + 1] - row_off[v];
        if (d > max_d) max_d = d;
        triads += d * (d - 1) / 2;
        if (d >= d_min) {
            ++tail;
            logs += log((double)d / ((double)d_min - 0.5));
        }
    }
    out_i[0] = row_off[n] - row_off[0];
    out_i[1] = max_d;
    out_i[2] = tail;
    out_i[3] = triads;
    out_d[0] = logs;
}

int64_t orc_triangles(int64_t n, const int64_t *row_off, const int32_t *col_idx, int64_t *t)
{
    int64_t total = 0;
    if (t)
        for (int64_t v = 0; v < n; ++v) t[v] = 0;
    for (int64_t u = 0; u < n; ++u) {
        const int64_t ub = row_off[u], ue = row_off[u + 1];
        for (int64_t a = ub; a < ue; ++a) {
            const int32_t v = col_idx[a];
            if (v <= u) continue;
            /* common neighbours w > v: N(u) after v, N(v) from its first entry above v */
            int64_t i = a + 1, j = row_off[v];
            const int64_t je = row_off[v + 1];
            while (j < je && col_idx[j] <= v) ++j;
            while (i < ue && j < je) {
                if (col_idx[i] < col_idx[j]) ++i;
                else if (col_idx[i] > col_idx[j]) ++j;
                else {
                    ++total;
                    if (t) {
                        ++t[u];
                        ++t[v];
                        ++t[col_idx[i]];
                    }
                    ++i;
                    ++j;
                }
            }
        }
    }
    return total;
}

/* ---------------------------------------------------------------------------
 * Random long-range edges (Sec. 4.2 and the appendix on additional random
 * edges: "adding 0.5 % of edges randomly").  Pair k draws the Philox4x32-10
 * block at counter 2^63 + k, i.e. (k_lo, k_hi + 2^31, 0, 0), key (seed_lo,
 * seed_hi) -- the point draws use counters below 2^31, so the two streams
 * never meet -- and maps each 64-bit half w to the vertex floor(w n / 2^64)
 * (the high word of the 128-bit product).  Self-pairs come out as u == v; the caller drops
 * them, repeats and pairs already in the graph.
 * ------------------------------------------------------------------------- */
void orc_random_pairs(int64_t n, int64_t count, uint64_t seed, int64_t *u, int64_t *v)
{
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    for (int64_t k = 0; k < count; ++k) {
        uint32_t ctr[4] = {(uint32_t)((uint64_t)k & 0xffffffffu), (uint32_t)((uint64_t)k >> 32) | 0x80000000u, 0u, 0u};
        uint32_t x[4];
        orc_philox4x32_10(ctr, key, x);
        uint64_t a = ((uint64_t)x[0] << 32) | (uint64_t)x[1];
        uint64_t b = ((uint64_t)x[2] << 32) | (uint64_t)x[3];
        u[k] = (int64_t)(((unsigned __int128)a * (uint64_t)n) >> 64);
        v[k] = (int64_t)(((unsigned __int128)b * (uint64_t)n) >> 64);
    }
}

/* ---------------------------------------------------------------------------
 * Breadth-first search (Sec. 4.1: the diameter is the longest shortest path;
 * Sec. 4.2: long-range edges shorten it).  dist[v] = hops from source, -1
 * where unreached; returns the eccentricity of source in its component.
 * ------------------------------------------------------------------------- */
int32_t orc_bfs(int64_t n, const int64_t *row_off, const int32_t *col_idx, int64_t source, int32_t *dist)
{
    for (int64_t v = 0; v < n; ++v) dist[v] = -1;
    if (n == 0) return 0;
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int64_t head = 0, tail = 0;
    dist[source] = 0;
    queue[tail++] = (int32_t)source;
    int32_t ecc = 0;
    while (head < tail) {
        const int32_t u = queue[head++];
        const int32_t du = dist[u];
        if (du > ecc) ecc = du;
        for (int64_t k = row_off[u]; k < row_off[u + 1]; ++k) {
            const int32_t w = col_idx[k];
            if (dist[w] < 0) {
                dist[w] = du + 1;
                queue[tail++] = w;
            }
        }
    }
    free(queue);
    return ecc;
}
