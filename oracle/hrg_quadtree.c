/* hrg_quadtree.c -- the paper's own generator (Algorithm 1 with the polar
 * quadtree of Sec. 3) on the CPU -- TEST AND BASELINE INFRASTRUCTURE.
 *
 * A second CPU program beside the oracle: bench.py times it as the paper's
 * method on the host cores, and tests check it against the oracle's brute
 * force.  It is not the parity reference (its Euclidean test in the Poincare
 * disk carries the rounding of that model, which grows with R), and it shares
 * no code with the generator library.
 *
 * Following Algorithm 1 and Sec. 3:
 *   - mapToPoincare (Appendix B.2): r_E = sqrt((cosh r - 1)/(cosh r + 1)),
 *     computed as tanh(r / 2) (the same value without the cancellation);
 *   - a polar quadtree over [0, 2pi) x [0, r_E(R)): a node is responsible for
 *     the points with min_phi <= phi < max_phi and min_r <= r_E < max_r; a
 *     leaf holding more than `capacity` points splits into four children, the
 *     angle range halved and the radial range split where the probability
 *     mass is halved (Eq. (3), in native coordinates, then mapped);
 *   - the points inserted one by one in vertex order;
 *   - for every vertex (in parallel) the query circle of Proposition 1:
 *     centre (phi_h, 2 r_h / (ab + 2)), radius
 *     sqrt((2 r_h / (ab + 2))^2 - (2 r_h^2 - ab) / (ab + 2)), a = cosh R - 1,
 *     b = 1 - r_h^2; the tree is searched from the root, every cell whose
 *     closest point to the centre lies within the radius is visited, and a
 *     leaf point is a neighbour when its Euclidean distance to the centre is
 *     below the radius (the vertex itself excluded).
 * The paper leaves the leaf capacity and the cell-circle test open (its
 * proofs take capacity 1); the capacity is a parameter here, and the cell
 * test is the exact distance from the centre to the cell (an annular
 * sector), with the radius widened by 1e-12 relative so that rounding never
 * drops a cell.  Rows are sorted ascending (canonical CSR).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    double min_phi, max_phi, min_r, max_r;  /* Poincare radii */
    double min_rh, max_rh;                  /* the same radial bounds, native */
    int32_t child;                          /* first of four children, -1 for a leaf */
    int32_t depth;
    int32_t cnt, cap;
    int32_t *ids;
} qt_node;

typedef struct {
    qt_node *nodes;
    int32_t n_nodes, cap_nodes;
    int32_t leaf_capacity;
    double alpha;
    const double *phi, *re;  /* per vertex: angle and Poincare radius */
    double *x, *y;           /* per vertex: Cartesian position in the disk */
} qt_tree;

enum { kMaxDepth = 48 };  /* the search stack below holds 3 * kMaxDepth + 4 nodes */

static int32_t qt_new_node(qt_tree *T, double p0, double p1, double rh0, double rh1, int32_t depth)
{
    if (T->n_nodes == T->cap_nodes) {
        T->cap_nodes = T->cap_nodes ? 2 * T->cap_nodes : 64;
        T->nodes = (qt_node *)realloc(T->nodes, sizeof(qt_node) * (size_t)T->cap_nodes);
    }
    qt_node *c = &T->nodes[T->n_nodes];
    memset(c, 0, sizeof *c);
    c->min_phi = p0;
    c->max_phi = p1;
    c->min_rh = rh0;
    c->max_rh = rh1;
    c->min_r = tanh(rh0 / 2.0);
    c->max_r = tanh(rh1 / 2.0);
    c->child = -1;
    c->depth = depth;
    return T->n_nodes++;
}

static void qt_leaf_push(qt_node *L, int32_t id)
{
    if (L->cnt == L->cap) {
        L->cap = L->cap ? 2 * L->cap : 16;
        L->ids = (int32_t *)realloc(L->ids, sizeof(int32_t) * (size_t)L->cap);
    }
    L->ids[L->cnt++] = id;
}

static int qt_quadrant(const qt_node *nd, const qt_node *c0, double phi, double re)
{
    /* children: 0 = (low phi, low r), 1 = (low phi, high r), 2 = (high phi, low r), 3 = (high phi, high r) */
    (void)nd;
    const int hi_phi = phi >= c0[2].min_phi;
    const int hi_r = re >= c0[1].min_r;
    return 2 * hi_phi + hi_r;
}

static void qt_insert(qt_tree *T, int32_t node, int32_t id);

static void qt_split(qt_tree *T, int32_t node)
{
    qt_node nd = T->nodes[node];
    const double mid_phi = 0.5 * (nd.min_phi + nd.max_phi);
    /* Eq. (3): the radius that halves the probability mass of the cell */
    const double mid_rh = acosh(0.5 * (cosh(T->alpha * nd.max_rh) + cosh(T->alpha * nd.min_rh))) / T->alpha;
    const int32_t c = qt_new_node(T, nd.min_phi, mid_phi, nd.min_rh, mid_rh, nd.depth + 1);
    qt_new_node(T, nd.min_phi, mid_phi, mid_rh, nd.max_rh, nd.depth + 1);
    qt_new_node(T, mid_phi, nd.max_phi, nd.min_rh, mid_rh, nd.depth + 1);
    qt_new_node(T, mid_phi, nd.max_phi, mid_rh, nd.max_rh, nd.depth + 1);
    int32_t *ids = T->nodes[node].ids;
    const int32_t cnt = T->nodes[node].cnt;
    T->nodes[node].ids = NULL;
    T->nodes[node].cnt = T->nodes[node].cap = 0;
    T->nodes[node].child = c;
    for (int32_t k = 0; k < cnt; ++k) qt_insert(T, node, ids[k]);
    free(ids);
}

static void qt_insert(qt_tree *T, int32_t node, int32_t id)
{
    const double phi = T->phi[id], re = T->re[id];
    while (T->nodes[node].child >= 0) {
        const int32_t c = T->nodes[node].child;
        node = c + qt_quadrant(&T->nodes[node], &T->nodes[c], phi, re);
    }
    qt_leaf_push(&T->nodes[node], id);
    /* a leaf at depth kMaxDepth keeps any number of points (coinciding points
     * would otherwise split forever) */
    if (T->nodes[node].cnt > T->leaf_capacity && T->nodes[node].depth < kMaxDepth) qt_split(T, node);
}

/* squared distance from the point (pc, rc) (polar) to the annular sector of nd */
static double qt_cell_dist2(const qt_node *nd, double pc, double rc)
{
    if (pc >= nd->min_phi && pc <= nd->max_phi) {
        const double d = rc < nd->min_r ? nd->min_r - rc : (rc > nd->max_r ? rc - nd->max_r : 0.0);
        return d * d;
    }
    double best = INFINITY;
    const double rays[2] = {nd->min_phi, nd->max_phi};
    for (int k = 0; k < 2; ++k) {
        double dphi = fabs(pc - rays[k]);
        if (dphi > M_PI) dphi = 2.0 * M_PI - dphi;
        const double cs = cos(dphi);
        double t = rc * cs;
        if (t < nd->min_r) t = nd->min_r;
        if (t > nd->max_r) t = nd->max_r;
        const double d2 = rc * rc + t * t - 2.0 * rc * t * cs;
        if (d2 < best) best = d2;
    }
    return best < 0.0 ? 0.0 : best;
}

typedef struct {
    double pc, rc, cx, cy, rad2, rad2_cells;
    int32_t self;
} qt_query;

/* neighbours of one query into out (when non-null); returns their number */
static int64_t qt_search(const qt_tree *T, const qt_query *q, int32_t *out)
{
    int32_t stack[256];
    int sp = 0;
    int64_t found = 0;
    stack[sp++] = 0;
    while (sp > 0) {
        const qt_node *nd = &T->nodes[stack[--sp]];
        if (qt_cell_dist2(nd, q->pc, q->rc) > q->rad2_cells) continue;
        if (nd->child >= 0) {
            for (int k = 3; k >= 0; --k) stack[sp++] = nd->child + k;
            continue;
        }
        for (int32_t k = 0; k < nd->cnt; ++k) {
            const int32_t id = nd->ids[k];
            if (id == q->self) continue;
            const double dx = T->x[id] - q->cx, dy = T->y[id] - q->cy;
            if (dx * dx + dy * dy < q->rad2) {
                if (out) out[found] = id;
                ++found;
            }
        }
    }
    return found;
}

static void qt_make_query(double R, double phi, double rh, int32_t self, qt_query *q)
{
    /* Proposition 1 */
    const double r_h = tanh(rh / 2.0);
    const double a = cosh(R) - 1.0, b = 1.0 - r_h * r_h;
    const double c = 2.0 * r_h / (a * b + 2.0);
    double rad2 = c * c - (2.0 * r_h * r_h - a * b) / (a * b + 2.0);
    if (rad2 < 0.0) rad2 = 0.0;
    q->pc = phi;
    q->rc = c;
    q->cx = c * cos(phi);
    q->cy = c * sin(phi);
    q->rad2 = rad2;
    const double wide = sqrt(rad2) * (1.0 + 1e-12) + 1e-15;
    q->rad2_cells = wide * wide;
    q->self = self;
}

static int cmp_id(const void *a, const void *b)
{
    const int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

typedef struct {
    qt_tree T;
    int64_t n;
    const double *r, *phi;
    double R;
    double *re;
} qt_handle;

/* Builds the tree: mapToPoincare, then insertion in vertex order.  The
 * handle keeps r and phi (caller owned) until orc_quadtree_free. */
void *orc_quadtree_build(int64_t n, const double *r, const double *phi, double R, double alpha, int32_t capacity)
{
    qt_handle *h = (qt_handle *)calloc(1, sizeof(qt_handle));
    h->n = n;
    h->r = r;
    h->phi = phi;
    h->R = R;
    h->T.leaf_capacity = capacity > 0 ? capacity : 1;
    h->T.alpha = alpha;
    h->re = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    h->T.x = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    h->T.y = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    h->T.phi = phi;
    h->T.re = h->re;
    for (int64_t i = 0; i < n; ++i) {
        h->re[i] = tanh(r[i] / 2.0); /* mapToPoincare */
        h->T.x[i] = h->re[i] * cos(phi[i]);
        h->T.y[i] = h->re[i] * sin(phi[i]);
    }
    qt_new_node(&h->T, 0.0, 2.0 * M_PI, 0.0, R, 0);
    for (int64_t i = 0; i < n; ++i) qt_insert(&h->T, 0, (int32_t)i);
    return h;
}

void orc_quadtree_free(void *hv)
{
    qt_handle *h = (qt_handle *)hv;
    if (!h) return;
    for (int32_t k = 0; k < h->T.n_nodes; ++k) free(h->T.nodes[k].ids);
    free(h->T.nodes);
    free(h->re);
    free(h->T.x);
    free(h->T.y);
    free(h);
}

/* Every vertex's range query (parallel over vertices): deg[n]; returns 2m. */
int64_t orc_quadtree_degrees(void *hv, int64_t *deg)
{
    qt_handle *h = (qt_handle *)hv;
    int64_t total = 0;
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : total)
    for (int64_t i = 0; i < h->n; ++i) {
        qt_query q;
        qt_make_query(h->R, h->phi[i], h->r[i], (int32_t)i, &q);
        deg[i] = qt_search(&h->T, &q, NULL);
        total += deg[i];
    }
    return total;
}

/* The queries again, every row written at row_off and sorted ascending. */
void orc_quadtree_fill(void *hv, const int64_t *row_off, int32_t *col_idx)
{
    qt_handle *h = (qt_handle *)hv;
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < h->n; ++i) {
        qt_query q;
        qt_make_query(h->R, h->phi[i], h->r[i], (int32_t)i, &q);
        int32_t *row = col_idx + row_off[i];
        const int64_t d = qt_search(&h->T, &q, row);
        qsort(row, (size_t)d, sizeof(int32_t), cmp_id);
    }
}

int32_t orc_quadtree_depth_counts(int64_t n, const double *r, const double *phi, double R, double alpha,
                                  int32_t capacity, int32_t depth, int64_t *counts)
{
    /* points per cell of the complete depth-`depth` level (4^depth cells in
     * the order (phi half, r half) per level), for Lemma 4 checks; returns the
     * number of nodes the tree grew to */
    qt_tree T;
    memset(&T, 0, sizeof T);
    T.leaf_capacity = capacity > 0 ? capacity : 1;
    T.alpha = alpha;
    double *re = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    T.x = T.y = NULL;
    T.phi = phi;
    T.re = re;
    for (int64_t i = 0; i < n; ++i) re[i] = tanh(r[i] / 2.0);
    qt_new_node(&T, 0.0, 2.0 * M_PI, 0.0, R, 0);
    for (int64_t i = 0; i < n; ++i) qt_insert(&T, 0, (int32_t)i);
    int64_t cells = 1;
    for (int32_t k = 0; k < depth; ++k) cells *= 4;
    for (int64_t c = 0; c < cells; ++c) counts[c] = 0;
    for (int64_t i = 0; i < n; ++i) {
        int32_t node = 0;
        int64_t cell = 0;
        for (int32_t k = 0; k < depth; ++k) {
            const int32_t c = T.nodes[node].child;
            if (c < 0) {
                cell = -1;
                break;
            }
            const int quad = qt_quadrant(&T.nodes[node], &T.nodes[c], phi[i], re[i]);
            cell = 4 * cell + quad;
            node = c + quad;
        }
        if (cell >= 0) ++counts[cell];
    }
    const int32_t nodes = T.n_nodes;
    for (int32_t k = 0; k < T.n_nodes; ++k) free(T.nodes[k].ids);
    free(T.nodes);
    free(re);
    return nodes;
}

/* Proposition 1's Euclidean circle for the query (phi, rh): out[0] = centre
 * radius (on the ray at phi), out[1] = circle radius (test access). */
void orc_quadtree_circle(double R, double phi, double rh, double *out)
{
    qt_query q;
    qt_make_query(R, phi, rh, -1, &q);
    out[0] = q.rc;
    out[1] = sqrt(q.rad2);
}
