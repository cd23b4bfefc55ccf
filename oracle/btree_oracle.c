/*
 * btree_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously-correct CPU statement of the b-tree of
 * "Finding Neighbors in a Forest: A b-tree for SPH Simulations"
 * (arXiv:1910.02639): BuildTree (Algorithm 1, Eqs. 1-4), FindNeighbors
 * (Algorithm 2, Eqs. 5-6), a brute-force O(n^2) neighbour search (the
 * definition of the result), and the FP64 SPH density sum with the M4
 * cubic spline that consumes the lists.
 *
 * Only the tests, the package's smoke check and the benchmark's CPU-baseline
 * leg may load this file.  It shares no code, header or constant with the
 * CUDA library; the library never calls it.
 *
 * Arithmetic: IEEE binary64, round to nearest, no FMA contraction (build with
 * -ffp-contract=off, never -ffast-math), so every expression is evaluated in
 * the order written.
 *
 * Readings of the paper taken here (the paper is silent, garbled or
 * self-contradictory on these points):
 *   - Eq. 1 is evaluated in exact integers: b = smallest integer >= 2 with
 *     b^3 * s >= n (a floating cube root misrounds at perfect cubes).
 *   - Eq. 2 coordinates are clamped to [0, b-1]; a cell whose upper and lower
 *     bound coincide in a dimension puts every particle at coordinate 0 there.
 *   - Eq. 4: u = #{j : n_j <= alpha*s} (empty cells count); the branching
 *     factor is halved (b <- max(2, floor(b/2))) while u > beta*b^3 and b > 2,
 *     i.e. the prose test "r larger than beta" of Sec. 3.1 step 3, not the
 *     inverted test printed in Algorithm 1.  b = 2 is always accepted.
 *   - Child boxes (Sec. 3.1 step 2, equal-size sub-cells): w = (hi-lo)/b,
 *     lo' = lo + c*w, hi' = lo + (c+1)*w, except hi' = hi for c = b-1.
 *   - A cell with more than s particles is a leaf ("oversized") when its depth
 *     has reached 32, or when all its particles fall into one child whose box
 *     equals its own (coincident particles would otherwise recurse forever).
 *   - Leaves are marked by a flag, not by n_j <= s (Algorithm 2), because of
 *     oversized leaves.
 *   - The neighbour predicate is strict: D < R with
 *     D = ((dx*dx + dy*dy) + dz*dz), dx = x_j - x_i in binary64 from the
 *     float inputs, R = (2 h_i)^2 (exact in binary64).  A particle is not its
 *     own neighbour.  Lists hold the min(count, ngmax) smallest indices in
 *     ascending order; unused row entries are -1; counts are uncapped.
 *   - Eqs. 5-6 are applied to the interval [x - Rs, x + Rs] with
 *     Rs = 2h(1 + 2^-30), each end moved one ulp outward, so that the walk
 *     visits every cell that can hold a particle with D < R.
 */
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_DEPTH_MAX 32
static const double ORC_PI = 3.14159265358979323846;

/* ------------------------------------------------------------------ */
/* Eq. 1: branching factor                                            */
/* ------------------------------------------------------------------ */
/* b = ceil((n/s)^(1/k)), k = 3, as the smallest integer b >= 2 with
 * b^3 * s >= n.  Plain linear search: b never exceeds ~1300 for n < 2^31. */
int64_t orc_branching_factor(int64_t n, int64_t s)
{
    int64_t b = 2;
    while (b * b * b * s < n)
        b++;
    return b;
}

/* The same for k = 2 (a two-dimensional tree, Table 1): the smallest b >= 2
 * with b^2 * s >= n. */
int64_t orc_branching_factor2(int64_t n, int64_t s)
{
    int64_t b = 2;
    while (b * b * s < n)
        b++;
    return b;
}

/* ------------------------------------------------------------------ */
/* Eq. 2: sub-cell coordinate of one particle in one dimension        */
/* ------------------------------------------------------------------ */
int64_t orc_child_coord(double x, double lo, double hi, int64_t b)
{
    if (hi == lo)
        return 0;
    double t = (x - lo) / (hi - lo);   /* normalise to the cell */
    double v = t * (double)b;          /* scale by b            */
    double f = floor(v);               /* round down            */
    if (f < 0.0)
        return 0;
    if (f > (double)(b - 1))
        return b - 1;
    return (int64_t)f;
}

/* Eq. 3: sub-cell id, x fastest (W = b). */
int64_t orc_child_id(int64_t c1, int64_t c2, int64_t c3, int64_t b)
{
    return c1 + c2 * b + c3 * b * b;
}

/* ------------------------------------------------------------------ */
/* Eqs. 5-6: range of sub-cells to visit in one dimension             */
/* ------------------------------------------------------------------ */
void orc_cell_range(double x, double two_h, double lo, double hi, int64_t b,
                    int64_t *rmin, int64_t *rmax)
{
    if (hi == lo) {
        *rmin = 0;
        *rmax = 0;
        return;
    }
    double rs = two_h * (1.0 + 0x1p-30);
    double ql = nextafter(x - rs, -INFINITY);
    double qh = nextafter(x + rs, INFINITY);
    double vl = floor(((ql - lo) / (hi - lo)) * (double)b);
    double vh = floor(((qh - lo) / (hi - lo)) * (double)b);
    if (vl < 0.0) vl = 0.0;
    if (vl > (double)(b - 1)) vl = (double)(b - 1);
    if (vh < 0.0) vh = 0.0;
    if (vh > (double)(b - 1)) vh = (double)(b - 1);
    *rmin = (int64_t)vl;
    *rmax = (int64_t)vh;
}

/* ------------------------------------------------------------------ */
/* Neighbour predicate (Algorithm 2, Sec. 3.2)                        */
/* ------------------------------------------------------------------ */
double orc_distance2(float xi, float yi, float zi, float xj, float yj, float zj)
{
    double dx = (double)xj - (double)xi;
    double dy = (double)yj - (double)yi;
    double dz = (double)zj - (double)zi;
    double d = dx * dx + dy * dy;
    d = d + dz * dz;
    return d;
}

double orc_radius2(float h)
{
    double two_h = 2.0 * (double)h;
    return two_h * two_h;
}

static int is_neighbor(const float *x, const float *y, const float *z,
                       int64_t i, int64_t j, double R)
{
    return orc_distance2(x[i], y[i], z[i], x[j], y[j], z[j]) < R;
}

/* ------------------------------------------------------------------ */
/* The tree                                                           */
/* ------------------------------------------------------------------ */
typedef struct {
    double lo[3], hi[3];
    int64_t start, count; /* particles perm[start .. start+count)        */
    int32_t depth;
    int32_t b;            /* branching factor; 0 for a leaf               */
    int64_t slot0;        /* children are nodes child[slot0 .. slot0+b^3) */
    int32_t oversized;    /* leaf holding more than s particles           */
} orc_node;

typedef struct {
    int64_t n, s;
    double alpha, beta;
    int octree;           /* b fixed to 2 at every split (no Eq. 1 / Eq. 4) */
    int dim;              /* k = 3, or 2: cells split in x and y only */
    const float *x, *y, *z;
    int64_t *perm;        /* original particle indices in tree order */
    orc_node *nodes;
    int64_t nnodes, cap_nodes;
    int64_t *child;       /* node index of every sub-cell */
    int64_t nslots, cap_slots;
    int64_t *scratch_perm;
    int64_t *cell;        /* per-particle sub-cell id (scratch) */
    int32_t max_depth;
    int32_t n_oversized;
} orc_tree;

static int64_t push_node(orc_tree *t)
{
    if (t->nnodes == t->cap_nodes) {
        t->cap_nodes = t->cap_nodes ? 2 * t->cap_nodes : 1024;
        t->nodes = (orc_node *)realloc(t->nodes, (size_t)t->cap_nodes * sizeof(orc_node));
    }
    memset(&t->nodes[t->nnodes], 0, sizeof(orc_node));
    return t->nnodes++;
}

static int64_t push_slots(orc_tree *t, int64_t k)
{
    while (t->nslots + k > t->cap_slots) {
        t->cap_slots = t->cap_slots ? 2 * t->cap_slots : 4096;
        t->child = (int64_t *)realloc(t->child, (size_t)t->cap_slots * sizeof(int64_t));
    }
    int64_t base = t->nslots;
    t->nslots += k;
    return base;
}

static double pcoord(const orc_tree *t, int64_t p, int l)
{
    const float *a = l == 0 ? t->x : (l == 1 ? t->y : t->z);
    return (double)a[p];
}

/* Algorithm 1, BuildTree(n, i) for node index ni. */
static void build_node(orc_tree *t, int64_t ni)
{
    orc_node nd = t->nodes[ni];
    if (nd.depth > t->max_depth)
        t->max_depth = nd.depth;
    if (nd.count <= t->s) {
        return; /* leaf */
    }
    if (nd.depth >= ORC_DEPTH_MAX) {
        t->nodes[ni].oversized = 1;
        t->n_oversized++;
        return;
    }

    /* Step 1: branching factor (Eq. 1, k = dim); the octree always halves. */
    int64_t b = t->octree ? 2 : (t->dim == 2 ? orc_branching_factor2(nd.count, t->s)
                                             : orc_branching_factor(nd.count, t->s));
    int64_t *counts = NULL;
    const double under = t->alpha * (double)t->s;
    for (;;) {
        /* Step 2: distribute the particles (Eqs. 2-3) and count n_j; with
         * k = 2 the z coordinate is not split (sub-cell coordinate 0). */
        int64_t ncell = t->dim == 2 ? b * b : b * b * b;
        counts = (int64_t *)realloc(counts, (size_t)ncell * sizeof(int64_t));
        memset(counts, 0, (size_t)ncell * sizeof(int64_t));
        for (int64_t k = 0; k < nd.count; k++) {
            int64_t p = t->perm[nd.start + k];
            int64_t c[3];
            for (int l = 0; l < 3; l++)
                c[l] = (t->dim == 2 && l == 2) ? 0
                                               : orc_child_coord(pcoord(t, p, l), nd.lo[l], nd.hi[l], b);
            int64_t j = orc_child_id(c[0], c[1], c[2], b);
            t->cell[nd.start + k] = j;
            counts[j]++;
        }
        /* Step 3: distribution ratio (Eq. 4) and redistribution. */
        int64_t u = 0;
        for (int64_t j = 0; j < ncell; j++)
            if ((double)counts[j] <= under)
                u++;
        if ((double)u > t->beta * (double)ncell && b > 2) {
            b = b / 2;
            if (b < 2)
                b = 2;
            continue;
        }
        break;
    }
    int64_t ncell = t->dim == 2 ? b * b : b * b * b;

    /* Child boxes: equal-size sub-cells of this cell (bl sub-cells along
     * dimension l: b, or 1 for the unsplit z of k = 2). */
    int64_t bl[3];
    double w[3];
    for (int l = 0; l < 3; l++) {
        bl[l] = (t->dim == 2 && l == 2) ? 1 : b;
        w[l] = (nd.hi[l] - nd.lo[l]) / (double)bl[l];
    }

    /* No-progress guard: everything in one child whose box is this box. */
    int64_t nonempty = 0, only = -1;
    for (int64_t j = 0; j < ncell; j++)
        if (counts[j] > 0) {
            nonempty++;
            only = j;
        }
    if (nonempty == 1) {
        int64_t c[3] = {only % b, (only / b) % b, only / (b * b)};
        int same = 1;
        for (int l = 0; l < 3; l++) {
            double clo = nd.lo[l] + (double)c[l] * w[l];
            double chi = (c[l] == bl[l] - 1) ? nd.hi[l] : nd.lo[l] + (double)(c[l] + 1) * w[l];
            if (clo != nd.lo[l] || chi != nd.hi[l])
                same = 0;
        }
        if (same) {
            t->nodes[ni].oversized = 1;
            t->n_oversized++;
            free(counts);
            return;
        }
    }

    /* Add each particle to its sub-cell: stable counting sort by cell id. */
    int64_t *offs = (int64_t *)malloc((size_t)(ncell + 1) * sizeof(int64_t));
    offs[0] = 0;
    for (int64_t j = 0; j < ncell; j++)
        offs[j + 1] = offs[j] + counts[j];
    int64_t *cursor = (int64_t *)malloc((size_t)ncell * sizeof(int64_t));
    memcpy(cursor, offs, (size_t)ncell * sizeof(int64_t));
    for (int64_t k = 0; k < nd.count; k++) {
        int64_t j = t->cell[nd.start + k];
        t->scratch_perm[nd.start + cursor[j]++] = t->perm[nd.start + k];
    }
    memcpy(t->perm + nd.start, t->scratch_perm + nd.start, (size_t)nd.count * sizeof(int64_t));
    free(cursor);

    int64_t slot0 = push_slots(t, ncell);
    t->nodes[ni].b = (int32_t)b;
    t->nodes[ni].slot0 = slot0;
    for (int64_t j = 0; j < ncell; j++) {
        int64_t c[3] = {j % b, (j / b) % b, j / (b * b)};
        int64_t ci = push_node(t);
        orc_node *ch = &t->nodes[ci];
        for (int l = 0; l < 3; l++) {
            ch->lo[l] = nd.lo[l] + (double)c[l] * w[l];
            ch->hi[l] = (c[l] == bl[l] - 1) ? nd.hi[l] : nd.lo[l] + (double)(c[l] + 1) * w[l];
        }
        ch->start = nd.start + offs[j];
        ch->count = counts[j];
        ch->depth = nd.depth + 1;
        t->child[slot0 + j] = ci;
    }
    free(offs);
    free(counts);
    /* Recurse into every sub-cell holding more than s particles. */
    for (int64_t j = 0; j < ncell; j++) {
        int64_t ci = t->child[slot0 + j];
        if (t->nodes[ci].count > t->s)
            build_node(t, ci);
        else if (t->nodes[ci].depth > t->max_depth)
            t->max_depth = t->nodes[ci].depth;
    }
}

/* octree != 0: the classical octree the paper compares with (Sec. 2: b = 2
 * in every dimension at every level; with b = 2 the ratio test of Eq. 4
 * never halves, so the same BuildTree steps apply). */
orc_tree *orc_build_ex(const float *x, const float *y, const float *z, int64_t n,
                       int64_t s, double alpha, double beta, int octree, int dim)
{
    if (n < 0 || s < 1 || (dim != 2 && dim != 3))
        return NULL;
    orc_tree *t = (orc_tree *)calloc(1, sizeof(orc_tree));
    t->octree = octree;
    t->dim = dim;
    t->n = n;
    t->s = s;
    t->alpha = alpha;
    t->beta = beta;
    t->x = x;
    t->y = y;
    t->z = z;
    size_t np = (size_t)(n > 0 ? n : 1);
    t->perm = (int64_t *)malloc(np * sizeof(int64_t));
    t->scratch_perm = (int64_t *)malloc(np * sizeof(int64_t));
    t->cell = (int64_t *)malloc(np * sizeof(int64_t));
    for (int64_t i = 0; i < n; i++)
        t->perm[i] = i;
    int64_t r = push_node(t);
    /* Root: the bounding box of the input (Eq. 2 "bounds of the domain"). */
    for (int l = 0; l < 3; l++) {
        double lo = INFINITY, hi = -INFINITY;
        for (int64_t i = 0; i < n; i++) {
            double v = pcoord(t, i, l);
            if (v < lo) lo = v;
            if (v > hi) hi = v;
        }
        if (n == 0) {
            lo = 0.0;
            hi = 0.0;
        }
        t->nodes[r].lo[l] = lo;
        t->nodes[r].hi[l] = hi;
    }
    t->nodes[r].start = 0;
    t->nodes[r].count = n;
    t->nodes[r].depth = 0;
    build_node(t, r);
    free(t->scratch_perm);
    free(t->cell);
    t->scratch_perm = NULL;
    t->cell = NULL;
    return t;
}

orc_tree *orc_build2(const float *x, const float *y, const float *z, int64_t n,
                     int64_t s, double alpha, double beta, int octree)
{
    return orc_build_ex(x, y, z, n, s, alpha, beta, octree, 3);
}

orc_tree *orc_build(const float *x, const float *y, const float *z, int64_t n,
                    int64_t s, double alpha, double beta)
{
    return orc_build_ex(x, y, z, n, s, alpha, beta, 0, 3);
}

void orc_free(orc_tree *t)
{
    if (!t)
        return;
    free(t->perm);
    free(t->nodes);
    free(t->child);
    free(t);
}

int64_t orc_num_nodes(const orc_tree *t) { return t->nnodes; }
int64_t orc_num_slots(const orc_tree *t) { return t->nslots; }
int32_t orc_max_depth(const orc_tree *t) { return t->max_depth; }
int32_t orc_num_oversized(const orc_tree *t) { return t->n_oversized; }

/* Export the tree: per node lo[3], hi[3], start, count, depth, b, slot0,
 * oversized; the child table and the particle order. */
void orc_export(const orc_tree *t, double *lo, double *hi, int64_t *start,
                int64_t *count, int32_t *depth, int32_t *b, int64_t *slot0,
                int32_t *oversized, int64_t *child, int64_t *perm)
{
    for (int64_t i = 0; i < t->nnodes; i++) {
        const orc_node *nd = &t->nodes[i];
        for (int l = 0; l < 3; l++) {
            lo[3 * i + l] = nd->lo[l];
            hi[3 * i + l] = nd->hi[l];
        }
        start[i] = nd->start;
        count[i] = nd->count;
        depth[i] = nd->depth;
        b[i] = nd->b;
        slot0[i] = nd->slot0;
        oversized[i] = nd->oversized;
    }
    if (child)
        memcpy(child, t->child, (size_t)t->nslots * sizeof(int64_t));
    if (perm)
        memcpy(perm, t->perm, (size_t)t->n * sizeof(int64_t));
}

/* ------------------------------------------------------------------ */
/* Neighbour lists                                                    */
/* ------------------------------------------------------------------ */
typedef struct {
    int64_t *v;
    int64_t n, cap;
} ivec;

static void ivec_push(ivec *a, int64_t x)
{
    if (a->n == a->cap) {
        a->cap = a->cap ? 2 * a->cap : 256;
        a->v = (int64_t *)realloc(a->v, (size_t)a->cap * sizeof(int64_t));
    }
    a->v[a->n++] = x;
}

static int cmp_i64(const void *a, const void *b)
{
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

/* Algorithm 2, FindNeighbors(p, h_p, i), appending to out. */
static void walk(const orc_tree *t, int64_t ni, int64_t p, double two_h,
                 double R, ivec *out)
{
    const orc_node *nd = &t->nodes[ni];
    if (nd->b == 0) {
        for (int64_t k = 0; k < nd->count; k++) {
            int64_t q = t->perm[nd->start + k];
            if (q != p && is_neighbor(t->x, t->y, t->z, p, q, R))
                ivec_push(out, q);
        }
        return;
    }
    int64_t b = nd->b;
    int64_t rmin[3], rmax[3];
    for (int l = 0; l < 3; l++) {
        if (t->dim == 2 && l == 2) {  /* k = 2: z is one unsplit sub-cell */
            rmin[l] = 0;
            rmax[l] = 0;
            continue;
        }
        orc_cell_range(pcoord(t, p, l), two_h, nd->lo[l], nd->hi[l], b, &rmin[l], &rmax[l]);
    }
    for (int64_t c3 = rmin[2]; c3 <= rmax[2]; c3++)
        for (int64_t c2 = rmin[1]; c2 <= rmax[1]; c2++)
            for (int64_t c1 = rmin[0]; c1 <= rmax[0]; c1++) {
                int64_t j = orc_child_id(c1, c2, c3, b);
                walk(t, t->child[nd->slot0 + j], p, two_h, R, out);
            }
}

/* Sort ascending, write the capped row and the uncapped count. */
static void emit_row(ivec *a, int64_t ngmax, int32_t *row, int32_t *count)
{
    qsort(a->v, (size_t)a->n, sizeof(int64_t), cmp_i64);
    *count = (int32_t)a->n;
    for (int64_t k = 0; k < ngmax; k++)
        row[k] = k < a->n ? (int32_t)a->v[k] : -1;
}

/* Tree-walk neighbour lists for query particles [q0, q1); row k of nbrs
 * belongs to particle q0 + k. */
void orc_find_tree(const orc_tree *t, const float *h, int64_t q0, int64_t q1,
                   int64_t ngmax, int32_t *nbrs, int32_t *counts)
{
#pragma omp parallel
    {
        ivec a = {0, 0, 0};
#pragma omp for schedule(dynamic, 256)
        for (int64_t p = q0; p < q1; p++) {
            a.n = 0;
            if (t->nnodes > 0 && t->n > 0)
                walk(t, 0, p, 2.0 * (double)h[p], orc_radius2(h[p]), &a);
            emit_row(&a, ngmax, nbrs + (p - q0) * ngmax, counts + (p - q0));
        }
        free(a.v);
    }
}

/* Brute-force O(n^2) lists: the definition of the result. */
void orc_find_brute(const float *x, const float *y, const float *z,
                    const float *h, int64_t n, int64_t q0, int64_t q1,
                    int64_t ngmax, int32_t *nbrs, int32_t *counts)
{
#pragma omp parallel
    {
        ivec a = {0, 0, 0};
#pragma omp for schedule(dynamic, 64)
        for (int64_t p = q0; p < q1; p++) {
            a.n = 0;
            double R = orc_radius2(h[p]);
            for (int64_t q = 0; q < n; q++)
                if (q != p && is_neighbor(x, y, z, p, q, R))
                    ivec_push(&a, q);
            emit_row(&a, ngmax, nbrs + (p - q0) * ngmax, counts + (p - q0));
        }
        free(a.v);
    }
}

/* ------------------------------------------------------------------ */
/* SPH density with the M4 cubic spline (support 2h)                  */
/* ------------------------------------------------------------------ */
/* Dimensionless M4 shape: 1 - 1.5 q^2 + 0.75 q^3 on [0,1),
 * 0.25 (2-q)^3 on [1,2), 0 beyond. */
double orc_m4_shape(double q)
{
    if (q < 1.0)
        return 1.0 - 1.5 * q * q + 0.75 * q * q * q;
    if (q < 2.0) {
        double a = 2.0 - q;
        return 0.25 * a * a * a;
    }
    return 0.0;
}

/* W(r, h) = shape(r/h) / (pi h^3). */
double orc_kernel_w(double r, double h)
{
    return orc_m4_shape(r / h) / (ORC_PI * h * h * h);
}

/* rho_i = m_i W(0, h_i) + sum_{j in N(i)} m_j W(r_ij, h_i), with N(i) the
 * uncapped neighbour set found by the tree walk; gather form with h_i. */
void orc_density(const orc_tree *t, const float *h, const float *m,
                 int64_t q0, int64_t q1, double *rho)
{
#pragma omp parallel
    {
        ivec a = {0, 0, 0};
#pragma omp for schedule(dynamic, 256)
        for (int64_t p = q0; p < q1; p++) {
            a.n = 0;
            if (t->nnodes > 0 && t->n > 0)
                walk(t, 0, p, 2.0 * (double)h[p], orc_radius2(h[p]), &a);
            qsort(a.v, (size_t)a.n, sizeof(int64_t), cmp_i64);
            double hp = (double)h[p];
            double sum = (double)m[p] * orc_kernel_w(0.0, hp);
            for (int64_t k = 0; k < a.n; k++) {
                int64_t q = a.v[k];
                double d = orc_distance2(t->x[p], t->y[p], t->z[p], t->x[q], t->y[q], t->z[q]);
                sum += (double)m[q] * orc_kernel_w(sqrt(d), hp);
            }
            rho[p - q0] = sum;
        }
        free(a.v);
    }
}

int orc_num_threads(void)
{
    int n = 1;
#pragma omp parallel
    {
#pragma omp single
        {
#ifdef _OPENMP
            n = omp_get_num_threads();
#endif
        }
    }
    return n;
}
